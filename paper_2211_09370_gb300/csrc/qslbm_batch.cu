// Batched stepping: many independent pipes of uneven size and parameters
// advance together, every phase of a flow step being one fused launch over all
// instances' work.  The time loop is captured into a CUDA graph (one graph per
// step, replayed); ping-pong parities live in device memory so the same graph
// serves every step.  Instances are ordered by N_mag (descending): sweep s only
// touches the prefix of instances with N_mag > s.  The node-parallel sweep
// kernel is persistent (grid-stride over the work list) with its block size
// and grid chosen by a timing autotuner when the batch is built.
//
// The per-node arithmetic is the single-instance code (march_tile, the IB sums
// of ib_plane, force_node, flow_node), so a batched instance follows the same
// expressions as one stepped alone with the split sweep kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "qslbm.h"
#include "qslbm_groups.cuh"
#include "qslbm_internal.h"
#include "qslbm_kernels.cuh"

namespace qslbm {

void set_last_error(const std::string& msg);
State& handle_state_mut(qslbm_handle* h);

template <typename T>
struct InstDesc {
    Geo g;
    int n_mag;
    int flow_q;      // 19 or 27: the instance's 3-D flow lattice
    int bpar, fpar;  // parity of b and of (drho, u) at the start of the current step
    int bpp;         // node blocks per plane
    T* b[2];
    T* u[2];
    T* drho[2];
    T* F;
    long long* tdev;
    SweepCoef<T> sc;
    ForceCoef<T> fc;
    FlowCoef<T> flc;
    IBView<T> ibm, ibu;
};

// instance owning work item w of a prefix table first[0..k]
__device__ __forceinline__ int find_inst(const int* __restrict__ first, int k, int w) {
    int lo = 0, hi = k;  // first[lo] <= w < first[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (first[mid] <= w)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Persistent z-marching sweep over every active instance's tiles: work item w
// is (instance, tile x, tile y, z chunk of `chunk` planes) in the prefix table
// `first`.
// XY: some instance has an in-plane applied field (QSLBM_B0_FIELD); TY: rows
// of the tile (the autotuner's choice; results do not depend on it).
template <typename T, bool XY, int TY>
__global__ void __launch_bounds__(kMarchTX* TY) k_batch_sweep(const InstDesc<T>* __restrict__ d,
                                                              const int* __restrict__ first, int kact, int s,
                                                              int chunk) {
    __shared__ MarchTile<T, TY> tile;
    pdl_trigger();  // the IB pass may be scheduled as these CTAs exit
    pdl_wait();     // b comes from the kernel before this one
    const int total = first[kact];
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int i = find_inst(first, kact, w);
        const InstDesc<T>& D = d[i];
        const int local = w - first[i];
        const int tiles_x = (D.g.nx + kMarchTX - 1) / kMarchTX;
        const int tiles_y = (D.g.ny + TY - 1) / TY;
        const int bz = local / (tiles_x * tiles_y);
        const int r = local - bz * tiles_x * tiles_y;
        const int by = r / tiles_x, bx = r - by * tiles_x;
        const int par = (D.bpar + s) & 1;
        march_tile<T, XY, TY>(D.g, D.b[par], D.b[par ^ 1], D.u[D.fpar], D.sc, bx, by, bz, chunk, tile);
        __syncthreads();
    }
}

// Two-phase IB over every active instance: markers, then (next launch) shell
// nodes; w indexes the prefix tables of markers / shell nodes.
template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_batch_ib_markers(const InstDesc<T>* __restrict__ d,
                                                                   const int* __restrict__ mfirst, int kact, int s) {
    const int w = blockIdx.x * kNodeThreads + threadIdx.x;
    if (w >= mfirst[kact]) return;
    const int i = find_inst(mfirst, kact, w);
    const InstDesc<T>& D = d[i];
    ib_marker<T>(D.ibm, D.b[((D.bpar + s) & 1) ^ 1], (int)D.g.n, w - mfirst[i]);
}

template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_batch_ib_shell(const InstDesc<T>* __restrict__ d,
                                                                 const int* __restrict__ sfirst, int kact, int s) {
    const int w = blockIdx.x * kNodeThreads + threadIdx.x;
    if (w >= sfirst[kact]) return;
    const int i = find_inst(sfirst, kact, w);
    const InstDesc<T>& D = d[i];
    ib_shell<T>(D.ibm, D.b[((D.bpar + s) & 1) ^ 1], (int)D.g.n, w - sfirst[i]);
}

// The staged IB corrector over every active instance: one CTA per
// (instance, plane) in the plane prefix table; shared memory for the largest
// ring and shell of the batch.
template <typename T, int U>
__global__ void __launch_bounds__(kNodeThreads, (kIbStagedMinBlocks<T, U>)) k_batch_ib_staged(const InstDesc<T>* __restrict__ d,
                                                                  const int* __restrict__ pfirst, int kact, int s,
                                                                  int max_ring, int max_shell) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();  // the next sweep may be scheduled as these CTAs exit
    const int i = find_inst(pfirst, kact, blockIdx.x);
    const InstDesc<T>& D = d[i];
    const int z = blockIdx.x - pfirst[i];
    T* f = D.b[((D.bpar + s) & 1) ^ 1];
    ib_staged_plane<T, kNodeThreads, U>(D.ibm, f, (int)D.g.n, z * D.g.nx * D.g.ny, D.ibm.zinv ? 0 : z, max_ring,
                                     max_shell, smem_raw);
}

template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_batch_ib(const InstDesc<T>* __restrict__ d,
                                                           const int* __restrict__ pfirst, int kact, int s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sdelta = reinterpret_cast<T*>(smem_raw);
    const int i = find_inst(pfirst, kact, blockIdx.x);
    const InstDesc<T>& D = d[i];
    const int z = blockIdx.x - pfirst[i];
    T* f = D.b[((D.bpar + s) & 1) ^ 1];
    const long long n = D.g.n;
    ib_plane<T>(D.ibm, f, f + n, f + 2 * n, (long long)z * D.g.nx * D.g.ny, D.ibm.zinv ? 0 : z, sdelta);
}

template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_batch_force(const InstDesc<T>* __restrict__ d,
                                                              const int* __restrict__ pfirst, int k) {
    const int i = find_inst(pfirst, k, blockIdx.x);
    const InstDesc<T>& D = d[i];
    const int z = blockIdx.x - pfirst[i];
    const int nx = D.g.nx, ny = D.g.ny, P = nx * ny;
    const T fb = body_force_at(D.fc, *D.tdev);
    const T* b = D.b[(D.bpar + D.n_mag) & 1];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int y = p / nx;
        const int x = p - y * nx;
        if (D.flow_q == 27)  // uniform across the CTA (one instance plane)
            force_node<T, 3, 27>(b, D.F, D.g.n, nx, ny, D.g.nz, x, y, z, (long long)z * P + p, D.fc, fb);
        else
            force_node<T, 3>(b, D.F, D.g.n, nx, ny, D.g.nz, x, y, z, (long long)z * P + p, D.fc, fb);
    }
}

template <typename T>
__global__ void __launch_bounds__(kPlaneThreads) k_batch_flow(InstDesc<T>* __restrict__ d, const int* __restrict__ pfirst,
                                                              int k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sdelta = reinterpret_cast<T*>(smem_raw);
    const int i = find_inst(pfirst, k, blockIdx.x);
    const InstDesc<T>& D = d[i];
    const int z = blockIdx.x - pfirst[i];
    const int nx = D.g.nx, ny = D.g.ny, nz = D.g.nz;
    const long long n = D.g.n, P = (long long)nx * ny, base = (long long)z * P;
    const T* dr = D.drho[D.fpar];
    const T* u = D.u[D.fpar];
    T* dro = D.drho[D.fpar ^ 1];
    T* uo = D.u[D.fpar ^ 1];
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int y = p / nx;
        const int x = p - y * nx;
        if (D.flow_q == 27)
            flow_node<T, 3, 27>(dr, u, D.F, dro, uo, n, nx, ny, nz, x, y, z, base + p, D.flc);
        else
            flow_node<T, 3>(dr, u, D.F, dro, uo, n, nx, ny, nz, x, y, z, base + p, D.flc);
    }
    ib_plane<T>(D.ibu, uo, uo + n, uo + 2 * n, base, D.ibu.zinv ? 0 : z, sdelta);
    if (z == 0 && threadIdx.x == 0) *D.tdev += 1;
}

template <typename T>
__global__ void k_batch_advance(InstDesc<T>* d, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    d[i].bpar ^= d[i].n_mag & 1;
    d[i].fpar ^= 1;
}

}  // namespace qslbm

using qslbm::State;

struct qslbm_batch {
    std::vector<qslbm_handle*> members;  // marching members by N_mag (descending), then the resident groups' members
    std::vector<int> order;              // order[k] = caller's index of member k
    std::vector<int> rank;               // rank[caller index] = k
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int precision = QSLBM_FP32;
    void* desc = nullptr;                // InstDesc<T>[K]
    int* first = nullptr;                // node-block prefix [K + 1]
    int* pfirst = nullptr;               // plane prefix [K + 1]
    int* mfirst = nullptr;               // marker prefix [K + 1]
    int* sfirst = nullptr;               // shell-node prefix [K + 1]
    std::vector<int> h_first, h_pfirst, h_mfirst, h_sfirst;
    std::vector<int> active;             // active[s] = instances with N_mag > s
    int max_nmag = 0;
    int capacity = 0;                    // instances the device tables can hold
    bool owns_members = true;
    bool tuned = false;
    size_t ib_smem = 0;
    size_t ib_staged_smem = 0;  // shared memory of k_batch_ib_staged, 0 when it does not fit
    int max_ring = 1;           // largest ring of the batch (layout of that shared memory)
    int max_shell = 1;          // largest shell of the batch
    int chunk = 16;             // z planes per work item of the marching sweep
    int sms = 1;                // SMs of the device
    bool has_field = false;     // some member has an in-plane applied field
    int threads = 256, grid = 0;         // autotuned sweep launch
    bool pdl = false;                    // autotuned: programmatic dependent launches of the marching route
    cudaGraphExec_t graph = nullptr;        // one flow step
    cudaGraphExec_t graph_chunk = nullptr;  // chunk_steps flow steps
    int chunk_steps = 1;
    int chunk_target = 1000;                // steps a chunk graph should hold
    long long steps = 0;
    long long device_bytes = 0;
    std::vector<double> tune_us;         // timing of each candidate
    // resident groups (FP32): members [kmarch, K) run all their sweeps in one
    // cooperative launch of k_batch_resident, a group of whole planes per CTA
    int kmarch = 0;
    std::vector<int> gplanes;            // per member: planes per group (0: marching)
    int ngroups = 0;
    size_t group_smem = 0;
    std::vector<qslbm::GroupDesc> h_groups;
    qslbm::GroupDesc* groups = nullptr;
    int groups_cap = 0;
    float* xbuf = nullptr;               // exchange planes of every group
    long long xbuf_cap = 0;              // floats
    unsigned* gflags = nullptr;          // [groups_cap] sweep counters
    int* gerr = nullptr;                 // 1: a neighbour wait timed out
    int gcap = -1, goptin = 0;           // co-resident CTAs of the group kernel and its shared memory (bytes)
    cudaError_t launch_err = cudaSuccess;  // a launch of the group kernel that failed
};

namespace {

// An argument refused on the host, with its reason left in qslbm_last_error.
int refuse(const char* why) {
    qslbm::set_last_error(why);
    return QSLBM_EINVAL;
}

int fail(cudaError_t e, const char* what) {
    qslbm::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return QSLBM_ECUDA;
}

#define BCHK(call)                                        \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fail(e_, #call);    \
    } while (0)

template <typename T>
qslbm::InstDesc<T> make_desc(const State& s) {
    qslbm::InstDesc<T> D;
    std::memset(&D, 0, sizeof(D));
    D.g = qslbm::Geo{s.nx, s.ny, s.nz, s.n};
    D.n_mag = s.units.n_mag;
    D.flow_q = s.units.flow_q;
    D.bpar = s.bcur;
    D.fpar = s.fcur;
    D.bpp = (s.nx * s.ny + qslbm::kNodeThreads - 1) / qslbm::kNodeThreads;
    for (int a = 0; a < 2; ++a) {
        D.b[a] = (T*)s.b[a];
        D.u[a] = (T*)s.u[a];
        D.drho[a] = (T*)s.drho[a];
    }
    D.F = (T*)s.F;
    D.tdev = s.tdev;
    sweep_weights(s, D.sc.w0, D.sc.w1, D.sc.kappa);
    for (int a = 0; a < 3; ++a) D.sc.be[a] = (T)s.be[a];
    D.sc.bext_z = (const T*)s.bext_z;
    D.sc.bext_xy = (const T*)s.bext_xy;
    D.sc.strict_qs = s.p.strict_qs;
    D.sc.sq = s.p.strict_qs ? T(0) : T(1);
    D.fc.F0 = s.units.F0;
    D.fc.amp = s.p.force_amp;
    D.fc.omega = s.omega;
    D.fc.axis = s.axis;
    for (int a = 0; a < 3; ++a) D.fc.be[a] = (T)s.be[a];
    D.fc.bext_z = (const T*)s.bext_z;
    D.fc.bext_xy = (const T*)s.bext_xy;
    D.flc.tau = (T)s.units.tau;
    D.flc.kforce = (T)(1.0 - 1.0 / (2.0 * s.units.tau));
    D.flc.mac = s.p.flow_scheme == QSLBM_FLOW_MACROSCOPIC;
    D.flc.ig = (T)s.ig;
    D.flc.ig2 = (T)(s.ig * s.ig);
    for (int m = 0; m < 2; ++m) {
        qslbm::IBView<T>& v = m ? D.ibu : D.ibm;
        v.ring_off = s.ib.ring_off;
        v.mk_q = s.ib.mk_q;
        v.mk_w = (const T*)s.ib.mk_w;
        v.mk_s = (const T*)(m ? s.ib.mk_s : s.ib.mk_sm);
        v.shell_off = s.ib.shell_off;
        v.shell_xy = s.ib.shell_xy;
        v.csr_off = s.ib.csr_off;
        v.csr_m = s.ib.csr_m;
        v.csr_w = (const T*)s.ib.csr_w;
        v.mk_base = s.ib.mk_base;
        v.shell_node = s.ib.shell_node;
        v.csr_mg = s.ib.csr_mg;
        v.delta = (T*)s.ib.delta;
        v.nm = s.ib.nm;
        v.ns = s.ib.ns;
        v.zinv = s.ib.zinv;
        v.mk_slot = s.ib.mk_slot;
        v.pad_m = s.ib.pad_m;
        v.pad_w = (const T*)s.ib.pad_w;
        v.pad_k = s.ib.pad_k;
    }
    return D;
}

// A launch that may begin while the previous kernel in the stream finishes
// (programmatic dependent launch; the kernel waits for that kernel's results).
template <typename... KArgs, typename... Args>
void launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);  // errors end the graph capture
}

template <typename T>
void launch_sweep(qslbm_batch& B, int s, int threads, int grid, cudaStream_t st) {
    const int kact = B.active[s];
    if (kact == 0) return;
    const int total = B.h_first[kact];
    const int g = grid > 0 ? std::min(grid, total) : total;
    const auto* d = (const qslbm::InstDesc<T>*)B.desc;
    // threads = kMarchTX x the tile's rows (4, 8 or 16)
    auto run = [&](auto kernel) {
        launch_pdl(B.pdl, kernel, dim3(g), dim3(threads), 0, st, d, (const int*)B.first, kact, s, B.chunk);
    };
    if (B.has_field) {
        if (threads == qslbm::kMarchTX * 4) run(qslbm::k_batch_sweep<T, true, 4>);
        else if (threads == qslbm::kMarchTX * 16) run(qslbm::k_batch_sweep<T, true, 16>);
        else run(qslbm::k_batch_sweep<T, true, 8>);
    } else {
        if (threads == qslbm::kMarchTX * 4) run(qslbm::k_batch_sweep<T, false, 4>);
        else if (threads == qslbm::kMarchTX * 16) run(qslbm::k_batch_sweep<T, false, 16>);
        else run(qslbm::k_batch_sweep<T, false, 8>);
    }
    const int nm = B.h_mfirst[kact], ns = B.h_sfirst[kact];
    if (nm > 0 && B.ib_staged_smem > 0) {
        const int np = B.h_pfirst[kact], R = B.max_ring, S = B.max_shell;
        const size_t sm = B.ib_staged_smem;
        const dim3 ig((unsigned)np), ib(qslbm::kNodeThreads);
        const int* pf = B.pfirst;
        switch (qslbm::ib_staged_unroll(S, np, B.sms)) {
            case 1: launch_pdl(B.pdl, qslbm::k_batch_ib_staged<T, 1>, ig, ib, sm, st, d, pf, kact, s, R, S); break;
            case 2: launch_pdl(B.pdl, qslbm::k_batch_ib_staged<T, 2>, ig, ib, sm, st, d, pf, kact, s, R, S); break;
            case 4: launch_pdl(B.pdl, qslbm::k_batch_ib_staged<T, 4>, ig, ib, sm, st, d, pf, kact, s, R, S); break;
            default: launch_pdl(B.pdl, qslbm::k_batch_ib_staged<T, 5>, ig, ib, sm, st, d, pf, kact, s, R, S); break;
        }
    } else if (nm > 0) {
        qslbm::k_batch_ib_markers<T><<<(nm + qslbm::kNodeThreads - 1) / qslbm::kNodeThreads, qslbm::kNodeThreads, 0,
                                        st>>>(d, B.mfirst, kact, s);
        qslbm::k_batch_ib_shell<T><<<(ns + qslbm::kNodeThreads - 1) / qslbm::kNodeThreads, qslbm::kNodeThreads, 0,
                                      st>>>(d, B.sfirst, kact, s);
    }
}

// Every sweep of the resident groups' members: one cooperative launch (its
// CTAs wait on one another, so all must be co-resident).
template <typename T>
void launch_groups(qslbm_batch& B, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (B.ngroups == 0) return;
        const auto* d = (const qslbm::InstDesc<float>*)B.desc;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(B.ngroups);
        cfg.blockDim = dim3(qslbm::kGroupThreads);
        cfg.dynamicSmemBytes = B.group_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e;
        if (B.has_field)
            e = cudaLaunchKernelEx(&cfg, qslbm::k_batch_resident<qslbm::InstDesc<float>, true>, d,
                                   (const qslbm::GroupDesc*)B.groups, B.xbuf, B.gflags, B.gerr);
        else
            e = cudaLaunchKernelEx(&cfg, qslbm::k_batch_resident<qslbm::InstDesc<float>, false>, d,
                                   (const qslbm::GroupDesc*)B.groups, B.xbuf, B.gflags, B.gerr);
        if (e != cudaSuccess) B.launch_err = e;
    }
}

template <typename T>
void launch_step(qslbm_batch& B, cudaStream_t st) {
    launch_groups<T>(B, st);
    for (int s = 0; s < B.max_nmag; ++s) launch_sweep<T>(B, s, B.threads, B.grid, st);
    const int K = (int)B.members.size();
    auto* d = (qslbm::InstDesc<T>*)B.desc;
    qslbm::k_batch_force<T><<<B.h_pfirst[K], qslbm::kNodeThreads, 0, st>>>(d, B.pfirst, K);
    qslbm::k_batch_flow<T><<<B.h_pfirst[K], qslbm::kPlaneThreads, B.ib_smem, st>>>(d, B.pfirst, K);
    qslbm::k_batch_advance<T><<<(K + 127) / 128, 128, 0, st>>>(d, K);
}

// Planes per group for a member that the resident group kernel can hold (0:
// it cannot): FP32, a wall ring with the same tables on every plane, planes of
// at most kGroupMaxNodes nodes, and a group's b, e and IB tables within the
// opt-in shared memory.  The planes are split into the fewest groups, of
// nearly equal size.
int group_planes(const State& s, int optin) {
    if (s.esz != 4 || s.dim != 3 || s.ib.nm == 0 || !s.ib.zinv || s.units.n_mag < 1) return 0;
    const int P = s.nx * s.ny;
    if (P > qslbm::kGroupMaxNodes) return 0;
    int G = std::min(s.nz, qslbm::kGroupMaxNodes / P);
    while (G > 0 && qslbm::group_smem_bytes(s.ib.max_ring, s.ib.max_shell, s.ib.max_nnz, G) > (size_t)optin) --G;
    if (G == 0) return 0;
    const int ng = (s.nz + G - 1) / G;
    return (s.nz + ng - 1) / ng;  // the largest group of the balanced split
}

int group_count(const State& s, int G) { return G > 0 ? (s.nz + G - 1) / G : 0; }

// Device tables of the resident groups (members kmarch .. K-1): the groups of
// each member (balanced split of its planes), their neighbours, exchange
// areas; the counters and the error flag start at zero.
int build_groups(qslbm_batch& B) {
    const int K = (int)B.members.size();
    B.h_groups.clear();
    long long xoff = 0;
    size_t smem = 0;
    for (int k = B.kmarch; k < K; ++k) {
        const State& s = qslbm::handle_state_mut(B.members[k]);
        const int P = s.nx * s.ny;
        const int ng = group_count(s, B.gplanes[k]);
        const int first = (int)B.h_groups.size();
        int z0 = 0;
        for (int j = 0; j < ng; ++j) {
            const int G = s.nz / ng + (j < s.nz % ng ? 1 : 0);
            qslbm::GroupDesc g;
            g.inst = k;
            g.z0 = z0;
            g.G = G;
            g.prev = first + (j == 0 ? ng - 1 : j - 1);
            g.next = first + (j == ng - 1 ? 0 : j + 1);
            g.xoff = xoff;
            xoff += 12LL * P;
            z0 += G;
            B.h_groups.push_back(g);
            smem = std::max(smem, qslbm::group_smem_bytes(s.ib.max_ring, s.ib.max_shell, s.ib.max_nnz, G));
        }
    }
    B.ngroups = (int)B.h_groups.size();
    B.group_smem = smem;
    if (B.ngroups == 0) return QSLBM_OK;
    if (B.ngroups > B.groups_cap) {
        if (B.groups) cudaFree(B.groups);
        if (B.gflags) cudaFree(B.gflags);
        B.groups = nullptr;
        B.gflags = nullptr;
        const int cap = std::max(B.ngroups, 2 * B.groups_cap);
        BCHK(cudaMalloc((void**)&B.groups, sizeof(qslbm::GroupDesc) * cap));
        BCHK(cudaMalloc((void**)&B.gflags, sizeof(unsigned) * cap));
        B.groups_cap = cap;
    }
    if (xoff > B.xbuf_cap) {
        if (B.xbuf) cudaFree(B.xbuf);
        B.xbuf = nullptr;
        const long long cap = std::max(xoff, 2 * B.xbuf_cap);
        BCHK(cudaMalloc((void**)&B.xbuf, sizeof(float) * cap));
        B.xbuf_cap = cap;
    }
    if (!B.gerr) BCHK(cudaMalloc((void**)&B.gerr, sizeof(int)));
    BCHK(cudaMemcpyAsync(B.groups, B.h_groups.data(), sizeof(qslbm::GroupDesc) * B.ngroups, cudaMemcpyHostToDevice,
                         B.stream));
    BCHK(cudaMemsetAsync(B.gflags, 0, sizeof(unsigned) * B.ngroups, B.stream));
    BCHK(cudaMemsetAsync(B.gerr, 0, sizeof(int), B.stream));
    for (bool xy : {false, true}) {
        const void* fn = xy ? (const void*)qslbm::k_batch_resident<qslbm::InstDesc<float>, true>
                            : (const void*)qslbm::k_batch_resident<qslbm::InstDesc<float>, false>;
        BCHK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    return QSLBM_OK;
}

// The work list depends on the sweep's tile: kMarchTX x (threads / kMarchTX)
// columns per item.
template <typename T>
int build_tables(qslbm_batch& B, int threads) {
    const int TY = threads / qslbm::kMarchTX;
    const int K = (int)B.members.size();
    std::vector<qslbm::InstDesc<T>> h(K);
    B.h_first.assign(K + 1, 0);
    B.h_pfirst.assign(K + 1, 0);
    B.h_mfirst.assign(K + 1, 0);
    B.h_sfirst.assign(K + 1, 0);
    size_t ring = 1, shell = 1;
    bool padded = true;
    {
        // z planes per work item of the marching sweep: 16, halved while the
        // batch would give fewer than 8 work items per SM (small instances:
        // shorter serial chains, more of them)
        int dev = 0, sms = 0;
        BCHK(cudaGetDevice(&dev));
        BCHK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        auto items = [&](int chunk) {
            long long w = 0;
            for (int k = 0; k < B.kmarch; ++k) {
                const State& s = qslbm::handle_state_mut(B.members[k]);
                w += (long long)((s.nx + qslbm::kMarchTX - 1) / qslbm::kMarchTX) * ((s.ny + TY - 1) / TY) *
                     ((s.nz + chunk - 1) / chunk);
            }
            return w;
        };
        B.sms = sms;
        B.chunk = qslbm::kMarchChunk;
        while (B.chunk > 2 && items(B.chunk) < 8LL * sms) B.chunk /= 2;
    }
    B.has_field = false;
    for (int k = 0; k < K; ++k) {
        const State& s = qslbm::handle_state_mut(B.members[k]);
        h[k] = make_desc<T>(s);
        if (s.bext_xy) B.has_field = true;
        const int tiles = ((s.nx + qslbm::kMarchTX - 1) / qslbm::kMarchTX) * ((s.ny + TY - 1) / TY) *
                          ((s.nz + B.chunk - 1) / B.chunk);
        h[k].bpp = tiles;
        B.h_first[k + 1] = B.h_first[k] + tiles;
        B.h_pfirst[k + 1] = B.h_pfirst[k] + s.nz;
        B.h_mfirst[k + 1] = B.h_mfirst[k] + s.ib.nm;
        B.h_sfirst[k + 1] = B.h_sfirst[k] + s.ib.ns;
        ring = std::max(ring, (size_t)std::max(1, s.ib.max_ring));
        shell = std::max(shell, (size_t)std::max(1, s.ib.max_shell));
        if (s.ib.nm > 0 && s.ib.pad_k == 0) padded = false;
    }
    B.ib_smem = 3 * ring * sizeof(T);
    // the staged IB corrector, when the largest plane's ring and shell fit
    // and every member's shell nodes have padded marker lists
    B.max_ring = (int)ring;
    B.max_shell = (int)shell;
    B.ib_staged_smem = 0;
    if (padded) {
        const size_t smem = qslbm::ib_staged_smem_bytes<T>((int)ring, (int)shell);
        int dev = 0, optin = 0;
        BCHK(cudaGetDevice(&dev));
        BCHK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (smem <= (size_t)optin) {
            // the launch picks U per active set (ib_staged_unroll)
            BCHK(cudaFuncSetAttribute(qslbm::k_batch_ib_staged<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
            BCHK(cudaFuncSetAttribute(qslbm::k_batch_ib_staged<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
            BCHK(cudaFuncSetAttribute(qslbm::k_batch_ib_staged<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
            BCHK(cudaFuncSetAttribute(qslbm::k_batch_ib_staged<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
            B.ib_staged_smem = smem;
        }
    }
    if (K > B.capacity) {
        if (B.desc) cudaFree(B.desc);
        if (B.first) cudaFree(B.first);
        if (B.pfirst) cudaFree(B.pfirst);
        if (B.mfirst) cudaFree(B.mfirst);
        if (B.sfirst) cudaFree(B.sfirst);
        B.desc = nullptr;
        B.first = B.pfirst = B.mfirst = B.sfirst = nullptr;
        const int cap = std::max(K, 2 * B.capacity);
        BCHK(cudaMalloc(&B.desc, sizeof(qslbm::InstDesc<T>) * cap));
        BCHK(cudaMalloc((void**)&B.first, sizeof(int) * (cap + 1)));
        BCHK(cudaMalloc((void**)&B.pfirst, sizeof(int) * (cap + 1)));
        BCHK(cudaMalloc((void**)&B.mfirst, sizeof(int) * (cap + 1)));
        BCHK(cudaMalloc((void**)&B.sfirst, sizeof(int) * (cap + 1)));
        B.device_bytes = (long long)(sizeof(qslbm::InstDesc<T>) * cap + 4 * sizeof(int) * (cap + 1));
        B.capacity = cap;
    }
    BCHK(cudaMemcpyAsync(B.desc, h.data(), sizeof(qslbm::InstDesc<T>) * K, cudaMemcpyHostToDevice, B.stream));
    BCHK(cudaMemcpyAsync(B.first, B.h_first.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, B.stream));
    BCHK(cudaMemcpyAsync(B.pfirst, B.h_pfirst.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, B.stream));
    BCHK(cudaMemcpyAsync(B.mfirst, B.h_mfirst.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, B.stream));
    BCHK(cudaMemcpyAsync(B.sfirst, B.h_sfirst.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, B.stream));
    if (sizeof(T) == 4) {
        const int rc = build_groups(B);
        if (rc) return rc;
    }
    BCHK(cudaStreamSynchronize(B.stream));
    return QSLBM_OK;
}

// Autotuner: time the first sweep of the batch for each (block size, grid)
// candidate on the real instances and keep the fastest: the marching tile's
// rows (4, 8 or 16, i.e. 128, 256 or 512 threads) and the persistent grid (1,
// 2, 4 or 8 CTAs per SM, or one CTA per work item).  The sweeps do not advance
// the solution (below).
template <typename T>
int autotune(qslbm_batch& B) {
    int dev = 0, sms = 0;
    BCHK(cudaGetDevice(&dev));
    BCHK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    struct Cand {
        int threads, grid;
        bool pdl;
    };
    std::vector<Cand> cands;
    for (int pdl : {0, 1})
        for (int ty : {4, 8, 16})
            for (int per_sm : {1, 2, 4, 8, 0})
                cands.push_back({qslbm::kMarchTX * ty, per_sm ? per_sm * sms : 0, pdl != 0});
    // the tuning sweeps write b[other parity]; they read b[current] and u only,
    // so the state the batch starts from is untouched
    cudaEvent_t e0, e1;
    BCHK(cudaEventCreate(&e0));
    BCHK(cudaEventCreate(&e1));
    float best = 1e30f;
    B.tune_us.clear();
    bool best_pdl = false;
    for (const Cand& c : cands) {
        int rc = build_tables<T>(B, c.threads);
        if (rc) return rc;
        B.pdl = c.pdl;
        launch_sweep<T>(B, 0, c.threads, c.grid, B.stream);  // warm-up
        BCHK(cudaEventRecord(e0, B.stream));
        for (int r = 0; r < 3; ++r) launch_sweep<T>(B, 0, c.threads, c.grid, B.stream);
        BCHK(cudaEventRecord(e1, B.stream));
        BCHK(cudaEventSynchronize(e1));
        float ms = 0;
        BCHK(cudaEventElapsedTime(&ms, e0, e1));
        B.tune_us.push_back(ms * 1e3 / 3);
        if (ms < best) {
            best = ms;
            B.threads = c.threads;
            B.grid = c.grid;
            best_pdl = c.pdl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B.pdl = best_pdl;
    return build_tables<T>(B, B.threads);
}

// Capture `steps` flow steps into one graph (the parities live in device
// memory, so a graph replays any steps).
template <typename T>
int capture_steps(qslbm_batch& B, int steps, cudaGraphExec_t* out) {
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaGraph_t g = nullptr;
    B.launch_err = cudaSuccess;
    BCHK(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < steps; ++i) launch_step<T>(B, B.stream);
    cudaError_t e = cudaStreamEndCapture(B.stream, &g);
    if (e == cudaSuccess && B.launch_err != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(B.launch_err, "cudaLaunchKernelEx (k_batch_resident)");
    }
    if (e != cudaSuccess) return fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(e, "cudaGraphInstantiate");
    return QSLBM_OK;
}

// Launches of one flow step: the group kernel, each marching sweep with its
// IB pass (or two), force, flow, parity advance.
int step_launches(const qslbm_batch& B) {
    int n = 3 + (B.ngroups > 0 ? 1 : 0);
    for (int s = 0; s < B.max_nmag; ++s)
        if (B.active[s] > 0) n += 1 + (B.h_mfirst[B.active[s]] > 0 ? (B.ib_staged_smem ? 1 : 2) : 0);
    return n;
}

// The one-step graph and a graph of many steps (chunk_target, or as many as
// keep it near kChunkLaunches launches), which qslbm_batch_step replays.
constexpr int kChunkLaunches = 4096;

template <typename T>
int capture(qslbm_batch& B) {
    int rc = capture_steps<T>(B, 1, &B.graph);
    if (rc) return rc;
    B.chunk_steps = std::max(1, std::min(B.chunk_target, kChunkLaunches / step_launches(B)));
    if (B.chunk_steps == 1) {
        if (B.graph_chunk) cudaGraphExecDestroy(B.graph_chunk);
        B.graph_chunk = nullptr;
        return QSLBM_OK;
    }
    return capture_steps<T>(B, B.chunk_steps, &B.graph_chunk);
}

// A timed-out neighbour wait of the group kernel, seen after the stream's
// work: restart the counters and report it.
int check_groups(qslbm_batch& B) {
    if (B.ngroups == 0 || !B.gerr) return QSLBM_OK;
    int bad = 0;
    BCHK(cudaMemcpyAsync(&bad, B.gerr, sizeof(int), cudaMemcpyDeviceToHost, B.stream));
    BCHK(cudaStreamSynchronize(B.stream));
    if (!bad) return QSLBM_OK;
    BCHK(cudaMemsetAsync(B.gflags, 0, sizeof(unsigned) * B.ngroups, B.stream));
    BCHK(cudaMemsetAsync(B.gerr, 0, sizeof(int), B.stream));
    BCHK(cudaStreamSynchronize(B.stream));
    qslbm::set_last_error("batched resident sweep: a neighbour wait timed out");
    return QSLBM_ETIMEOUT;
}

// Mirror the device-side parity updates on the members' host state.
void advance_host(qslbm_batch& B, long long nsteps) {
    for (qslbm_handle* h : B.members) {
        State& s = qslbm::handle_state_mut(h);
        s.fcur ^= (int)(nsteps & 1);
        s.bcur ^= (int)((nsteps * s.units.n_mag) & 1);
        s.t += nsteps;
    }
    B.steps += nsteps;
}

void destroy_batch(qslbm_batch* B) {
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->graph_chunk) cudaGraphExecDestroy(B->graph_chunk);
    if (B->desc) cudaFree(B->desc);
    if (B->groups) cudaFree(B->groups);
    if (B->gflags) cudaFree(B->gflags);
    if (B->gerr) cudaFree(B->gerr);
    if (B->xbuf) cudaFree(B->xbuf);
    if (B->first) cudaFree(B->first);
    if (B->pfirst) cudaFree(B->pfirst);
    if (B->mfirst) cudaFree(B->mfirst);
    if (B->sfirst) cudaFree(B->sfirst);
    if (B->owns_members)
        for (qslbm_handle* h : B->members) qslbm_destroy(h);
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    delete B;
}

// CTAs of the group kernel the device holds at once (one per SM) and the
// dynamic shared memory one may take (the opt-in limit less the kernel's
// static shared memory), computed once per batch.
int group_capacity(qslbm_batch& B) {
    if (B.gcap >= 0) return QSLBM_OK;
    int dev = 0, sms = 0, optin = 0, occ = 0;
    BCHK(cudaGetDevice(&dev));
    BCHK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BCHK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const void* fn = (const void*)qslbm::k_batch_resident<qslbm::InstDesc<float>, true>;
    cudaFuncAttributes fa;
    BCHK(cudaFuncGetAttributes(&fa, fn));
    optin -= (int)fa.sharedSizeBytes;
    BCHK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    BCHK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, qslbm::kGroupThreads, optin));
    B.gcap = occ * sms;
    B.goptin = optin;
    return QSLBM_OK;
}

// (Re)build the batch over the given handles: choose the members the
// resident group kernel holds (allowed ones that fit, smallest first, while
// their groups fit co-resident on the device), order the marching members by
// N_mag, device tables, autotune (first time only) and the per-step graph.
// The handles' host parity must match their device buffers (true for handles
// created by this library).  allow[i] (empty: all) lets handle i run in the
// group kernel.
int set_members(qslbm_batch* B, const std::vector<qslbm_handle*>& hs, const std::vector<char>& allow) {
    const int count = (int)hs.size();
    B->members.clear();
    B->order.assign(count, 0);
    B->rank.assign(count, 0);
    B->gplanes.clear();
    B->kmarch = 0;
    B->ngroups = 0;
    if (count == 0) {
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
        }
        if (B->graph_chunk) {
            cudaGraphExecDestroy(B->graph_chunk);
            B->graph_chunk = nullptr;
        }
        B->max_nmag = 0;
        B->active.clear();
        return QSLBM_OK;
    }
    // planes per group of each handle, and the members the launch can hold
    std::vector<int> gp(count, 0);
    if (B->precision == QSLBM_FP32) {
        int rc0 = group_capacity(*B);
        if (rc0) return rc0;
        const int cap = B->gcap, optin = B->goptin;
        std::vector<int> cand;
        for (int i = 0; i < count; ++i) {
            if (!allow.empty() && !allow[i]) continue;
            gp[i] = group_planes(qslbm::handle_state_mut(hs[i]), optin);
            if (gp[i] > 0) cand.push_back(i);
        }
        std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
            return qslbm::handle_state_mut(hs[a]).n < qslbm::handle_state_mut(hs[b]).n;
        });
        int used = 0;
        std::vector<int> adm;
        for (int i : cand) {
            const int ng = group_count(qslbm::handle_state_mut(hs[i]), gp[i]);
            if (used + ng <= cap) {
                used += ng;
                adm.push_back(i);
            } else {
                gp[i] = 0;
            }
        }
        // spread the admitted members over every co-resident CTA: the
        // smallest group size (nodes) at which their groups still fit
        auto planes_at = [&](int i, int T) {
            const State& s = qslbm::handle_state_mut(hs[i]);
            const int G = std::max(1, std::min(gp[i], T / (s.nx * s.ny)));
            return (s.nz + group_count(s, G) - 1) / group_count(s, G);
        };
        auto groups_at = [&](int T) {
            int tot = 0;
            for (int i : adm) tot += group_count(qslbm::handle_state_mut(hs[i]), planes_at(i, T));
            return tot;
        };
        int lo = 1, hi = qslbm::kGroupMaxNodes;  // groups_at(hi) <= cap
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (groups_at(mid) <= cap)
                hi = mid;
            else
                lo = mid + 1;
        }
        std::vector<int> spread(count, 0);
        for (int i : adm) spread[i] = planes_at(i, lo);
        for (int i : adm) gp[i] = spread[i];
    }
    std::vector<int> idx(count);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        if ((gp[a] > 0) != (gp[b] > 0)) return gp[b] > 0;  // marching members first
        return qslbm::handle_state_mut(hs[a]).units.n_mag > qslbm::handle_state_mut(hs[b]).units.n_mag;
    });
    B->order = idx;
    for (int k = 0; k < count; ++k) {
        B->members.push_back(hs[idx[k]]);
        B->rank[idx[k]] = k;
        B->gplanes.push_back(gp[idx[k]]);
        if (gp[idx[k]] == 0) B->kmarch = k + 1;
    }
    B->max_nmag = 0;
    for (qslbm_handle* h : B->members) B->max_nmag = std::max(B->max_nmag, qslbm::handle_state_mut(h).units.n_mag);
    // active[s]: marching members with N_mag > s (a prefix)
    B->active.assign(B->max_nmag, 0);
    for (int s = 0; s < B->max_nmag; ++s) {
        int a = 0;
        while (a < B->kmarch && qslbm::handle_state_mut(B->members[a]).units.n_mag > s) ++a;
        B->active[s] = a;
    }
    int rc;
    if (!B->tuned && B->kmarch > 0) {  // (no marching member: nothing to time yet)
        rc = B->precision == QSLBM_FP64 ? autotune<double>(*B) : autotune<float>(*B);
        B->tuned = true;
    } else {
        rc = B->precision == QSLBM_FP64 ? build_tables<double>(*B, B->threads) : build_tables<float>(*B, B->threads);
    }
    if (!rc) rc = B->precision == QSLBM_FP64 ? capture<double>(*B) : capture<float>(*B);
    return rc;
}

int create_batch(const qslbm_params* params, int32_t count, void* stream, qslbm_batch** out) {
    if (!params || !out || count <= 0) {
        qslbm::set_last_error("qslbm_batch_create: NULL argument or a count below one");
        return QSLBM_EINVAL;
    }
    *out = nullptr;
    const int prec = params[0].precision;
    for (int i = 0; i < count; ++i)
        if (params[i].precision != prec || params[i].dim != 3) {
            qslbm::set_last_error("qslbm_batch_create: member " + std::to_string(i) +
                                  (params[i].dim != 3 ? " is not 3-D" : " has another precision than member 0"));
            return QSLBM_EINVAL;
        }
    qslbm_batch* B = new (std::nothrow) qslbm_batch();
    if (!B) return QSLBM_ENOMEM;
    B->precision = prec;
    if (stream) {
        B->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreate(&B->stream);
        if (e != cudaSuccess) {
            delete B;
            return fail(e, "cudaStreamCreate");
        }
        B->own_stream = true;
    }
    std::vector<qslbm_handle*> hs(count, nullptr);
    for (int i = 0; i < count; ++i) {
        qslbm_params p = params[i];
        p.sweep_kernel = QSLBM_SWEEP_SPLIT;
        p.stream = B->stream;
        int rc = qslbm_create(&p, &hs[i]);
        if (rc) {
            for (qslbm_handle* h : hs)
                if (h) qslbm_destroy(h);
            if (B->own_stream) cudaStreamDestroy(B->stream);
            delete B;
            return rc;
        }
    }
    // QSLBM_SWEEP_SPLIT keeps a member on the marching sweep; any other choice
    // lets it run in the resident group kernel when it fits
    std::vector<char> allow(count);
    for (int i = 0; i < count; ++i) allow[i] = params[i].sweep_kernel != QSLBM_SWEEP_SPLIT;
    int rc = set_members(B, hs, allow);
    if (rc) {
        destroy_batch(B);
        return rc;
    }
    *out = B;
    return QSLBM_OK;
}

}  // namespace

extern "C" {

int qslbm_batch_create(const qslbm_params* params, int32_t count, void* stream, qslbm_batch** out) {
    try {
        return create_batch(params, count, stream, out);
    } catch (...) {
        return QSLBM_ENOMEM;
    }
}

int qslbm_batch_step(qslbm_batch* B, int64_t nsteps) {
    if (!B || nsteps < 0) return refuse("qslbm_batch_step: NULL batch or negative step count");
    if (B->members.empty()) return QSLBM_OK;
    long long i = 0;
    if (B->graph_chunk)
        for (; i + B->chunk_steps <= nsteps; i += B->chunk_steps) BCHK(cudaGraphLaunch(B->graph_chunk, B->stream));
    for (; i < nsteps; ++i) BCHK(cudaGraphLaunch(B->graph, B->stream));
    advance_host(*B, nsteps);
    return QSLBM_OK;
}

int qslbm_batch_handle(qslbm_batch* B, int32_t i, qslbm_handle** out) {
    if (!B || !out || i < 0 || i >= (int)B->members.size())
        return refuse("qslbm_batch_handle: NULL argument or member index out of range");
    BCHK(cudaStreamSynchronize(B->stream));
    const int rc = check_groups(*B);
    if (rc) return rc;
    *out = B->members[B->rank[i]];
    return QSLBM_OK;
}

int qslbm_batch_info(const qslbm_batch* B, qslbm_batch_info_t* info) {
    if (!B || !info) return refuse("qslbm_batch_info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->count = (int32_t)B->members.size();
    info->max_n_mag = B->max_nmag;
    info->sweep_threads = B->threads;
    info->sweep_grid = B->grid;
    long long nodes = 0, sweeps = 0;
    long long bytes = B->device_bytes + (long long)B->groups_cap * (sizeof(qslbm::GroupDesc) + sizeof(unsigned)) +
                      B->xbuf_cap * (long long)sizeof(float) + (B->gerr ? (long long)sizeof(int) : 0);
    for (qslbm_handle* h : B->members) {
        const State& s = qslbm::handle_state_mut(h);
        nodes += s.n;
        bytes += s.device_bytes;
        sweeps += s.n * (long long)s.units.n_mag;
    }
    info->nodes = nodes;
    info->node_sweeps_per_step = sweeps;
    info->device_bytes = bytes;
    info->launches_per_step = B->members.empty() ? 0 : step_launches(*B);
    info->resident_instances = (int32_t)B->members.size() - B->kmarch;
    info->resident_groups = B->ngroups;
    info->graph_steps = B->chunk_steps;
    info->march_chunk = B->chunk;
    info->steps = B->steps;
    for (size_t c = 0; c < B->tune_us.size() && c < 32; ++c) info->tune_us[c] = B->tune_us[c];
    info->sweep_pdl = B->pdl ? 1 : 0;
    return QSLBM_OK;
}

int qslbm_batch_destroy(qslbm_batch* B) {
    if (!B) return refuse("qslbm_batch_destroy: NULL batch");
    destroy_batch(B);
    return QSLBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: a request loop over the batched engine.  Requests (a problem and a
// stop tolerance) are queued from any thread; each call of qslbm_server_run
// admits the queued requests whose device memory fits the budget (first fit),
// rebuilds the batch when its membership changed, advances every admitted
// instance by one chunk of steps in the fused launches, then checks each
// instance's FP64 steady residual and retires those that converged (or hit
// their step cap, or went non-finite).  New requests join between chunks while
// others keep running: continuous batching.
#include <chrono>
#include <deque>
#include <mutex>

namespace {

struct Request {
    int64_t id;
    qslbm_params p;
    double tol;
    int64_t max_steps;
    int32_t keep;
    double t_submit;
};

struct Running {
    Request r;
    qslbm_handle* h;
    double t_admit;
    int64_t steps;
    long long bytes;
    double residual;
};

}  // namespace

struct qslbm_server {
    std::mutex mu;  // guards pending and next_id (submit may come from other threads)
    std::deque<Request> pending;
    int64_t next_id = 1;
    std::vector<Running> running;
    std::vector<qslbm_result> done;
    std::vector<std::pair<int64_t, qslbm_handle*>> kept;
    qslbm_batch* batch = nullptr;
    qslbm_server_config cfg{};
    long long used = 0;
    std::chrono::steady_clock::time_point t0;
    long long chunks = 0, rebuilds = 0, steps = 0, node_steps = 0;
};

namespace {

double now_s(const qslbm_server& S) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t0).count();
}

// Groups of the resident group kernel a request would take at the largest
// group size (-1: the kernel does not hold it: 2-D, no wall, planes above
// kGroupMaxNodes nodes).
int groups_needed(const qslbm_params& p) {
    if (p.dim != 3 || p.geometry == QSLBM_PERIODIC) return -1;
    const long long P = (long long)p.nx * p.ny;
    if (P > qslbm::kGroupMaxNodes || p.nz < 1) return -1;
    const int G = std::max(1, std::min(p.nz, (int)(qslbm::kGroupMaxNodes / P)));
    return (p.nz + G - 1) / G;
}

// Device bytes a request will hold (fields, double buffers, scratch, tables).
long long estimate_bytes(const qslbm_params& p) {
    const long long n = (long long)p.nx * p.ny * (p.dim == 2 ? 1 : p.nz);
    const long long esz = p.precision == QSLBM_FP64 ? 8 : 4;
    return n * esz * 20 + n * 8 / 16 + (1 << 20);
}

void finish(qslbm_server& S, Running& r, int32_t status) {
    qslbm_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = r.r.id;
    res.status = status;
    res.steps = r.steps;
    res.residual = r.residual;
    res.t_submit = r.r.t_submit;
    res.t_admit = r.t_admit;
    res.t_done = now_s(S);
    res.nodes = qslbm::handle_state_mut(r.h).n;
    qslbm_observables(r.h, &res.obs, nullptr, nullptr, nullptr);
    S.done.push_back(res);
    if (r.r.keep) {
        S.kept.push_back({r.r.id, r.h});
    } else {
        S.used -= r.bytes;
        qslbm_destroy(r.h);
    }
    r.h = nullptr;
}

int server_run(qslbm_server& S, int32_t* n_running, int32_t* n_pending) {
    bool changed = false;
    // admission (first fit under the budget)
    {
        std::lock_guard<std::mutex> lock(S.mu);
        // smallest first in FP32: keep the running requests within the group
        // kernel's capacity (a request beyond it would put the whole batch on
        // the marching route's launches every step)
        const bool hold = S.cfg.admit == QSLBM_ADMIT_SMALLEST && S.cfg.precision == QSLBM_FP32;
        int used_groups = 0;
        // a request larger than the whole budget is answered at once
        for (auto it = S.pending.begin(); it != S.pending.end();) {
            if (estimate_bytes(it->p) > S.cfg.hbm_budget_bytes) {
                qslbm_result res;
                std::memset(&res, 0, sizeof(res));
                res.id = it->id;
                res.status = QSLBM_EBUDGET;
                res.t_submit = it->t_submit;
                res.t_admit = res.t_done = now_s(S);
                S.done.push_back(res);
                it = S.pending.erase(it);
            } else {
                ++it;
            }
        }
        if (hold) {
            std::stable_sort(S.pending.begin(), S.pending.end(), [](const Request& a, const Request& b) {
                return estimate_bytes(a.p) < estimate_bytes(b.p);
            });
            int rc0 = group_capacity(*S.batch);
            if (rc0) return rc0;
            for (const Running& r : S.running) used_groups += std::max(0, groups_needed(r.r.p));
        }
        for (auto it = S.pending.begin(); it != S.pending.end();) {
            if (S.cfg.max_running > 0 && (int)S.running.size() >= S.cfg.max_running) break;
            const long long est = estimate_bytes(it->p);
            if (hold) {
                const int ng = groups_needed(it->p);
                if (!S.running.empty() && (ng < 0 || used_groups + ng > S.batch->gcap)) break;
                if (S.used + est <= S.cfg.hbm_budget_bytes) used_groups += std::max(0, ng);
            }
            if (S.used + est > S.cfg.hbm_budget_bytes) {
                ++it;
                continue;
            }
            qslbm_params p = it->p;
            p.precision = S.cfg.precision;
            p.sweep_kernel = QSLBM_SWEEP_SPLIT;
            p.stream = S.batch->stream;
            qslbm_handle* h = nullptr;
            int rc = qslbm_create(&p, &h);
            if (rc) {
                qslbm_result res;
                std::memset(&res, 0, sizeof(res));
                res.id = it->id;
                res.status = rc;
                res.t_submit = it->t_submit;
                res.t_admit = res.t_done = now_s(S);
                S.done.push_back(res);
                it = S.pending.erase(it);
                continue;
            }
            const long long bytes = qslbm::handle_state_mut(h).device_bytes;
            S.used += bytes;
            qslbm_obs o;
            qslbm_observables(h, &o, nullptr, nullptr, nullptr);  // reference velocity for the residual
            S.running.push_back({*it, h, now_s(S), 0, bytes, 0.0});
            it = S.pending.erase(it);
            changed = true;
        }
    }
    if (changed) {
        std::vector<qslbm_handle*> hs;
        std::vector<char> allow;
        for (const Running& r : S.running) {
            hs.push_back(r.h);
            allow.push_back(r.r.p.sweep_kernel != QSLBM_SWEEP_SPLIT);
        }
        int rc = set_members(S.batch, hs, allow);
        if (rc) return rc;
        ++S.rebuilds;
    }
    if (!S.running.empty()) {
        int rc = qslbm_batch_step(S.batch, S.cfg.chunk_steps);
        if (!rc) rc = check_groups(*S.batch);
        if (rc) return rc;
        ++S.chunks;
        S.steps += S.cfg.chunk_steps;
        bool retired = false;
        for (Running& r : S.running) {
            r.steps += S.cfg.chunk_steps;
            S.node_steps += qslbm::handle_state_mut(r.h).n * (long long)S.cfg.chunk_steps;
            qslbm_obs o;
            rc = qslbm_observables(r.h, &o, nullptr, nullptr, nullptr);
            r.residual = o.steady_residual;
            if (rc == QSLBM_EUNSTABLE || o.nan_flag) {
                finish(S, r, QSLBM_EUNSTABLE);
                retired = true;
            } else if (rc) {
                return rc;
            } else if (o.steady_residual < r.r.tol) {
                finish(S, r, QSLBM_OK);
                retired = true;
            } else if (r.steps >= r.r.max_steps) {
                finish(S, r, QSLBM_ETIMEOUT);
                retired = true;
            }
        }
        if (retired) {
            std::vector<Running> keep;
            for (Running& r : S.running)
                if (r.h) keep.push_back(r);
            S.running.swap(keep);
            std::vector<qslbm_handle*> hs;
            std::vector<char> allow;
            for (const Running& r : S.running) {
                hs.push_back(r.h);
                allow.push_back(r.r.p.sweep_kernel != QSLBM_SWEEP_SPLIT);
            }
            rc = set_members(S.batch, hs, allow);
            if (rc) return rc;
            ++S.rebuilds;
        }
    }
    if (n_running) *n_running = (int32_t)S.running.size();
    if (n_pending) {
        std::lock_guard<std::mutex> lock(S.mu);
        *n_pending = (int32_t)S.pending.size();
    }
    return QSLBM_OK;
}

}  // namespace

extern "C" {

int qslbm_server_create(const qslbm_server_config* cfg, qslbm_server** out) {
    const char* why = nullptr;
    if (!cfg || !out)
        why = "NULL argument";
    else if (cfg->chunk_steps <= 0 || cfg->hbm_budget_bytes <= 0)
        why = "chunk_steps and hbm_budget_bytes must be positive";
    else if (cfg->precision != QSLBM_FP32 && cfg->precision != QSLBM_FP64)
        why = "unknown precision";
    else if (cfg->admit != QSLBM_ADMIT_FIFO && cfg->admit != QSLBM_ADMIT_SMALLEST)
        why = "unknown admission order";
    if (why) {
        qslbm::set_last_error(std::string("qslbm_server_create: ") + why);
        return QSLBM_EINVAL;
    }
    *out = nullptr;
    qslbm_server* S = new (std::nothrow) qslbm_server();
    if (!S) return QSLBM_ENOMEM;
    S->cfg = *cfg;
    S->t0 = std::chrono::steady_clock::now();
    qslbm_batch* B = new (std::nothrow) qslbm_batch();
    if (!B) {
        delete S;
        return QSLBM_ENOMEM;
    }
    B->owns_members = false;
    B->precision = cfg->precision;
    B->chunk_target = (int)std::min<int64_t>(cfg->chunk_steps, 1000);
    if (cfg->stream) {
        B->stream = (cudaStream_t)cfg->stream;
    } else {
        cudaError_t e = cudaStreamCreate(&B->stream);
        if (e != cudaSuccess) {
            delete B;
            delete S;
            return fail(e, "cudaStreamCreate");
        }
        B->own_stream = true;
    }
    S->batch = B;
    *out = S;
    return QSLBM_OK;
}

int qslbm_server_submit(qslbm_server* S, const qslbm_params* p, double tol, int64_t max_steps, int32_t keep_fields,
                        int64_t* id) {
    if (!S || !p || !(tol > 0) || max_steps <= 0 || p->dim != 3) {
        qslbm::set_last_error("qslbm_server_submit: NULL argument, tol or max_steps not positive, or a 2-D problem");
        return QSLBM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    Request r{S->next_id++, *p, tol, max_steps, keep_fields, now_s(*S)};
    S->pending.push_back(r);
    if (id) *id = r.id;
    return QSLBM_OK;
}

int qslbm_server_run(qslbm_server* S, int32_t* n_running, int32_t* n_pending) {
    if (!S) return refuse("qslbm_server_run: NULL server");
    try {
        return server_run(*S, n_running, n_pending);
    } catch (...) {
        return QSLBM_ENOMEM;
    }
}

int qslbm_server_poll(qslbm_server* S, qslbm_result* out, int32_t max, int32_t* n) {
    if (!S || !n || max < 0 || (max > 0 && !out)) return refuse("qslbm_server_poll: NULL argument or max < 0");
    const int k = std::min<int>(max, (int)S->done.size());
    for (int i = 0; i < k; ++i) out[i] = S->done[i];
    S->done.erase(S->done.begin(), S->done.begin() + k);
    *n = k;
    return QSLBM_OK;
}

int qslbm_server_fields(qslbm_server* S, int64_t id, double* rho, double* u, double* b) {
    if (!S) return refuse("qslbm_server_fields: NULL server");
    for (auto& kv : S->kept)
        if (kv.first == id) {
            // the first host copy allocates the handle's staging buffer; it is
            // held until the release, so it counts against the budget
            const long long before = qslbm::handle_state_mut(kv.second).device_bytes;
            const int rc = qslbm_get_state(kv.second, rho, u, b, nullptr);
            S->used += qslbm::handle_state_mut(kv.second).device_bytes - before;
            return rc;
        }
    return QSLBM_ENOTFOUND;
}

int qslbm_server_release(qslbm_server* S, int64_t id) {
    if (!S) return refuse("qslbm_server_release: NULL server");
    for (size_t i = 0; i < S->kept.size(); ++i)
        if (S->kept[i].first == id) {
            S->used -= qslbm::handle_state_mut(S->kept[i].second).device_bytes;
            qslbm_destroy(S->kept[i].second);
            S->kept.erase(S->kept.begin() + i);
            return QSLBM_OK;
        }
    return QSLBM_ENOTFOUND;
}

int qslbm_server_stats(const qslbm_server* S, qslbm_server_stats_t* st) {
    if (!S || !st) return refuse("qslbm_server_stats: NULL argument");
    std::memset(st, 0, sizeof(*st));
    st->running = (int32_t)S->running.size();
    st->pending = (int32_t)S->pending.size();
    st->chunks = S->chunks;
    st->rebuilds = S->rebuilds;
    st->steps = S->steps;
    st->node_steps = S->node_steps;
    st->device_bytes = S->used;
    st->sweep_threads = S->batch->threads;
    st->sweep_grid = S->batch->grid;
    return QSLBM_OK;
}

int qslbm_server_destroy(qslbm_server* S) {
    if (!S) return refuse("qslbm_server_destroy: NULL server");
    if (S->batch->stream) cudaStreamSynchronize(S->batch->stream);
    for (Running& r : S->running)
        if (r.h) qslbm_destroy(r.h);
    for (auto& kv : S->kept) qslbm_destroy(kv.second);
    S->batch->members.clear();
    destroy_batch(S->batch);
    delete S;
    return QSLBM_OK;
}

}  // extern "C"
