// Internal host-side structures of the qslbm library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "qslbm.h"

namespace qslbm {

// Diagnostics slots and the reduction block size (see k_observe).
constexpr int kObs = 11;
constexpr int kReduceThreads = 256;

// Marker and shell tables of the IB corrector (device pointers).  The same
// tables serve u and b; only the per-marker scaling differs (mk_s, mk_sm).
struct DeviceIB {
    int *ring_off = nullptr, *mk_q = nullptr;
    int *shell_off = nullptr, *shell_xy = nullptr, *csr_off = nullptr, *csr_m = nullptr;
    void *mk_w = nullptr, *mk_s = nullptr, *mk_sm = nullptr, *csr_w = nullptr;
    int *mk_base = nullptr, *shell_node = nullptr, *csr_mg = nullptr;
    void *delta = nullptr;  // [3 nm] markers' corrections (two-phase corrector)
    int nm = 0, ns = 0, nnz = 0, max_ring = 0, max_shell = 0, max_nnz = 0;
    int zinv = 0;  // 1: every z plane carries plane 0's ring and shell tables
    int* mk_slot = nullptr;  // [9 nm] shell-list position of each support node
    int* pad_m = nullptr;    // [nsp pad_k] padded marker lists of the shell nodes
    void* pad_w = nullptr;   // [nsp pad_k] and their weights
    int pad_k = 0;           // list length, a multiple of 4 (0: none)
};

// The fused sweep + IB kernel (FP32): a plane slot holds, per field and
// component, the 3 rows above a band, its TY rows and the 3 rows below, each
// block padded to 128 bytes.
constexpr int kFusedMaxThreads = 768;  // threads of a CTA of the fused kernel, at most
__host__ __device__ inline int fused_pad32(int v) { return (v + 31) / 32 * 32; }
inline size_t fused_slot_floats(int nx, int TY) {
    return (size_t)6 * (2 * fused_pad32(3 * nx) + fused_pad32(TY * nx));
}
// Shared memory (bytes): `slots` plane slots, two buffers of b* of TY + 4
// rows (three components), two buffers of deltas and the tables of up to
// Mmax markers and
// Smax shell nodes with K list entries (Mmax, Smax multiples of 4), one
// mbarrier per slot, and 128 bytes of room to align the region's start.
inline size_t fused_smem_bytes(int nx, int TY, int Mmax, int Smax, int K, int slots) {
    const size_t f = (size_t)slots * fused_slot_floats(nx, TY) + (size_t)6 * (TY + 4) * nx + (size_t)25 * Mmax +
                     (size_t)Smax * (2 + 2 * K) + 1;
    return f * sizeof(float) + (size_t)slots * sizeof(unsigned long long) + 128;
}

// Longest padded marker list of a shell node (longer lists: the staged IB
// corrector is not used).
constexpr int kMaxPadK = 16;

// Host copy of the marker geometry and IB weights (binary64).
struct HostIB {
    std::vector<double> X, Y;   // marker positions
    std::vector<int> zplane;    // plane of each marker
    std::vector<int> ring_off;  // [nz + 1]
    std::vector<int> ix, iy;    // [3 nm] wrapped node indices
    std::vector<double> wx, wy; // [3 nm] 1-D kernel weights
    std::vector<double> d, s, sm;
    std::vector<int> shell_off, shell_xy, csr_off, csr_m;
    std::vector<double> csr_w;
    int max_ring = 0, max_shell = 0, max_nnz = 0;
};

struct State {
    qslbm_params p{};
    qslbm_units units{};
    int dim = 3, nx = 0, ny = 0, nz = 0;
    long long n = 0;
    size_t esz = 4;
    double cx = 0, cy = 0, R = 0;
    double w0 = 0, w1 = 0, kappa = 0;  // field lattice weights, 1/(2 eta)
    double alpha = 1.0;                // accelerated-sweep coefficient (1: plain sweep)
    double ig = 1.0;                   // 1/gamma: the time step in physical time
    double be[3] = {0, 0, 0};          // uniform B^ext
    int axis = 2;                      // body-force direction
    double omega = 0;                  // 2 pi / period
    void *drho[2] = {nullptr, nullptr}, *u[2] = {nullptr, nullptr}, *b[2] = {nullptr, nullptr};
    void *F = nullptr, *usnap = nullptr, *bext_z = nullptr;
    void* bext_xy = nullptr;  // [3][nx ny] B0 times the in-plane applied field (QSLBM_B0_FIELD)
    long long* tdev = nullptr;
    double *partial = nullptr, *obs_dev = nullptr, *staging = nullptr;
    int nblocks_obs = 0;
    int fcur = 0, bcur = 0;
    long long t = 0, tsnap = 0;
    double mass0 = 0;
    std::vector<double> bext_host;  // [3 nz] when the field is a ramp
    HostIB hib;
    DeviceIB ib;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int graph_next[2][2][2] = {};  // ping-pong parity (bcur, fcur) after each graph
    // resident sub-iteration (all sweeps of a step in one cooperative launch)
    bool resident = false;
    bool launch_error = false;  // a cudaLaunchKernelEx call failed
    int march_chunk = 16;       // z planes per CTA of the marching sweep (one wave)
    size_t ib_staged_smem = 0;  // shared memory of k_ib_staged, 0 when it does not fit
    int ib_staged_u = 1;        // its shell nodes per thread per batch of loads (1, 2 or 5)
    bool resident_uhalo = false;
    size_t resident_smem = 0;
    void* xbuf = nullptr;   // [2][nz][3][P] plane exchange
    void* rsync = nullptr;  // ResidentSync + flags[nz]
    int graph_steps = 0;
    // fused sweep + IB (FP32 planes beyond the resident kernel): bands of
    // fu_TY rows, fu_chunk z planes per CTA, per-band IB tables
    bool fused = false;
    int fu_TY = 0, fu_bands = 0, fu_chunk = 0, fu_chunks = 0, fu_threads = 0, fu_slots = 4;
    size_t fu_smem = 0;
    int fu_Mmax = 0, fu_Smax = 0, fu_K = 0;
    int *fu_mk_cnt = nullptr, *fu_mk_off = nullptr, *fu_sh_cnt = nullptr, *fu_sh_off = nullptr, *fu_sh_m = nullptr,
        *fu_sh_ce = nullptr;
    float *fu_mk_w = nullptr, *fu_mk_s = nullptr, *fu_sh_w = nullptr;
    int* fu_err = nullptr;  // 1: a copy wait timed out
    // b[i], u[i] as (x, y, z, component) tensors: boxes of 3 rows and of TY rows of one component
    CUtensorMap fu_map_b3[2], fu_map_bt[2], fu_map_u3[2], fu_map_ut[2];
    std::vector<void*> allocations;
    long long device_bytes = 0;
};

// Weights of the magnetic update as the sweep kernels use them,
//   b <- w0 b + w1 sum_{axis nbrs} b + (w1 kappa) D   (D: the flux differences),
// covering three forms of the same sum:
//   - the tau_m = 1 sweep (Sec. V.G): w_0, w_axis, 1/(c c_m^2);
//   - the accelerated sweep (Sec. V.H): (w_0 - 1 + alpha)/alpha, w_axis/alpha;
//   - the time-resolved update for any tau_m (Sec. III.D, de Rosis form), whose
//     sum_i {g_i(x - e_i) + (tau_m - 1)[g_i(x + e_i) - 2 g_i(x) + g_i(x - e_i)]}
//     is (2 tau_m - 1) times the plain neighbour sum of b, plus the plain flux
//     sum, minus 2 (tau_m - 1) b, since the flux terms of g_i(x + e_i) are
//     those of g_i(x - e_i) with the sign reversed and sum_i g_i(x) = b.
// With the time step rescaled by gamma (Sec. VII) the flux carries 1/gamma.
// At alpha = 1, tau_m = 1 and gamma = 1 every weight is exactly the plain one.
template <typename T>
inline void sweep_weights(const State& s, T& w0, T& w1, T& kappa) {
    const double tm = s.units.tau_m, a = s.alpha;
    w0 = (T)(((2.0 * tm - 1.0) * s.w0 - 2.0 * (tm - 1.0) + (a - 1.0)) / a);
    w1 = (T)((2.0 * tm - 1.0) * s.w1 / a);
    kappa = (T)(s.kappa / (2.0 * tm - 1.0) * s.ig);  // flux over gamma (Sec. VII)
}

// Kernel launchers, one table per storage precision.
struct Ops {
    void (*init)(State&, cudaStream_t);
    void (*sweeps)(State&, int nsweeps, cudaStream_t);  // flips bcur per sweep
    void (*force_flow)(State&, cudaStream_t);           // flips fcur
    void (*observe)(State&, double fb, cudaStream_t);   // obs_dev[0..10]
    // the same reduction over caller-held fields (drho, u, b, u_prev in the
    // handle's layout and precision): `blocks` partial sums into partial
    // [blocks * kObs], folded into sums[kObs]
    void (*observe_fields)(const State&, const void* drho, const void* u, const void* b, const void* u_prev,
                           double fb, int blocks, double* partial, double* sums, cudaStream_t);
    void (*to_f64)(State&, cudaStream_t);               // staging <- state
    void (*from_f64)(State&, int mask, cudaStream_t);   // state <- staging
    // decide whether the resident sweep kernel fits this domain; sets
    // s.resident, s.resident_uhalo, s.resident_smem (no allocation)
    cudaError_t (*plan_resident)(State&);
    cudaError_t (*plan_march)(State&);  // sets s.march_chunk and s.ib_staged_smem
    // launch shape of the fused sweep for the tables already in s (fu_TY,
    // fu_bands, fu_smem): sets fu_threads, fu_chunk, fu_chunks, or clears
    // s.fused when it cannot run here
    cudaError_t (*plan_fused)(State&);
    // one sweep of each of the fused kernel and the split path timed on the
    // handle's fields; keeps the faster (s.fused, s.p.sweep_kernel)
    cudaError_t (*tune_fused)(State&, double* us_fused, double* us_split);
};

const Ops& ops_f32();
const Ops& ops_f64();

}  // namespace qslbm
