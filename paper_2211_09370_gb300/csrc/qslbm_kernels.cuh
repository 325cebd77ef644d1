// CUDA kernels of the single-step simplified LBM for quasi-static MHD pipe flow
// (arXiv 2211.09370), written for sm_103a.  Templated on the storage/arithmetic
// type T (float or double) and the dimension DIM (2: D2Q9 + D2Q5, 3: D3Q19 +
// D3Q7).
//
// Layout in device memory: structure of arrays, one array per component,
// index k = (z * ny + y) * nx + x (x fastest), periodic in every direction.
// The density is stored as drho = rho - 1 so that FP32 keeps the small density
// variations; the field evolved by the magnetic sweep is the induced part b of
// B = B^ext + b, B^ext being analytic (uniform, or a tanh ramp in z held as one
// value per z plane).
//
// Wall markers sit on integer z planes (rings of a pipe, lines of a channel),
// so the z factor of the interpolation kernel D = D_x D_y D_z is a Kronecker
// delta and the immersed-boundary operator couples nodes of one plane only.
// Every kernel that applies the IB therefore gives one CTA a whole z plane: the
// CTA first writes the plane's predictor values, then interpolates them at the
// plane's markers (all markers before any spreading, as the explicit scheme
// requires), then adds the spread corrections to the plane's shell nodes with
// a node-side gather (node -> marker list), which needs no atomics and is
// deterministic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "qslbm_internal.h"

namespace qslbm {

constexpr int kPlaneThreads = 512;

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may start while the previous kernel in
// its stream is still running, once every CTA of that kernel has called
// pdl_trigger (or exited); pdl_wait then blocks until the previous kernel has
// completed and its memory is visible.  Every read of data another kernel
// writes, and every global write, comes after pdl_wait; only reads of
// constant tables may come before it.  Both are no-ops in a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

struct Geo {
    int nx, ny, nz;
    long long n;  // nx * ny * nz
};

// Marker / shell tables of one field's IB corrector, in device memory.
template <typename T>
struct IBView {
    const int* ring_off;   // [nz + 1]: markers of plane z are ring_off[z] .. ring_off[z+1]-1
    const int* mk_q;       // [9 * nm]: in-plane index y * nx + x of the marker's 3 x 3 support
    const T* mk_w;         // [9 * nm]: D(x_k - X_j) = D_x D_y there (Sec. V.B)
    const T* mk_s;         // [nm]: lambda / (d (1 + d (lambda - 1)))
    const int* shell_off;  // [nz + 1]: shell nodes of plane z
    const int* shell_xy;   // [ns]: in-plane index y * nx + x of each shell node
    const int* csr_off;    // [ns + 1]: entries of shell node s
    const int* csr_m;      // [nnz]: marker index relative to its ring
    const T* csr_w;        // [nnz]: D(x_k - X_j) for that pair
    const int* mk_base;    // [nm]: first node of the marker's plane (z * nx * ny)
    const int* shell_node; // [ns]: node index of each shell node
    const int* csr_mg;     // [nnz]: marker index in the whole domain
    T* delta;              // [3 * nm]: delta_j of the two-phase corrector
    const int* mk_slot;    // [9 * nm]: position of each support node in its plane's shell list
                           //           (0 where the weight is zero)
    const int* pad_m;      // [ns_pad * pad_k]: each shell node's markers (ring-relative, CSR order)
    const T* pad_w;        //   and weights, padded with (0, 0.0) to pad_k entries
    int pad_k;             // a multiple of 4 (0: no padded lists; the staged corrector is not used)
    int nm, ns;
    int zinv;              // 1: every plane has plane 0's ring and shell tables (straight pipe)
};

// Coefficients of the tau_m = 1 magnetic sweep (Sec. V.G).
template <typename T>
struct SweepCoef {
    // The accelerated sweep of Sec. V.H, b <- (1/alpha) [(w_0 - 1 + alpha) b +
    // sum_{i>0} g_i(x - e_i)], is carried by the weights: w0 = (w_0 - 1 +
    // alpha)/alpha, w1 = w_axis/alpha (the plain weights, exactly, at alpha = 1).
    T w0, w1;      // scaled field-lattice weights: rest, axis
    T kappa;       // 1 / (c c_m^2) = 1 / (2 eta)
    T be[3];       // uniform B^ext (used when bext_z == nullptr)
    const T* bext_z;  // [3 * nz] B^ext per plane for the ramp, or nullptr
    int strict_qs;
    T sq;          // weight of b in the flux's B: 1, or 0 for the strict QS flux
    const T* bext_xy;  // [3][nx ny] in-plane applied field (QSLBM_B0_FIELD), or nullptr
};

// Coefficients of the flow update (Sec. III.E, V.A).
template <typename T>
struct FlowCoef {
    T tau;        // relaxation time
    T kforce;     // 1 - 1/(2 tau)
    T ig, ig2;    // 1/gamma, 1/gamma^2 (time step rescaled, Sec. VII; 1 by default)
    int mac;      // 1: density of the macroscopic scheme, sum_i f_i^eq(x - c_i) (Sec. V.G)
};

template <typename T>
struct ForceCoef {
    double F0, amp, omega;  // F_body(t) = F0 (1 + amp sin(omega t))
    int axis;               // direction of the body force
    T be[3];
    const T* bext_z;
    const T* bext_xy;  // [3][nx ny] in-plane applied field, or nullptr
};

__device__ __forceinline__ int wrap_dec(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_inc(int i, int n) { return i == n - 1 ? 0 : i + 1; }
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ void bext_at(const T* bext_z, const T* be, int z, T out[3]) {
    if (bext_z) {
        out[0] = bext_z[3 * z + 0];
        out[1] = bext_z[3 * z + 1];
        out[2] = bext_z[3 * z + 2];
    } else {
        out[0] = be[0];
        out[1] = be[1];
        out[2] = be[2];
    }
}

// Adds the in-plane applied field of node p (QSLBM_B0_FIELD) to a plane's value.
template <typename T>
__device__ __forceinline__ void bext_add_xy(const T* bxy, int P, int p, T out[3]) {
    if (bxy) {
        out[0] += bxy[p];
        out[1] += bxy[P + p];
        out[2] += bxy[2 * P + p];
    }
}

// ---------------------------------------------------------------------------
// IB corrector on plane z of field f[3] (f[c] + k), run by a whole CTA after
// the plane's predictor values are written.  sdelta: shared [3 * ring size].
// Sec. V.C-V.F: delta_j = s_j (0 - D f*), then f += D^T delta.
template <typename T>
__device__ __forceinline__ void ib_plane(const IBView<T>& ib, T* f0, T* f1, T* f2, long long plane_base,
                                         int z, T* sdelta) {
    const int m0 = ib.ring_off[z], m1 = ib.ring_off[z + 1];
    if (m1 == m0) return;  // uniform across the CTA: no divergence around barriers
    __syncthreads();
    for (int m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
        T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const T w = ib.mk_w[9 * m + j];
            const long long q = plane_base + ib.mk_q[9 * m + j];
            a0 += w * f0[q];
            a1 += w * f1[q];
            a2 += w * f2[q];
        }
        const T s = ib.mk_s[m];
        const int l = m - m0;
        sdelta[3 * l + 0] = -s * a0;
        sdelta[3 * l + 1] = -s * a1;
        sdelta[3 * l + 2] = -s * a2;
    }
    __syncthreads();
    const int s0 = ib.shell_off[z], s1 = ib.shell_off[z + 1];
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        T c0 = T(0), c1 = T(0), c2 = T(0);
        const int e0 = ib.csr_off[s], e1 = ib.csr_off[s + 1];
        for (int e = e0; e < e1; ++e) {
            const T w = ib.csr_w[e];
            const int l = ib.csr_m[e];
            c0 += w * sdelta[3 * l + 0];
            c1 += w * sdelta[3 * l + 1];
            c2 += w * sdelta[3 * l + 2];
        }
        const long long q = plane_base + ib.shell_xy[s];
        f0[q] += c0;
        f1[q] += c1;
        f2[q] += c2;
    }
}

// ---------------------------------------------------------------------------
// Magnetic sweep + IB on b for one z plane per CTA.
// b_alpha(x) <- w0 b_alpha(x) + w1 sum_beta [ b_alpha(x - e_beta) + b_alpha(x + e_beta)
//               + kappa (Phi_ab(x - e_beta) - Phi_ab(x + e_beta)) ],
// Phi_ab = u_beta B_alpha - u_alpha B_beta, B = B^ext + b (B^ext only if
// strict_qs).  This is sum_i g^eq_i(x - e_i) of Sec. V.G written per axis.
// diff[alpha] += sgn Phi_{alpha beta}, Phi_{alpha beta} = u_beta B_alpha - u_alpha B_beta,
// for alpha != beta (Phi_{beta beta} is zero).  beta is a constant after the
// callers' loops are unrolled, so the skipped component costs nothing.
template <typename T>
__device__ __forceinline__ void flux_acc(const T u[3], const T B[3], int beta, T sgn, T diff[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a != beta) diff[a] += sgn * (u[beta] * B[a] - u[a] * B[beta]);
}

// One node of the sweep: in-plane index p of the plane at base, z neighbours
// at zmbase / zpbase.  Neighbours enter in the order -x, +x, -y, +y, -z, +z.
// Indices are 32-bit (the library keeps 3 n below 2^31) so that every load is
// one pointer + offset.
template <typename T, int DIM>
__device__ __forceinline__ void sweep_node(const T* __restrict__ bin, const T* __restrict__ u, long long n_, int nx,
                                           int ny, long long base_, long long zmbase_, long long zpbase_, int p,
                                           const SweepCoef<T>& c, const T be_c[3], const T be_m[3],
                                           const T be_p[3], T out[3]) {
    const int n = (int)n_, base = (int)base_;
    const int y = p / nx;
    const int x = p - y * nx;
    const int k = base + p;
    int nb[6];  // -x, +x, -y, +y, -z, +z
    const int row = base + y * nx;
    nb[0] = row + wrap_dec(x, nx);
    nb[1] = row + wrap_inc(x, nx);
    nb[2] = base + wrap_dec(y, ny) * nx + x;
    nb[3] = base + wrap_inc(y, ny) * nx + x;
    nb[4] = (int)zmbase_ + p;
    nb[5] = (int)zpbase_ + p;
    const T* b0 = bin;
    const T* b1 = bin + n;
    const T* b2 = bin + 2 * n;
    const T* u0 = u;
    const T* u1 = u + n;
    const T* u2 = u + 2 * n;
    T acc[3] = {c.w0 * b0[k], c.w0 * b1[k], c.w0 * b2[k]};
    T diff[3] = {T(0), T(0), T(0)};  // sum_beta Phi_ab(x - e_beta) - Phi_ab(x + e_beta)
#pragma unroll
    for (int d = 0; d < 2 * DIM; ++d) {
        const int q = nb[d];
        const T bq[3] = {b0[q], b1[q], b2[q]};
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] += c.w1 * bq[a];
        const T uq[3] = {u0[q], u1[q], u2[q]};
        const T* bez = (d < 4) ? be_c : (d == 4 ? be_m : be_p);
        T Bx[3] = {bez[0], bez[1], bez[2]};
        bext_add_xy(c.bext_xy, nx * ny, d < 4 ? q - base : p, Bx);
        T B[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) B[a] = Bx[a] + c.sq * bq[a];
        // x - e_beta enters with +, x + e_beta with -
        flux_acc(uq, B, d >> 1, (d & 1) ? T(-1) : T(1), diff);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = acc[a] + c.w1 * c.kappa * diff[a];
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kPlaneThreads) k_sweep_ib(Geo g, const T* __restrict__ bin, T* bout,
                                                            const T* __restrict__ u, SweepCoef<T> c,
                                                            IBView<T> ib) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sdelta = reinterpret_cast<T*>(smem_raw);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int z = blockIdx.x;
    const long long n = g.n;
    const long long P = (long long)nx * ny;
    const long long base = (long long)z * P;
    const int zm = DIM == 3 ? wrap_dec(z, nz) : z, zp = DIM == 3 ? wrap_inc(z, nz) : z;
    T be_c[3], be_m[3], be_p[3];
    bext_at(c.bext_z, c.be, z, be_c);
    bext_at(c.bext_z, c.be, zm, be_m);
    bext_at(c.bext_z, c.be, zp, be_p);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        T o[3];
        sweep_node<T, DIM>(bin, u, n, nx, ny, base, (long long)zm * P, (long long)zp * P, p, c, be_c, be_m, be_p, o);
        bout[base + p] = o[0];
        bout[base + p + n] = o[1];
        bout[base + p + 2 * n] = o[2];
    }
    ib_plane<T>(ib, bout, bout + n, bout + 2 * n, base, ib.zinv ? 0 : z, sdelta);
}

// Node-parallel sweep without the IB (grid: in-plane blocks x z planes); the
// IB then runs as k_ib_planes.  For domains above L2 this keeps every SM busy
// regardless of the plane count.
constexpr int kNodeThreads = 256;

template <typename T, int DIM>
__global__ void __launch_bounds__(kNodeThreads) k_sweep_nodes(Geo g, const T* __restrict__ bin,
                                                              T* __restrict__ bout, const T* __restrict__ u,
                                                              SweepCoef<T> c) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int z = blockIdx.y;
    const int P = nx * ny;
    const int p = blockIdx.x * kNodeThreads + threadIdx.x;
    if (p >= P) return;
    const long long n = g.n;
    const long long base = (long long)z * P;
    const int zm = DIM == 3 ? wrap_dec(z, nz) : z, zp = DIM == 3 ? wrap_inc(z, nz) : z;
    T be_c[3], be_m[3], be_p[3];
    bext_at(c.bext_z, c.be, z, be_c);
    bext_at(c.bext_z, c.be, zm, be_m);
    bext_at(c.bext_z, c.be, zp, be_p);
    T o[3];
    sweep_node<T, DIM>(bin, u, n, nx, ny, base, (long long)zm * P, (long long)zp * P, p, c, be_c, be_m, be_p, o);
    bout[base + p] = o[0];
    bout[base + p + n] = o[1];
    bout[base + p + 2 * n] = o[2];
}

// z-marching sweep without the IB (3-D): a CTA owns an (x, y) tile of
// kMarchTX x kMarchTY columns and walks a chunk of z planes.  Each thread keeps
// its column's values at z - 1, z, z + 1 in registers, so a node costs one new
// load of (b, u) from HBM plus the tile's halo; the in-plane neighbours come
// from the tile of plane z staged in shared memory.
constexpr int kMarchTX = 32, kMarchTY = 8, kMarchChunk = 16;

// Halo cell of a march tile of TY rows handled by thread hid: the ring of
// (kMarchTX + 2) x (TY + 2) tile cells around the interior.  hp is the
// in-plane index of the node it stages (periodic image), -1 for no cell.
template <int TY = kMarchTY>
__device__ __forceinline__ void march_halo(int hid, int x0, int y0, int nx, int ny, int& hx, int& hy, int& hp) {
    constexpr int W = kMarchTX + 2, H = TY + 2, NH = 2 * W + 2 * TY;
    hx = 0;
    hy = 0;
    hp = -1;
    if (hid >= NH) return;
    if (hid < W) {
        hx = hid;
        hy = 0;
    } else if (hid < 2 * W) {
        hx = hid - W;
        hy = H - 1;
    } else {
        const int r = hid - 2 * W;
        hx = (r & 1) ? W - 1 : 0;
        hy = 1 + (r >> 1);
    }
    const int gx = (x0 + hx - 1 + nx) % nx, gy = (y0 + hy - 1 + ny) % ny;
    hp = gy * nx + gx;
}

// The flux Phi_{ab} = u_b B_a - u_a B_b is antisymmetric, so a node carries
// three numbers of it: e1 = Phi_yx, e2 = Phi_zx, e3 = Phi_zy (B = B^ext + sq b).
// Written over them, the neighbour sum of the sweep is
//   b_a <- w0 b_a + w1 (sum_{6 nbrs} b_a + kappa D_a),
//   D_x = e1(+y) - e1(-y) + e2(+z) - e2(-z),
//   D_y = e1(-x) - e1(+x) + e3(+z) - e3(-z),
//   D_z = e2(-x) - e2(+x) + e3(-y) - e3(+y),
// where D_a = sum_b [Phi_ab(x - e_b) - Phi_ab(x + e_b)] as in sweep_node.
// node_emf turns a node's (b, u) into (b, e) in place.
// The EMF form is the FP32 path; its roundings are spelled out (fused
// multiply-adds where written, nothing left to contraction) so that every
// kernel using it (march_tile, the node-pair sweep, the batched sweep)
// produces bitwise the same values.
__device__ __forceinline__ void node_emf(float r[6], const float be[3], float sq) {
    const float B0 = __fmaf_rn(sq, r[0], be[0]), B1 = __fmaf_rn(sq, r[1], be[1]), B2 = __fmaf_rn(sq, r[2], be[2]);
    const float u0 = r[3], u1 = r[4], u2 = r[5];
    r[3] = __fmaf_rn(u0, B1, -__fmul_rn(u1, B0));
    r[4] = __fmaf_rn(u0, B2, -__fmul_rn(u2, B0));
    r[5] = __fmaf_rn(u1, B2, -__fmul_rn(u2, B1));
}

// New b of one node in the EMF form: w0 b + (w1 s + w1 kappa D).
__device__ __forceinline__ float emf_update(float w0, float w1, float w1k, float b, float s, float d) {
    return __fmaf_rn(w0, b, __fmaf_rn(w1k, d, __fmul_rn(w1, s)));
}

// Shared tile of one march plane: six fields of (TY + 2) x (kMarchTX + 2)
// cells, the tile and its one-cell halo.
template <typename T, int TY = kMarchTY>
using MarchTile = T[6][TY + 2][kMarchTX + 2];

// The sweep over one tile and z chunk, one node per thread.  FP32 (EMF form):
// each node's (e1, e2, e3) is formed once, where its (b, u) is loaded, and the
// tile and the column registers hold (b, e); about half the arithmetic and
// shared-memory traffic of forming the flux per neighbour, the same sweep up
// to the order of rounding.  FP64 (direct form): the tile holds (b, u) and
// every neighbour's flux is formed as in sweep_node, with the same
// expressions and neighbour order, so that it rounds like the other FP64 sweep
// kernels.  The column's plane z + 2 is loaded one plane ahead of its use.
// TY: rows of the tile (the CTA has kMarchTX * TY threads); the results do not
// depend on it.
template <typename T, bool XY = true, int TY = kMarchTY>
__device__ __forceinline__ void march_tile(const Geo& g, const T* __restrict__ bin, T* __restrict__ bout,
                                           const T* __restrict__ u, const SweepCoef<T>& c, int bx, int by, int bz,
                                           int chunk, MarchTile<T, TY>& tile) {
    static_assert(kMarchTX * TY >= 2 * (kMarchTX + 2) + 2 * TY, "every halo cell needs a thread");
    constexpr bool EMF = sizeof(T) == 4;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int n = (int)g.n, P = nx * ny;
    const int tx = threadIdx.x % kMarchTX, ty = threadIdx.x / kMarchTX;
    const int x0 = bx * kMarchTX, y0 = by * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < nx && y < ny;
    // columns past the domain edge stage the periodic images their neighbours need
    const int xc = x % nx, yc = y % ny;
    const int p = yc * nx + xc;
    const int z0 = bz * chunk;
    const int z1 = min(z0 + chunk, nz);
    const T* src[6] = {bin, bin + n, bin + 2 * n, u, u + n, u + 2 * n};
    int hx, hy, hp;
    march_halo<TY>(threadIdx.x, x0, y0, nx, ny, hx, hy, hp);
    // prv / cur / nxt: the column at z - 1, z, z + 1 ((b, e) or (b, u)); ahd:
    // raw (b, u) of plane z + 2
    T prv[6], cur[6], nxt[6], ahd[6];
    {
        const int zm = wrap_dec(z0, nz), zn = wrap_inc(z0, nz);
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            prv[v] = src[v][zm * P + p];
            cur[v] = src[v][z0 * P + p];
            nxt[v] = src[v][zn * P + p];
        }
        if constexpr (EMF) {
            T be[3];
            bext_at(c.bext_z, c.be, zm, be);
            if constexpr (XY) bext_add_xy(c.bext_xy, P, p, be);
            node_emf(prv, be, c.sq);
            bext_at(c.bext_z, c.be, z0, be);
            if constexpr (XY) bext_add_xy(c.bext_xy, P, p, be);
            node_emf(cur, be, c.sq);
            bext_at(c.bext_z, c.be, zn, be);
            if constexpr (XY) bext_add_xy(c.bext_xy, P, p, be);
            node_emf(nxt, be, c.sq);
        }
    }
    const T w1k = c.w1 * c.kappa;
    for (int z = z0; z < z1; ++z) {
        const int zn = wrap_inc(z, nz);
        const int za = wrap_inc(zn, nz);
        if (z + 1 < z1) {
#pragma unroll
            for (int v = 0; v < 6; ++v) ahd[v] = src[v][za * P + p];
        }
        // stage plane z: interior from the column registers, halo from global
#pragma unroll
        for (int v = 0; v < 6; ++v) tile[v][ty + 1][tx + 1] = cur[v];
        if (hp >= 0) {
            T r[6];
#pragma unroll
            for (int v = 0; v < 6; ++v) r[v] = src[v][z * P + hp];
            if constexpr (EMF) {
                T be[3];
                bext_at(c.bext_z, c.be, z, be);
                if constexpr (XY) bext_add_xy(c.bext_xy, P, hp, be);
                node_emf(r, be, c.sq);
            }
#pragma unroll
            for (int v = 0; v < 6; ++v) tile[v][hy][hx] = r[v];
        }
        __syncthreads();
        if (active) {
            const int cx = tx + 1, cy = ty + 1;
            const int k = z * P + p;
            if constexpr (EMF) {
                T s[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    s[a] = (tile[a][cy][cx - 1] + tile[a][cy][cx + 1]) + (tile[a][cy - 1][cx] + tile[a][cy + 1][cx]) +
                           (prv[a] + nxt[a]);
                const T dx = (tile[3][cy + 1][cx] - tile[3][cy - 1][cx]) + (nxt[4] - prv[4]);
                const T dy = (tile[3][cy][cx - 1] - tile[3][cy][cx + 1]) + (nxt[5] - prv[5]);
                const T dz =
                    (tile[4][cy][cx - 1] - tile[4][cy][cx + 1]) + (tile[5][cy - 1][cx] - tile[5][cy + 1][cx]);
                bout[k] = emf_update(c.w0, c.w1, w1k, cur[0], s[0], dx);
                bout[k + n] = emf_update(c.w0, c.w1, w1k, cur[1], s[1], dy);
                bout[k + 2 * n] = emf_update(c.w0, c.w1, w1k, cur[2], s[2], dz);
            } else {
                T be_c[3], be_m[3], be_p[3];
                bext_at(c.bext_z, c.be, z, be_c);
                bext_at(c.bext_z, c.be, wrap_dec(z, nz), be_m);
                bext_at(c.bext_z, c.be, zn, be_p);
                T acc[3] = {c.w0 * cur[0], c.w0 * cur[1], c.w0 * cur[2]};
                T diff[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    T bq[3], uq[3];
                    if (d < 4) {
                        const int ix = cx + (d == 0 ? -1 : d == 1 ? 1 : 0);
                        const int iy = cy + (d == 2 ? -1 : d == 3 ? 1 : 0);
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            bq[a] = tile[a][iy][ix];
                            uq[a] = tile[3 + a][iy][ix];
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            bq[a] = d == 4 ? prv[a] : nxt[a];
                            uq[a] = d == 4 ? prv[3 + a] : nxt[3 + a];
                        }
                    }
                    const T* bez = (d < 4) ? be_c : (d == 4 ? be_m : be_p);
#pragma unroll
                    for (int a = 0; a < 3; ++a) acc[a] += c.w1 * bq[a];
                    T Bx[3] = {bez[0], bez[1], bez[2]};
                    if constexpr (XY) {
                        if (c.bext_xy) {
                            const int xq = d == 0 ? wrap_dec(xc, nx) : d == 1 ? wrap_inc(xc, nx) : xc;
                            const int yq = d == 2 ? wrap_dec(yc, ny) : d == 3 ? wrap_inc(yc, ny) : yc;
                            bext_add_xy(c.bext_xy, P, yq * nx + xq, Bx);
                        }
                    }
                    T B[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) B[a] = Bx[a] + c.sq * bq[a];
                    flux_acc(uq, B, d >> 1, (d & 1) ? T(-1) : T(1), diff);
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) bout[k + a * n] = acc[a] + c.w1 * c.kappa * diff[a];
            }
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            prv[v] = cur[v];
            cur[v] = nxt[v];
        }
        if (z + 1 < z1) {
            if constexpr (EMF) {
                T be[3];
                bext_at(c.bext_z, c.be, za, be);
                if constexpr (XY) bext_add_xy(c.bext_xy, P, p, be);
                node_emf(ahd, be, c.sq);
            }
#pragma unroll
            for (int v = 0; v < 6; ++v) nxt[v] = ahd[v];
        }
    }
}

// XY: the domain has an in-plane applied field (QSLBM_B0_FIELD)
template <typename T, bool XY>
__global__ void __launch_bounds__(kMarchTX* kMarchTY) k_sweep_march(Geo g, const T* __restrict__ bin,
                                                                    T* __restrict__ bout, const T* __restrict__ u,
                                                                    SweepCoef<T> c, int chunk) {
    __shared__ MarchTile<T> tile;
    march_tile<T, XY>(g, bin, bout, u, c, blockIdx.x, blockIdx.y, blockIdx.z, chunk, tile);
}

// FP32 z-marching sweep on x-adjacent node pairs (nx even): a CTA of 256
// threads owns a tile of kPairTXP pairs (32 nodes) x kPairTY rows and walks a
// chunk of z planes; every global access moves two nodes (8 bytes), so the
// address arithmetic, loads, stores and loop overhead per node are half those
// of march_tile.  EMF form as in march_tile.  The staged plane is
// double-buffered (one barrier per plane) and every global load is issued one
// plane ahead of its use: the column's plane z + 2, the halo's plane z + 1.
constexpr int kPairTXP = 16, kPairTY = 16;
constexpr int kPairThreads = kPairTXP * kPairTY;
// tile row: pad, left halo, 32 nodes, right halo, pad (pairs start at even columns)
constexpr int kPairW = 2 * kPairTXP + 4;
using PairTile = float[2][6][kPairTY + 2][kPairW];

// Halo item hid of a pair tile (64 items): 0-15 the pairs of the row above,
// 16-31 the row below, 32-47 the column left of the tile, 48-63 the column
// right of it (corners are not needed by the 5-point in-plane stencil).
// kind: 0 none, 1 pair, 2 single node; gp: in-plane index (periodic image).
__device__ __forceinline__ void pair_halo(int hid, int x0, int y0, int nx, int ny, int& kind, int& row, int& col,
                                          int& gp) {
    kind = 0;
    row = 0;
    col = 0;
    gp = 0;
    if (hid >= 64) return;
    int gx, gy;
    if (hid < 32) {
        const int j = hid & 15;
        kind = 1;
        row = hid < 16 ? 0 : kPairTY + 1;
        col = 2 + 2 * j;
        gx = (x0 + 2 * j) % nx;
        gy = hid < 16 ? (y0 - 1 + ny) % ny : (y0 + kPairTY) % ny;
    } else {
        const int i = hid & 15;
        kind = 2;
        row = 1 + i;
        col = hid < 48 ? 1 : 2 * kPairTXP + 2;
        gx = hid < 48 ? (x0 - 1 + nx) % nx : (x0 + 2 * kPairTXP) % nx;
        gy = (y0 + i) % ny;
    }
    gp = gy * nx + gx;
}

__device__ __forceinline__ void pair_emf(float2 r[6], const float beA[3], const float beB[3], float sq) {
    float a[6] = {r[0].x, r[1].x, r[2].x, r[3].x, r[4].x, r[5].x};
    float b[6] = {r[0].y, r[1].y, r[2].y, r[3].y, r[4].y, r[5].y};
    node_emf(a, beA, sq);
    node_emf(b, beB, sq);
#pragma unroll
    for (int v = 0; v < 6; ++v) r[v] = make_float2(a[v], b[v]);
}

template <typename F, bool XY>
__global__ void __launch_bounds__(kPairThreads) k_sweep_march_pair(Geo g, const F* __restrict__ bin,
                                                                   F* __restrict__ bout, const F* __restrict__ u,
                                                                   SweepCoef<F> c, int chunk) {
    static_assert(sizeof(F) == 4, "the pair sweep is the FP32 path");
    __shared__ __align__(16) PairTile tile;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int n = (int)g.n, P = nx * ny;
    const int tx = threadIdx.x % kPairTXP, ty = threadIdx.x / kPairTXP;
    const int x0 = blockIdx.x * 2 * kPairTXP, y0 = blockIdx.y * kPairTY;
    const int x = x0 + 2 * tx, y = y0 + ty;
    const bool active = x < nx && y < ny;
    const int p = (y % ny) * nx + (x % nx);  // even: a pair never straddles a row end
    const int z0 = blockIdx.z * chunk;
    const int z1 = min(z0 + chunk, nz);
    const float* src[6] = {bin, bin + n, bin + 2 * n, u, u + n, u + 2 * n};
    int hkind, hrow, hcol, hp;
    pair_halo(threadIdx.x, x0, y0, nx, ny, hkind, hrow, hcol, hp);
    auto ld2 = [](const float* q) { return *reinterpret_cast<const float2*>(q); };
    // halo values of plane zz (raw), pair or single node (in .x)
    auto load_halo = [&](int zz, float2 h[6]) {
        if (hkind == 1) {
#pragma unroll
            for (int v = 0; v < 6; ++v) h[v] = ld2(src[v] + zz * P + hp);
        } else if (hkind == 2) {
#pragma unroll
            for (int v = 0; v < 6; ++v) h[v] = make_float2(src[v][zz * P + hp], 0.f);
        }
    };
    // (b, u) -> (b, e) of the nodes pp and pp + 1 of plane zz
    auto emf2 = [&](float2 r[6], int zz, int pp) {
        float be[3];
        bext_at(c.bext_z, c.be, zz, be);
        if constexpr (XY) {
            float bA[3] = {be[0], be[1], be[2]}, bB[3] = {be[0], be[1], be[2]};
            bext_add_xy(c.bext_xy, P, pp, bA);
            bext_add_xy(c.bext_xy, P, pp + 1 < P ? pp + 1 : pp, bB);
            pair_emf(r, bA, bB, c.sq);
        } else {
            pair_emf(r, be, be, c.sq);
        }
    };
    float2 prv[6], cur[6], nxt[6], ahd[6], hcur[6], hnxt[6];
    // the IB pass after this sweep may be scheduled as this grid's CTAs exit;
    // b comes from the kernel before this one
    pdl_trigger();
    pdl_wait();
    {
        const int zm = wrap_dec(z0, nz), zn = wrap_inc(z0, nz);
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            prv[v] = ld2(src[v] + zm * P + p);
            cur[v] = ld2(src[v] + z0 * P + p);
            nxt[v] = ld2(src[v] + zn * P + p);
        }
        load_halo(z0, hcur);
        emf2(prv, zm, p);
        emf2(cur, z0, p);
        emf2(nxt, zn, p);
    }
    const float w0 = c.w0, w1 = c.w1, w1k = c.w1 * c.kappa;
    const int r = ty + 1, cc = 2 + 2 * tx;
    for (int z = z0; z < z1; ++z) {
        const int zn = wrap_inc(z, nz);
        const int za = wrap_inc(zn, nz);
        const int buf = z & 1;
        if (z + 1 < z1) {
#pragma unroll
            for (int v = 0; v < 6; ++v) ahd[v] = ld2(src[v] + za * P + p);
            load_halo(zn, hnxt);
        }
        auto& t = tile[buf];
#pragma unroll
        for (int v = 0; v < 6; ++v) *reinterpret_cast<float2*>(&t[v][r][cc]) = cur[v];
        if (hkind != 0) {
            emf2(hcur, z, hp);  // a single halo node uses .x only
            if (hkind == 1) {
#pragma unroll
                for (int v = 0; v < 6; ++v) *reinterpret_cast<float2*>(&t[v][hrow][hcol]) = hcur[v];
            } else {
#pragma unroll
                for (int v = 0; v < 6; ++v) t[v][hrow][hcol] = hcur[v].x;
            }
        }
        __syncthreads();
        if (active) {
            float lf[6], rt[6];
            float2 up[6], dn[6];
#pragma unroll
            for (int v = 0; v < 6; ++v) {
                if (v != 5) {  // x neighbours: b, e1, e2
                    lf[v] = t[v][r][cc - 1];
                    rt[v] = t[v][r][cc + 2];
                }
                if (v != 4) {  // y neighbours: b, e1, e3
                    up[v] = *reinterpret_cast<const float2*>(&t[v][r - 1][cc]);
                    dn[v] = *reinterpret_cast<const float2*>(&t[v][r + 1][cc]);
                }
            }
            const int k = z * P + p;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float sL = (lf[a] + cur[a].y) + (up[a].x + dn[a].x) + (prv[a].x + nxt[a].x);
                const float sR = (cur[a].x + rt[a]) + (up[a].y + dn[a].y) + (prv[a].y + nxt[a].y);
                float dL, dR;
                if (a == 0) {
                    dL = (dn[3].x - up[3].x) + (nxt[4].x - prv[4].x);
                    dR = (dn[3].y - up[3].y) + (nxt[4].y - prv[4].y);
                } else if (a == 1) {
                    dL = (lf[3] - cur[3].y) + (nxt[5].x - prv[5].x);
                    dR = (cur[3].x - rt[3]) + (nxt[5].y - prv[5].y);
                } else {
                    dL = (lf[4] - cur[4].y) + (up[5].x - dn[5].x);
                    dR = (cur[4].x - rt[4]) + (up[5].y - dn[5].y);
                }
                *reinterpret_cast<float2*>(bout + k + a * n) =
                    make_float2(emf_update(w0, w1, w1k, cur[a].x, sL, dL), emf_update(w0, w1, w1k, cur[a].y, sR, dR));
            }
        }
#pragma unroll
        for (int v = 0; v < 6; ++v) {
            prv[v] = cur[v];
            cur[v] = nxt[v];
            hcur[v] = hnxt[v];
        }
        if (z + 1 < z1) {
            emf2(ahd, za, p);
#pragma unroll
            for (int v = 0; v < 6; ++v) nxt[v] = ahd[v];
        }
    }
}

// Two-phase IB corrector over the whole domain (Sec. V.C-V.F): first one
// thread per marker forms delta_j = s_j (0 - D f*) from the predictor field,
// then (next launch, so every delta is ready) one thread per shell node adds
// sum_j D(x_k - X_j) delta_j.  Same sums, in the same order, as ib_plane.
template <typename T>
__device__ __forceinline__ void ib_marker(const IBView<T>& ib, const T* __restrict__ f, int n, int m) {
    T a0 = T(0), a1 = T(0), a2 = T(0);
    const int base = ib.mk_base[m];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const T w = ib.mk_w[9 * m + j];
        const int q = base + ib.mk_q[9 * m + j];
        a0 += w * f[q];
        a1 += w * f[q + n];
        a2 += w * f[q + 2 * n];
    }
    const T sm = ib.mk_s[m];
    ib.delta[3 * m + 0] = -sm * a0;
    ib.delta[3 * m + 1] = -sm * a1;
    ib.delta[3 * m + 2] = -sm * a2;
}

template <typename T>
__device__ __forceinline__ void ib_shell(const IBView<T>& ib, T* __restrict__ f, int n, int i) {
    T c0 = T(0), c1 = T(0), c2 = T(0);
    const int e0 = ib.csr_off[i], e1 = ib.csr_off[i + 1];
    for (int e = e0; e < e1; ++e) {
        const T w = ib.csr_w[e];
        const int m = ib.csr_mg[e];
        c0 += w * ib.delta[3 * m + 0];
        c1 += w * ib.delta[3 * m + 1];
        c2 += w * ib.delta[3 * m + 2];
    }
    const int q = ib.shell_node[i];
    f[q] += c0;
    f[q + n] += c1;
    f[q + 2 * n] += c2;
}

template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_ib_markers(Geo g, const T* __restrict__ f, IBView<T> ib) {
    const int m = blockIdx.x * kNodeThreads + threadIdx.x;
    if (m < ib.nm) ib_marker<T>(ib, f, (int)g.n, m);
}

template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_ib_shell(Geo g, T* __restrict__ f, IBView<T> ib) {
    const int i = blockIdx.x * kNodeThreads + threadIdx.x;
    if (i < ib.ns) ib_shell<T>(ib, f, (int)g.n, i);
}

// IB corrector alone, one CTA per z plane, after a sweep kernel without the
// IB (k_sweep_march, k_sweep_nodes).  With z-invariant tables (a straight
// pipe) every CTA reads plane 0's tables, which then stay in cache.
template <typename T>
__global__ void __launch_bounds__(kNodeThreads) k_ib_planes(Geo g, T* f, IBView<T> ib) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sdelta = reinterpret_cast<T*>(smem_raw);
    const long long n = g.n;
    const long long base = (long long)blockIdx.x * g.nx * g.ny;
    ib_plane<T>(ib, f, f + n, f + 2 * n, base, ib.zinv ? 0 : (int)blockIdx.x, sdelta);
}

// Shared memory of the staged IB corrector for a plane of R markers and S
// shell nodes: 3 R deltas, 3 S staged values, the markers' 9 R weights and R
// scalings, then 9 R shell slots (int).
template <typename T>
__host__ __device__ inline size_t ib_staged_smem_bytes(int max_ring, int max_shell) {
    return (size_t)(13 * max_ring + 3 * max_shell) * sizeof(T) + (size_t)9 * max_ring * sizeof(int);
}

// Shell nodes a thread of the staged corrector loads at once (U), and the CTAs
// kept resident per SM at that U (bounds the registers).  When the launch's
// planes fit one wave at four CTAs per SM, U is chosen for the largest shell
// so that one batch of loads covers it (U = 4 for shells of up to 1024 nodes,
// as on the 96x96x512 pipe, where four CTAs per SM cover a plane per CTA; 5
// above that); with more planes than that, U = 1 keeps eight CTAs per SM in
// flight.
inline int ib_staged_unroll(int max_shell, long long planes, int sms) {
    if (planes > 4LL * sms) return 1;
    return max_shell <= kNodeThreads ? 1
                                      : (max_shell <= 2 * kNodeThreads ? 2 : (max_shell <= 4 * kNodeThreads ? 4 : 5));
}
template <typename T, int U>
constexpr int kIbStagedMinBlocks = (sizeof(T) == 4 ? 8 : 4) / (U == 1 ? 1 : 2);

// Four consecutive weights of a padded marker list (16-byte aligned rows).
__device__ __forceinline__ void ld4(const float* p, float (&w)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&w)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}

// The IB corrector with the plane's shell nodes staged in shared memory, on
// plane `base` of f (three components n apart).  Three phases, each one
// round trip to memory: (A) the shell values and the markers' tables are
// read with independent loads into shared memory; (B) each marker
// interpolates from the staged copy through mk_slot; (C) each shell node adds
// the spread of its markers' deltas, read from its padded marker list
// (pad_k entries, weight 0 past its own), and is written once.  Same sums in
// the same order as ib_plane (the padding adds exact zeros).  tz: the plane
// whose tables apply; smem as ib_staged_smem_bytes.  Called by every thread
// of the CTA.
template <typename T, int THREADS, int U>
__device__ __forceinline__ void ib_staged_plane(const IBView<T>& ib, T* f, int n, int base, int tz, int max_ring,
                                                int max_shell, unsigned char* smem) {
    const int m0 = ib.ring_off[tz], R = ib.ring_off[tz + 1] - m0;
    if (R == 0) return;  // uniform across the CTA
    const int s0 = ib.shell_off[tz], S = ib.shell_off[tz + 1] - s0;
    T* sdelta = reinterpret_cast<T*>(smem);  // [3 R]
    T* sf = sdelta + 3 * max_ring;           // [3 S]
    T* tw = sf + 3 * max_shell;              // [9 R]
    T* tsc = tw + 9 * max_ring;              // [R]
    int* tslot = reinterpret_cast<int*>(tsc + max_ring);  // [9 R]
    T* f0 = f + base;
    T* f1 = f0 + n;
    T* f2 = f1 + n;
    const int tid = threadIdx.x;
    // (A) the markers' tables (constant: read before the wait for the
    // sweep that wrote f), then the shell values (in-plane index, then value)
    for (int e = tid; e < 9 * R; e += THREADS) {
        tw[e] = __ldg(ib.mk_w + 9 * m0 + e);
        tslot[e] = __ldg(ib.mk_slot + 9 * m0 + e);
    }
    for (int m = tid; m < R; m += THREADS) tsc[m] = __ldg(ib.mk_s + m0 + m);
    pdl_wait();
    for (int i0 = 0; i0 < S; i0 += U * THREADS) {
        int q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * THREADS + tid;
            q[u] = i < S ? __ldg(ib.shell_xy + s0 + i) : 0;
        }
        T v[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * THREADS + tid < S) {
                v[u][0] = f0[q[u]];
                v[u][1] = f1[q[u]];
                v[u][2] = f2[q[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * THREADS + tid;
            if (i < S) {
                sf[i] = v[u][0];
                sf[S + i] = v[u][1];
                sf[2 * S + i] = v[u][2];
            }
        }
    }
    __syncthreads();
    // (B) delta_j = -s_j D f* at every marker
    for (int m = tid; m < R; m += THREADS) {
        T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const T w = tw[9 * m + j];
            const int q = tslot[9 * m + j];
            a0 += w * sf[q];
            a1 += w * sf[S + q];
            a2 += w * sf[2 * S + q];
        }
        const T sm = tsc[m];
        sdelta[3 * m + 0] = -sm * a0;
        sdelta[3 * m + 1] = -sm * a1;
        sdelta[3 * m + 2] = -sm * a2;
    }
    __syncthreads();
    // (C) f += D^T delta on the shell, four list entries per load
    const int K = ib.pad_k;
    for (int i0 = 0; i0 < S; i0 += U * THREADS) {
        T c[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u][0] = c[u][1] = c[u][2] = T(0);
        for (int k0 = 0; k0 < K; k0 += 4) {
            int4 mm[U];
            T ww[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * THREADS + tid;
                if (i < S) {
                    const long long r = (long long)(s0 + i) * K + k0;
                    mm[u] = __ldg(reinterpret_cast<const int4*>(ib.pad_m + r));
                    ld4(ib.pad_w + r, ww[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + u * THREADS + tid < S) {
                    const int l[4] = {mm[u].x, mm[u].y, mm[u].z, mm[u].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        c[u][0] += ww[u][e] * sdelta[3 * l[e] + 0];
                        c[u][1] += ww[u][e] * sdelta[3 * l[e] + 1];
                        c[u][2] += ww[u][e] * sdelta[3 * l[e] + 2];
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * THREADS + tid;
            if (i < S) {
                const int q = __ldg(ib.shell_xy + s0 + i);
                f0[q] = sf[i] + c[u][0];
                f1[q] = sf[S + i] + c[u][1];
                f2[q] = sf[2 * S + i] + c[u][2];
            }
        }
    }
}

// The staged corrector as a launch of its own, one CTA per plane; shared
// memory ib_staged_smem_bytes(max_ring, max_shell).
template <typename T, int U>
__global__ void __launch_bounds__(kNodeThreads, (kIbStagedMinBlocks<T, U>))
    k_ib_staged(Geo g, T* f, IBView<T> ib, int max_ring, int max_shell) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z = blockIdx.x;
    pdl_trigger();  // the next sweep may be scheduled as these CTAs exit
    ib_staged_plane<T, kNodeThreads, U>(ib, f, (int)g.n, z * g.nx * g.ny, ib.zinv ? 0 : z, max_ring, max_shell,
                                     smem_raw);
}

// ---------------------------------------------------------------------------
// Lattice tables for the flow update: D2Q9, D3Q19, and the paper's own D3Q27
// (Sec. III.A, Table I).  Q is the number of velocities; the 3-D tables list
// the rest velocity, the 6 axis, the 12 edge (D3Q19 ends here) and the 8
// corner velocities.
template <int DIM>
constexpr int kDefaultFlowQ = DIM == 3 ? 19 : 9;

__device__ __forceinline__ void flow_dir3(int j, int& cx, int& cy, int& cz) {
    const int tx[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    const int ty[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    const int tz[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, 1, -1, -1, -1, -1};
    cx = tx[j];
    cy = ty[j];
    cz = tz[j];
}
__device__ __forceinline__ void flow_dir2(int j, int& cx, int& cy, int& cz) {
    const int tx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ty[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    cx = tx[j];
    cy = ty[j];
    cz = 0;
}
template <int Q>
__device__ __forceinline__ void flow_dir(int j, int& cx, int& cy, int& cz) {
    if constexpr (Q == 9)
        flow_dir2(j, cx, cy, cz);
    else
        flow_dir3(j, cx, cy, cz);
}

template <int Q>
__device__ __forceinline__ double flow_w(int j) {
    static_assert(Q == 9 || Q == 19 || Q == 27, "flow lattices: D2Q9, D3Q19, D3Q27");
    if (Q == 27) return j == 0 ? 8.0 / 27.0 : (j <= 6 ? 2.0 / 27.0 : (j <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
    if (Q == 19) return j == 0 ? 1.0 / 3.0 : (j <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    return j == 0 ? 4.0 / 9.0 : (j <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------
// Force: J = curl b by isotropic differences on the flow lattice
// (d_beta phi = 3 sum_i w_i c_i,beta phi(x + c_i)), F = F_body(t) e_axis +
// J x (B^ext + b).  One thread per node.
template <typename T, int DIM, int Q = kDefaultFlowQ<DIM>>
__device__ __forceinline__ void force_node(const T* __restrict__ b, T* __restrict__ F, long long n, int nx, int ny,
                                           int nz, int x, int y, int z, long long k, const ForceCoef<T>& c,
                                           T fb) {
    const T* b1 = b + n;
    const T* b2 = b + 2 * n;
    T db[3][3];  // db[beta][alpha] = d_beta b_alpha
#pragma unroll
    for (int be = 0; be < 3; ++be)
#pragma unroll
        for (int a = 0; a < 3; ++a) db[be][a] = T(0);
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        int cx, cy, cz;
        flow_dir<Q>(j, cx, cy, cz);
        const int q = (wrapi(z + cz, nz) * ny + wrapi(y + cy, ny)) * nx + wrapi(x + cx, nx);
        const T w = (T)(3.0 * flow_w<Q>(j));
        const T bq[3] = {b[q], b1[q], b2[q]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (cx) db[0][a] += (w * (T)cx) * bq[a];
            if (cy) db[1][a] += (w * (T)cy) * bq[a];
            if (cz) db[2][a] += (w * (T)cz) * bq[a];
        }
    }
    const T J[3] = {db[1][2] - db[2][1], db[2][0] - db[0][2], db[0][1] - db[1][0]};
    T Be[3];
    bext_at(c.bext_z, c.be, z, Be);
    bext_add_xy(c.bext_xy, nx * ny, y * nx + x, Be);
    const T B[3] = {Be[0] + b[k], Be[1] + b[k + n], Be[2] + b[k + 2 * n]};
    T L[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
    L[c.axis] += fb;
    F[k] = L[0];
    F[k + n] = L[1];
    F[k + 2 * n] = L[2];
}

template <typename T>
__device__ __forceinline__ T body_force_at(const ForceCoef<T>& c, long long t) {
    const double fb_d = c.amp != 0.0 ? c.F0 * (1.0 + c.amp * sin(c.omega * (double)t)) : c.F0;
    return (T)fb_d;
}

template <typename T, int DIM, int Q = kDefaultFlowQ<DIM>>
__global__ void __launch_bounds__(256) k_force(Geo g, const T* __restrict__ b, T* __restrict__ F,
                                               ForceCoef<T> c, const long long* __restrict__ tstep) {
    const long long n = g.n;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const T fb = body_force_at(c, *tstep);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx);
        const int y = (int)((k / nx) % ny);
        const int z = (int)(k / ((long long)nx * ny));
        force_node<T, DIM, Q>(b, F, n, nx, ny, nz, x, y, z, k, c, fb);
    }
}

// ---------------------------------------------------------------------------
// Single-step flow update + IB on u, one z plane per CTA.  For each neighbour
// y = x + c_j the equilibria of direction j (as f_j(x + c_j)) and of the
// opposite direction (as f_jbar(x - c_jbar)) are formed from one load of y:
//   drho* = 2 f~_0(x) - drho(x) + sum_j [ 0.5 f~_j(y) + 1.5 f~_jbar(y) ]
//   m*    = sum_j c_j [ (tau - 1) f~_j(y) - tau f~_jbar(y) ] - 2 (tau - 1) rho u(x)
//           - (tau/2) sum_j c_j [ F_j(y) + F_jbar(y) ] + F(x)
// with f~_i = f_i^eq - w_i = w_i (drho + q_i + drho q_i),
// q_i = 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u, and the GZS terms
// F_j + F_jbar = (1 - 1/2tau) w_j (-6 u.F + 18 (c_j.u)(c_j.F)).  This uses
// sum_i f_i^eq(x) = rho and sum_i c_i f_i^eq(x) = rho u, exact on the lattice.
template <typename T, int DIM, int Q = kDefaultFlowQ<DIM>>
__device__ __forceinline__ void flow_node(const T* __restrict__ drho, const T* __restrict__ u,
                                          const T* __restrict__ F, T* __restrict__ drho_out, T* uout, long long n,
                                          int nx, int ny, int nz, int x, int y, int z, long long k,
                                          const FlowCoef<T>& c) {
    const T* u1 = u + n;
    const T* u2 = u + 2 * n;
    const T* F1 = F + n;
    const T* F2 = F + 2 * n;
    const T tau = c.tau, tm1 = c.tau - T(1), half_tau = T(0.5) * c.tau;
    const T dr0 = drho[k];
    const T ux0 = u[k], uy0 = u[k + n], uz0 = u[k + 2 * n];
    const T uu0 = ux0 * ux0 + uy0 * uy0 + uz0 * uz0;
    const T q0 = T(-1.5) * uu0 * c.ig;
    const T w0 = (T)flow_w<Q>(0);
    // single-step density (Sec. III.E) or the macroscopic scheme's (Sec. V.G);
    // c.mac is uniform across the launch
    T rho_acc = c.mac ? w0 * (dr0 + q0 + dr0 * q0) : T(2) * w0 * (dr0 + q0 + dr0 * q0) - dr0;
    T m[3] = {T(0), T(0), T(0)};
    T corr[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int j = 1; j < Q; ++j) {
        int cx, cy, cz;
        flow_dir<Q>(j, cx, cy, cz);
        const int q = (wrapi(z + cz, nz) * ny + wrapi(y + cy, ny)) * nx + wrapi(x + cx, nx);
        const T dr = drho[q];
        const T uq[3] = {u[q], u1[q], u2[q]};
        const T Fq[3] = {F[q], F1[q], F2[q]};
        const T a = (T)cx * uq[0] + (T)cy * uq[1] + (T)cz * uq[2];
        const T uu = uq[0] * uq[0] + uq[1] * uq[1] + uq[2] * uq[2];
        const T cF = (T)cx * Fq[0] + (T)cy * Fq[1] + (T)cz * Fq[2];
        const T uF = uq[0] * Fq[0] + uq[1] * Fq[1] + uq[2] * Fq[2];
        const T w = (T)flow_w<Q>(j);
        const T sq = (T(4.5) * a * a - T(1.5) * uu) * c.ig;
        const T qp = T(3) * a + sq, qm = T(-3) * a + sq;
        const T fj = w * (dr + qp + dr * qp);
        const T fjb = w * (dr + qm + dr * qm);
        if (c.mac)
            rho_acc += fjb;  // f^eq of direction -c_j at x + c_j
        else
            rho_acc += T(0.5) * fj + T(1.5) * fjb;
        const T mom = tm1 * fj - tau * fjb;
        const T fs = c.kforce * w * (T(-6) * uF + T(18) * a * cF) * c.ig2;
        if (cx) {
            m[0] += (T)cx * mom;
            corr[0] += (T)cx * fs;
        }
        if (cy) {
            m[1] += (T)cy * mom;
            corr[1] += (T)cy * fs;
        }
        if (cz) {
            m[2] += (T)cz * mom;
            corr[2] += (T)cz * fs;
        }
    }
    const T rho0 = T(1) + dr0;
    const T rho_new = T(1) + rho_acc;
    const T inv = T(1) / rho_new;
    const T Fk[3] = {F[k], F[k + n], F[k + 2 * n]};
    const T u0v[3] = {ux0, uy0, uz0};
    drho_out[k] = rho_acc;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T mm = m[a] - T(2) * tm1 * rho0 * u0v[a] - half_tau * corr[a] + Fk[a] * c.ig;
        uout[k + a * n] = mm * inv;
    }
}

template <typename T, int DIM, int Q = kDefaultFlowQ<DIM>>
__global__ void __launch_bounds__(kPlaneThreads) k_flow_ib(Geo g, const T* __restrict__ drho,
                                                           const T* __restrict__ u, const T* __restrict__ F,
                                                           T* __restrict__ drho_out, T* uout, FlowCoef<T> c,
                                                           IBView<T> ib, long long* tstep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sdelta = reinterpret_cast<T*>(smem_raw);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int z = blockIdx.x;
    const long long n = g.n;
    const long long P = (long long)nx * ny;
    const long long base = (long long)z * P;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int y = p / nx;
        const int x = p - y * nx;
        flow_node<T, DIM, Q>(drho, u, F, drho_out, uout, n, nx, ny, nz, x, y, z, base + p, c);
    }
    ib_plane<T>(ib, uout, uout + n, uout + 2 * n, base, ib.zinv ? 0 : z, sdelta);
    if (blockIdx.x == 0 && threadIdx.x == 0) *tstep += 1;
}

// ---------------------------------------------------------------------------
// Initial state: drho = 0, b = 0, u = splitmix64 noise (Steele, Lea, Flood)
// of the counter seed ^ (3 k + component), top 53 bits to [-1, 1), times amp,
// on nodes within radius R of the wall centre (between the walls for a channel).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void k_init(Geo g, T* drho, T* u, T* b, unsigned long long seed, double amp, int ncomp,
                       int geometry, double cx, double cy, double R, int poiseuille, double U0, int axis) {
    const long long n = g.n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        drho[k] = T(0);
        const int x = (int)(k % g.nx);
        const int y = (int)((k / g.nx) % g.ny);
        bool inside;
        if (geometry == 2)
            inside = true;
        else if (geometry == 0)
            inside = fabs((double)y - cy) <= R;
        else
            inside = sqrt(((double)x - cx) * ((double)x - cx) + ((double)y - cy) * ((double)y - cy)) <= R;
        for (int a = 0; a < 3; ++a) {
            b[k + a * n] = T(0);
            double v = 0.0;
            if (amp != 0.0 && inside && a < ncomp) {
                const unsigned long long r = splitmix64(seed ^ (unsigned long long)(3 * k + a));
                v = amp * ((double)(r >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
            }
            if (poiseuille && inside && a == axis && geometry != 2) {
                const double d2 = geometry == 0 ? ((double)y - cy) * ((double)y - cy)
                                                : ((double)x - cx) * ((double)x - cx) + ((double)y - cy) * ((double)y - cy);
                v += U0 * (1.0 - d2 / (R * R));
            }
            u[k + a * n] = (T)v;
        }
    }
}

// Conversions between the device state and binary64 staging arrays.
template <typename T>
__global__ void k_to_f64(long long n, const T* drho, const T* u, const T* b, double* out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        out[k] = 1.0 + (double)drho[k];
        for (int a = 0; a < 3; ++a) {
            out[(1 + a) * n + k] = (double)u[a * n + k];
            out[(4 + a) * n + k] = (double)b[a * n + k];
        }
    }
}

template <typename T>
__global__ void k_from_f64(long long n, const double* in, T* drho, T* u, T* b, int mask) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        if (mask & 1) drho[k] = (T)(in[k] - 1.0);
        for (int a = 0; a < 3; ++a) {
            if (mask & 2) u[a * n + k] = (T)in[(1 + a) * n + k];
            if (mask & 4) b[a * n + k] = (T)in[(4 + a) * n + k];
        }
    }
}

// ---------------------------------------------------------------------------
// Diagnostics in binary64: per-block partial sums, then one block folds them
// in a fixed order (deterministic).  Slots:
// 0 mass, 1 E_k, 2 E_m, 3 pump, 4 visc (u . lap u), 5 joule, 6 qs^2,
// 7 |u - usnap|^2, 8 |u|^2, 9 count, 10 non-finite count.
template <typename T>
struct ObsCoef {
    double eta, fb;  // resistivity, F_body at the current step
    int axis, geometry, strict_qs, dim;
    double cx, cy, rin;  // region: distance from the centre <= rin
    T be[3];
    const T* bext_z;
    const T* bext_xy;  // [3][nx ny] in-plane applied field, or nullptr
};

template <typename T, int DIM, int Q = kDefaultFlowQ<DIM>>
__global__ void __launch_bounds__(kReduceThreads) k_observe(Geo g, const T* __restrict__ drho,
                                                            const T* __restrict__ u, const T* __restrict__ b,
                                                            const T* __restrict__ usnap, ObsCoef<T> c,
                                                            double* partial) {
    __shared__ double red[kObs][kReduceThreads / 32];
    // The node-local derivatives (flow-lattice Laplacian of u, gradient of b,
    // the field lattice's QS operators) are formed in the fields' own
    // precision; every product that enters a sum, and the sums, are FP64.
    using L = typename std::conditional<sizeof(T) == 4, float, double>::type;
    double acc[kObs];
#pragma unroll
    for (int i = 0; i < kObs; ++i) acc[i] = 0.0;
    const int n = (int)g.n;  // the library keeps 3 n below 2^31
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int x = k % nx;
        const int t = k / nx;
        const int y = t % ny;
        const int z = t / ny;
        const double rho = 1.0 + (double)drho[k];
        const T ut[3] = {u[k], u[k + n], u[k + 2 * n]};
        const T bt[3] = {b[k], b[k + n], b[k + 2 * n]};
        const double uk[3] = {(double)ut[0], (double)ut[1], (double)ut[2]};
        const double bk[3] = {(double)bt[0], (double)bt[1], (double)bt[2]};
        acc[0] += rho;
        bool bad = !isfinite(rho);
#pragma unroll
        for (int a = 0; a < 3; ++a) bad = bad || !isfinite(uk[a]) || !isfinite(bk[a]);
        if (bad) acc[10] += 1.0;
        bool inside;
        if (c.geometry == 2)
            inside = true;
        else if (c.geometry == 0)
            inside = fabs((double)y - c.cy) <= c.rin;
        else
            inside = sqrt(((double)x - c.cx) * ((double)x - c.cx) + ((double)y - c.cy) * ((double)y - c.cy)) <= c.rin;
        if (!inside) continue;
        acc[9] += 1.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double du = uk[a] - (double)usnap[k + a * n];
            acc[7] += du * du;
            acc[8] += uk[a] * uk[a];
        }
        T Be_t[3];
        bext_at(c.bext_z, c.be, z, Be_t);
        bext_add_xy(c.bext_xy, nx * ny, y * nx + x, Be_t);
        const double Be[3] = {(double)Be_t[0], (double)Be_t[1], (double)Be_t[2]};
        const double B[3] = {Be[0] + bk[0], Be[1] + bk[1], Be[2] + bk[2]};
        acc[1] += 0.5 * rho * (uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
        acc[2] += 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        acc[3] += c.fb * uk[c.axis];
        // flow-lattice Laplacian of u and isotropic gradient of b
        L lap[3] = {L(0), L(0), L(0)};
        L db[3][3] = {{L(0), L(0), L(0)}, {L(0), L(0), L(0)}, {L(0), L(0), L(0)}};
#pragma unroll
        for (int j = 1; j < Q; ++j) {
            int cx, cy, cz;
            flow_dir<Q>(j, cx, cy, cz);
            const int q = (wrapi(z + cz, nz) * ny + wrapi(y + cy, ny)) * nx + wrapi(x + cx, nx);
            const L w = (L)flow_w<Q>(j);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lap[a] += w * ((L)u[q + a * n] - (L)ut[a]);
                const L bq = (L)b[q + a * n];
                db[0][a] += L(3) * w * L(cx) * bq;
                db[1][a] += L(3) * w * L(cy) * bq;
                db[2][a] += L(3) * w * L(cz) * bq;
            }
        }
        double ulap = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) ulap += uk[a] * 6.0 * (double)lap[a];
        acc[4] += ulap;
        const double J[3] = {(double)db[1][2] - (double)db[2][1], (double)db[2][0] - (double)db[0][2],
                             (double)db[0][1] - (double)db[1][0]};
        const double Lf[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
        acc[5] += -(uk[0] * Lf[0] + uk[1] * Lf[1] + uk[2] * Lf[2]);
        // QS residual with the field lattice's operators
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            L lapb = L(0), div = L(0);
#pragma unroll
            for (int be = 0; be < DIM; ++be) {
                const int ex = be == 0, ey = be == 1, ez = be == 2;
                const int zpp = wrapi(z + ez, nz), zmm = wrapi(z - ez, nz);
                const int kp = (zpp * ny + wrapi(y + ey, ny)) * nx + wrapi(x + ex, nx);
                const int km = (zmm * ny + wrapi(y - ey, ny)) * nx + wrapi(x - ex, nx);
                lapb += (L)b[kp + a * n] + (L)b[km + a * n] - L(2) * (L)bt[a];
                T Bep_t[3], Bem_t[3];
                bext_at(c.bext_z, c.be, zpp, Bep_t);
                bext_at(c.bext_z, c.be, zmm, Bem_t);
                bext_add_xy(c.bext_xy, nx * ny, kp - zpp * nx * ny, Bep_t);
                bext_add_xy(c.bext_xy, nx * ny, km - zmm * nx * ny, Bem_t);
                L Bp[3], Bm[3];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    Bp[cc] = (L)Bep_t[cc] + (c.strict_qs ? L(0) : (L)b[kp + cc * n]);
                    Bm[cc] = (L)Bem_t[cc] + (c.strict_qs ? L(0) : (L)b[km + cc * n]);
                }
                const L phip = (L)u[kp + be * n] * Bp[a] - (L)u[kp + a * n] * Bp[be];
                const L phim = (L)u[km + be * n] * Bm[a] - (L)u[km + a * n] * Bm[be];
                div += L(0.5) * (phip - phim);
            }
            const double r = c.eta * (double)lapb - (double)div;
            acc[6] += r * r;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kObs; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kObs) {
        double v = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) v += red[threadIdx.x][w];
        partial[(long long)blockIdx.x * kObs + threadIdx.x] = v;
    }
}

template <typename T>
__global__ void k_fold(const double* partial, int nblocks, double* out) {
    // one warp per slot, fixed order within each lane, fixed shuffle tree
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (i >= kObs) return;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += partial[(long long)b * kObs + i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[i] = v;
}

}  // namespace qslbm
