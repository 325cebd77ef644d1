// Resident magnetic sub-iteration: one launch runs all N_mag sweeps (Sec. V.G)
// with the IB corrector on b after each (Sec. V.D, V.F), for domains whose z
// planes fit one per CTA with every CTA co-resident (cooperative launch).
//
// Each CTA keeps its plane's b and u in shared memory for the whole launch.
// Per sweep it needs only the two neighbouring planes' b from the previous
// sweep; those travel through a double-buffered exchange array in global
// memory.  A CTA publishes its plane by bumping a per-plane counter with a
// release store after writing it, and waits (acquire loads, bounded by a
// one-second timeout that raises an error flag instead of hanging) for its two
// neighbours' counters before reading their planes.  Plane-local IB (markers on
// integer z) runs entirely in shared memory.
#pragma once

#include "qslbm_kernels.cuh"

namespace qslbm {

// Launch shape: a thread holds its NPT nodes' new values in registers until
// the whole plane has been read.  Planes of up to 4096 nodes (SMALL) take
// 1024 threads x 4 nodes in both precisions (64 registers a thread; the most
// warps to hide each sweep's latencies); larger planes, up to 8192 nodes, take
// 512 x 16 in FP32 and 1024 x 8 in FP64.
template <typename T, bool SMALL>
struct ResidentShape {
    static constexpr int threads = (sizeof(T) == 4 && !SMALL) ? 512 : 1024;
    static constexpr int npt = SMALL ? 4 : (sizeof(T) == 4 ? 16 : 8);
};
constexpr int kResidentSmallPlane = 4096;
constexpr int kResidentMaxPlane = 8192;
constexpr unsigned long long kWaitTimeoutNs = 1000000000ULL;

// Counters in device memory: flags[z] counts the planes CTA z has published;
// epoch is the count at the start of the current launch.
struct ResidentSync {
    unsigned int epoch;
    unsigned int done;
    int err;   // 1: a wait timed out
    int pad;
    unsigned int flags[1];  // [nz]
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (one thread) until the counters *fa and *fb reach target, comparing
// modulo 2^32.  Gives up after timeout_ns of the GPU's global timer and
// returns false, so that no wait outlasts its limit.
__device__ __forceinline__ bool wait_counters(const unsigned int* fa, const unsigned int* fb, unsigned int target,
                                              unsigned long long timeout_ns) {
    const unsigned long long t0 = globaltimer_ns();
    while ((int)(ld_acquire_u32(fa) - target) < 0 || (int)(ld_acquire_u32(fb) - target) < 0) {
        if (globaltimer_ns() - t0 > timeout_ns) return false;
        __nanosleep(16);
    }
    return true;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
    return __ldcg(p);
}

// Two adjacent values (8-byte float2 or 16-byte double2 accesses).
template <typename T>
struct Two;
template <>
struct Two<float> {
    using V = float2;
};
template <>
struct Two<double> {
    using V = double2;
};
template <typename T>
__device__ __forceinline__ typename Two<T>::V ld2(const T* p) {
    return *reinterpret_cast<const typename Two<T>::V*>(p);
}
template <typename T>
__device__ __forceinline__ typename Two<T>::V ldcg2(const T* p) {
    return __ldcg(reinterpret_cast<const typename Two<T>::V*>(p));
}
template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
    typename Two<T>::V v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<typename Two<T>::V*>(p) = v;
}
template <typename T>
__device__ __forceinline__ void stcg2(T* p, T a, T b) {
    typename Two<T>::V v;
    v.x = a;
    v.y = b;
    __stcg(reinterpret_cast<typename Two<T>::V*>(p), v);
}

// Shared-memory copy of one plane's IB tables (ring markers and shell CSR).
template <typename T>
struct LocalIB {
    int R, S;               // markers in the ring, shell nodes of the plane
    const int* q;           // [9 R] in-plane support indices
    const T* w;             // [9 R] weights
    const T* sc;            // [R] scaling s^m_j
    const int* shell;       // [S] in-plane index of each shell node
    const int* off;         // [S + 1] CSR offsets (local)
    const int* cm;          // CSR marker (local to the ring)
    const T* cw;            // CSR weight
};

// Explicit IB corrector on a plane held in shared memory (Sec. V.D, V.F):
// delta_j = s_j (0 - D f*) for every marker first, then f += D^T delta.
// With pub set, each corrected shell value is also written to pub (three
// components P apart), by the thread that corrected it.
template <typename T, int THREADS>
__device__ __forceinline__ void ib_local(const LocalIB<T>& t, T* f0, T* f1, T* f2, T* sdelta, T* pub, int P) {
    if (t.R == 0) return;
    __syncthreads();
    for (int m = threadIdx.x; m < t.R; m += THREADS) {
        T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const T w = t.w[9 * m + j];
            const int q = t.q[9 * m + j];
            a0 += w * f0[q];
            a1 += w * f1[q];
            a2 += w * f2[q];
        }
        const T sm = t.sc[m];
        sdelta[3 * m + 0] = -sm * a0;
        sdelta[3 * m + 1] = -sm * a1;
        sdelta[3 * m + 2] = -sm * a2;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < t.S; i += THREADS) {
        T c0 = T(0), c1 = T(0), c2 = T(0);
        for (int e = t.off[i]; e < t.off[i + 1]; ++e) {
            const T w = t.cw[e];
            const int l = t.cm[e];
            c0 += w * sdelta[3 * l + 0];
            c1 += w * sdelta[3 * l + 1];
            c2 += w * sdelta[3 * l + 2];
        }
        const int q = t.shell[i];
        const T v0 = f0[q] + c0, v1 = f1[q] + c1, v2 = f2[q] + c2;
        f0[q] = v0;
        f1[q] = v1;
        f2[q] = v2;
        if (pub) {
            __stcg(pub + q, v0);
            __stcg(pub + P + q, v1);
            __stcg(pub + 2 * P + q, v2);
        }
    }
}

// Bytes of shared memory the resident kernel needs (the host uses the same
// function to plan the launch).
template <typename T>
__host__ __device__ inline size_t resident_smem_bytes(int P, bool uhalo, int max_ring, int max_shell, int max_nnz) {
    size_t nT = (size_t)6 * P + (uhalo ? (size_t)6 * P : 0) + (size_t)3 * max_ring + (size_t)9 * max_ring +
                (size_t)max_ring + (size_t)max_nnz;
    size_t nI = (size_t)9 * max_ring + (size_t)max_shell + (size_t)max_shell + 1 + (size_t)max_nnz;
    return nT * sizeof(T) + nI * sizeof(int);
}

// PAIR: each thread takes x-adjacent node pairs (nx even), so that own-row,
// y-neighbour and z-neighbour values move two at a time.
template <typename T, int DIM, bool UHALO, int kResidentThreads, int kResidentMaxNpt, bool PAIR>
__global__ void __launch_bounds__(kResidentThreads, 1)
    k_sweeps_resident(Geo g, const T* __restrict__ b_in, T* __restrict__ b_out, const T* __restrict__ u,
                      SweepCoef<T> c, IBView<T> ib, T* xbuf, ResidentSync* sync, int nsweeps, int max_ring,
                      int max_shell, int max_nnz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned int s_epoch;
    __shared__ int s_abort;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int P = nx * ny;
    const long long n = g.n;
    const int z = blockIdx.x;
    const int zm = DIM == 3 ? wrap_dec(z, nz) : z, zp = DIM == 3 ? wrap_inc(z, nz) : z;
    // shared memory: values of type T first, then int tables
    T* sb = reinterpret_cast<T*>(smem_raw);   // [3][P] own b
    T* su = sb + 3 * P;                       // [3][P] own u
    T* suh = su + 3 * P;                      // [2][3][P] u of planes zm, zp (UHALO)
    T* sdelta = UHALO ? suh + 6 * P : suh;    // [3 R]
    T* tw = sdelta + 3 * max_ring;            // [9 R]
    T* tsc = tw + 9 * max_ring;               // [R]
    T* tcw = tsc + max_ring;                  // [E]
    int* tq = reinterpret_cast<int*>(tcw + max_nnz);  // [9 R]
    int* tshell = tq + 9 * max_ring;          // [S]
    int* toff = tshell + max_shell;           // [S + 1]
    int* tcm = toff + max_shell + 1;          // [E]
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_epoch = *(volatile unsigned int*)&sync->epoch;
        s_abort = 0;
    }
    const long long base = (long long)z * P;
    for (int p = tid; p < P; p += kResidentThreads) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sb[a * P + p] = b_in[a * n + base + p];
            su[a * P + p] = u[a * n + base + p];
            if (UHALO) {
                suh[a * P + p] = u[a * n + (long long)zm * P + p];
                suh[(3 + a) * P + p] = u[a * n + (long long)zp * P + p];
            }
        }
    }
    LocalIB<T> lib;
    {
        const int tz = ib.zinv ? 0 : z;
        const int m0 = ib.ring_off[tz];
        lib.R = ib.ring_off[tz + 1] - m0;
        const int s0 = ib.shell_off[tz];
        lib.S = ib.shell_off[tz + 1] - s0;
        const int e0 = lib.S > 0 ? ib.csr_off[s0] : 0;
        const int E = lib.S > 0 ? ib.csr_off[s0 + lib.S] - e0 : 0;
        for (int i = tid; i < 9 * lib.R; i += kResidentThreads) {
            tq[i] = ib.mk_q[9 * m0 + i];
            tw[i] = ib.mk_w[9 * m0 + i];
        }
        for (int i = tid; i < lib.R; i += kResidentThreads) tsc[i] = ib.mk_s[m0 + i];
        for (int i = tid; i < lib.S; i += kResidentThreads) tshell[i] = ib.shell_xy[s0 + i];
        for (int i = tid; i <= lib.S; i += kResidentThreads) toff[i] = ib.csr_off[s0 + i] - e0;
        for (int i = tid; i < E; i += kResidentThreads) {
            tcm[i] = ib.csr_m[e0 + i];
            tcw[i] = ib.csr_w[e0 + i];
        }
        lib.q = tq;
        lib.w = tw;
        lib.sc = tsc;
        lib.shell = tshell;
        lib.off = toff;
        lib.cm = tcm;
        lib.cw = tcw;
    }
    T be_c[3], be_m[3], be_p[3];
    bext_at(c.bext_z, c.be, z, be_c);
    bext_at(c.bext_z, c.be, zm, be_m);
    bext_at(c.bext_z, c.be, zp, be_p);
    __syncthreads();
    const unsigned int epoch = s_epoch;
    const long long xplane = 3LL * P;
    for (int s = 0; s < nsweeps; ++s) {
        const bool publish = DIM == 3 && s + 1 < nsweeps;
        T* xout = xbuf + (long long)(s & 1) * nz * xplane + (long long)z * xplane;
        if constexpr (PAIR) {
        constexpr int NPAIR = kResidentMaxNpt / 2;
        // (1) in-plane part, pairs (x, x + 1) with x even
        T nv[NPAIR][2][3];
#pragma unroll
        for (int k = 0; k < NPAIR; ++k) {
            const int p0 = 2 * (tid + k * kResidentThreads);
            if (p0 < P) {
                const int y = p0 / nx;
                const int x0 = p0 - y * nx;
                const int rc = y * nx, rm = wrap_dec(y, ny) * nx, rp = wrap_inc(y, ny) * nx;
                const int xl = wrap_dec(x0, nx), xr = x0 + 2 == nx ? 0 : x0 + 2;
                T bC[2][3], bN[2][4][3], uN[2][4][3];  // own b; neighbours -x, +x, -y, +y
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const auto cb = ld2(sb + a * P + rc + x0), cu = ld2(su + a * P + rc + x0);
                    const auto mb = ld2(sb + a * P + rm + x0), mu = ld2(su + a * P + rm + x0);
                    const auto pb = ld2(sb + a * P + rp + x0), pu = ld2(su + a * P + rp + x0);
                    const T lb = sb[a * P + rc + xl], lu = su[a * P + rc + xl];
                    const T rb = sb[a * P + rc + xr], ru = su[a * P + rc + xr];
                    bC[0][a] = cb.x;
                    bC[1][a] = cb.y;
                    bN[0][0][a] = lb;   uN[0][0][a] = lu;
                    bN[0][1][a] = cb.y; uN[0][1][a] = cu.y;
                    bN[0][2][a] = mb.x; uN[0][2][a] = mu.x;
                    bN[0][3][a] = pb.x; uN[0][3][a] = pu.x;
                    bN[1][0][a] = cb.x; uN[1][0][a] = cu.x;
                    bN[1][1][a] = rb;   uN[1][1][a] = ru;
                    bN[1][2][a] = mb.y; uN[1][2][a] = mu.y;
                    bN[1][3][a] = pb.y; uN[1][3][a] = pu.y;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    T acc[3], dif[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        acc[a] = c.w0 * bC[h][a];
                        dif[a] = T(0);
                    }
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        T B[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            acc[a] += c.w1 * bN[h][d][a];
                            B[a] = be_c[a] + c.sq * bN[h][d][a];
                        }
                        flux_acc(uN[h][d], B, d >> 1, (d & 1) ? T(-1) : T(1), dif);
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a) nv[k][h][a] = acc[a] + c.w1 * c.kappa * dif[a];
                }
            }
        }
        // (2) neighbour planes of the previous sweep
        if (DIM == 3 && s > 0) {
            if (tid == 0 &&
                !wait_counters(&sync->flags[zm], &sync->flags[zp], epoch + (unsigned int)s, kWaitTimeoutNs)) {
                atomicExch(&sync->err, 1);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
        }
        // (3) the z terms, two nodes at a time.  All neighbour-plane loads of
        // the thread are issued before any is used: one L2 round trip per sweep.
        if constexpr (DIM == 3) {
            const T* xin = xbuf + (long long)((s - 1) & 1) * nz * xplane;
            const T* zsrc[2];
            long long cs;  // stride between components
            if (s == 0) {
                zsrc[0] = b_in + (long long)zm * P;
                zsrc[1] = b_in + (long long)zp * P;
                cs = n;
            } else {
                zsrc[0] = xin + (long long)zm * xplane;
                zsrc[1] = xin + (long long)zp * xplane;
                cs = P;
            }
            // groups of up to 4 pairs (FP32; one pair in FP64, whose 1024-thread
            // CTAs have half the registers) bound the registers holding loads in flight
            constexpr int G = sizeof(T) == 8 ? 1 : (NPAIR < 4 ? NPAIR : 4);
#pragma unroll
            for (int g0 = 0; g0 < NPAIR; g0 += G) {
                typename Two<T>::V zb[G][2][3];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int p0 = 2 * (tid + (g0 + j) * kResidentThreads);
                    if (p0 < P) {
#pragma unroll
                        for (int d = 0; d < 2; ++d)
#pragma unroll
                            for (int a = 0; a < 3; ++a) zb[j][d][a] = ldcg2(zsrc[d] + a * cs + p0);
                    }
                }
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int k = g0 + j;
                    const int p0 = 2 * (tid + k * kResidentThreads);
                    if (p0 < P) {
#pragma unroll
                        for (int d = 0; d < 2; ++d) {
                            const int zn = d == 0 ? zm : zp;
                            const T* bez = d == 0 ? be_m : be_p;
                            T bq[2][3], uq[2][3];
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                const auto vu = UHALO ? ld2(suh + (3 * d + a) * P + p0)
                                                      : ld2(u + a * n + (long long)zn * P + p0);
                                bq[0][a] = zb[j][d][a].x;
                                bq[1][a] = zb[j][d][a].y;
                                uq[0][a] = vu.x;
                                uq[1][a] = vu.y;
                            }
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                T B[3];
#pragma unroll
                                for (int a = 0; a < 3; ++a) B[a] = bez[a] + c.sq * bq[h][a];
                                T phz[3] = {T(0), T(0), T(0)};
                                flux_acc(uq[h], B, 2, d == 1 ? -c.w1 * c.kappa : c.w1 * c.kappa, phz);
#pragma unroll
                                for (int a = 0; a < 3; ++a) nv[k][h][a] += c.w1 * bq[h][a] + phz[a];
                            }
                        }
                    }
                }
            }
        }
        // every read of the old plane is done (after a wait, its barrier did that)
        if (!(DIM == 3 && s > 0)) __syncthreads();
#pragma unroll
        for (int k = 0; k < NPAIR; ++k) {
            const int p0 = 2 * (tid + k * kResidentThreads);
            if (p0 < P) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    st2(sb + a * P + p0, nv[k][0][a], nv[k][1][a]);
                    if (publish) stcg2(xout + a * P + p0, nv[k][0][a], nv[k][1][a]);
                }
            }
        }
        } else {
        // (1) in-plane part of the sweep from this CTA's own plane; it overlaps
        // the neighbours' publication of the previous sweep
        T nv[kResidentMaxNpt][3];
#pragma unroll
        for (int k = 0; k < kResidentMaxNpt; ++k) {
            const int p = tid + k * kResidentThreads;
            if (p < P) {
                const int y = p / nx;
                const int x = p - y * nx;
                const int qn[4] = {y * nx + wrap_dec(x, nx), y * nx + wrap_inc(x, nx),
                                   wrap_dec(y, ny) * nx + x, wrap_inc(y, ny) * nx + x};
                T acc[3], dif[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc[a] = c.w0 * sb[a * P + p];
                    dif[a] = T(0);
                }
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    const int q = qn[d];
                    T uq[3], B[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const T bq = sb[a * P + q];
                        uq[a] = su[a * P + q];
                        acc[a] += c.w1 * bq;
                        B[a] = be_c[a] + c.sq * bq;
                    }
                    flux_acc(uq, B, d >> 1, (d & 1) ? T(-1) : T(1), dif);
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) nv[k][a] = acc[a] + c.w1 * c.kappa * dif[a];
            }
        }
        // (2) neighbour planes of the previous sweep
        if (DIM == 3 && s > 0) {
            if (tid == 0 &&
                !wait_counters(&sync->flags[zm], &sync->flags[zp], epoch + (unsigned int)s, kWaitTimeoutNs)) {
                atomicExch(&sync->err, 1);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
        }
        // (3) the z terms: w1 b(z -/+ 1) and w1 kappa (+/-) Phi_az(z -/+ 1)
        const T* xin = xbuf + (long long)((s - 1) & 1) * nz * xplane;
#pragma unroll
        for (int k = 0; k < kResidentMaxNpt; ++k) {
            const int p = tid + k * kResidentThreads;
            if (p < P) {
                if (DIM == 3) {
#pragma unroll
                    for (int d = 4; d < 6; ++d) {
                        const int zn = d == 4 ? zm : zp;
                        const T* bez = d == 4 ? be_m : be_p;
                        T uq[3], B[3], bq[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            bq[a] = s == 0 ? b_in[a * n + (long long)zn * P + p]
                                           : ldcg(xin + (long long)zn * xplane + (long long)a * P + p);
                            uq[a] = UHALO ? suh[((d == 4 ? 0 : 3) + a) * P + p] : u[a * n + (long long)zn * P + p];
                            B[a] = bez[a] + c.sq * bq[a];
                        }
                        T phz[3] = {T(0), T(0), T(0)};
                        flux_acc(uq, B, 2, d == 5 ? -c.w1 * c.kappa : c.w1 * c.kappa, phz);
#pragma unroll
                        for (int a = 0; a < 3; ++a) nv[k][a] += c.w1 * bq[a] + phz[a];
                    }
                }
            }
        }
        // every read of the old plane is done (after a wait, its barrier did that)
        if (!(DIM == 3 && s > 0)) __syncthreads();
#pragma unroll
        for (int k = 0; k < kResidentMaxNpt; ++k) {
            const int p = tid + k * kResidentThreads;
            if (p < P) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sb[a * P + p] = nv[k][a];
                    // nodes off the wall shell are final now; shell nodes are
                    // rewritten after the IB correction below
                    if (publish) __stcg(xout + a * P + p, nv[k][a]);
                }
            }
        }
        }
        ib_local<T, kResidentThreads>(lib, sb, sb + P, sb + 2 * P, sdelta, publish ? xout : nullptr, P);
        __syncthreads();  // the plane is final in shared memory and in xout
        if (publish && tid == 0) {
            __threadfence();
            st_release_u32(&sync->flags[z], epoch + (unsigned int)s + 1u);
        }
    }
    for (int p = tid; p < P; p += kResidentThreads) {
#pragma unroll
        for (int a = 0; a < 3; ++a) b_out[a * n + base + p] = sb[a * P + p];
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&sync->done, 1u);
        if (prev == gridDim.x - 1) {
            sync->done = 0;
            sync->epoch = epoch + (unsigned int)nsweeps;
            __threadfence();
        }
    }
}

}  // namespace qslbm
