// Resident sub-iteration for a batch of small instances (FP32): one
// cooperative launch per flow step runs all N_mag sweeps (Sec. V.G) with the
// IB on b after each (Sec. V.D, V.F) for every instance whose planes are
// small, each CTA holding a group of consecutive z planes of one instance in
// shared memory for the whole launch.
//
// A group is G planes of an instance (G P <= kGroupMaxNodes nodes).  Per
// sweep the CTA forms every node's (e1, e2, e3) (the EMF form of
// k_sweep_march_pair; u is read from L2, it does not change during the
// sweeps), writes the new b of its nodes into the second of two b buffers
// (z neighbours inside the group from shared memory, those across its ends
// from the neighbouring groups' end planes of the previous sweep), applies
// the plane-local IB to each of its planes, and publishes its first and last
// planes to a double-buffered exchange array in global memory with a release
// store of its counter.  A group waits (acquire loads, bounded by one second
// of the GPU's global timer, after which it raises an error flag and ends the
// sweeps early) for its two neighbours' counters before reading their planes.
// All groups of one instance do the same number of sweeps, so the counters of
// an instance stay equal between launches.  The arithmetic is that of the
// split path (march_tile's EMF form, the staged IB's sums in the same order).
#pragma once

#include "qslbm_kernels.cuh"
#include "qslbm_resident.cuh"

namespace qslbm {

constexpr int kGroupThreads = 1024;
constexpr int kGroupNpt = 5;                                  // nodes per thread, at most
constexpr int kGroupMaxNodes = kGroupThreads * kGroupNpt;     // nodes a CTA holds, at most
// Shared-memory stride of one field component (nodes): a compile-time
// constant, so that the components of a node are one base address apart by
// immediate offsets.
constexpr int kGS = kGroupMaxNodes;

// One CTA's group: planes z0 .. z0 + G - 1 of instance inst; prev / next: the
// groups holding planes z0 - 1 and z0 + G (periodic; possibly itself); xoff:
// its exchange area, [2 parities][first, last][3][P] floats.
struct GroupDesc {
    int inst, z0, G, prev, next;
    long long xoff;
};

// Shared memory of one group (bytes): two buffers of b and one of e (kGS
// nodes each), B^ext of its G planes and their two neighbours, the IB tables
// of one ring (R markers, S shell nodes, E list entries) and the deltas of
// its G rings.  A launch gives every CTA the largest group's size.
inline size_t group_smem_bytes(int R, int S, int E, int G) {
    const size_t f = (size_t)9 * kGS + (size_t)3 * (G + 2) + (size_t)10 * R + E + (size_t)3 * G * R;
    const size_t i = (size_t)9 * R + S + (S + 1) + E;
    return f * sizeof(float) + i * sizeof(int) + 16;
}

// t / d for t d < 2^32 as a high multiply, m = group_magic(d) (exact in that
// range: m d - 2^32 < d).
__host__ __device__ inline unsigned group_magic(unsigned d) { return d > 1 ? 0xFFFFFFFFu / d + 1u : 0u; }
__device__ __forceinline__ int group_div(int t, int d, unsigned m) {
    return d > 1 ? (int)__umulhi((unsigned)t, m) : t;
}

// XY: some instance has an in-plane applied field (QSLBM_B0_FIELD).
template <typename Desc, bool XY>
__global__ void __launch_bounds__(kGroupThreads, 1)
    k_batch_resident(const Desc* __restrict__ d, const GroupDesc* __restrict__ groups, float* xbuf, unsigned* flags,
                     int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned int s_base;
    __shared__ int s_abort;
    __shared__ float s_w[4];  // w0, w1, w1 kappa, sq
    const GroupDesc gd = groups[blockIdx.x];
    const Desc& D = d[gd.inst];
    const int nmag = D.n_mag;
    if (nmag == 0) return;  // uniform: b keeps its parity
    const int nx = D.g.nx, ny = D.g.ny, nz = D.g.nz;
    const int P = nx * ny, n = (int)D.g.n;
    const int G = gd.G, z0 = gd.z0, GN = G * P;
    const unsigned mP = group_magic(P), mX = group_magic(nx);
    const bool whole = G == nz;  // the group holds every plane: no exchange
    const int tid = threadIdx.x;
    // the ring and shell of plane 0, which every plane carries (z-invariant tables)
    const int m0 = D.ibm.ring_off[0], R = D.ibm.ring_off[1] - m0;
    const int s0 = D.ibm.shell_off[0], S = D.ibm.shell_off[1] - s0;
    const int e0 = S > 0 ? D.ibm.csr_off[s0] : 0;
    const int E = S > 0 ? D.ibm.csr_off[s0 + S] - e0 : 0;
    const int zm = z0 == 0 ? nz - 1 : z0 - 1;  // plane below the group
    const int zp = z0 + G == nz ? 0 : z0 + G;  // plane above it
    // shared memory: b [2][3][kGS] (sweep s reads b[s % 2], writes b[(s + 1) % 2]),
    // e [3][kGS], B^ext [G + 2][3], tables, deltas
    float* sb0 = reinterpret_cast<float*>(smem_raw);
    float* se = sb0 + 6 * kGS;
    float* sbz = se + 3 * kGS;           // B^ext of planes zm, z0 .. z0 + G - 1, zp
    float* tw = sbz + 3 * (G + 2);      // [9 R] weights D(x_k - X_j)
    float* tsc = tw + 9 * R;            // [R]   s^m_j
    float* tcw = tsc + R;               // [E]   list weights
    float* sdelta = tcw + E;            // [G][R][3]
    int* tq = reinterpret_cast<int*>(sdelta + 3 * G * R);  // [9 R] support (in-plane index)
    int* tshell = tq + 9 * R;           // [S] shell nodes (in-plane index)
    int* toff = tshell + S;             // [S + 1] list offsets
    int* tcm = toff + S + 1;            // [E] markers (ring-relative)
    {
        const SweepCoef<float>& c = D.sc;
        if (tid == 0) {
            s_base = *(volatile unsigned int*)&flags[blockIdx.x];
            s_abort = 0;
            s_w[0] = c.w0;
            s_w[1] = c.w1;
            s_w[2] = c.w1 * c.kappa;
            s_w[3] = c.sq;
        }
        if (tid < G + 2) {
            const int zz = tid == 0 ? zm : (tid == G + 1 ? zp : z0 + tid - 1);
            float be[3];
            bext_at(c.bext_z, c.be, zz, be);
            sbz[3 * tid + 0] = be[0];
            sbz[3 * tid + 1] = be[1];
            sbz[3 * tid + 2] = be[2];
        }
    }
    for (int i = tid; i < 9 * R; i += kGroupThreads) {
        tq[i] = D.ibm.mk_q[9 * m0 + i];
        tw[i] = D.ibm.mk_w[9 * m0 + i];
    }
    for (int i = tid; i < R; i += kGroupThreads) tsc[i] = D.ibm.mk_s[m0 + i];
    for (int i = tid; i < S; i += kGroupThreads) tshell[i] = D.ibm.shell_xy[s0 + i];
    for (int i = tid; i <= S; i += kGroupThreads) toff[i] = D.ibm.csr_off[s0 + i] - e0;
    for (int i = tid; i < E; i += kGroupThreads) {
        tcm[i] = D.ibm.csr_m[e0 + i];
        tcw[i] = D.ibm.csr_w[e0 + i];
    }
    {
        const float* __restrict__ bin = D.b[D.bpar];
        for (int i = tid; i < GN; i += kGroupThreads)
#pragma unroll
            for (int a = 0; a < 3; ++a) sb0[a * kGS + i] = bin[a * n + z0 * P + i];
    }
    __syncthreads();
    const unsigned int base = s_base;
    const int xs = 2 * 3 * P;  // floats per parity of an exchange area
    const unsigned long long xown = gd.xoff;
    const unsigned long long xprev = groups[gd.prev].xoff + 3 * P;  // its last plane
    const unsigned long long xnext = groups[gd.next].xoff;          // its first plane
    const float* bxy = XY ? D.sc.bext_xy : nullptr;

    int s = 0;  // sweeps done
    for (; s < nmag; ++s) {
        const float* __restrict__ u = D.u[D.fpar];
        const float* sb = sb0 + (s & 1) * 3 * kGS;      // b after sweep s - 1
        float* sn = sb0 + ((s + 1) & 1) * 3 * kGS;      // b after sweep s
        // (a) every node's e from its b (shared memory) and u (L2); the loads
        // of u are issued kGroupNpt / 2 nodes at a time before their first use
#pragma unroll 1
        for (int k0 = 0; k0 < kGroupNpt; k0 += kGroupNpt / 2) {
            if (tid + k0 * kGroupThreads >= GN) break;
            float ur[kGroupNpt / 2][3];
#pragma unroll
            for (int k = 0; k < kGroupNpt / 2; ++k) {
                const int i = tid + (k0 + k) * kGroupThreads;
                if (i < GN) {
                    const int q = z0 * P + i;
                    ur[k][0] = __ldg(u + q);
                    ur[k][1] = __ldg(u + n + q);
                    ur[k][2] = __ldg(u + 2 * n + q);
                }
            }
            const float sq = s_w[3];
#pragma unroll
            for (int k = 0; k < kGroupNpt / 2; ++k) {
                const int i = tid + (k0 + k) * kGroupThreads;
                if (i < GN) {
                    const int g = group_div(i, P, mP);
                    float be[3] = {sbz[3 * g + 3], sbz[3 * g + 4], sbz[3 * g + 5]};
                    if constexpr (XY) bext_add_xy(bxy, P, i - g * P, be);
                    float r[6] = {sb[i], sb[kGS + i], sb[2 * kGS + i], ur[k][0], ur[k][1], ur[k][2]};
                    node_emf(r, be, sq);
                    se[i] = r[3];
                    se[kGS + i] = r[4];
                    se[2 * kGS + i] = r[5];
                }
            }
        }
        // the neighbours' end planes of sweep s - 1
        if (!whole && s > 0 && tid == 0 &&
            !wait_counters(&flags[gd.prev], &flags[gd.next], base + (unsigned int)s, kWaitTimeoutNs)) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;  // uniform: read by every thread after the barrier
        // (b) the new b of this thread's nodes into the other buffer
        // (march_tile's expressions in its order)
        {
            const float* __restrict__ bin = D.b[D.bpar];
            const float* xp = xbuf + xprev + (size_t)((s + 1) & 1) * xs;  // parity written at sweep s - 1
            const float* xq = xbuf + xnext + (size_t)((s + 1) & 1) * xs;
            const float w0 = s_w[0], w1 = s_w[1], w1k = s_w[2];
            // (b, u) of node p of the plane zz next to the group (table row t) -> (b, e)
            auto halo = [&](const float* src, int stride, int zz, int t, int p, float r[6]) {
                float be[3] = {sbz[3 * t], sbz[3 * t + 1], sbz[3 * t + 2]};
                if constexpr (XY) bext_add_xy(bxy, P, p, be);
                r[0] = __ldcg(src + p);
                r[1] = __ldcg(src + stride + p);
                r[2] = __ldcg(src + 2 * stride + p);
                r[3] = __ldg(u + zz * P + p);
                r[4] = __ldg(u + n + zz * P + p);
                r[5] = __ldg(u + 2 * n + zz * P + p);
                node_emf(r, be, s_w[3]);
            };
            const float* E1 = se;
            const float* E2 = se + kGS;
            const float* E3 = se + 2 * kGS;
            // each thread walks whole z columns of the group: the column's
            // (b, e) at planes g - 1, g, g + 1 stay in registers
#pragma unroll 1
            for (int p = tid; p < P; p += kGroupThreads) {
                const int y = group_div(p, nx, mX), x = p - y * nx;
                const int dl = x == 0 ? nx - 1 : -1, dr = x == nx - 1 ? 1 - nx : 1;
                const int du = y == 0 ? P - nx : -nx, dd = y == ny - 1 ? nx - P : nx;
                float prv[6], cur[6], nxt[6];
                if (whole) {
                    const int j = (G - 1) * P + p;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        prv[a] = sb[a * kGS + j];
                        prv[3 + a] = se[a * kGS + j];
                    }
                } else {
                    halo(s == 0 ? bin + zm * P : xp, s == 0 ? n : P, zm, 0, p, prv);
                }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cur[a] = sb[a * kGS + p];
                    cur[3 + a] = se[a * kGS + p];
                }
#pragma unroll 1
                for (int g = 0; g < G; ++g) {
                    const int i = g * P + p;
                    if (g < G - 1 || whole) {
                        const int j = g < G - 1 ? i + P : p;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            nxt[a] = sb[a * kGS + j];
                            nxt[3 + a] = se[a * kGS + j];
                        }
                    } else {
                        halo(s == 0 ? bin + zp * P : xq, s == 0 ? n : P, zp, G + 1, p, nxt);
                    }
                    const int il = i + dl, ir = i + dr, iu = i + du, id = i + dd;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float* Ba = sb + a * kGS;
                        const float sa = (Ba[il] + Ba[ir]) + (Ba[iu] + Ba[id]) + (prv[a] + nxt[a]);
                        float da;
                        if (a == 0)
                            da = (E1[id] - E1[iu]) + (nxt[4] - prv[4]);
                        else if (a == 1)
                            da = (E1[il] - E1[ir]) + (nxt[5] - prv[5]);
                        else
                            da = (E2[il] - E2[ir]) + (E3[iu] - E3[id]);
                        sn[a * kGS + i] = emf_update(w0, w1, w1k, cur[a], sa, da);
                    }
#pragma unroll
                    for (int v = 0; v < 6; ++v) {
                        prv[v] = cur[v];
                        cur[v] = nxt[v];
                    }
                }
            }
        }
        __syncthreads();  // the new b is complete
        // (c) IB on each plane of the group: delta_j = -s^m_j D b* at every
        // marker, then b = b* + D^T delta on the shell (ib_plane's sums in its
        // order; the planes are independent)
        if (R > 0) {
            const unsigned mR = group_magic(R), mS = group_magic(S);
            for (int t = tid; t < G * R; t += kGroupThreads) {
                const int g = group_div(t, R, mR), m = t - g * R;
                const float* f = sn + g * P;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const float w = tw[9 * m + j];
                    const int q = tq[9 * m + j];
                    a0 += w * f[q];
                    a1 += w * f[kGS + q];
                    a2 += w * f[2 * kGS + q];
                }
                const float sm = tsc[m];
                sdelta[3 * t + 0] = -sm * a0;
                sdelta[3 * t + 1] = -sm * a1;
                sdelta[3 * t + 2] = -sm * a2;
            }
            __syncthreads();
            for (int t = tid; t < G * S; t += kGroupThreads) {
                const int g = group_div(t, S, mS), k = t - g * S;
                const float* dl = sdelta + 3 * g * R;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                const int ea = toff[k], eb = toff[k + 1];
                for (int e = ea; e < eb; ++e) {
                    const float w = tcw[e];
                    const int l = tcm[e];
                    c0 += w * dl[3 * l + 0];
                    c1 += w * dl[3 * l + 1];
                    c2 += w * dl[3 * l + 2];
                }
                const int q = g * P + tshell[k];
                sn[q] += c0;
                sn[kGS + q] += c1;
                sn[2 * kGS + q] += c2;
            }
            __syncthreads();
        }
        // (d) publish the first and last planes for the neighbours' sweep s + 1
        if (!whole) {
            if (s + 1 < nmag) {
                float* xo = xbuf + xown + (size_t)(s & 1) * xs;
                for (int t = tid; t < 2 * P; t += kGroupThreads) {
                    const int h = t >= P, p = t - h * P;
                    const int i = h ? (G - 1) * P + p : p;
#pragma unroll
                    for (int a = 0; a < 3; ++a) __stcg(xo + h * 3 * P + a * P + p, sn[a * kGS + i]);
                }
                __syncthreads();
            }
            if (tid == 0) {
                __threadfence();
                st_release_u32(&flags[blockIdx.x], base + (unsigned int)s + 1u);
            }
        }
    }
    // the b of the last sweep done (all of them unless a wait gave up)
    const float* sb = sb0 + (s & 1) * 3 * kGS;
    float* __restrict__ bfin = D.b[(D.bpar + nmag) & 1];
    for (int i = tid; i < GN; i += kGroupThreads)
#pragma unroll
        for (int a = 0; a < 3; ++a) bfin[a * n + z0 * P + i] = sb[a * kGS + i];
}

}  // namespace qslbm
