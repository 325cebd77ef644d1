// Fused magnetic sweep + IB corrector on b for planes too large for the
// resident kernel (FP32, 3-D, the same wall ring on every plane): one launch
// per sweep (Sec. V.G) with the explicit IB on b (Sec. V.D, V.F) applied to
// every plane inside the same launch, so that the swept field b* never goes
// back to memory before its wall correction.
//
// A CTA owns a band of TY rows of every plane of a z chunk and marches the
// chunk plane by plane.  The markers sit on integer z, so the IB couples the
// nodes of one plane only, and locally: a node's corrected value depends on
// the deltas of the markers whose support is centred within one row of it,
// and those deltas on b* within one further row.  So the CTA sweeps its rows
// and two halo rows on each side (b* of rows y0 - 2 .. y0 + TY + 1, computed
// redundantly with the neighbouring bands, bitwise alike), interpolates the
// markers centred on rows y0 - 1 .. y0 + TY, and corrects and writes its own
// rows.  It reads b and u of rows y0 - 3 .. y0 + TY + 2.  No CTA waits for
// another.  Bands have TY rows; when TY does not divide ny the last band
// starts at ny - TY and shares rows with the one before it (both compute and
// write them, bitwise alike).
//
// Shared memory holds a ring of NS = 4 or 5 plane slots.  The tensor memory
// accelerator fills a slot (cp.async.bulk.tensor, completion on an mbarrier)
// NS - 1 planes ahead: per field and component three boxes, the 3 rows above
// the band, its TY rows and the 3 rows below, each starting on a 128-byte
// boundary and taken across the periodic y boundary by its own coordinate.
// Each thread owns one node pair of the swept rows for the whole chunk: it
// turns its pair of every staged plane in place from (b, u) into (b, e) (the
// EMF form of k_sweep_march_pair) and keeps the pair's planes z - 1, z, z + 1
// in registers, so that only in-plane neighbours come from shared memory.
// Plane iteration i (plane z = z0 + i), two barriers:
//   1. sweep of the own pair of plane z into S[i % 2]; the own rows of plane
//      z - 1 (S[(i - 1) % 2]) to b_out                               | barrier
//      (the slot of plane z is free: one warp refills it with plane z + NS)
//   2. interpolate delta_j = -s_j D b* for the band's markers of plane z
//      (into D[i % 2]); at the same time the own shell nodes of plane z - 1
//      take sum_j D delta_j (from D[(i - 1) % 2] and S[(i - 1) % 2]) and
//      replace their swept values in b_out; convert the own pair of plane
//      z + 2                                                         | barrier
// The arithmetic is that of k_sweep_march_pair (explicit fused multiply-adds)
// and of k_ib_staged (the same sums in the same order), so the results are
// bitwise those of the split path.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "qslbm_kernels.cuh"

namespace qslbm {

constexpr unsigned long long kFusedWaitNs = 1000000000ULL;  // bounded copy wait: 1 s

// Per-band IB tables (z-invariant).  Offsets are row * nx + x in the band's
// swept rows (row 0 = y0 - 2).
struct FusedIB {
    const int* mk_cnt;   // [bands] markers centred on rows y0 - 1 .. y0 + TY
    const int* mk_off;   // [bands][Mmax][9] support nodes
    const float* mk_w;   // [bands][Mmax][9] D(x_k - X_j) = D_x D_y
    const float* mk_s;   // [bands][Mmax]    s^m_j
    const int* sh_cnt;   // [bands] shell nodes in the band's own rows
    const int* sh_off;   // [bands][Smax]
    const int* sh_m;     // [bands][Smax][K] marker index in the band's list (padding: 0)
    const float* sh_w;   // [bands][Smax][K] weight (padding: 0)
    const int* sh_cnt_e; // [bands][Smax] entries of each list before the padding
    int Mmax, Smax, K;   // K a multiple of 4
};

struct FusedGeo {
    int nx, ny, nz;
    int TY;      // rows per band
    int chunk;   // z planes per CTA
    int n;       // nx ny nz
    int slots;   // plane slots in the ring (4 or 5)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the mbarrier to complete; gives up after
// kFusedWaitNs of the GPU's global timer and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > kFusedWaitNs) return false;
    }
}

// A box of the 4-D (x, y, z, component) tensor map starting at row y of
// plane z, component cc: (nx, 3, 1, 1) or (nx, TY, 1, 1); it lands as
// [row][x].
__device__ __forceinline__ void tma_box(const CUtensorMap* map, float* dst, int y, int z, int cc,
                                        unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(y), "r"(z), "r"(cc), "r"(smem_u32(bar))
        : "memory");
}

// Slot layout (floats): [field][component] areas of CA floats; within an
// area the 3 rows above the band at 0, its TY rows at P1, the 3 rows below at
// P2 (P1, P2 and CA multiples of 32 floats, so that every box lands on a
// 128-byte boundary).  Staged row r (0 .. TY + 5) of a component sits at
// row_off(r).
struct SlotLayout {
    int nx, TY, P1, P2, CA;
    __device__ __forceinline__ int row_off(int r) const {
        return r < 3 ? r * nx : (r < TY + 3 ? P1 + (r - 3) * nx : P2 + (r - TY - 3) * nx);
    }
};

// Issue the copies of plane zz into `slot`: for b and u and each component the
// rows above (from yA), the band (from y0) and the rows below (from yB): 18
// boxes, one per lane of the calling warp; lane 0 arms the mbarrier first.
__device__ __forceinline__ void fused_load_plane(const CUtensorMap* mb3, const CUtensorMap* mbt,
                                                 const CUtensorMap* mu3, const CUtensorMap* mut, float* slot,
                                                 const SlotLayout& sl, int zz, int yA, int y0, int yB,
                                                 unsigned long long* bar, int lane) {
    if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, 2u * 3u * (unsigned)(sl.TY + 6) * (unsigned)sl.nx * 4u);
    }
    __syncwarp();
    if (lane < 18) {
        const int f = lane / 9, cc = (lane / 3) % 3, part = lane % 3;
        float* area = slot + (size_t)(3 * f + cc) * sl.CA;
        const CUtensorMap* m = part == 1 ? (f ? mut : mbt) : (f ? mu3 : mb3);
        tma_box(m, area + (part == 0 ? 0 : (part == 1 ? sl.P1 : sl.P2)), part == 0 ? yA : (part == 1 ? y0 : yB), zz,
                cc, bar);
    }
}

// grid: (bands, z chunks); block: kFusedMaxThreads or fewer (whole warps)
// Thread t owns the node pair t of the band's swept rows for every plane of
// the chunk (swept row t / (nx/2), x = 2 (t mod nx/2)): it converts that
// pair in each staged plane and keeps the pair's values of planes z - 1, z
// and z + 1 in registers; the threads of the first and last swept rows also
// convert the outermost staged row next to them.
// NXc, TYc, NSc: the width, band height and slot count as compile-time
// constants (instantiations for common plane widths: every shared-memory
// offset folds into the instruction), or 0 to take them from g.
template <bool XY, int NXc = 0, int TYc = 0, int NSc = 0>
__global__ void __launch_bounds__(kFusedMaxThreads, 1)
    k_sweep_fused(const __grid_constant__ CUtensorMap tm_b3, const __grid_constant__ CUtensorMap tm_bt,
                  const __grid_constant__ CUtensorMap tm_u3, const __grid_constant__ CUtensorMap tm_ut,
                  float* __restrict__ bout, SweepCoef<float> c, FusedIB ib, FusedGeo g, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_bad;
    // the copies land on 128-byte boundaries: align the dynamic region's start
    // at run time (the host adds 128 bytes of room)
    unsigned char* smem_al = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int nx = NXc ? NXc : g.nx, ny = g.ny, nz = g.nz, TY = TYc ? TYc : g.TY;
    const int P = nx * ny, n = g.n;
    const int band = blockIdx.x;
    const int y0 = min(band * TY, ny - TY);  // the last band ends at ny
    const int yA = y0 >= 3 ? y0 - 3 : y0 - 3 + ny, yB = y0 + TY < ny ? y0 + TY : y0 + TY - ny;
    const int z0 = blockIdx.y * g.chunk;
    const int z1 = min(z0 + g.chunk, nz);
    const int L = z1 - z0;
    if (L <= 0) return;
    SlotLayout lay;
    lay.nx = nx;
    lay.TY = TY;
    lay.P1 = fused_pad32(3 * nx);
    lay.P2 = lay.P1 + fused_pad32(TY * nx);
    lay.CA = lay.P2 + fused_pad32(3 * nx);
    const int slot_f = 6 * lay.CA;
    const int NS = NSc ? NSc : g.slots;
    const int SC = (TY + 4) * nx;        // component stride of S
    const int Mm = ib.Mmax, Sm = ib.Smax, K = ib.K;
    // shared memory: ring, S[2], deltas, the band's IB tables, mbarriers
    float* ring = reinterpret_cast<float*>(smem_al);
    float* S0 = ring + (size_t)NS * slot_f;  // [2][3][TY + 4][nx]: b* of the swept rows
    float* D0 = S0 + 2 * 3 * SC;             // [2][3][Mmax] deltas
    int* t_mo = reinterpret_cast<int*>(D0 + 2 * 3 * Mm);  // [Mmax][9] support offsets
    float* t_mw = reinterpret_cast<float*>(t_mo + 9 * Mm);  // [Mmax][9] weights
    float* t_ms = t_mw + 9 * Mm;                      // [Mmax] s^m_j
    int* t_so = reinterpret_cast<int*>(t_ms + Mm);    // [Smax] shell offsets
    int* t_sm = t_so + Sm;                            // [Smax][K] markers
    float* t_sw = reinterpret_cast<float*>(t_sm + Sm * K);  // [Smax][K] weights
    int* t_sc = reinterpret_cast<int*>(t_sw + Sm * K);       // [Smax] entries of each list
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(t_sc + Sm + ((reinterpret_cast<float*>(t_sc + Sm) - ring) & 1));
    const int tid = threadIdx.x, nthr = blockDim.x;
    const float w0 = c.w0, w1 = c.w1, w1k = c.w1 * c.kappa;
    const int half = nx / 2;
    const int npairs = (TY + 4) * half;
    const bool owner = tid < npairs;

    auto slot_of = [&](int j) { return ring + (size_t)(j % NS) * slot_f; };
    auto zwrap = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };

    if (tid == 0) {
        s_bad = 0;
        for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the next sweep may be scheduled as these CTAs exit; the band's IB
    // tables (constant) are read while the previous sweep finishes, b only
    // after it has
    pdl_trigger();
    // the band's IB tables, once
    const int Mr = ib.mk_cnt[band], Sr = ib.sh_cnt[band];
    for (int e = tid; e < 9 * Mr; e += nthr) {
        t_mo[e] = ib.mk_off[(size_t)band * Mm * 9 + e];
        t_mw[e] = ib.mk_w[(size_t)band * Mm * 9 + e];
    }
    for (int e = tid; e < Mr; e += nthr) t_ms[e] = ib.mk_s[(size_t)band * Mm + e];
    for (int e = tid; e < Sr; e += nthr) {
        t_so[e] = ib.sh_off[(size_t)band * Sm + e];
        t_sc[e] = ib.sh_cnt_e[(size_t)band * Sm + e];
    }
    for (int e = tid; e < Sr * K; e += nthr) {
        t_sm[e] = ib.sh_m[(size_t)band * Sm * K + e];
        t_sw[e] = ib.sh_w[(size_t)band * Sm * K + e];
    }
    pdl_wait();
    __syncthreads();
    // planes z0 - 1 .. z1 are needed (relative index j: plane z0 - 1 + j, in
    // slot j % NS, completing phase (j / NS) & 1 of that slot's mbarrier)
    // the warp that issues the copies: one in the middle, away from the
    // interpolation (first threads) and the spread (last threads)
    const int warp = tid >> 5, lane = tid & 31, copy_warp = (nthr >> 5) / 2;
    if (warp == copy_warp)
        for (int j = 0; j < NS && j <= L + 1; ++j)
            fused_load_plane(&tm_b3, &tm_bt, &tm_u3, &tm_ut, slot_of(j), lay, zwrap(z0 - 1 + j), yA, y0, yB,
                             &bars[j % NS], lane);

    // this thread's pair: swept row r (staged row r + 1), columns x, x + 1
    const int r = owner ? tid / half : 0;
    const int x = 2 * (tid - r * half);
    const int xl = x == 0 ? nx - 1 : x - 1, xr = x + 2 == nx ? 0 : x + 2;
    const int ou = lay.row_off(r), oc = lay.row_off(r + 1), od = lay.row_off(r + 2);
    // the outermost staged row converted by this thread too (-1: none)
    const int ox = !owner ? -1 : (r == 0 ? lay.row_off(0) : (r == TY + 3 ? lay.row_off(TY + 5) : -1));
    const int xs = (ox >= 0 && r == 0) ? -1 : ((ox >= 0) ? 1 : 0);  // row offset of that row from y (for XY)

    // (b, u) of the pair at offset o of plane slot sl -> (b, e) in place and in v
    auto convert_at = [&](float* sl, int o, int zz, int ydy, float2 v[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = *reinterpret_cast<const float2*>(sl + k * lay.CA + o);
        float be[3];
        bext_at(c.bext_z, c.be, zz, be);
        if constexpr (XY) {
            int y = ydy;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            const int pp = y * nx + x;
            float bA[3] = {be[0], be[1], be[2]}, bB[3] = {be[0], be[1], be[2]};
            bext_add_xy(c.bext_xy, P, pp, bA);
            bext_add_xy(c.bext_xy, P, pp + 1, bB);
            pair_emf(v, bA, bB, c.sq);
        } else {
            pair_emf(v, be, be, c.sq);
        }
#pragma unroll
        for (int k = 3; k < 6; ++k) *reinterpret_cast<float2*>(sl + k * lay.CA + o) = v[k];
    };
    // plane j: wait for its copy, convert this thread's pair (and its extra row)
    auto convert = [&](int j, float2 v[6]) {
        float* sl = slot_of(j);
        const int zz = zwrap(z0 - 1 + j);
        if (!mbar_wait_bounded(&bars[j % NS], (unsigned)((j / NS) & 1))) s_bad = 1;
        if (owner) {
            if (ox >= 0) {
                float2 t[6];
                convert_at(sl, ox + x, zz, y0 - 2 + r + xs, t);
            }
            convert_at(sl, oc + x, zz, y0 - 2 + r, v);
        }
    };

    // register pipeline of the pair: planes z - 1 (b, e2, e3), z (b, e), z + 1
    float2 prv[6], cur[6], nxt[6];
    convert(0, prv);
    convert(1, cur);
    convert(2, nxt);
    __syncthreads();  // the in-plane reads of plane z0 come next (and S is free)

    // own rows of the plane in S buffer ib_ (plane zp) to b_out: per component
    // one contiguous run of TY nx values, 16-byte aligned on both sides
    auto write_out = [&](int ib_, int zp) {
        const float* S = S0 + (size_t)ib_ * 3 * SC;
        const int run4 = TY * nx / 4;
        const size_t g0 = (size_t)zp * P + (size_t)y0 * nx;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float4* src = reinterpret_cast<const float4*>(S + a * SC + 2 * nx);
            float4* dst = reinterpret_cast<float4*>(bout + (size_t)a * n + g0);
            for (int v = tid; v < run4; v += nthr) dst[v] = src[v];
        }
    };
    // shell nodes of the plane in S buffer ib_ (plane zp) take the spread of
    // the deltas in D buffer ib_ and go to b_out, replacing the swept value
    // write_out put there before the last barrier; threads from the top down
    auto spread = [&](int ib_, int zp) {
        const float* S = S0 + (size_t)ib_ * 3 * SC;
        const float* D = D0 + (size_t)ib_ * 3 * Mm;
        const long long g0 = (long long)zp * P + (long long)(y0 - 2) * nx;  // row y0 - 2 (o >= 2 nx)
        for (int k = nthr - 1 - tid; k < Sr; k += nthr) {
            float c0 = 0.f, c1 = 0.f, c2 = 0.f;
            // the node's own entries (the zero-weight padding past them adds
            // exact zeros, so stopping there changes nothing)
            const int ke = t_sc[k];
            for (int e0 = 0; e0 < ke; e0 += 4) {
                const int4 mm = *reinterpret_cast<const int4*>(t_sm + k * K + e0);
                const float4 ww = *reinterpret_cast<const float4*>(t_sw + k * K + e0);
                const int ms[4] = {mm.x, mm.y, mm.z, mm.w};
                const float ws[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    c0 = __fmaf_rn(ws[e], D[ms[e]], c0);
                    c1 = __fmaf_rn(ws[e], D[Mm + ms[e]], c1);
                    c2 = __fmaf_rn(ws[e], D[2 * Mm + ms[e]], c2);
                }
            }
            const int o = t_so[k];
            float* q = bout + (g0 + o);
            q[0] = S[o] + c0;
            q[n] = S[SC + o] + c1;
            q[2 * (size_t)n] = S[2 * SC + o] + c2;
        }
    };
    // plane z0 - 1 is held in registers only: its slot takes plane z0 - 1 + NS
    if (warp == copy_warp && NS <= L + 1)
        fused_load_plane(&tm_b3, &tm_bt, &tm_u3, &tm_ut, slot_of(NS), lay, zwrap(z0 - 1 + NS), yA, y0, yB,
                         &bars[0], lane);

    for (int i = 0; i < L; ++i) {
        const int z = z0 + i;
        float* S = S0 + (size_t)(i & 1) * 3 * SC;
        // 1. sweep of this thread's pair of plane z: in-plane neighbours from
        // the slot of plane z, z neighbours from the registers
        if (owner) {
            const float* pc = slot_of(i + 1);
            float lf[6], rt[6];
            float2 up[6], dn[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float* a = pc + k * lay.CA;
                if (k != 5) {  // x neighbours: b, e1, e2
                    lf[k] = a[oc + xl];
                    rt[k] = a[oc + xr];
                }
                if (k != 4) {  // y neighbours: b, e1, e3
                    up[k] = *reinterpret_cast<const float2*>(a + ou + x);
                    dn[k] = *reinterpret_cast<const float2*>(a + od + x);
                }
            }
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
                const float2 o = make_float2(emf_update(w0, w1, w1k, cur[a].x, sL, dL),
                                             emf_update(w0, w1, w1k, cur[a].y, sR, dR));
                *reinterpret_cast<float2*>(S + a * SC + r * nx + x) = o;
            }
        }
        // plane z - 1's own rows as swept (b* of the wall shell is replaced
        // after the barrier)
        if (i >= 1) write_out((i - 1) & 1, z - 1);
        __syncthreads();
        // the slot of plane z (read for the last time above) takes plane
        // z + NS, NS - 1 planes ahead of its conversion
        if (warp == copy_warp && i + 1 + NS <= L + 1)
            fused_load_plane(&tm_b3, &tm_bt, &tm_u3, &tm_ut, slot_of(i + 1 + NS), lay, zwrap(z0 + i + NS), yA, y0,
                             yB, &bars[(i + 1 + NS) % NS], lane);
        // 2. deltas of the band's markers of plane z (threads from 0 up), the
        // shell nodes of plane z - 1 (threads from the top down), this
        // thread's pair of plane z + 2
        {
            float* D = D0 + (size_t)(i & 1) * 3 * Mm;
            for (int m = tid; m < Mr; m += nthr) {
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const int o = t_mo[m * 9 + j];
                    const float w = t_mw[m * 9 + j];
                    a0 = __fmaf_rn(w, S[o], a0);
                    a1 = __fmaf_rn(w, S[SC + o], a1);
                    a2 = __fmaf_rn(w, S[2 * SC + o], a2);
                }
                const float sm = t_ms[m];
                D[m] = -sm * a0;
                D[Mm + m] = -sm * a1;
                D[2 * Mm + m] = -sm * a2;
            }
        }
        if (i >= 1) spread((i - 1) & 1, z - 1);
        float2 ahd[6];
        if (i + 3 <= L + 1) convert(i + 3, ahd);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            prv[k] = cur[k];
            cur[k] = nxt[k];
            nxt[k] = ahd[k];
        }
    }
    // the last plane: its rows, then (after a barrier, so that the corrected
    // shell values come last) its shell nodes
    write_out((L - 1) & 1, z1 - 1);
    __syncthreads();
    spread((L - 1) & 1, z1 - 1);
    if (tid == 0 && s_bad) atomicExch(err, 1);
}

}  // namespace qslbm
