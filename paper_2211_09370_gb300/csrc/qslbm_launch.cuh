// Kernel launchers for one storage precision T; included by qslbm_f32.cu and
// qslbm_f64.cu, which instantiate it for float and double.
#pragma once

#include <algorithm>

#include "qslbm_fused.cuh"
#include "qslbm_internal.h"
#include "qslbm_kernels.cuh"
#include "qslbm_resident.cuh"

namespace qslbm {

template <typename T>
struct Launch {
    static Geo geo(const State& s) { return Geo{s.nx, s.ny, s.nz, s.n}; }

    static IBView<T> view(const State& s, bool magnetic) {
        IBView<T> v;
        v.ring_off = s.ib.ring_off;
        v.mk_q = s.ib.mk_q;
        v.mk_w = static_cast<const T*>(s.ib.mk_w);
        v.mk_s = static_cast<const T*>(magnetic ? s.ib.mk_sm : s.ib.mk_s);
        v.shell_off = s.ib.shell_off;
        v.shell_xy = s.ib.shell_xy;
        v.csr_off = s.ib.csr_off;
        v.csr_m = s.ib.csr_m;
        v.csr_w = static_cast<const T*>(s.ib.csr_w);
        v.mk_base = s.ib.mk_base;
        v.shell_node = s.ib.shell_node;
        v.csr_mg = s.ib.csr_mg;
        v.delta = static_cast<T*>(s.ib.delta);
        v.nm = s.ib.nm;
        v.ns = s.ib.ns;
        v.zinv = s.ib.zinv;
        v.mk_slot = s.ib.mk_slot;
        v.pad_m = s.ib.pad_m;
        v.pad_w = static_cast<const T*>(s.ib.pad_w);
        v.pad_k = s.ib.pad_k;
        return v;
    }

    // A launch that may begin while the previous kernel in the stream finishes
    // (programmatic dependent launch; the kernel calls pdl_wait before it
    // touches that kernel's results).
    template <typename... KArgs, typename... Args>
    static void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
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
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, kernel, args...);  // errors surface at the next synchronising call
    }

    static size_t ib_smem(const State& s) { return (size_t)3 * (s.ib.max_ring > 0 ? s.ib.max_ring : 1) * sizeof(T); }

    static int grid_for(long long n, int threads) {
        long long b = (n + threads - 1) / threads;
        if (b > 152LL * 16) b = 152LL * 16;
        if (b < 1) b = 1;
        return (int)b;
    }

    static void init(State& s, cudaStream_t st) {
        int ncomp = s.dim == 3 ? 3 : 2;
        k_init<T><<<grid_for(s.n, 256), 256, 0, st>>>(geo(s), (T*)s.drho[0], (T*)s.u[0], (T*)s.b[0], s.p.seed,
                                                       s.p.perturb * s.units.U0, ncomp, s.p.geometry, s.cx,
                                                       s.cy, s.R, s.p.init_kind == QSLBM_INIT_POISEUILLE,
                                                       s.units.U0, s.axis);
    }

    static void sweeps(State& s, int nsweeps, cudaStream_t st) {
        SweepCoef<T> c;
        sweep_weights(s, c.w0, c.w1, c.kappa);
        for (int a = 0; a < 3; ++a) c.be[a] = (T)s.be[a];
        c.bext_z = static_cast<const T*>(s.bext_z);
        c.bext_xy = static_cast<const T*>(s.bext_xy);
        c.strict_qs = s.p.strict_qs;
        c.sq = s.p.strict_qs ? T(0) : T(1);
        const IBView<T> v = view(s, true);
        const size_t smem = ib_smem(s);
        if (s.resident && nsweeps > 0) {
            launch_resident(s, nsweeps, c, v, st);
            s.bcur ^= 1;
            return;
        }
        if (s.fused) {
            for (int i = 0; i < nsweeps; ++i) {
                launch_fused(s, c, st);
                s.bcur ^= 1;
            }
            return;
        }
        if (s.p.sweep_kernel == QSLBM_SWEEP_SPLIT) {
            const int P = s.nx * s.ny;
            const dim3 grid((unsigned)((P + kNodeThreads - 1) / kNodeThreads), (unsigned)s.nz);
            const int chunk = s.march_chunk;
            const dim3 mgrid((unsigned)((s.nx + kMarchTX - 1) / kMarchTX), (unsigned)((s.ny + kMarchTY - 1) / kMarchTY),
                             (unsigned)((s.nz + chunk - 1) / chunk));
            for (int i = 0; i < nsweeps; ++i) {
                const T* bin = (const T*)s.b[s.bcur];
                T* bout = (T*)s.b[1 - s.bcur];
                const T* u = (const T*)s.u[s.fcur];
                if (pair_march(s)) {
                    const dim3 pgrid((unsigned)((s.nx + 2 * kPairTXP - 1) / (2 * kPairTXP)),
                                     (unsigned)((s.ny + kPairTY - 1) / kPairTY), (unsigned)((s.nz + chunk - 1) / chunk));
                    if (s.bext_xy)
                        launch_pdl(k_sweep_march_pair<float, true>, pgrid, dim3(kPairThreads), 0, st, geo(s),
                                   (const float*)bin, (float*)bout, (const float*)u, fcoef(c), chunk);
                    else
                        launch_pdl(k_sweep_march_pair<float, false>, pgrid, dim3(kPairThreads), 0, st, geo(s),
                                   (const float*)bin, (float*)bout, (const float*)u, fcoef(c), chunk);
                } else if (s.dim == 3)
                {
                    if (s.bext_xy)
                        k_sweep_march<T, true><<<mgrid, kMarchTX * kMarchTY, 0, st>>>(geo(s), bin, bout, u, c, chunk);
                    else
                        k_sweep_march<T, false><<<mgrid, kMarchTX * kMarchTY, 0, st>>>(geo(s), bin, bout, u, c, chunk);
                }
                else
                    k_sweep_nodes<T, 2><<<grid, kNodeThreads, 0, st>>>(geo(s), bin, bout, u, c);
                if (s.ib.nm > 0 && s.ib_staged_smem > 0) {
                    const int R = s.ib.max_ring, S = s.ib.max_shell;
                    const size_t sm = s.ib_staged_smem;
                    const dim3 ig((unsigned)s.nz), ib(kNodeThreads);
                    switch (s.ib_staged_u) {
                        case 1: launch_pdl(k_ib_staged<T, 1>, ig, ib, sm, st, geo(s), bout, v, R, S); break;
                        case 2: launch_pdl(k_ib_staged<T, 2>, ig, ib, sm, st, geo(s), bout, v, R, S); break;
                        case 4: launch_pdl(k_ib_staged<T, 4>, ig, ib, sm, st, geo(s), bout, v, R, S); break;
                        default: launch_pdl(k_ib_staged<T, 5>, ig, ib, sm, st, geo(s), bout, v, R, S); break;
                    }
                } else if (s.ib.nm > 0) {
                    k_ib_markers<T><<<(s.ib.nm + kNodeThreads - 1) / kNodeThreads, kNodeThreads, 0, st>>>(geo(s), bout, v);
                    k_ib_shell<T><<<(s.ib.ns + kNodeThreads - 1) / kNodeThreads, kNodeThreads, 0, st>>>(geo(s), bout, v);
                }
                s.bcur ^= 1;
            }
            return;
        }
        for (int i = 0; i < nsweeps; ++i) {
            const T* bin = (const T*)s.b[s.bcur];
            T* bout = (T*)s.b[1 - s.bcur];
            const T* u = (const T*)s.u[s.fcur];
            if (s.dim == 3)
                k_sweep_ib<T, 3><<<s.nz, kPlaneThreads, smem, st>>>(geo(s), bin, bout, u, c, v);
            else
                k_sweep_ib<T, 2><<<s.nz, kPlaneThreads, smem, st>>>(geo(s), bin, bout, u, c, v);
            s.bcur ^= 1;
        }
    }

    template <int DIM, bool UHALO, bool SMALL>
    static void resident_launch_one(State& s, int nsweeps, const SweepCoef<T>& c, const IBView<T>& v,
                                    cudaStream_t st) {
        constexpr int RT = ResidentShape<T, SMALL>::threads, NPT = ResidentShape<T, SMALL>::npt;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)s.nz);
        cfg.blockDim = dim3(RT);
        cfg.dynamicSmemBytes = s.resident_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const T* bin = (const T*)s.b[s.bcur];
        T* bout = (T*)s.b[1 - s.bcur];
        const T* u = (const T*)s.u[s.fcur];
        cudaError_t e;
        if (s.nx % 2 == 0)
            e = cudaLaunchKernelEx(&cfg, k_sweeps_resident<T, DIM, UHALO, RT, NPT, true>, geo(s), bin, bout, u, c, v,
                                   (T*)s.xbuf, (ResidentSync*)s.rsync, nsweeps, s.ib.max_ring, s.ib.max_shell,
                                   s.ib.max_nnz);
        else
            e = cudaLaunchKernelEx(&cfg, k_sweeps_resident<T, DIM, UHALO, RT, NPT, false>, geo(s), bin, bout, u, c,
                                   v, (T*)s.xbuf, (ResidentSync*)s.rsync, nsweeps, s.ib.max_ring, s.ib.max_shell,
                                   s.ib.max_nnz);
        // a failed launch is recorded for the caller
        if (e != cudaSuccess) s.launch_error = true;
    }

    static FusedIB fused_ib(const State& s) {
        FusedIB t;
        t.mk_cnt = s.fu_mk_cnt;
        t.mk_off = s.fu_mk_off;
        t.mk_w = s.fu_mk_w;
        t.mk_s = s.fu_mk_s;
        t.sh_cnt = s.fu_sh_cnt;
        t.sh_off = s.fu_sh_off;
        t.sh_m = s.fu_sh_m;
        t.sh_w = s.fu_sh_w;
        t.sh_cnt_e = s.fu_sh_ce;
        t.Mmax = s.fu_Mmax;
        t.Smax = s.fu_Smax;
        t.K = s.fu_K;
        return t;
    }

    // the instantiation for this handle's shape: compile-time (nx, rows per
    // band, slots) for common plane widths, the general one otherwise
    static decltype(&k_sweep_fused<false>) fused_kernel(const State& s) {
        if (s.bext_xy) return k_sweep_fused<true>;
        if (s.nx == 96 && s.fu_TY == 12 && s.fu_slots == 4) return k_sweep_fused<false, 96, 12, 4>;
        if (s.nx == 64 && s.fu_TY == 20 && s.fu_slots == 4) return k_sweep_fused<false, 64, 20, 4>;
        if (s.nx == 128 && s.fu_TY == 8 && s.fu_slots == 4) return k_sweep_fused<false, 128, 8, 4>;
        return k_sweep_fused<false>;
    }

    // one sweep + IB on b, bin = b[bcur] -> b[1 - bcur], u = u[fcur]
    static void launch_fused(State& s, const SweepCoef<T>& c, cudaStream_t st) {
        if constexpr (sizeof(T) == 4) {
            const dim3 grid((unsigned)s.fu_bands, (unsigned)s.fu_chunks);
            const FusedGeo g{s.nx, s.ny, s.nz, s.fu_TY, s.fu_chunk, (int)s.n, s.fu_slots};
            const int bc = s.bcur, fc = s.fcur;
            launch_pdl(fused_kernel(s), grid, dim3(s.fu_threads), s.fu_smem, st, s.fu_map_b3[bc], s.fu_map_bt[bc],
                       s.fu_map_u3[fc], s.fu_map_ut[fc], (float*)s.b[1 - bc], c, fused_ib(s), g, s.fu_err);
        } else {
            s.launch_error = true;  // never planned: the fused sweep is the FP32 path
        }
    }

    // threads, and z planes per CTA so that the grid is one CTA per SM
    static cudaError_t plan_fused(State& s) {
        if constexpr (sizeof(T) != 4) {
            s.fused = false;
            return cudaSuccess;
        } else {
            // one node pair per thread and pass over the band's swept rows
            const int pairs = (s.fu_TY + 4) * s.nx / 2;
            s.fu_threads = std::min(kFusedMaxThreads, (pairs + 31) / 32 * 32);
            auto kern = fused_kernel(s);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.fu_smem);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s.fused = false;
                return cudaSuccess;
            }
            int dev = 0, sms = 0, per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.fu_threads, s.fu_smem)) !=
                cudaSuccess)
                return e;
            if (per_sm < 1) {
                s.fused = false;
                return cudaSuccess;
            }
            const int slots_total = per_sm * sms;
            const int chunks = std::max(1, slots_total / s.fu_bands);
            s.fu_chunk = (s.nz + chunks - 1) / chunks;
            s.fu_chunks = (s.nz + s.fu_chunk - 1) / s.fu_chunk;
            return cudaSuccess;
        }
    }

    // Times one sweep of the fused kernel and one of the split path (each
    // reads b[bcur] and writes b[1 - bcur], which holds no state) on this
    // handle's own fields: two sweeps to warm up, then four, CUDA events on
    // the handle's stream.  Leaves the fused kernel in use when it is the
    // faster one.
    // Times both routes (two interleaved rounds of 8 sweeps each after a
    // warm-up, the faster round kept) and takes the fused kernel only when it
    // is at least 2 % faster: the split path is the simpler one and wins
    // ties, so that the choice does not flip on timing noise.  Every timed
    // sweep reads b[bcur] and writes the other buffer, so the state is left
    // as it was.
    static cudaError_t tune_fused(State& s, double* us_fused, double* us_split) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        double us[2] = {1e300, 1e300};
        for (int round = 0; round < 2; ++round) {
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                s.fused = k == 0;
                s.p.sweep_kernel = k == 0 ? QSLBM_SWEEP_FUSED : QSLBM_SWEEP_SPLIT;
                for (int r = 0; r < 2; ++r) {
                    sweeps(s, 1, s.stream);
                    s.bcur ^= 1;  // undo the sweep's swap: the next reads the same b
                }
                e = cudaEventRecord(e0, s.stream);
                for (int r = 0; r < 8 && e == cudaSuccess; ++r) {
                    sweeps(s, 1, s.stream);
                    s.bcur ^= 1;
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, s.stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                us[k] = std::min(us[k], 1e3 * ms / 8);
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        *us_fused = us[0];
        *us_split = us[1];
        s.fused = e == cudaSuccess && us[0] < 0.98 * us[1];
        s.p.sweep_kernel = s.fused ? QSLBM_SWEEP_FUSED : QSLBM_SWEEP_SPLIT;
        return e;
    }

    static bool small_plane(const State& s) { return (long long)s.nx * s.ny <= (long long)kResidentSmallPlane; }

    static void launch_resident(State& s, int nsweeps, const SweepCoef<T>& c, const IBView<T>& v,
                                cudaStream_t st) {
        const bool small = small_plane(s);
        if (s.dim == 3) {
            if (s.resident_uhalo) {
                if (small)
                    resident_launch_one<3, true, true>(s, nsweeps, c, v, st);
                else
                    resident_launch_one<3, true, false>(s, nsweeps, c, v, st);
            } else {
                if (small)
                    resident_launch_one<3, false, true>(s, nsweeps, c, v, st);
                else
                    resident_launch_one<3, false, false>(s, nsweeps, c, v, st);
            }
        } else {
            if (small)
                resident_launch_one<2, false, true>(s, nsweeps, c, v, st);
            else
                resident_launch_one<2, false, false>(s, nsweeps, c, v, st);
        }
    }

    template <int DIM, bool UHALO, bool SMALL>
    static cudaError_t try_resident_shape(State& s, size_t smem, bool& ok) {
        constexpr int RT = ResidentShape<T, SMALL>::threads, NPT = ResidentShape<T, SMALL>::npt;
        ok = false;
        auto kern = k_sweeps_resident<T, DIM, UHALO, RT, NPT, false>;
        auto kern2 = k_sweeps_resident<T, DIM, UHALO, RT, NPT, true>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cudaSuccess;  // too much shared memory: not resident
        }
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        ok = per_sm >= 1 && (long long)per_sm * sms >= s.nz;
        return cudaSuccess;
    }

    template <int DIM, bool UHALO>
    static cudaError_t try_resident(State& s, size_t smem, bool& ok) {
        if (small_plane(s)) return try_resident_shape<DIM, UHALO, true>(s, smem, ok);
        return try_resident_shape<DIM, UHALO, false>(s, smem, ok);
    }

    // The FP32 pair kernel serves 3-D domains with an even nx.
    static bool pair_march(const State& s) { return sizeof(T) == 4 && s.dim == 3 && s.nx % 2 == 0; }
    static SweepCoef<float> fcoef(const SweepCoef<T>& c) {
        if constexpr (sizeof(T) == 4)
            return c;
        else
            return SweepCoef<float>{};  // never launched: the pair kernel is FP32 only
    }

    // z planes per CTA of the marching sweep such that the grid fills one wave
    static cudaError_t plan_march(State& s) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const bool pair = pair_march(s);
        if (e == cudaSuccess)
            e = pair ? (s.bext_xy ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_march_pair<float, true>,
                                                                                  kPairThreads, 0)
                                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                        &per_sm, k_sweep_march_pair<float, false>, kPairThreads, 0))
                     : (s.bext_xy ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_march<T, true>,
                                                                                  kMarchTX * kMarchTY, 0)
                                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_march<T, false>,
                                                                                  kMarchTX * kMarchTY, 0));
        if (e != cudaSuccess) return e;
        const long long tiles =
            pair ? (long long)((s.nx + 2 * kPairTXP - 1) / (2 * kPairTXP)) * ((s.ny + kPairTY - 1) / kPairTY)
                 : (long long)((s.nx + kMarchTX - 1) / kMarchTX) * ((s.ny + kMarchTY - 1) / kMarchTY);
        const long long slots = (long long)std::max(1, per_sm) * std::max(1, sms);
        const long long per_column = std::max<long long>(1, slots / std::max<long long>(1, tiles));
        long long chunk = (s.nz + per_column - 1) / per_column;
        chunk = std::max<long long>(chunk, 4);  // keep the z halo overhead small
        s.march_chunk = (int)std::min<long long>(chunk, s.nz);
        // the staged IB corrector, when the plane's shell fits shared memory
        // and the shell nodes' marker lists are padded
        s.ib_staged_smem = 0;
        if (s.ib.nm > 0 && s.ib.pad_k > 0) {
            const size_t smem = ib_staged_smem_bytes<T>(s.ib.max_ring, s.ib.max_shell);
            int max_optin = 0;
            e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (e != cudaSuccess) return e;
            if (smem <= (size_t)max_optin) {
                s.ib_staged_u = ib_staged_unroll(s.ib.max_shell, s.nz, sms);
                const int U = s.ib_staged_u;
                e = cudaFuncSetAttribute(U == 1   ? k_ib_staged<T, 1>
                                         : U == 2 ? k_ib_staged<T, 2>
                                         : U == 4 ? k_ib_staged<T, 4>
                                                  : k_ib_staged<T, 5>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                s.ib_staged_smem = smem;
            }
        }
        return cudaSuccess;
    }

    static cudaError_t plan_resident(State& s) {
        s.resident = false;
        const long long P = (long long)s.nx * s.ny;
        if (P > (long long)kResidentMaxPlane) return cudaSuccess;
        if (s.bext_xy) return cudaSuccess;  // an in-plane applied field takes the split path
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return e;
        const size_t base = resident_smem_bytes<T>((int)P, false, s.ib.max_ring, s.ib.max_shell, s.ib.max_nnz);
        const size_t halo = (size_t)6 * P * sizeof(T);
        const size_t reserve = 1024;  // static shared variables and the runtime's own share
        bool ok = false;
        if (s.dim == 3 && base + halo + reserve <= (size_t)optin) {
            if ((e = try_resident<3, true>(s, base + halo, ok)) != cudaSuccess) return e;
            if (ok) {
                s.resident = true;
                s.resident_uhalo = true;
                s.resident_smem = base + halo;
                return cudaSuccess;
            }
        }
        if (base + reserve > (size_t)optin) return cudaSuccess;
        if (s.dim == 3)
            e = try_resident<3, false>(s, base, ok);
        else
            e = try_resident<2, false>(s, base, ok);
        if (e != cudaSuccess) return e;
        if (ok) {
            s.resident = true;
            s.resident_uhalo = false;
            s.resident_smem = base;
        }
        return cudaSuccess;
    }

    static void force_flow(State& s, cudaStream_t st) {
        ForceCoef<T> fc;
        fc.F0 = s.units.F0;
        fc.amp = s.p.force_amp;
        fc.omega = s.omega;
        fc.axis = s.axis;
        for (int a = 0; a < 3; ++a) fc.be[a] = (T)s.be[a];
        fc.bext_z = static_cast<const T*>(s.bext_z);
        fc.bext_xy = static_cast<const T*>(s.bext_xy);
        FlowCoef<T> c;
        c.tau = (T)s.units.tau;
        c.kforce = (T)(1.0 - 1.0 / (2.0 * s.units.tau));
        c.mac = s.p.flow_scheme == QSLBM_FLOW_MACROSCOPIC;
        c.ig = (T)s.ig;
        c.ig2 = (T)(s.ig * s.ig);
        const IBView<T> v = view(s, false);
        const T* b = (const T*)s.b[s.bcur];
        const T* dr = (const T*)s.drho[s.fcur];
        const T* u = (const T*)s.u[s.fcur];
        T* dro = (T*)s.drho[1 - s.fcur];
        T* uo = (T*)s.u[1 - s.fcur];
        T* F = (T*)s.F;
        if (s.dim == 3 && s.units.flow_q == 27) {
            k_force<T, 3, 27><<<grid_for(s.n, 256), 256, 0, st>>>(geo(s), b, F, fc, s.tdev);
            k_flow_ib<T, 3, 27><<<s.nz, kPlaneThreads, ib_smem(s), st>>>(geo(s), dr, u, F, dro, uo, c, v, s.tdev);
        } else if (s.dim == 3) {
            k_force<T, 3><<<grid_for(s.n, 256), 256, 0, st>>>(geo(s), b, F, fc, s.tdev);
            k_flow_ib<T, 3><<<s.nz, kPlaneThreads, ib_smem(s), st>>>(geo(s), dr, u, F, dro, uo, c, v, s.tdev);
        } else {
            k_force<T, 2><<<grid_for(s.n, 256), 256, 0, st>>>(geo(s), b, F, fc, s.tdev);
            k_flow_ib<T, 2><<<s.nz, kPlaneThreads, ib_smem(s), st>>>(geo(s), dr, u, F, dro, uo, c, v, s.tdev);
        }
        s.fcur ^= 1;
    }

    static ObsCoef<T> obs_coef(const State& s, double fb) {
        ObsCoef<T> c;
        c.eta = s.units.eta;
        c.fb = fb;
        c.axis = s.axis;
        c.geometry = s.p.geometry;
        c.strict_qs = s.p.strict_qs;
        c.dim = s.dim;
        c.cx = s.cx;
        c.cy = s.cy;
        c.rin = s.R - 2.0;
        for (int a = 0; a < 3; ++a) c.be[a] = (T)s.be[a];
        c.bext_z = static_cast<const T*>(s.bext_z);
        c.bext_xy = static_cast<const T*>(s.bext_xy);
        return c;
    }

    static void observe_fields(const State& s, const void* drho, const void* u, const void* b, const void* usnap,
                               double fb, int blocks, double* partial, double* sums, cudaStream_t st) {
        const ObsCoef<T> c = obs_coef(s, fb);
        const T* dr = (const T*)drho;
        const T* uu = (const T*)u;
        const T* bb = (const T*)b;
        const T* us = (const T*)usnap;
        if (s.dim == 3 && s.units.flow_q == 27)
            k_observe<T, 3, 27><<<blocks, kReduceThreads, 0, st>>>(geo(s), dr, uu, bb, us, c, partial);
        else if (s.dim == 3)
            k_observe<T, 3><<<blocks, kReduceThreads, 0, st>>>(geo(s), dr, uu, bb, us, c, partial);
        else
            k_observe<T, 2><<<blocks, kReduceThreads, 0, st>>>(geo(s), dr, uu, bb, us, c, partial);
        k_fold<T><<<1, 32 * kObs, 0, st>>>(partial, blocks, sums);
    }

    static void observe(State& s, double fb, cudaStream_t st) {
        observe_fields(s, s.drho[s.fcur], s.u[s.fcur], s.b[s.bcur], s.usnap, fb, s.nblocks_obs, s.partial,
                       s.obs_dev, st);
    }

    static void to_f64(State& s, cudaStream_t st) {
        k_to_f64<T><<<grid_for(s.n, 256), 256, 0, st>>>(s.n, (const T*)s.drho[s.fcur], (const T*)s.u[s.fcur],
                                                        (const T*)s.b[s.bcur], s.staging);
    }

    static void from_f64(State& s, int mask, cudaStream_t st) {
        k_from_f64<T><<<grid_for(s.n, 256), 256, 0, st>>>(s.n, s.staging, (T*)s.drho[s.fcur], (T*)s.u[s.fcur],
                                                          (T*)s.b[s.bcur], mask);
    }

    static const Ops& table() {
        static const Ops o = {&init,     &sweeps,        &force_flow, &observe,     &observe_fields,
                              &to_f64,   &from_f64,      &plan_resident, &plan_march, &plan_fused,
                              &tune_fused};
        return o;
    }
};

}  // namespace qslbm
