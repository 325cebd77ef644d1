// Allocation-free diagnostics: qslbm_observables_static.
//
// Some callers cannot allocate device memory at the moment they want the
// diagnostics: code that is recording a CUDA graph (cudaMalloc is refused
// while a stream is being captured), code whose device memory is handed out by
// another allocator that already owns the pool (a framework's caching
// allocator), or a loop with latency limits that must stay out of the CUDA
// driver's allocator.  This file gives them the same FP64 diagnostic reduction as
// qslbm_observables, over fields they pass in, with the per-block partial sums
// kept in a fixed array compiled into the library instead of allocated memory.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "qslbm.h"
#include "qslbm_internal.h"

namespace {

// One block of the reduction per z plane; its 11 partial sums per block, the
// 11 folded sums, in one array that every call on this device shares.
constexpr int kStaticMaxPlanes = QSLBM_STATIC_MAX_PLANES;
static __device__ __align__(256) double g_static_scratch[(kStaticMaxPlanes + 1) * qslbm::kObs];

std::mutex g_mutex;
double* g_scratch_addr[64] = {};  // device address of g_static_scratch, per device ordinal

// Turn the folded sums into the qslbm_obs quantities (same formulas as the
// host side of qslbm_observables).
__global__ void k_static_finish(const double* sums, double mass0, double nu, long long dt, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double inv = sums[9] > 0 ? 1.0 / sums[9] : 0.0;
    out[0] = sums[0];
    out[1] = (sums[0] - mass0) / mass0;
    out[2] = sums[1] * inv;
    out[3] = sums[2] * inv;
    out[4] = sums[3] * inv;
    out[5] = -nu * sums[4] * inv;
    out[6] = sums[5] * inv;
    out[7] = sqrt(sums[6] * inv);
    out[8] = (dt > 0 && sums[8] > 0) ? sqrt(sums[7]) / ((double)dt * sqrt(sums[8])) : 0.0;
    out[9] = sums[10] > 0 ? 1.0 : 0.0;
}

// The reduction runs through the handle's per-precision launcher table, so the
// diagnostics kernels exist once per precision in the library (the FP64 ones
// compiled without contraction) and the flow lattice is chosen as in
// qslbm_observables.
void launch(const qslbm::State& s, const void* drho, const void* u, const void* b, const void* u_prev, double fb,
            long long dt, double* out, double* scratch, cudaStream_t st) {
    const qslbm::Ops& ops = s.p.precision == QSLBM_FP64 ? qslbm::ops_f64() : qslbm::ops_f32();
    double* partial = scratch;
    double* sums = scratch + (size_t)kStaticMaxPlanes * qslbm::kObs;
    ops.observe_fields(s, drho, u, b, u_prev, fb, s.nz, partial, sums, st);
    k_static_finish<<<1, 32, 0, st>>>(sums, s.mass0, s.units.nu, dt, out);
}

// Device address of the scratch array for the current device, looked up once.
int scratch_for_current_device(double** out, std::string& err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return QSLBM_ECUDA;
    }
    if (dev < 0 || dev >= 64) {
        err = "device ordinal out of range";
        return QSLBM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return QSLBM_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return QSLBM_OK;
}

}  // namespace

namespace qslbm {
// The ABI's error text lives in qslbm_api.cu; this file reports through it.
void set_last_error(const std::string& msg);
const State& handle_state(const qslbm_handle* h);
}  // namespace qslbm

extern "C" int qslbm_observables_static(const qslbm_handle* h, const void* drho, const void* u, const void* b,
                                        const void* u_prev, double fb, int64_t steps_since_prev, double* out,
                                        void* stream) {
    if (!h || !drho || !u || !b || !u_prev || !out) {
        qslbm::set_last_error("qslbm_observables_static: a handle, field or output pointer is NULL");
        return QSLBM_EINVAL;
    }
    if (steps_since_prev < 0) {
        qslbm::set_last_error("qslbm_observables_static: steps_since_prev is negative");
        return QSLBM_EINVAL;
    }
    const qslbm::State& s = qslbm::handle_state(h);
    if (s.nz > kStaticMaxPlanes) {
        qslbm::set_last_error("qslbm_observables_static: " + std::to_string(s.nz) + " z planes exceed the limit of " +
                              std::to_string(kStaticMaxPlanes));
        return QSLBM_EINVAL;
    }
    std::string err;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch, err);
    if (rc) {
        qslbm::set_last_error(err);
        return rc;
    }
    launch(s, drho, u, b, u_prev, fb, steps_since_prev, out, scratch, static_cast<cudaStream_t>(stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        qslbm::set_last_error(std::string("qslbm_observables_static: ") + cudaGetErrorString(e));
        return QSLBM_ECUDA;
    }
    return QSLBM_OK;
}
