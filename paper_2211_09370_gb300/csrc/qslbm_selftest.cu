// Self-check of the bounded wait used by the resident sweep kernel: a single
// warp waits on a counter in device memory with the same routine
// (wait_counters) and reports whether it gave up.  With the counter left at
// zero nothing ever satisfies the wait, so a correct routine must return
// after its limit; with the counter already set it must return at once.
#include <cuda_runtime.h>

#include <string>

#include "qslbm.h"
#include "qslbm_resident.cuh"

namespace qslbm {
void set_last_error(const std::string& msg);
}

namespace {

__global__ void k_wait_probe(const unsigned int* counter, unsigned long long limit_ns, int* gave_up,
                             unsigned long long* waited_ns) {
    if (threadIdx.x != 0) return;
    const unsigned long long t0 = qslbm::globaltimer_ns();
    const bool ok = qslbm::wait_counters(counter, counter, 1u, limit_ns);
    *waited_ns = qslbm::globaltimer_ns() - t0;
    *gave_up = ok ? 0 : 1;
}

int fail(cudaError_t e, const char* what) {
    qslbm::set_last_error(std::string("qslbm_check_bounded_wait: ") + what + ": " + cudaGetErrorString(e));
    return QSLBM_ECUDA;
}

}  // namespace

extern "C" int qslbm_check_bounded_wait(double limit_s, int32_t counter_set, int32_t* gave_up, double* waited_s) {
    if (!gave_up || !waited_s || !(limit_s > 0.0) || limit_s > 2.0) return QSLBM_EINVAL;
    struct Buf {
        unsigned int counter;
        int gave_up;
        unsigned long long waited_ns;
    };
    Buf* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(Buf));
    if (e != cudaSuccess) return fail(e, "cudaMalloc");
    Buf h{};
    h.counter = counter_set ? 1u : 0u;
    h.gave_up = -1;
    e = cudaMemcpy(d, &h, sizeof(Buf), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32>>>(&d->counter, (unsigned long long)(limit_s * 1e9), &d->gave_up, &d->waited_ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(Buf), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(e, "launch");
    *gave_up = h.gave_up;
    *waited_s = (double)h.waited_ns * 1e-9;
    return QSLBM_OK;
}
