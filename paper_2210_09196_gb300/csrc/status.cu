// Failure reporting of the C ABI: the kernels' error words folded into the caller's status words, the
// synchronous status check (pusch_status_check) and the bounded-wait self-test (pusch_selftest_wait).
//
// Numeric failures of the detector (Eq. 2: a Cholesky pivot that is not a positive finite number, a
// non-finite detected symbol) are counted by the detection kernels in the status words. Kernels that wait
// on asynchronous copies or MMAs give up after a bounded time (bounded_wait.cuh) and set a bit in an error
// word; the fold kernel moves that word into status[0] (PUSCH_STATUS_TIMEOUT) and status[3] at the end of
// every chain call, so that one read of the status words reports both kinds of failure.
#include <stdio.h>

#include "bounded_wait.cuh"
#include "internal.cuh"

namespace pusch {
namespace {

__global__ void status_fold_kernel(uint32_t *status, uint32_t *err) {
    const uint32_t e = *err;
    if (e != 0u) {
        status[0] |= (uint32_t)PUSCH_STATUS_TIMEOUT;
        status[3] |= e;
        *err = 0u;
    }
}

// One thread waits on a barrier that nothing arrives on (its phase 0 never completes) with the library's
// bounded wait and the given limit, then records the expiry. No copy, MMA or TMEM allocation is issued, so
// nothing is left in flight when the thread gives up.
__global__ void selftest_wait_kernel(uint32_t *err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    bw::mbar_init(a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!bw::mbar_wait_for(a, 0u, limit_ns)) atomicOr(err, kErrSelftest);
}

thread_local char g_msg[256];

pusch_status sfail(pusch_status st, const char *msg) {
    set_last_error(msg);
    return st;
}

}  // namespace

cudaError_t launch_status_fold(uint32_t *status, uint32_t *err, cudaStream_t st) {
    status_fold_kernel<<<1, 1, 0, st>>>(status, err);
    return cudaGetLastError();
}

}  // namespace pusch

extern "C" {

pusch_status pusch_status_check(pusch_handle *h, const uint32_t *status, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t st[4] = {0u, 0u, 0xffffffffu, 0u};
    uint32_t err = 0u;
    cudaError_t e = cudaSuccess;
    if (status) e = cudaMemcpyAsync(st, status, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h) e = cudaMemcpyAsync(&err, h->kernel_err, sizeof err, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(h->kernel_err, 0, sizeof err, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(pusch::g_msg, sizeof pusch::g_msg, "pusch_status_check: %s (%s)", cudaGetErrorName(e),
                 cudaGetErrorString(e));
        return pusch::sfail(PUSCH_ERR_CUDA, pusch::g_msg);
    }
    const uint32_t timeout_bits = err | ((st[0] & PUSCH_STATUS_TIMEOUT) ? (st[3] ? st[3] : 1u) : 0u);
    if (timeout_bits) {
        snprintf(pusch::g_msg, sizeof pusch::g_msg,
                 "a bounded device wait expired (error bits 0x%x: 1 tensor-core kernel, 2 FFT copy ring, 4 self-test); "
                 "the outputs of the calls since the last check are not valid",
                 timeout_bits);
        return pusch::sfail(PUSCH_ERR_TIMEOUT, pusch::g_msg);
    }
    if (st[0] & (PUSCH_STATUS_PIVOT | PUSCH_STATUS_NONFINITE)) {
        snprintf(pusch::g_msg, sizeof pusch::g_msg,
                 "detection: %u factorisation(s) met a pivot that is not a positive finite number (first at index "
                 "%u)%s",
                 st[1], st[2], (st[0] & PUSCH_STATUS_NONFINITE) ? "; a detected symbol is not finite" : "");
        return pusch::sfail(PUSCH_ERR_NUMERIC, pusch::g_msg);
    }
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_selftest_wait(pusch_handle *h, unsigned limit_us, void *stream) {
    if (!h) return pusch::sfail(PUSCH_ERR_ARG, "pusch_selftest_wait: handle is NULL");
    if (limit_us < 1u || limit_us > 1000000u)
        return pusch::sfail(PUSCH_ERR_ARG, "pusch_selftest_wait: limit_us out of [1, 1000000]");
    pusch::selftest_wait_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(h->kernel_err,
                                                                                 1000ull * limit_us);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(pusch::g_msg, sizeof pusch::g_msg, "pusch_selftest_wait launch: %s", cudaGetErrorString(e));
        return pusch::sfail(PUSCH_ERR_CUDA, pusch::g_msg);
    }
    pusch::set_last_error("");
    return PUSCH_OK;
}

}  // extern "C"
