// selftest.cu -- check of the bounded-wait path that every TMA-staged step
// kernel relies on: a wait on an mbarrier that nothing ever completes must
// give up after its limit, report the timeout to the host, and leave the
// context usable.  No fault, trap or endless loop is involved.
#include <cuda_runtime.h>

#include <string>

#include "pact.h"
#include "tma.cuh"

void pact_note_error(const std::string& msg);

namespace {

__global__ void k_wait_probe(unsigned long long limit_ns, int* timed_out) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // nothing arrives on the barrier, so its phase 0 never completes
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(timed_out, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&bar);
}

}  // namespace

extern "C" int pact_check_bounded_wait(unsigned int limit_us, void* stream) {
    if (limit_us < 1 || limit_us > 2000000) {
        pact_note_error("pact_check_bounded_wait: limit_us must be in [1, 2e6]");
        return PACT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int* flag = nullptr;
    int host = 0;
    if (cudaMallocAsync(&flag, sizeof(int), st) != cudaSuccess) {
        pact_note_error("pact_check_bounded_wait: allocation failed");
        return PACT_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 128, 0, st>>>(1000ull * limit_us, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(flag, st);
    if (e != cudaSuccess) {
        pact_note_error(std::string("pact_check_bounded_wait: ") + cudaGetErrorString(e));
        return PACT_ECUDA;
    }
    if (host) {
        pact_note_error("pact_check_bounded_wait: the wait gave up after its limit (expected)");
        return PACT_ETIMEOUT;
    }
    return PACT_OK;
}
