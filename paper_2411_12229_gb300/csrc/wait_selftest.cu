// wait_selftest.cu -- the search kernel's bounded wait, made to run out.
//
// Every wait of the search kernel on a block copy goes through
// mbar_wait_bounded (search.cuh): it gives up after its time limit and the
// kernel records SQG_STATUS_TIMEOUT instead of hanging.  A copy that never
// completes cannot be produced without faulting the GPU, so this entry
// point waits, with the same function, on an mbarrier phase that nothing
// completes (no arrival, no copy in flight): the wait must return false
// after the limit, the status word must read SQG_STATUS_TIMEOUT, and the
// context must stay usable.
#include <cuda_runtime.h>

#include "../../include/sqg.h"
#include "search.cuh"

namespace {

__global__ void wait_selftest_kernel(uint32_t *status, unsigned long long *waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) sqg::mbar_init(&bar, 1);
    sqg::fence_mbar_init();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = sqg::global_ns();
        const bool done = sqg::mbar_wait_bounded(&bar, 0u);  // phase 0 never completes
        *waited_ns = sqg::global_ns() - t0;
        *status = done ? 0u : SQG_STATUS_TIMEOUT;
    }
}

}  // namespace

extern "C" int sqg_wait_selftest(int device, uint32_t *status, uint64_t *waited_ns) {
    if (!status || !waited_ns || device < 0) return SQG_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SQG_ERR_INVALID_ARG;
    }
    int rc = SQG_OK;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 16) != cudaSuccess) {
        rc = SQG_ERR_OOM;
    } else {
        uint32_t *d_status = static_cast<uint32_t *>(buf);
        unsigned long long *d_ns = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf) + 8);
        wait_selftest_kernel<<<1, 32>>>(d_status, d_ns);
        uint32_t s = 0;
        unsigned long long ns = 0;
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&s, d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&ns, d_ns, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SQG_ERR_CUDA;
        *status = s;
        *waited_ns = ns;
        cudaFree(buf);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
