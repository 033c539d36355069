// diag.cu -- failure-detection check of the bounded device waits.
//
// One block waits, through the same time-bounded mbarrier wait that the staged
// step kernels use, on a shared-memory barrier that nothing completes and
// against which no copy is issued.  The wait gives up after kWaitLimitNs, and
// the kernel records kErrTimeout in the device error word and returns, leaving
// nothing in flight.  The host then reads the word as after any step.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.cuh"

namespace lbm {

__global__ void __launch_bounds__(32) k_wait_probe(unsigned* __restrict__ err)
{
    __shared__ alignas(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0)) atomicOr(err, kErrTimeout);
}

cudaError_t launch_wait_probe(unsigned* err, cudaStream_t s)
{
    k_wait_probe<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

}  // namespace lbm
