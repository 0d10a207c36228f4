// selfcheck.cu -- failure-detection check of the bounded device waits.
//
// Every copy wait in the step kernels is bounded (tma_util.cuh,
// mbar_wait_bounded): a copy that never lands makes the kernel give up, set
// the timeout status bit and return, so the host sees FLOOD_ERR_TIMEOUT and
// the CUDA context stays usable.  This kernel exercises that path without a
// fault: one thread waits on a shared-memory mbarrier that nothing arrives at.
#include <cstdint>
#include <cuda_runtime.h>

#include "tma_util.cuh"

namespace flood {

namespace {

__global__ void wait_probe_kernel(const uint64_t budget_ns, int *gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);               // one arrival expected; none is made
        fence_mbar_init();
        *gave_up = mbar_wait_bounded(&bar, 0u, budget_ns) ? 0 : 1;
    }
}

}  // namespace

cudaError_t launch_wait_probe(uint64_t budget_ns, int *gave_up, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(budget_ns, gave_up);
    return cudaGetLastError();
}

}  // namespace flood
