// Failure-path diagnostics: a forced time-out of the bounded device wait that every tensor-core
// kernel uses (tc_prims.cuh), so that the path from a wait that runs out to the status word the
// host reads is exercised without faulting, trapping or hanging the GPU.
#include "common.cuh"
#include "kernels.cuh"
#include "tc_prims.cuh"

namespace rl {

namespace {

// One warp: an mbarrier that nothing arrives on, waited for by lane 0 with the bounded wait
// (2 s on the global timer), which records RL_ERR_TIMEOUT in *status and returns.
__global__ void forced_timeout_kernel(int* status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0) mbar_wait(b, 0u, status);
    __syncwarp();
}

}  // namespace

cudaError_t launch_forced_timeout(int* status, cudaStream_t s) {
    forced_timeout_kernel<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

}  // namespace rl
