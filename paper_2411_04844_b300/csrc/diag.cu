// dgr_test_bounded_wait: checks the failure detection of the library's
// asynchronous kernels without faulting or hanging the GPU.  Every kernel that
// waits for bulk copies or tensor-core MMAs waits on an mbarrier with a
// bounded number of polls (mbar_wait); when the limit runs out it ORs
// DGR_STATUS_TIMEOUT into the status word and returns, so the host reads the
// failure and the context stays usable.  This entry point makes such a wait
// run out on purpose: one CTA waits on an mbarrier that nothing ever arrives
// at (no copy or MMA is issued, so nothing is in flight when it gives up).
// The paper has no counterpart.
#include "async_ops.cuh"
#include "dgr_internal.cuh"

namespace {

__global__ void k_wait_nothing(int polls, int *status, int *gave_up) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        dgr::mbar_init(&bar, 1);  // one arrival would complete phase 0; none comes
        dgr::fence_barrier_init();
    }
    __syncthreads();
    const bool done = dgr::mbar_wait(&bar, 0, status, polls);
    if (threadIdx.x == 0) *gave_up = done ? 0 : 1;
}

}  // namespace

extern "C" int dgr_test_bounded_wait(int polls, int *status, int *gave_up, cudaStream_t stream) {
    if (polls < 1 || polls > dgr::MBAR_POLLS || !status || !gave_up) return DGR_ERR_ARG;
    k_wait_nothing<<<1, 32, 0, stream>>>(polls, status, gave_up);
    dgr::counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}
