// Check of the failure path that every wait in the library's kernels uses:
// a bounded mbarrier wait that runs out records QADIC_E_DEVICE_TIMEOUT in the
// per-device status word (read and cleared by qadic_sync_status) and the
// kernel returns, leaving the context usable.  The wait is on a barrier that
// nothing ever arrives on, with a small poll limit: no fault, trap or hang.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace qadic {

namespace {

constexpr int kSelftestSite = 9;

__global__ void bounded_wait_kernel(uint32_t polls, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !ptx::mbar_wait(&bar, 0, polls)) record_timeout(status, kSelftestSite);
}

}  // namespace

}  // namespace qadic

using namespace qadic;

extern "C" int qadic_selftest_bounded_wait(uint32_t polls, void *stream) {
    if (polls < 1 || polls > kSpinLimit)
        return set_error(QADIC_E_INVALID, "polls outside [1, %u]", kSpinLimit);
    int *status = device_status_word();
    if (!status) return set_error(QADIC_E_CUDA, "status word unavailable");
    bounded_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(polls, status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "selftest launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}
