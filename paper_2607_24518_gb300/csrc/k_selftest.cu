// Self-test of the bounded device waits: one thread waits, with the same
// bounded mbarrier wait the tensor-core kernels use, on a barrier that no
// one will complete.  The wait gives up after the given limit and the
// kernel records the error code the production kernels record, so a test
// can check that a wait that runs out reaches the host as a status and
// leaves the context usable.
#include "../../include/symnmf.h"
#include "tc_ptx.cuh"

namespace symnmf {
namespace {

using namespace tc;

__global__ void wait_selftest_kernel(uint64_t limit_ns, int *err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  // phase 0 never completes: nothing arrives
  if (!mbar_wait(&bar, 0u, reinterpret_cast<volatile int *>(&abort_flag), limit_ns))
    set_err(err, 99);
}

}  // namespace
}  // namespace symnmf

extern "C" int symnmf_selftest_wait_timeout(double limit_s) {
  if (!(limit_s > 0) || limit_s > 10.0) return SYMNMF_ERR_INVALID;
  int *derr = nullptr;
  int herr = 0;
  if (cudaMalloc((void **)&derr, sizeof(int)) != cudaSuccess) return SYMNMF_ERR_CUDA;
  cudaError_t e = cudaMemset(derr, 0, sizeof(int));
  if (e == cudaSuccess) {
    symnmf::wait_selftest_kernel<<<1, 32>>>((uint64_t)(limit_s * 1e9), derr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(derr);
  if (e != cudaSuccess) return SYMNMF_ERR_CUDA;
  return herr == 99 ? SYMNMF_ERR_TIMEOUT : SYMNMF_OK;
}
