// Self-test of the failure-detection path: a kernel waits, with the step kernels' own bounded
// mbarrier wait, on a barrier that nothing ever arrives on, so the wait must give up after its
// limit (about 2 s) and the kernel must return normally with the give-up recorded. No fault,
// trap or hang is involved: the context stays usable.
#include <cuda_runtime.h>

#include <chrono>

#include "mclbm_device.cuh"

namespace {

__device__ int g_selftest_status;  // 0 not run, 1 the wait completed (wrong), 2 it gave up

__global__ void wait_gives_up_kernel() {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    const uint32_t b = mcl::tma::smem_u32(&bar);
    mcl::tma::mbar_init(b, 1);
    mcl::tma::fence_barrier_init();
    g_selftest_status = mcl::tma::mbar_wait(b, 0) ? 1 : 2;
  }
}

}  // namespace

extern "C" int mclbm_selftest_wait_timeout(void* cuda_stream, double* seconds) {
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_selftest_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice,
                              st) != cudaSuccess)
    return MCLBM_ECUDA;
  const auto t0 = std::chrono::steady_clock::now();
  wait_gives_up_kernel<<<1, 32, 0, st>>>();
  if (cudaGetLastError() != cudaSuccess) return MCLBM_ECUDA;
  int status = 0;
  if (cudaMemcpyFromSymbolAsync(&status, g_selftest_status, sizeof(int), 0,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MCLBM_ECUDA;
  if (seconds)
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status == 2 ? MCLBM_ETIMEOUT : MCLBM_ECUDA;
}
