// mclbm_mass_noalloc: the component-mass reduction for callers that cannot allocate device
// memory. It reads a caller-owned population array and keeps its FP64 partial sums in a
// file-scope static device array instead of memory obtained from cudaMalloc or from a bound
// buffer. No other entry point uses this file.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mclbm_internal.h"

namespace {

// Largest ny the static scratch can serve: one FP64 pair of partial sums per lattice row.
constexpr int kNoallocMaxRows = 8192;
constexpr int kNoallocMaxCols = 32768;
constexpr int kNoallocDevices = 64;

// Scratch shared by every call on a device: [kNoallocMaxRows][2] row sums, then the [2] total.
// 128 KiB per device, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxRows + 2];

// One CTA per row (grid-stride over rows): FP64 sums of the f^w and f^p deviation planes of
// row j, written (not accumulated) to scratch[2j], scratch[2j+1].
__global__ void noalloc_row_sums(const float* __restrict__ st, int nx, int ny,
                                 double* __restrict__ scratch) {
  __shared__ double s[32][2];
  const size_t n = (size_t)nx * ny;
  for (int j = blockIdx.x; j < ny; j += gridDim.x) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const size_t o = (size_t)j * nx + i;
      for (int q = 0; q < mcl::kQ; ++q) {
        a += (double)st[(size_t)q * n + o];
        b += (double)st[(size_t)(mcl::kQ + q) * n + o];
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      b += __shfl_down_sync(0xffffffffu, b, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      s[warp][0] = a;
      s[warp][1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ra = 0.0, rb = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        ra += s[w][0];
        rb += s[w][1];
      }
      scratch[2 * j] = ra;
      scratch[2 * j + 1] = rb;
    }
    __syncthreads();
  }
}

// One CTA: thread t sums rows t, t + 256, ... in order, then a fixed-order tree; the total
// goes to scratch[2 * kNoallocMaxRows], scratch[2 * kNoallocMaxRows + 1]. Deterministic.
__global__ void noalloc_total(int ny, double* __restrict__ scratch) {
  __shared__ double s[256][2];
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    a += scratch[2 * j];
    b += scratch[2 * j + 1];
  }
  s[threadIdx.x][0] = a;
  s[threadIdx.x][1] = b;
  __syncthreads();
  for (int half = blockDim.x / 2; half > 0; half >>= 1) {
    if ((int)threadIdx.x < half) {
      s[threadIdx.x][0] += s[threadIdx.x + half][0];
      s[threadIdx.x][1] += s[threadIdx.x + half][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * kNoallocMaxRows] = s[0][0];
    scratch[2 * kNoallocMaxRows + 1] = s[0][1];
  }
}

// Device address of g_noalloc_scratch, looked up once per device with that device current.
// In host code the symbol name is only a host-side stand-in and must not be passed to a kernel.
std::mutex g_setup_mutex;
double* g_scratch_ptr[kNoallocDevices] = {nullptr};

cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int mclbm_mass_noalloc(const float* state_dev, int nx, int ny, double rho_w0,
                                  double rho_p0, double* mass_w, double* mass_p,
                                  void* cuda_stream) {
  if (!state_dev || !mass_w || !mass_p || nx < 2 || ny < 2) return MCLBM_EINVAL;
  if (ny > kNoallocMaxRows || nx > kNoallocMaxCols) return MCLBM_ETOOLARGE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return MCLBM_ECUDA;
  const int grid = ny < 1024 ? ny : 1024;
  noalloc_row_sums<<<grid, 256, 0, st>>>(state_dev, nx, ny, scratch);
  noalloc_total<<<1, 256, 0, st>>>(ny, scratch);
  if (cudaGetLastError() != cudaSuccess) return MCLBM_ECUDA;
  double tot[2];
  if (cudaMemcpyAsync(tot, scratch + 2 * kNoallocMaxRows, sizeof(tot), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess)
    return MCLBM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MCLBM_ECUDA;
  const double nodes = (double)nx * (double)ny;
  *mass_w = tot[0] + nodes * rho_w0;
  *mass_p = tot[1] + nodes * rho_p0;
  if (!std::isfinite(*mass_w) || !std::isfinite(*mass_p)) return MCLBM_EDIVERGED;
  return MCLBM_OK;
}
