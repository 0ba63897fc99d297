// Non-step kernels of libmclbm (initial fill, streaming-only test hook, fields, reductions,
// state copies), templated on the storage element type, and the host-side dispatch by
// storage type. The step kernels are in mclbm_device.cuh / mclbm_step_*.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "mclbm_device.cuh"

namespace mcl {

// ---- streaming only (test hook) -------------------------------------------------------------
template <class T>
__global__ void stream_only_kernel(const T* __restrict__ src, T* __restrict__ dst, const Layout L,
                                   float s) {
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<T, true>(src, L, i, j, fw, fp, g, s);
    const size_t o = (size_t)j * L.pitch + i;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      dst[(size_t)q * L.plane + o] = Elem<T>::put(fw[q]);
      dst[(size_t)(kQ + q) * L.plane + o] = Elem<T>::put(fp[q]);
      dst[(size_t)(2 * kQ + q) * L.plane + o] = Elem<T>::put(g[q]);
    }
    if (L.np == kPlanes2) {  // g^p
      pull_thermal<T>(src, L, i, j, 3 * kQ, g, s);
#pragma unroll
      for (int q = 0; q < kQ; ++q) dst[(size_t)(3 * kQ + q) * L.plane + o] = Elem<T>::put(g[q]);
    }
  }
}

// ---- initial equilibrium (Eqs 26-27) ---------------------------------------------------------
template <class T>
__global__ void init_kernel(T* __restrict__ dst, const Layout L, const StepConsts k,
                            const float* __restrict__ warm, int warm_rho) {
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    // FP64 here (once per run) so that the stored values are correctly rounded
    double ux = 0.0, uy = 0.0, th, drw = 0.0, drp = 0.0;
    if (warm) {
      ux = warm[t];
      uy = warm[n + t];
      th = warm[2 * n + t];
      const double phi = warm[3 * n + t];
      // rho^w = 1 - phi (or the caller's rho^w field), rho^p = phi rho_f / rho_p, as
      // deviations from the initial values
      drw = (warm_rho ? (double)warm[4 * n + t] : 1.0 - phi) - k.rho_w0_d;
      drp = phi / k.fr_d - k.rho_p0_d;
    } else {
      th = 0.5 - ((double)i + 0.5) / (double)L.nx;
    }
    const double dth = th - (0.5 - ((double)i + 0.5) / (double)L.nx);
    const double rw = k.rho_w0_d + drw, rp = k.rho_p0_d + drp;
    const double usq = 1.5 * (ux * ux + uy * uy);
    const size_t o = (size_t)j * L.pitch + i;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const double eu = (double)ex(q) * ux + (double)ey(q) * uy;
      const double P = eu * (3.0 + 4.5 * eu) - usq;
      const double W = q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
      dst[(size_t)q * L.plane + o] = Elem<T>::put((float)(W * (drw + rw * P)));
      dst[(size_t)(kQ + q) * L.plane + o] = Elem<T>::put((float)(W * (drp + rp * P)));
      dst[(size_t)(2 * kQ + q) * L.plane + o] = Elem<T>::put((float)(W * (dth + th * P)));
      if (L.np == kPlanes2)
        dst[(size_t)(3 * kQ + q) * L.plane + o] = Elem<T>::put((float)(W * (dth + th * P)));
    }
  }
}

// ---- macroscopic fields of the post-stream state ----------------------------------------------
// thp: the particles' thermal set's deviation (= m.th with one set); v[kFields].
__device__ __forceinline__ void node_fields(const StepConsts& k, const Moments& m, float thp,
                                            int i, float* v) {
  const float rw = k.rho_w0 + m.rw, rp = k.rho_p0 + m.rp;
  const float rho = rw + rp;
  const float tc = theta_c(k, i);
  v[0] = (m.mwx + m.mpx) / rho;
  v[1] = (m.mwy + m.mpy) / rho;
  v[2] = tc + (k.two_sets ? mixture_dev(k, rw, rp, m.th, thp) : m.th);
  v[8] = tc + m.th;
  v[9] = tc + thp;
  v[3] = rp * k.phi_per_rho_p;
  v[4] = rw;
  v[5] = rp;
  const bool has_p = k.has_p && rp > 1e-30f;
  v[6] = has_p ? m.mpx / rp : m.mwx / rw;
  v[7] = has_p ? m.mpy / rp : m.mwy / rw;
}

template <class T>
__global__ void fields_kernel(const T* __restrict__ src, const Layout L, const StepConsts k,
                              uint32_t which, float* __restrict__ out) {
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<T, true>(src, L, i, j, fw, fp, g, k.inv_nx);
    const Moments m = moments_of(fw, fp, g);
    float thp = m.th;
    if (k.two_sets) {
      pull_thermal<T>(src, L, i, j, 3 * kQ, g, k.inv_nx);
      thp = sum9(g);
    }
    float v[kFields];
    node_fields(k, m, thp, i, v);
    int slot = 0;
#pragma unroll
    for (int b = 0; b < kFields; ++b)
      if (which & (1u << b)) out[(int64_t)(slot++) * n + t] = v[b];
  }
}

// ---- deterministic FP64 block reduction -------------------------------------------------------
template <int N>
__device__ __forceinline__ void block_reduce_store(double (&acc)[N], double* out) {
  __shared__ double s[32][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < N; ++c)
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], off);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < N; ++c) s[warp][c] = acc[c];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < N; ++c) {
      double v = lane < nw ? s[lane][c] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) out[c] = v;
    }
  }
}

// Sums `count` partial rows of kRedWidth doubles in a fixed order into red[0..kRedWidth).
__global__ void final_reduce_kernel(const double* __restrict__ partials, int count,
                                    double* __restrict__ red) {
  double acc[kRedWidth];
#pragma unroll
  for (int c = 0; c < kRedWidth; ++c) acc[c] = 0.0;
  for (int r = threadIdx.x; r < count; r += blockDim.x)
#pragma unroll
    for (int c = 0; c < kRedWidth; ++c) acc[c] += partials[(size_t)r * kRedWidth + c];
  block_reduce_store<kRedWidth>(acc, red);
}

// Wall gradients from the theta deviations (the Eq 33 mixture's with two sets): with
// theta = theta_c + theta', (8 T_h - 9 theta_0 + theta_1)/3 = 1/nx + (theta'_1 - 9 theta'_0)/3
// and the cold-wall twin (9 theta_{n-1} - theta_{n-2} - 8 T_c)/3
// = 1/nx + (9 theta'_{n-1} - theta'_{n-2})/3.
template <class T>
__global__ void nusselt_kernel(const T* __restrict__ src, const Layout L, const StepConsts k,
                               double* __restrict__ red) {
  const float s = k.inv_nx;
  // the (mixture) temperature's deviation from theta_c at node (i, j) after streaming
  auto dev = [&](int i, int j) -> float {
    float fw[kQ], fp[kQ], g[kQ];
    if (!k.two_sets) {
      pull_node<T, false>(src, L, i, j, fw, fp, g, s);
      return sum9(g);
    }
    pull_node<T, true>(src, L, i, j, fw, fp, g, s);
    const float dw = sum9(g);
    pull_thermal<T>(src, L, i, j, 3 * kQ, g, s);
    return mixture_dev(k, k.rho_w0 + sum9(fw), k.rho_p0 + sum9(fp), dw, sum9(g));
  };
  double acc[2] = {0.0, 0.0};
  for (int j = threadIdx.x; j < L.ny; j += blockDim.x) {
    const double t0 = dev(0, j);
    const double t1 = dev(1, j);
    const double c0 = dev(L.nx - 1, j);
    const double c1 = dev(L.nx - 2, j);
    const double slope = 1.0 / (double)L.nx;
    acc[0] += slope + (t1 - 9.0 * t0) / 3.0;
    acc[1] += slope + (9.0 * c0 - c1) / 3.0;
  }
  block_reduce_store<2>(acc, red);
}

template <class T>
__global__ void mass_kernel(const T* __restrict__ src, const Layout L,
                            double* __restrict__ partials) {
  double acc[kRedWidth];
#pragma unroll
  for (int c = 0; c < kRedWidth; ++c) acc[c] = 0.0;
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    const size_t o = (size_t)j * L.pitch + i;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      acc[0] += (double)Elem<T>::ldg(src + (size_t)q * L.plane + o);
      acc[1] += (double)Elem<T>::ldg(src + (size_t)(kQ + q) * L.plane + o);
    }
  }
  block_reduce_store<kRedWidth>(acc, partials + (size_t)blockIdx.x * kRedWidth);
}

template <class T>
__global__ void residual_kernel(const T* __restrict__ src, const Layout L, const StepConsts k,
                                float* __restrict__ snap, int sums,
                                double* __restrict__ partials) {
  double acc[kRedWidth];
#pragma unroll
  for (int c = 0; c < kRedWidth; ++c) acc[c] = 0.0;
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<T, true>(src, L, i, j, fw, fp, g, k.inv_nx);
    const Moments m = moments_of(fw, fp, g);
    float thp = m.th;
    if (k.two_sets) {
      pull_thermal<T>(src, L, i, j, 3 * kQ, g, k.inv_nx);
      thp = sum9(g);
    }
    float v[kFields];
    node_fields(k, m, thp, i, v);
    if (sums) {
      const double now[4] = {v[0], v[1], v[2], v[3]};
      double d[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) d[f] = now[f] - (double)snap[f * n + t];
      acc[0] += d[0] * d[0] + d[1] * d[1];
      acc[1] += now[0] * now[0] + now[1] * now[1];
      acc[2] += d[2] * d[2];
      acc[3] += now[2] * now[2];
      acc[4] += d[3] * d[3];
      acc[5] += now[3] * now[3];
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) snap[f * n + t] = v[f];
  }
  if (sums) block_reduce_store<kRedWidth>(acc, partials + (size_t)blockIdx.x * kRedWidth);
}

template <class T>
__global__ void state_copy_kernel(const void* __restrict__ src_v, void* __restrict__ dst_v,
                                  const Layout L, int to_packed) {
  const int64_t n = (int64_t)L.nx * L.ny;
  const int64_t total = n * L.np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / n, r = t % n;
    const int i = (int)(r % L.nx), j = (int)(r / L.nx);
    const size_t po = (size_t)p * L.plane + (size_t)j * L.pitch + i;
    if (to_packed)
      static_cast<float*>(dst_v)[t] = Elem<T>::get(static_cast<const T*>(src_v)[po]);
    else
      static_cast<T*>(dst_v)[po] = Elem<T>::put(static_cast<const float*>(src_v)[t]);
  }
}

__global__ void epoch_advance_kernel(uint32_t* epoch) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *epoch += 1u;
}

// ---- launchers ------------------------------------------------------------------------------
namespace {
int grid_for(int64_t n, int block, int cap) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}
}  // namespace

// Calls f.template operator()<T>() with T the element type of the storage.
template <class F>
cudaError_t by_storage(int storage, F&& f) {
  switch (storage) {
    case MCLBM_STORE_F32:
      return f((float*)nullptr);
    case MCLBM_STORE_F16:
      return f((__half*)nullptr);
    case MCLBM_STORE_BF16:
      return f((__nv_bfloat16*)nullptr);
    default:
      return cudaErrorInvalidValue;
  }
}

StepConfig choose_step_config(int nx, int ny, int np) {
  StepConfig c;
  // default: TMA-staged tiles for lattices with a few tiles per SM, the plain tile kernel below.
  // MCLBM_STEP_VARIANT = tile | tma overrides (diagnostics and comparisons).
  c.variant = (nx >= 64 && ny >= 32) ? 2 : 0;
  const char* v = std::getenv("MCLBM_STEP_VARIANT");
  if (v && std::strcmp(v, "tile") == 0) c.variant = 0;
  if (v && (std::strcmp(v, "tma") == 0 || std::strcmp(v, "two") == 0)) c.variant = 2;
  c.grid = 0;
  c.sr = true;
  c.two = false;
  c.grid2 = 0;
  // MCLBM_STEP_VEC = 1 | 2 forces the nodes per thread (comparisons; default by lattice size)
  const char* vv = std::getenv("MCLBM_STEP_VEC");
  c.vec = (vv && (vv[0] == '1' || vv[0] == '2') && vv[1] == 0) ? vv[0] - '0' : 0;
  // MCLBM_STEP_TILE_H = 8 | 7 forces the TMA kernel's tile height with one node per thread
  // (comparisons; default: 7 where 32 x 8 tiles would leave some SMs with a second tile and
  // 32 x 7 tiles fit two per SM)
  const char* th = std::getenv("MCLBM_STEP_TILE_H");
  c.th = th && std::strcmp(th, "8") == 0 ? 8 : (th && std::strcmp(th, "7") == 0 ? 7 : 0);
  if (np != kPlanes) {  // two thermal sets: the plain tile kernel, one node per thread
    c.variant = 0;
    c.vec = 1;
  }
  return c;
}

cudaError_t prepare_step(StepConfig* c, const Layout& L) {
  if (c->variant != 2) return cudaSuccess;
  switch (L.storage) {
    case MCLBM_STORE_F32:
      return prepare_tma_f32(c, L);
    case MCLBM_STORE_F16:
      return prepare_tma_f16(c, L);
    case MCLBM_STORE_BF16:
      return prepare_tma_bf16(c, L);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                        cudaStream_t st) {
  switch (a.L.storage) {
    case MCLBM_STORE_F32:
      return launch_step_f32(a, c, map, st);
    case MCLBM_STORE_F16:
      return launch_step_f16(a, c, map, st);
    case MCLBM_STORE_BF16:
      return launch_step_bf16(a, c, map, st);
    default:
      return cudaErrorInvalidValue;
  }
}

int step_tile_width(const StepConfig&) { return 32; }

// maps[0]: window loads (box = window); maps[1]: output tile stores (box = tile).
cudaError_t make_state_tensor_map(CUtensorMap* maps, void* state0, const Layout& L, int tile_w,
                                  int tile_h) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMapDataType dt;
  switch (L.storage) {
    case MCLBM_STORE_F32:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
      break;
    case MCLBM_STORE_F16:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
      break;
    case MCLBM_STORE_BF16:
      dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if ((tile_w != 32 && tile_w != 64) || (tile_h != 8 && tile_h != 7)) return cudaErrorInvalidValue;
  const int wx = tile_w + 2 * (16 / L.elem);  // 16 bytes of halo columns on each side
  const cuuint64_t dims[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, (cuuint64_t)(2 * kPlanes)};
  const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * L.elem, (cuuint64_t)L.plane * L.elem};
  const cuuint32_t box[3] = {(cuuint32_t)wx, (cuuint32_t)(tile_h + 4), (cuuint32_t)kPlanes};
  const cuuint32_t tile[3] = {(cuuint32_t)tile_w, (cuuint32_t)tile_h, (cuuint32_t)kPlanes};
  const cuuint32_t elem[3] = {1, 1, 1};
  CUresult r = encode(&maps[0], dt, 3, state0, dims, strides, box, elem,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  r = encode(&maps[1], dt, 3, state0, dims, strides, tile, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_two_step_tensor_map(CUtensorMap* map, void* state0, const Layout& L) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if (L.storage != MCLBM_STORE_F32 || L.np != kPlanes) return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, (cuuint64_t)(2 * kPlanes)};
  const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4, (cuuint64_t)L.plane * 4};
  const cuuint32_t box[3] = {32 + 2 * 4, 16 + 2 * 4, (cuuint32_t)kPlanes};
  const cuuint32_t elem[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, state0, dims, strides, box,
                            elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_epoch_advance(uint32_t* epoch, cudaStream_t st) {
  epoch_advance_kernel<<<1, 32, 0, st>>>(epoch);
  return cudaGetLastError();
}

cudaError_t launch_stream_only(const void* src, void* dst, const Layout& L, const StepConsts& k,
                               cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    stream_only_kernel<T><<<grid_for(n, 256, 4096), 256, 0, st>>>(
        static_cast<const T*>(src), static_cast<T*>(dst), L, k.inv_nx);
    return cudaGetLastError();
  });
}

cudaError_t launch_init(void* dst, const Layout& L, const StepConsts& k, const float* warm,
                        int warm_rho, cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    init_kernel<T><<<grid_for(n, 256, 4096), 256, 0, st>>>(static_cast<T*>(dst), L, k, warm,
                                                            warm_rho);
    return cudaGetLastError();
  });
}

cudaError_t launch_fields(const void* src, const Layout& L, const StepConsts& k, uint32_t which,
                          float* out, cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    fields_kernel<T><<<grid_for(n, 256, 4096), 256, 0, st>>>(static_cast<const T*>(src), L, k,
                                                              which, out);
    return cudaGetLastError();
  });
}

cudaError_t launch_nusselt(const void* src, const Layout& L, const StepConsts& k, double* red,
                           cudaStream_t st) {
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    nusselt_kernel<T><<<1, 256, 0, st>>>(static_cast<const T*>(src), L, k, red);
    return cudaGetLastError();
  });
}

cudaError_t launch_mass(const void* src, const Layout& L, double* partials, double* red,
                        cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  const int g = grid_for(n, 256, kMaxRedBlocks);
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    mass_kernel<T><<<g, 256, 0, st>>>(static_cast<const T*>(src), L, partials);
    final_reduce_kernel<<<1, 256, 0, st>>>(partials, g, red);
    return cudaGetLastError();
  });
}

cudaError_t launch_residual(const void* src, const Layout& L, const StepConsts& k, float* snap,
                            bool sums, double* partials, double* red, cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  const int g = grid_for(n, 256, kMaxRedBlocks);
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    residual_kernel<T><<<g, 256, 0, st>>>(static_cast<const T*>(src), L, k, snap, sums ? 1 : 0,
                                           partials);
    if (sums) final_reduce_kernel<<<1, 256, 0, st>>>(partials, g, red);
    return cudaGetLastError();
  });
}

cudaError_t launch_state_copy(const void* src, void* dst, const Layout& L, bool to_packed,
                              cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny * L.np;
  return by_storage(L.storage, [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    state_copy_kernel<T><<<grid_for(n, 256, 8192), 256, 0, st>>>(src, dst, L, to_packed ? 1 : 0);
    return cudaGetLastError();
  });
}

}  // namespace mcl
