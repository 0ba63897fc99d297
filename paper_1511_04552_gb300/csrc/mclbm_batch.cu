// Batched stepping of many cavities in one persistent launch per time step (the parametric
// sweep: cavities of different sizes, Rayleigh numbers, volume fractions and particle sizes).
// A tile table lists the 64 x 8 tiles of every active cavity; the persistent CTAs walk it
// exactly like the single-cavity TMA kernel walks one cavity (the same tile loop), reading each
// tile's cavity arguments and tensor maps from device memory. A batched reduction gives every cavity's
// Nusselt numbers in one launch. The autotuner times a few tile orders and grid sizes.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "mclbm_pair.cuh"

namespace mcl {
static_assert(pair::kTY == kTmaTY && kBatchTileH == kTmaTY,
              "the tile table, the tensor maps and the kernels share the tile height");

// Tile table entry: cavity (10 bits) | tile column (11 bits) | tile row (11 bits).
__host__ __device__ constexpr uint32_t pack_tile(int c, int tx, int ty) {
  return ((uint32_t)c << 22) | ((uint32_t)tx << 11) | (uint32_t)ty;
}
__device__ __forceinline__ int tile_cav(uint32_t e) { return (int)(e >> 22); }
__device__ __forceinline__ int tile_x(uint32_t e) { return (int)((e >> 11) & 2047u); }
__device__ __forceinline__ int tile_y(uint32_t e) { return (int)(e & 2047u); }

// One time step of every tile in the table: the single-cavity TMA tile loop (two nodes per
// thread, one window per CTA reloaded as soon as the pulls have read it), with each tile's
// tensor maps, layout, constants and destination level taken from its cavity's entry.
template <class T, bool SR, bool ALLF>
__global__ void __launch_bounds__(pair::Threads<2, kBatchTileW>::value,
                                  pair::MinBlocks<2, kBatchTileW>::value)
    step_batch_kernel(const BatchCav* __restrict__ cavs, const uint32_t* __restrict__ tiles,
                      int n_tiles, int parity, uint32_t seed, const uint32_t* epoch, int* err) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  uint32_t sh = 0u;
  if (SR) {
    const uint32_t ep = epoch ? *(volatile const uint32_t*)epoch : 0u;
    sh = mix32(seed ^ mix32(ep + 0x632BE5ABu));
  }
  // the source level of cavity c this launch: its level at batch creation, flipped on odd
  // launches
  auto tile_of = [&](int tile) {
    const uint32_t e = tiles[tile];
    const int c = tile_cav(e);
    const BatchCav& cv = cavs[c];
    const int from = cv.cur ^ parity;
    return pair::TmaTileDesc{&cv.map, &cv.map_out, from * kPlanes, (from ^ 1) * kPlanes,
                             tile_x(e) * kBatchTileW, tile_y(e) * pair::kTY, cv.L, cv.k,
                             cv.level[from ^ 1], sh ^ ((uint32_t)c << 24)};
  };
  pair::tma_tile_loop<T, SR, ALLF, 2, kBatchTileW, pair::kTY>(tile_of, n_tiles, err);
}

// Nusselt sums of every cavity: block c reduces cavity c (the same sums as nusselt_kernel).
template <class T>
__global__ void batch_nusselt_kernel(const BatchCav* __restrict__ cavs, int parity,
                                     double* __restrict__ out) {
  const BatchCav& cv = cavs[blockIdx.x];
  const Layout L = cv.L;
  const T* src = static_cast<const T*>(cv.level[cv.cur ^ parity]);
  const float s = cv.k.inv_nx;
  double acc[2] = {0.0, 0.0};
  for (int j = threadIdx.x; j < L.ny; j += blockDim.x) {
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<T, false>(src, L, 0, j, fw, fp, g, s);
    const double t0 = sum9(g);
    pull_node<T, false>(src, L, 1, j, fw, fp, g, s);
    const double t1 = sum9(g);
    pull_node<T, false>(src, L, L.nx - 1, j, fw, fp, g, s);
    const double c0 = sum9(g);
    pull_node<T, false>(src, L, L.nx - 2, j, fw, fp, g, s);
    const double c1 = sum9(g);
    const double slope = 1.0 / (double)L.nx;
    acc[0] += slope + (t1 - 9.0 * t0) / 3.0;
    acc[1] += slope + (9.0 * c0 - c1) / 3.0;
  }
  __shared__ double sm[8][2];
  for (int c = 0; c < 2; ++c)
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sm[warp][0] = acc[0];
    sm[warp][1] = acc[1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
      a += sm[w2][0];
      b += sm[w2][1];
    }
    out[2 * blockIdx.x] = a;
    out[2 * blockIdx.x + 1] = b;
  }
}

namespace {
template <class T, bool SR, bool ALLF>
cudaError_t launch_batch_t3(const BatchLaunch& b, int parity, uint32_t seed, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(b.grid);
  cfg.blockDim = dim3(pair::Threads<2, kBatchTileW>::value);
  cfg.dynamicSmemBytes = pair::TmaPair<T, 2, kBatchTileW>::SMEM;
  return cudaLaunchKernelEx(&cfg, step_batch_kernel<T, SR, ALLF>,
                            (const BatchCav*)b.cavs, (const uint32_t*)b.tiles, b.n_tiles, parity,
                            seed, (const uint32_t*)b.epoch, b.err);
}

template <class T>
cudaError_t launch_batch_t(const BatchLaunch& b, int parity, uint32_t seed, cudaStream_t st) {
  const bool sr = b.sr && sizeof(T) == 2;
  if (sr)
    return b.all_forces ? launch_batch_t3<T, true, true>(b, parity, seed, st)
                        : launch_batch_t3<T, true, false>(b, parity, seed, st);
  return b.all_forces ? launch_batch_t3<T, false, true>(b, parity, seed, st)
                      : launch_batch_t3<T, false, false>(b, parity, seed, st);
}

template <class T>
cudaError_t prepare_batch_t(int* per_sm) {
  const size_t smem = pair::TmaPair<T, 2, kBatchTileW>::SMEM;
  const void* fns[4] = {(const void*)step_batch_kernel<T, false, false>,
                        (const void*)step_batch_kernel<T, false, true>,
                        (const void*)step_batch_kernel<T, true, false>,
                        (const void*)step_batch_kernel<T, true, true>};
  cudaError_t e;
  for (const void* fn : fns)
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_batch_kernel<T, true, true>,
                                                    pair::Threads<2, kBatchTileW>::value, smem);
  if (e == cudaSuccess && *per_sm > pair::MinBlocks<2, kBatchTileW>::value)
    *per_sm = pair::MinBlocks<2, kBatchTileW>::value;
  return e;
}
}  // namespace

cudaError_t launch_batch_step(const BatchLaunch& b, int parity, uint32_t seed, cudaStream_t st) {
  if (b.n_tiles < 1) return cudaSuccess;
  switch (b.storage) {
    case MCLBM_STORE_F32:
      return launch_batch_t<float>(b, parity, seed, st);
    case MCLBM_STORE_F16:
      return launch_batch_t<__half>(b, parity, seed, st);
    case MCLBM_STORE_BF16:
      return launch_batch_t<__nv_bfloat16>(b, parity, seed, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_nusselt(const BatchLaunch& b, int n_cav, int parity, double* out,
                                 cudaStream_t st) {
  switch (b.storage) {
    case MCLBM_STORE_F32:
      batch_nusselt_kernel<float><<<n_cav, 256, 0, st>>>((const BatchCav*)b.cavs, parity, out);
      break;
    case MCLBM_STORE_F16:
      batch_nusselt_kernel<__half><<<n_cav, 256, 0, st>>>((const BatchCav*)b.cavs, parity, out);
      break;
    case MCLBM_STORE_BF16:
      batch_nusselt_kernel<__nv_bfloat16>
          <<<n_cav, 256, 0, st>>>((const BatchCav*)b.cavs, parity, out);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t prepare_batch(int storage, int* per_sm) {
  switch (storage) {
    case MCLBM_STORE_F32:
      return prepare_batch_t<float>(per_sm);
    case MCLBM_STORE_F16:
      return prepare_batch_t<__half>(per_sm);
    case MCLBM_STORE_BF16:
      return prepare_batch_t<__nv_bfloat16>(per_sm);
    default:
      return cudaErrorInvalidValue;
  }
}

// Tile tables for the autotuner's orders. order 0: cavity by cavity in the given order;
// 1: largest cavity first; 2: tiles of all cavities interleaved round-robin (neighbouring
// CTAs work on different cavities at the same time).
void build_tile_table(const std::vector<int>& nx, const std::vector<int>& ny,
                      const std::vector<int>& active, int order, std::vector<uint32_t>* out) {
  out->clear();
  std::vector<int> ids;
  for (size_t c = 0; c < nx.size(); ++c)
    if (active[c]) ids.push_back((int)c);
  auto ntiles = [&](int c) { return ((nx[c] + kBatchTileW - 1) / kBatchTileW) * ((ny[c] + kTmaTY - 1) / kTmaTY); };
  if (order == 1)
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return ntiles(a) > ntiles(b); });
  if (order == 2) {
    std::vector<int> pos(ids.size(), 0);
    bool more = true;
    while (more) {
      more = false;
      for (size_t k = 0; k < ids.size(); ++k) {
        const int c = ids[k];
        const int tx_n = (nx[c] + kBatchTileW - 1) / kBatchTileW;
        if (pos[k] < ntiles(c)) {
          out->push_back(pack_tile(c, pos[k] % tx_n, pos[k] / tx_n));
          ++pos[k];
          more = true;
        }
      }
    }
    return;
  }
  for (int c : ids) {
    const int tx_n = (nx[c] + kBatchTileW - 1) / kBatchTileW, ty_n = (ny[c] + kTmaTY - 1) / kTmaTY;
    for (int y = 0; y < ty_n; ++y)
      for (int x = 0; x < tx_n; ++x) out->push_back(pack_tile(c, x, y));
  }
}

}  // namespace mcl
