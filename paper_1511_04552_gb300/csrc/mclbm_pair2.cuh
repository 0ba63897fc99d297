// Two time steps per launch (FP32 storage, lattices with at most one 32 x 16 tile per SM;
// selected with MCLBM_STEP_VARIANT=two).
//
// Each launch of the one-step kernels pays a fixed part (the launch gap, the window load from
// L2, barriers and the store drain). This kernel pays it once for two steps: one TMA load
// brings the tile's 27 planes with a halo of four nodes (the second step's pulls and its
// neighbours' moments need the first step's result two nodes around the tile, which needs the
// source two nodes further out). The first step is computed on the 36 x 20 region around the
// 32 x 16 tile (Steps A1-A7 on every node of the region that lies in the cavity, populations
// kept in shared memory), the second on the tile itself, stored to the other time level. Every
// node's arithmetic is that of the one-step kernels with one node per thread (the same pulls,
// moment sums and collide), so the states are bitwise those of two single steps. Measured on
// the 256 x 256 cavity it is no faster than single steps (9.6 us per pair against 2 x 4.9 us):
// the first step's 720 nodes per 512-node tile and the serial phases of one CTA per SM cost
// what the saved launch gains.
#pragma once

#include "mclbm_pair.cuh"

namespace mcl {
namespace pair {

constexpr int k2TX = 32, k2TY = 16;                          // tile
constexpr int k2H = 4;                                       // halo of the input window
constexpr int k2WX = k2TX + 2 * k2H, k2WY = k2TY + 2 * k2H;  // 40 x 24 window
constexpr int k2RX = k2TX + 4, k2RY = k2TY + 4;              // 36 x 20: the first step's nodes
constexpr int k2MX = k2TX + 6, k2MY = k2TY + 6;              // 38 x 22: their moments
constexpr int k2BX = k2TX + 2, k2BY = k2TY + 2;              // 34 x 18: the second step's moments
constexpr int k2Threads = k2TX * k2TY;                       // one tile node per thread
constexpr uint32_t k2WinBytes = (uint32_t)kPlanes * k2WX * k2WY * 4;
constexpr uint32_t k2MidBytes = (uint32_t)kPlanes * k2RX * k2RY * 4;
constexpr uint32_t k2MomBytes = 2u * k2MX * k2MY * 4;
constexpr size_t k2Smem = (size_t)k2WinBytes + k2MidBytes + k2MomBytes;
static_assert(k2WinBytes % 128 == 0 && k2MidBytes % 16 == 0, "aligned shared-memory regions");
static_assert(k2WX * 4 % 16 == 0, "TMA rows of 16-byte multiples");

// Accessor of an FP32 shared-memory array [27][rows][WX]; base = the node's element of plane 0.
template <int WX, int WPLANE>
struct SmemAcc {
  const float* base;
  __device__ __forceinline__ float a1(int p, int dx, int dy) const {
    return base[p * WPLANE + dy * WX + dx];
  }
  __device__ __forceinline__ float2 a2(int p, int dy) const {
    return *reinterpret_cast<const float2*>(base + p * WPLANE + dy * WX);
  }
};

// The first step's output of one node into the [27][20][36] shared-memory array.
struct MidSink {
  float* base;
  __device__ __forceinline__ void operator()(int p, float v) const {
    base[p * (k2RX * k2RY)] = v;
  }
};

// Steps A2-A7 of node (i, j) at region position (dx, dy) (one node per thread), its own and its
// neighbours' theta' and rho'^p at m[(dy + OY) * MW + dx + OX], with the ghosts of the one-step
// tile body (isothermal walls: -theta'; adiabatic walls and rho^p: the node's own value).
template <bool ALLF, int MW, int OX, int OY, class Sink>
__device__ __forceinline__ void collide_node(const StepConsts& k, const Layout& L, int i, int j,
                                             int dx, int dy, const float* mth, const float* mrp,
                                             const float* fw, const float* fp, const float* g,
                                             Sink& out) {
  const int c = (dy + OY) * MW + dx + OX;
  const float th = mth[c], rp = mrp[c];
  const float thN = j + 1 < L.ny ? mth[c + MW] : th;
  const float thS = j > 0 ? mth[c - MW] : th;
  const float rpN = j + 1 < L.ny ? mrp[c + MW] : rp;
  const float rpS = j > 0 ? mrp[c - MW] : rp;
  const float thW = i > 0 ? mth[c - 1] : -th;
  const float rpW = i > 0 ? mrp[c - 1] : rp;
  const float thE = i + 1 < L.nx ? mth[c + 1] : -th;
  const float rpE = i + 1 < L.nx ? mrp[c + 1] : rp;
  collide<1, ALLF, float, false>(k, L, out, i, j, fw, fp, g, nullptr, thE, thW, thN, thS, rpE,
                                 rpW, rpN, rpS);
}

template <bool ALLF>
__global__ void __launch_bounds__(k2Threads, 1)
    step_two_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs a) {
  // programmatic dependent launch, as the one-step kernels
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  extern __shared__ __align__(128) unsigned char smem2[];
  float* win = reinterpret_cast<float*>(smem2);                           // [27][24][40]
  float* mid = reinterpret_cast<float*>(smem2 + k2WinBytes);              // [27][20][36]
  float* mth = reinterpret_cast<float*>(smem2 + k2WinBytes + k2MidBytes);  // moments
  float* mrp = mth + k2MX * k2MY;
  __shared__ __align__(8) uint64_t bar_mem;
  __shared__ int s_abort;
  const Layout L = a.L;
  const int t = threadIdx.x;
  const int tiles_x = (L.nx + k2TX - 1) / k2TX;
  const int i0 = (blockIdx.x % tiles_x) * k2TX, j0 = (blockIdx.x / tiles_x) * k2TY;
  const uint32_t bar = tma::smem_u32(&bar_mem);
  if (t == 0) {
    tma::mbar_init(bar, 1);
    tma::fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  if (t == 0) {
    tma::mbar_expect_tx(bar, k2WinBytes);
    tma::load_3d(tma::smem_u32(win), &tmap, i0 - k2H, j0 - k2H, a.z_src, bar);
  }
  if (!tma::mbar_wait(bar, 0)) s_abort = 1;  // bounded (2 s)
  __syncthreads();
  if (s_abort) {
    if (t == 0) {
      atomicOr(a.err, 1);
      tma::mbar_wait(bar, 0);  // drain the copy (bounded)
    }
    return;
  }
  using WinA = SmemAcc<k2WX, k2WX * k2WY>;
  using MidA = SmemAcc<k2RX, k2RX * k2RY>;
  // first step: theta' and rho'^p of the 38 x 22 nodes around its region
  for (int n = t; n < k2MX * k2MY; n += k2Threads) {
    const int dx = n % k2MX - 3, dy = n / k2MX - 3;
    const int i = i0 + dx, j = j0 + dy;
    if ((unsigned)i < (unsigned)L.nx && (unsigned)j < (unsigned)L.ny) {
      float hp[kQ], hg[kQ];
      pull1<false>(WinA{win + (dy + k2H) * k2WX + dx + k2H}, L, i, j, 0, nullptr, hp, hg);
      mth[n] = sum9(hg);
      mrp[n] = sum9(hp);
    }
  }
  __syncthreads();
  // first step on the 36 x 20 region, into shared memory
  for (int n = t; n < k2RX * k2RY; n += k2Threads) {
    const int dx = n % k2RX - 2, dy = n / k2RX - 2;
    const int i = i0 + dx, j = j0 + dy;
    if ((unsigned)i < (unsigned)L.nx && (unsigned)j < (unsigned)L.ny) {
      float fw[kQ], fp[kQ], g[kQ];
      pull1<true>(WinA{win + (dy + k2H) * k2WX + dx + k2H}, L, i, j, 0, fw, fp, g);
      MidSink out{mid + n};
      collide_node<ALLF, k2MX, 3, 3>(a.k, L, i, j, dx, dy, mth, mrp, fw, fp, g, out);
    }
  }
  __syncthreads();
  // second step: theta' and rho'^p of the 34 x 18 nodes around the tile
  for (int n = t; n < k2BX * k2BY; n += k2Threads) {
    const int dx = n % k2BX - 1, dy = n / k2BX - 1;
    const int i = i0 + dx, j = j0 + dy;
    if ((unsigned)i < (unsigned)L.nx && (unsigned)j < (unsigned)L.ny) {
      float hp[kQ], hg[kQ];
      pull1<false>(MidA{mid + (dy + 2) * k2RX + dx + 2}, L, i, j, 0, nullptr, hp, hg);
      mth[n] = sum9(hg);
      mrp[n] = sum9(hp);
    }
  }
  __syncthreads();
  // second step on the tile, to the other time level
  {
    const int dx = t % k2TX, dy = t / k2TX;
    const int i = i0 + dx, j = j0 + dy;
    if (i < L.nx && j < L.ny) {
      float fw[kQ], fp[kQ], g[kQ];
      pull1<true>(MidA{mid + (dy + 2) * k2RX + dx + 2}, L, i, j, 0, fw, fp, g);
      GlobSink<float, false, 1> out{static_cast<float*>(a.dst) + (size_t)j * L.pitch + i,
                                    L.plane, 0u, true};
      collide_node<ALLF, k2BX, 1, 1>(a.k, L, i, j, dx, dy, mth, mrp, fw, fp, g, out);
    }
  }
}

// ---- host side ---------------------------------------------------------------------------------
// Enables the two-step kernel for a lattice whose 32 x 16 tiles fit one per SM.
inline cudaError_t prepare_two(StepConfig* c, const Layout& L) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int tiles = ((L.nx + k2TX - 1) / k2TX) * ((L.ny + k2TY - 1) / k2TY);
  if (tiles > sms) return cudaErrorNotSupported;
  const void* fns[2] = {(const void*)step_two_kernel<false>, (const void*)step_two_kernel<true>};
  for (const void* fn : fns)
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)k2Smem)) != cudaSuccess)
      return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_two_kernel<true>,
                                                         k2Threads, k2Smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  c->two = true;
  c->grid2 = tiles;
  return cudaSuccess;
}

inline cudaError_t launch_two(const StepArgs& a, const StepConfig& c, const CUtensorMap* map2,
                              cudaStream_t st) {
  if (!c.two || !map2 || c.grid2 < 1) return cudaErrorInvalidValue;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(c.grid2);
  cfg.blockDim = dim3(k2Threads);
  cfg.dynamicSmemBytes = k2Smem;
  if (a.k.mask == MCLBM_F_ALL)
    return cudaLaunchKernelEx(&cfg, step_two_kernel<true>, *map2, a);
  return cudaLaunchKernelEx(&cfg, step_two_kernel<false>, *map2, a);
}

}  // namespace pair
}  // namespace mcl
