// Device code shared by the kernels of libmclbm: the D2Q9 tables and equilibrium constants,
// the storage element types, the scalar pull of one node (initial fill, fields, reductions and
// the streaming test hook), the per-step rounding hash and the TMA / mbarrier helpers. The
// fused step kernels themselves are in mclbm_pair.cuh.
//
// State: 27 planes [ny][pitch] per time level (structure of arrays), f^w_0..8, f^p_0..8,
// g_0..8 in the direction order of Eq 21. The planes hold deviations from the initial
// conduction state: f_q - W_q rho_sigma0 and g_q - W_q theta_c(i), theta_c(i) = 1/2 - (i+1/2)/nx,
// so the stored mantissa resolves the small departures that carry the flow and the heat.
// Streaming a g deviation across x adds W_q e_qx / nx (the drop of theta_c over one link).
// Storage: FP32, or FP16 / BF16 holding the deviations times 2^12 (FP16's normal range then
// covers deviations from 1.5e-8 to 16); all arithmetic is FP32.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mclbm_internal.h"

namespace mcl {

// ---- D2Q9 tables as constexpr functions (indices are compile-time after unrolling) --------
__host__ __device__ constexpr int ex(int q) {
  return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int q) {
  return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int q) {
  return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 5 + 2) % 4) + 5);
}
// direction mirrored in a horizontal wall: (ex, ey) -> (ex, -ey)
__host__ __device__ constexpr int mir(int q) {
  return q == 2 ? 4 : q == 4 ? 2 : q == 5 ? 8 : q == 8 ? 5 : q == 6 ? 7 : q == 7 ? 6 : q;
}
__host__ __device__ constexpr float wq(int q) {
  return q == 0 ? 4.0f / 9.0f : (q <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// Equilibrium polynomial coefficients for q = 1..8: W_q rho P_q(u) with
// P_q = A_q e.u + B_q (e.u)^2 - C_q u.u, nominally A = 3 W, B = 4.5 W, C = 1.5 W (Eqs 26-28).
// FP32 cannot hold 1/3 and 1/12, and rounding them independently makes the equilibrium's
// first moment 3 (2 W_1 + 4 W_2) u = (1 + 7.5e-9) u: every collision then relaxes momentum
// and heat flux towards a target 1e-8 too large, a bias the slow large-scale modes of a cavity
// integrate into a ~1e-4 error. A_1 = 0.33333334 and A_2 = 0.08333333 are chosen so that
// 2 A_1 + 4 A_2 = 1 exactly; B is exact; the rest population's equilibrium is the remainder,
// so the zeroth moment is exact as well (up to unbiased rounding).
__host__ __device__ constexpr float aq(int q) {
  return q == 0 ? 0.0f : (q <= 4 ? 0x1.555556p-2f : 0x1.555554p-4f);
}
__host__ __device__ constexpr float bq(int q) { return q == 0 ? 0.0f : (q <= 4 ? 0.5f : 0.125f); }
__host__ __device__ constexpr float cq(int q) {
  return q == 0 ? 0.0f : (q <= 4 ? 1.0f / 6.0f : 1.0f / 24.0f);
}
static_assert(2.0f * aq(1) + 4.0f * aq(5) == 1.0f, "first moment of the equilibrium is exact");
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "axial opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "diagonal opposites");
static_assert(ex(opp(6)) == -ex(6) && ey(opp(6)) == -ey(6), "opposite of e_6");
static_assert(ex(mir(5)) == ex(5) && ey(mir(5)) == -ey(5), "mirror of e_5");


// ---- storage element types -------------------------------------------------------------------
// Elem<T>: how a stored deviation becomes an FP32 value and back (round to nearest) for the
// kernels outside the step. 16-bit types hold 2^12 times the deviation.
constexpr float kStoreScale = 4096.0f;
constexpr float kStoreInvScale = 1.0f / 4096.0f;

template <class T>
struct Elem;

template <>
struct Elem<float> {
  static constexpr int kBytes = 4;
  __device__ __forceinline__ static float get(float v) { return v; }
  __device__ __forceinline__ static float ldg(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static float put(float v) { return v; }
};

template <>
struct Elem<__half> {
  static constexpr int kBytes = 2;
  __device__ __forceinline__ static float get(__half v) {
    return __half2float(v) * kStoreInvScale;
  }
  __device__ __forceinline__ static float ldg(const __half* p) { return get(__ldg(p)); }
  __device__ __forceinline__ static __half put(float v) {
    return __float2half_rn(v * kStoreScale);
  }
};

template <>
struct Elem<__nv_bfloat16> {
  static constexpr int kBytes = 2;
  __device__ __forceinline__ static float get(__nv_bfloat16 v) {
    return __bfloat162float(v) * kStoreInvScale;
  }
  __device__ __forceinline__ static float ldg(const __nv_bfloat16* p) { return get(__ldg(p)); }
  __device__ __forceinline__ static __nv_bfloat16 put(float v) {
    return __float2bfloat16_rn(v * kStoreScale);
  }
};

// 32-bit integer hash (xor-shift-multiply finaliser with the "lowbias32" constants published
// by C. Wellons) used to seed the per-node rounding stream.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Pull streaming of node (i, j) from a state level in global memory. FULL: all 27
// populations; otherwise only f^p and g (the 18 planes the halo moments need). Wall rules, in
// absolute values:
//   f^w, f^p: link-wise bounce-back f_q(x) = f*_{-q}(x);
//   g through the hot/cold wall (corners included): g_q(x) = 2 W_q T_wall - g*_{-q}(x);
//   g through the top/bottom wall only: g_q(x) = g*_{mir q}(i - e_qx, j) (specular).
// For the stored g deviations every rule becomes g'_q(x) = W_q e_qx s + (source deviation),
// s = 1/nx: the interior and specular sources by the drop of theta_c over the link, the
// isothermal walls because 2 (T_wall - theta_c) = e_qx s at the outer columns.
template <class T, bool FULL>
__device__ __forceinline__ void pull_node(const T* __restrict__ src, const Layout& L, int i, int j,
                                          float* fw, float* fp, float* g, float s) {
  using E = Elem<T>;
  const size_t self = (size_t)j * L.pitch + i;
  if ((unsigned)(i - 1) < (unsigned)(L.nx - 2) && (unsigned)(j - 1) < (unsigned)(L.ny - 2)) {
    // no link of a node away from the walls leaves the cavity
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const size_t o = self - (size_t)((ptrdiff_t)ey(q) * L.pitch + ex(q));
      if (FULL) fw[q] = E::ldg(src + (size_t)q * L.plane + o);
      fp[q] = E::ldg(src + (size_t)(kQ + q) * L.plane + o);
      g[q] = E::ldg(src + (size_t)(2 * kQ + q) * L.plane + o);
      if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int si = i - ex(q), sj = j - ey(q);
    const bool inx = (unsigned)si < (unsigned)L.nx;
    const bool iny = (unsigned)sj < (unsigned)L.ny;
    if (inx && iny) {
      const size_t o = (size_t)sj * L.pitch + si;
      if (FULL) fw[q] = E::ldg(src + (size_t)q * L.plane + o);
      fp[q] = E::ldg(src + (size_t)(kQ + q) * L.plane + o);
      g[q] = E::ldg(src + (size_t)(2 * kQ + q) * L.plane + o);
    } else {
      if (FULL) fw[q] = E::ldg(src + (size_t)opp(q) * L.plane + self);
      fp[q] = E::ldg(src + (size_t)(kQ + opp(q)) * L.plane + self);
      if (!inx) {
        g[q] = -E::ldg(src + (size_t)(2 * kQ + opp(q)) * L.plane + self);
      } else {
        g[q] = E::ldg(src + (size_t)(2 * kQ + mir(q)) * L.plane + (size_t)j * L.pitch + si);
      }
    }
    if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
  }
}

// Pull of the thermal set whose planes start at `base` (18: g or g^w; 27: g^p), with the wall
// rules of pull_node.
template <class T>
__device__ __forceinline__ void pull_thermal(const T* __restrict__ src, const Layout& L, int i,
                                             int j, int base, float* g, float s) {
  using E = Elem<T>;
  const size_t self = (size_t)j * L.pitch + i;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int si = i - ex(q), sj = j - ey(q);
    const bool inx = (unsigned)si < (unsigned)L.nx;
    const bool iny = (unsigned)sj < (unsigned)L.ny;
    if (inx && iny)
      g[q] = E::ldg(src + (size_t)(base + q) * L.plane + (size_t)sj * L.pitch + si);
    else if (!inx)
      g[q] = -E::ldg(src + (size_t)(base + opp(q)) * L.plane + self);
    else
      g[q] = E::ldg(src + (size_t)(base + mir(q)) * L.plane + (size_t)j * L.pitch + si);
    if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
  }
}

// Eq 33 with two thermal sets: the mixture's deviation from theta_c, the heat-capacity
// weighted mean of the sets' deviations (rho_w, rho_p the absolute partial densities).
__device__ __forceinline__ float mixture_dev(const StepConsts& k, float rho_w, float rho_p,
                                             float dev_w, float dev_p) {
  const float cp = k.r_cp * rho_p;
  return (rho_w * dev_w + cp * dev_p) / (rho_w + cp);
}

// theta_c(i): the linear conduction profile the g deviations are taken from
__device__ __forceinline__ float theta_c(const StepConsts& k, int i) {
  return k.th_c0 - (float)i * k.inv_nx;
}

struct Moments {
  float rw, rp;    // partial density deviations from rho_w0, rho_p0
  float mwx, mwy;  // momenta (Eq 30)
  float mpx, mpy;
  float th;        // theta deviation from theta_c(i) (Eq 31)
};

__device__ __forceinline__ float sum9(const float* a) {
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])) + a[8];
}
__device__ __forceinline__ float mom_x(const float* a) {
  return (a[1] - a[3]) + (a[5] - a[6]) + (a[8] - a[7]);
}
__device__ __forceinline__ float mom_y(const float* a) {
  return (a[2] - a[4]) + (a[5] - a[8]) + (a[6] - a[7]);
}

__device__ __forceinline__ Moments moments_of(const float* fw, const float* fp, const float* g) {
  Moments m;
  m.rw = sum9(fw);
  m.rp = sum9(fp);
  m.mwx = mom_x(fw);
  m.mwy = mom_y(fw);
  m.mpx = mom_x(fp);
  m.mpy = mom_y(fp);
  m.th = sum9(g);
  return m;
}

// Per-step hash that seeds the rounding streams: the launch's seed and the graph epoch.
__device__ __forceinline__ uint32_t step_hash(const StepArgs& a) {
  const uint32_t ep = a.epoch ? *(volatile const uint32_t*)a.epoch : 0u;
  return mix32(a.seed ^ mix32(ep + 0x632BE5ABu));
}

// ---- TMA, bulk-copy and mbarrier helpers (inline PTX) ---------------------------------------
// Every mbarrier wait is bounded (2 s on %globaltimer); the caller decides what a timeout means.
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase with the given parity to complete; false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t k = 0; k < (1u << 26); ++k) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > 2000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void store_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(src)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// waits until at most one committed bulk store still has to read its shared-memory source
__device__ __forceinline__ void bulk_wait_read_1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// waits until no committed bulk store still has to read its shared-memory source
__device__ __forceinline__ void bulk_wait_read_0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// waits until every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

}  // namespace tma


constexpr int kTmaTY = 8;  // tile height of the step kernels' tensor maps

}  // namespace mcl
