// Device code of the fused MCLBM step, shared by the per-storage translation units
// (mclbm_step_f32.cu, mclbm_step_f16.cu, mclbm_step_bf16.cu) and by mclbm_kernels.cu.
//
// State: 27 planes [ny][pitch] per time level (structure of arrays), f^w_0..8, f^p_0..8,
// g_0..8 in the direction order of Eq 21. The planes hold deviations from the initial
// conduction state: f_q - W_q rho_sigma0 and g_q - W_q theta_c(i), theta_c(i) = 1/2 - (i+1/2)/nx,
// so the stored mantissa resolves the small departures that carry the flow and the heat.
// Streaming a g deviation across x adds W_q e_qx / nx (the drop of theta_c over one link).
// Storage: FP32, or FP16 / BF16 holding the deviations times 2^12 (FP16's normal range then
// covers deviations from 1.5e-8 to 16); all arithmetic is FP32. The 16-bit stores round
// stochastically by default: near a steady state round-to-nearest repeats the same rounding
// error every step, a constant forcing that the slow modes integrate; unbiased random rounding
// does not accumulate that way.
//
// The step is one fused kernel (one launch per time step): pull streaming with the wall rules
// (Eqs 18-19 LHS, 34-36), moments (Eqs 29-32), same-time-level gradients of theta and phi,
// the slip forces of Table 1 (Eqs 4, 6, 20), the exact drag impulse, BGK collision with
// forcing (Eqs 18-19 RHS, 26-28, 24) and the store. Same-time-level gradients need theta and
// rho^p of the neighbours after streaming: a CTA pulls its tile and the ring of nodes around
// it, puts their moments in shared memory, and then finishes its own nodes. Two variants:
// the TMA-staged persistent kernel (default) and a plain tile kernel for small lattices.
// No tensor cores: this is a memory-bound stencil.
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
// Elem<T>: how a stored deviation becomes an FP32 value and back. 16-bit types hold 2^12 times
// the deviation. put_sr rounds stochastically with 32 random bits r (only the low bits that
// fall below the 16-bit mantissa are used): adding them to the FP32 pattern and truncating
// rounds up with probability equal to the discarded fraction (sign-magnitude, so symmetric).
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
  __device__ __forceinline__ static float put_sr(float v, uint32_t) { return v; }
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
  // FP16 keeps 10 of FP32's 23 mantissa bits: 13 random bits below them, then truncate
  __device__ __forceinline__ static __half put_sr(float v, uint32_t r) {
    const uint32_t b = __float_as_uint(v * kStoreScale) + (r >> 19);
    return __float2half_rz(__uint_as_float(b));
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
  // BF16 is the upper half of FP32: 16 random bits below it, then truncate
  __device__ __forceinline__ static __nv_bfloat16 put_sr(float v, uint32_t r) {
    const uint32_t b = __float_as_uint(v * kStoreScale) + (r >> 16);
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
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

// Random bits for output plane p of a node: a Weyl sequence in p from the node's hashed seed,
// multiplied so that its high bits (the ones put_sr uses) mix.
__device__ __forceinline__ uint32_t plane_bits(uint32_t seed, int p) {
  return (seed + (uint32_t)p * 0x9E3779B9u) * 0x85EBCA6Bu;
}

// Writes one node's 27 results into a [27][STRIDE] shared-memory tile (TMA-stored afterwards).
template <class T, bool SR, int STRIDE>
struct TileSink {
  T* base;        // tile + node offset
  uint32_t seed;  // per-node rounding stream (SR only)
  __device__ __forceinline__ void operator()(int p, float v) const {
    base[p * STRIDE] = SR ? Elem<T>::put_sr(v, plane_bits(seed, p)) : Elem<T>::put(v);
  }
};

// Writes one node's 27 results to a state level in global memory.
template <class T, bool SR>
struct StoreSink {
  T* base;        // destination level + node offset
  size_t plane;   // elements per plane
  uint32_t seed;  // per-node rounding stream (SR only)
  __device__ __forceinline__ void operator()(int p, float v) const {
    base[(size_t)p * plane] = SR ? Elem<T>::put_sr(v, plane_bits(seed, p)) : Elem<T>::put(v);
  }
};

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

// Steps A2-A7 for one node: moments, forces, drag impulse, collision and store.
// thE, thW, thN, thS and rpE, ... are the neighbours' theta and rho^p deviations (ghosts
// already applied by the caller; theta_c's own slope -1/nx is added to d theta/dx here).
// ALLF: the force mask is known to be MCLBM_F_ALL at compile time (no per-node mask tests).
// The 27 results go to out(p, v), p the plane index (f^w_0..8, f^p_0..8, g_0..8).
template <bool ALLF, class Sink>
__device__ __forceinline__ void collide(const StepConsts& k, const Layout& L, Sink& out, int i,
                                        int j, const float* fw, const float* fp, const float* g,
                                        float thE, float thW, float thN, float thS, float rpE,
                                        float rpW, float rpN, float rpS) {
  const Moments m = moments_of(fw, fp, g);
  const float th = theta_c(k, i) + m.th;  // absolute temperature
  const float rw = k.rho_w0 + m.rw;
  const float rp = k.rho_p0 + m.rp;
  const float rho = rw + rp;
  const float inv_rho = 1.0f / rho;
  const float Yw = rw * inv_rho, Yp = rp * inv_rho;
  const float ux = (m.mwx + m.mpx) * inv_rho;  // Eq 32, barycentric
  const float uy = (m.mwy + m.mpy) * inv_rho;
  const float inv_rw = 1.0f / rw;
  const float uwx = m.mwx * inv_rw, uwy = m.mwy * inv_rw;
  const bool has_p = k.has_p && rp > 1e-30f;
  const float inv_rp = has_p ? 1.0f / rp : 0.0f;
  const float upx = has_p ? m.mpx * inv_rp : uwx;
  const float upy = has_p ? m.mpy * inv_rp : uwy;
  const uint32_t mask = ALLF ? MCLBM_F_ALL : k.mask;

  // external forces: Boussinesq buoyancy on the fluid, gravity pair (Eq 20, Table 1)
  float Fbuoy = (mask & MCLBM_F_BUOYANCY) ? rho * k.buoy * th : 0.0f;
  const bool grav = (mask & MCLBM_F_GRAVITY) != 0;
  float Fwx = 0.0f, Fwy = 0.0f, Fpx = 0.0f, Fpy = 0.0f;
  if (has_p) {
    // particle-fluid interaction forces on the particle phase (reaction on the fluid)
    float Fix = 0.0f, Fiy = 0.0f;
    const float TT0 = 1.0f + th * k.t_ratio;  // T / T0
    const float wx = uwx - upx, wy = uwy - upy;
    if (mask & MCLBM_F_BROWNIAN) {
      const float c = -k.cB * rp * TT0 * TT0 * 0.5f;
      Fix += c * (rpE - rpW);
      Fiy += c * (rpN - rpS);
    }
    if (mask & MCLBM_F_THERMOPHORESIS) {
      const float c = -k.cT * rp / TT0;
      Fix += c * (0.5f * (thE - thW) - k.inv_nx);
      Fiy += c * (0.5f * (thN - thS));
    }
    if (mask & MCLBM_F_SAFFMAN) {
      const float c = k.cS * rp * sqrtf(sqrtf(upx * upx + upy * upy));
      Fix -= c * wy;
      Fiy += c * wx;
    }
    if (mask & MCLBM_F_MAGNUS) {
      // nearest wall (ties: left, right, bottom, top) and its inward normal
      float z = (float)i + 0.5f, nrx = 1.0f, nry = 0.0f;
      const float dr = (float)(L.nx - i) - 0.5f, db = (float)j + 0.5f;
      const float dtp = (float)(L.ny - j) - 0.5f;
      if (dr < z) { z = dr; nrx = -1.0f; nry = 0.0f; }
      if (db < z) { z = db; nrx = 0.0f; nry = 1.0f; }
      if (dtp < z) { z = dtp; nrx = 0.0f; nry = -1.0f; }
      const float zH = z * k.two_over_ny;
      const float sx = uwx + upx, sy = uwy + upy;
      const float c = k.cM * rp * (sx * sx + sy * sy) * zH * (0.63f - zH);
      Fix += c * nrx;
      Fiy += c * nry;
    }
    // non-drag forces: particles F_int + F_G, fluid F_buoy + F_G0 - F_int
    const float FGp = grav ? -rp * k.gG : 0.0f;
    const float FG0w = grav ? k.rho_p0 * k.gG : 0.0f;
    const float Fpnx = Fix, Fpny = Fiy + FGp;
    const float Fwnx = -Fix, Fwny = Fbuoy + FG0w - Fiy;
    if (mask & MCLBM_F_DRAG) {
      // Exact drag impulse over the step (slip ODE dw/dt = -a w + b from the relaxed slip),
      // rearranged so that the large interaction forces cancel before rounding:
      // F^p = Y_p F_tot + mu_r [(1 - e^-a) w' - ((1 - e^-a)/a) b], F^w = F_tot - F^p.
      // Schiller-Naumann correction 0.15 Re^0.687: Re is 1e-8..1e-3 here, so the correction
      // is below 1e-3 of the Stokes rate and the hardware log/exp suffice
      const float Re = k.cRe * sqrtf(wx * wx + wy * wy);
      const float sn = Re > 0.0f ? __expf(0.687f * __logf(Re)) : 0.0f;
      const float beta = k.beta_dt * (1.0f + 0.15f * sn);
      const float a = beta * (1.0f + rp * inv_rw);
      // e^-a is below FP32 resolution of 1 for a > 20 (nanoparticles: a = 1e3..1e7)
      const float E = a > 20.0f ? 1.0f : -expm1f(-a);
      const float Ea = (a < 1e-2f) ? 1.0f - a * (0.5f - a * (1.0f / 6.0f - a * (1.0f / 24.0f)))
                                   : E / a;
      const float mu_r = rw * rp * inv_rho;
      const float relax = 1.0f - Yp * k.inv_tau_w - Yw * k.inv_tau_p;
      const float bx = Fwnx * inv_rw - Fpnx * inv_rp, by = Fwny * inv_rw - Fpny * inv_rp;
      // F_tot: the interaction forces cancel exactly; gravity pair = -(rho^p - rho_p0) gG
      const float Ftx = 0.0f;
      const float Fty = Fbuoy + (grav ? -m.rp * k.gG : 0.0f);
      Fpx = Yp * Ftx + mu_r * (E * relax * wx - Ea * bx);
      Fpy = Yp * Fty + mu_r * (E * relax * wy - Ea * by);
      Fwx = Ftx - Fpx;
      Fwy = Fty - Fpy;
    } else {
      Fpx = Fpnx;
      Fpy = Fpny;
      Fwx = Fwnx;
      Fwy = Fwny;
    }
  } else {
    Fwy = Fbuoy + (grav ? k.rho_p0 * k.gG : 0.0f);
  }

  // BGK collision with forcing 3 W_q e_q.F on the common velocity (Eqs 18, 26), in deviation
  // form: f' <- (1 - 1/tau) f' + (W_q rho' + rho P_q) / tau + A_q e_q.F; g likewise with theta.
  // Opposite directions share the even part of P_q (B (e.u)^2 - C u.u) and negate the odd part
  // (A e.u) and the forcing, so the loop runs over the four pairs (q, -q).
  const float tau_t = Yw * k.tau_tw + Yp * k.tau_tp;  // Eq 24 with local mass fractions
  const float om_t = 1.0f / tau_t;
  const float om_w = k.inv_tau_w, om_p = k.inv_tau_p;
  const float keep_w = 1.0f - om_w, keep_p = 1.0f - om_p, keep_t = 1.0f - om_t;
  const float usq = ux * ux + uy * uy;
  float sw = 0.0f, sp = 0.0f, sg = 0.0f;  // half the sum of the moving equilibria
#pragma unroll
  for (int pr = 0; pr < 4; ++pr) {
    const int q = pr == 0 ? 1 : (pr == 1 ? 2 : (pr == 2 ? 5 : 6));
    const int qo = opp(q);
    const float eu = (float)ex(q) * ux + (float)ey(q) * uy;
    const float even = bq(q) * eu * eu - cq(q) * usq;
    const float odd = aq(q) * eu;
    const float W = wq(q);
    const float tw = W * m.rw + rw * even, dw = rw * odd;
    const float tp = W * m.rp + rp * even, dp = rp * odd;
    const float tg = W * m.th + th * even, dg = th * odd;
    sw += tw;
    sp += tp;
    sg += tg;
    const float Sw = aq(q) * ((float)ex(q) * Fwx + (float)ey(q) * Fwy);
    const float Sp = aq(q) * ((float)ex(q) * Fpx + (float)ey(q) * Fpy);
    out(q, fmaf(fw[q], keep_w, fmaf(om_w, tw + dw, Sw)));
    out(qo, fmaf(fw[qo], keep_w, fmaf(om_w, tw - dw, -Sw)));
    out(kQ + q, fmaf(fp[q], keep_p, fmaf(om_p, tp + dp, Sp)));
    out(kQ + qo, fmaf(fp[qo], keep_p, fmaf(om_p, tp - dp, -Sp)));
    out(2 * kQ + q, fmaf(g[q], keep_t, om_t * (tg + dg)));
    out(2 * kQ + qo, fmaf(g[qo], keep_t, om_t * (tg - dg)));
  }
  // rest populations: equilibrium = zeroth moment minus the moving equilibria
  out(0, fmaf(fw[0], keep_w, om_w * (m.rw - 2.0f * sw)));
  out(kQ, fmaf(fp[0], keep_p, om_p * (m.rp - 2.0f * sp)));
  out(2 * kQ, fmaf(g[0], keep_t, om_t * (m.th - 2.0f * sg)));
}


// Per-step hash that seeds the rounding streams: the launch's seed and the graph epoch.
__device__ __forceinline__ uint32_t step_hash(const StepArgs& a) {
  const uint32_t ep = a.epoch ? *(volatile const uint32_t*)a.epoch : 0u;
  return mix32(a.seed ^ mix32(ep + 0x632BE5ABu));
}

// ---- the fused step, tile variant --------------------------------------------------------------
// One node per thread on a TX x TY tile. Every thread pulls its node's 27 populations; the
// first 2 TX + 2 TY threads also pull the 18 f^p and g populations of one node of the ring
// around the tile, all in the same load phase, so each CTA has all its loads in flight at once
// and the next CTA on the SM overlaps its compute. theta' and rho'^p of the tile and ring go to
// shared memory; one barrier; then every thread finishes its node.
template <class T, bool SR, bool ALLF>
__global__ void __launch_bounds__(256, 2) step_tile_kernel(const StepArgs a) {
  constexpr int TX = 32, TY = 8;
  constexpr int NRING = 2 * TX + 2 * TY;
  __shared__ float s_th[TY + 2][TX + 2];
  __shared__ float s_rp[TY + 2][TX + 2];
  const Layout L = a.L;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < L.nx && j < L.ny;

  // this thread's ring node, tile coordinates in [-1, TX] x [-1, TY] without the corners
  int hx = 0, hy = 0;
  bool ring = false;
  if (t < NRING) {
    if (t < TX) {
      hx = t;
      hy = -1;
    } else if (t < 2 * TX) {
      hx = t - TX;
      hy = TY;
    } else if (t < 2 * TX + TY) {
      hx = -1;
      hy = t - 2 * TX;
    } else {
      hx = TX;
      hy = t - 2 * TX - TY;
    }
    const int gi = i0 + hx, gj = j0 + hy;
    ring = gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny;
  }
  float fw[kQ], fp[kQ], g[kQ];
  float hw[kQ], hp[kQ], hg[kQ];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous step has completed
  if (active) pull_node<T, true>(src, L, i, j, fw, fp, g, a.k.inv_nx);
  if (ring) pull_node<T, false>(src, L, i0 + hx, j0 + hy, hw, hp, hg, a.k.inv_nx);
  if (active) {
    s_th[ty + 1][tx + 1] = sum9(g);
    s_rp[ty + 1][tx + 1] = sum9(fp);
  }
  if (ring) {
    s_th[hy + 1][hx + 1] = sum9(hg);
    s_rp[hy + 1][hx + 1] = sum9(hp);
  }
  __syncthreads();
  if (!active) return;
  const float th = s_th[ty + 1][tx + 1], rp = s_rp[ty + 1][tx + 1];
  // theta deviations: the isothermal ghost 2 T_wall - theta is -theta' in deviation form
  const float thW = (i > 0) ? s_th[ty + 1][tx] : -th;
  const float thE = (i + 1 < L.nx) ? s_th[ty + 1][tx + 2] : -th;
  const float thS = (j > 0) ? s_th[ty][tx + 1] : th;
  const float thN = (j + 1 < L.ny) ? s_th[ty + 2][tx + 1] : th;
  const float rpW = (i > 0) ? s_rp[ty + 1][tx] : rp;
  const float rpE = (i + 1 < L.nx) ? s_rp[ty + 1][tx + 2] : rp;
  const float rpS = (j > 0) ? s_rp[ty][tx + 1] : rp;
  const float rpN = (j + 1 < L.ny) ? s_rp[ty + 2][tx + 1] : rp;
  const size_t o = (size_t)j * L.pitch + i;
  StoreSink<T, SR> out{static_cast<T*>(a.dst) + o, L.plane,
                       SR ? mix32((uint32_t)o ^ step_hash(a)) : 0u};
  collide<ALLF>(a.k, L, out, i, j, fw, fp, g, thE, thW, thN, thS, rpE, rpW, rpN, rpS);
}

// ---- the fused step, TMA-staged persistent variant -------------------------------------------
// Each persistent CTA walks tiles of 32 x 8 nodes. For every tile one TMA tensor load brings
// the tile's window of all 27 planes (2 rows and 16 bytes of columns of halo on each side; the
// domain outside reads as zeros and is never used) into shared memory, double-buffered: while a
// tile is computed from one buffer the next tile's window streams into the other, so the HBM
// stays busy without the compute warps waiting on their own loads. Completion is tracked by one
// mbarrier per buffer; every wait on it is bounded (2 s on %globaltimer), after which the
// kernel sets bit 0 of the error word, drains its copies (bounded) and returns.
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


constexpr int kTmaTX = 32;  // tile width
constexpr int kTmaTY = 8;   // tile height
template <class T>
struct TmaTile {
  static constexpr int XO = 16 / Elem<T>::kBytes;  // halo columns per side: 16 bytes (x alignment)
  static constexpr int WX = kTmaTX + 2 * XO;      // window width
  static constexpr int WY = kTmaTY + 4;           // window height: 2 rows each side
  static constexpr int WPLANE = WX * WY;
  static constexpr uint32_t BYTES = (uint32_t)kPlanes * WPLANE * Elem<T>::kBytes;
  // 16-bit storage leaves room for two output tiles, written by TMA stores; FP32 stores from
  // registers (two FP32 windows already fill the shared memory of two CTAs per SM)
  static constexpr bool STORE_TMA = Elem<T>::kBytes == 2;
  static constexpr uint32_t OUT_BYTES =
      STORE_TMA ? (uint32_t)kPlanes * kTmaTX * kTmaTY * Elem<T>::kBytes : 0u;
  static constexpr size_t SMEM = 2 * (size_t)BYTES + 2 * (size_t)OUT_BYTES;
  static_assert(BYTES % 128 == 0 && OUT_BYTES % 128 == 0, "buffers stay 128-byte aligned");
};

// Pull of node (i, j) from a window whose element (wx, wy) of plane p is
// w[p * WPLANE + wy * WX + wx]; (wx, wy) is the node's own position in the window.
template <class T, bool FULL>
__device__ __forceinline__ void pull_window(const T* w, const Layout& L, int i, int j, int wx,
                                            int wy, float* fw, float* fp, float* g, float s) {
  using E = Elem<T>;
  constexpr int WX = TmaTile<T>::WX, WPLANE = TmaTile<T>::WPLANE;
  const int self = wy * WX + wx;
  if ((unsigned)(i - 1) < (unsigned)(L.nx - 2) && (unsigned)(j - 1) < (unsigned)(L.ny - 2)) {
    // no link of a node away from the walls leaves the cavity
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int src = self - ey(q) * WX - ex(q);
      if (FULL) fw[q] = E::get(w[q * WPLANE + src]);
      fp[q] = E::get(w[(kQ + q) * WPLANE + src]);
      g[q] = E::get(w[(2 * kQ + q) * WPLANE + src]);
      if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int si = i - ex(q), sj = j - ey(q);
    const bool inx = (unsigned)si < (unsigned)L.nx;
    const bool iny = (unsigned)sj < (unsigned)L.ny;
    const int src = self - ey(q) * WX - ex(q);
    if (inx && iny) {
      if (FULL) fw[q] = E::get(w[q * WPLANE + src]);
      fp[q] = E::get(w[(kQ + q) * WPLANE + src]);
      g[q] = E::get(w[(2 * kQ + q) * WPLANE + src]);
    } else {
      if (FULL) fw[q] = E::get(w[opp(q) * WPLANE + self]);
      fp[q] = E::get(w[(kQ + opp(q)) * WPLANE + self]);
      if (!inx)
        g[q] = -E::get(w[(2 * kQ + opp(q)) * WPLANE + self]);
      else
        g[q] = E::get(w[(2 * kQ + mir(q)) * WPLANE + self - ex(q)]);
    }
    if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
  }
}

template <class T, bool SR, bool ALLF>
__global__ void __launch_bounds__(kTmaTX * kTmaTY, 2)
    step_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                    const __grid_constant__ CUtensorMap tmap_out, const StepArgs a) {
  constexpr int TX = kTmaTX, TY = kTmaTY;
  constexpr int NRING = 2 * TX + 2 * TY;
  constexpr int XO = TmaTile<T>::XO;
  constexpr uint32_t BYTES = TmaTile<T>::BYTES;
  constexpr uint32_t OUT_BYTES = TmaTile<T>::OUT_BYTES;
  constexpr bool STORE_TMA = TmaTile<T>::STORE_TMA;
  static_assert(NRING <= TX * TY, "at most one ring node per thread");
  extern __shared__ __align__(128) unsigned char win_raw[];
  __shared__ float s_th[TY + 2][TX + 2];
  __shared__ float s_rp[TY + 2][TX + 2];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_abort;

  const Layout L = a.L;
  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int tiles_x = (L.nx + TX - 1) / TX;
  const int n_tiles = tiles_x * ((L.ny + TY - 1) / TY);
  const uint32_t bar0 = tma::smem_u32(&bars[0]);
  const uint32_t win0 = tma::smem_u32(win_raw);

  if (t == 0) {
    tma::mbar_init(bar0, 1);
    tma::mbar_init(bar0 + 8, 1);
    tma::fence_barrier_init();
    s_abort = 0;
  }
  // Programmatic dependent launch: let the next step's CTAs start their prologue while this
  // grid drains, and do not read the state before the previous step has completed.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const uint32_t sh = SR ? step_hash(a) : 0u;
  __syncthreads();

  // this thread's ring node (tile coordinates, corners excluded)
  int hx = 0, hy = 0;
  if (t < NRING) {
    if (t < TX) {
      hx = t;
      hy = -1;
    } else if (t < 2 * TX) {
      hx = t - TX;
      hy = TY;
    } else if (t < 2 * TX + TY) {
      hx = -1;
      hy = t - 2 * TX;
    } else {
      hx = TX;
      hy = t - 2 * TX - TY;
    }
  }

  // tile coordinates, advanced by gridDim.x tiles per iteration without divisions
  const int step_y = (int)gridDim.x / tiles_x, step_x = (int)gridDim.x - step_y * tiles_x;
  int tile = blockIdx.x;
  int tcx = tile % tiles_x, tcy = tile / tiles_x;            // current tile
  int ncx = tcx + step_x, ncy = tcy + step_y;                // next tile
  if (ncx >= tiles_x) {
    ncx -= tiles_x;
    ++ncy;
  }
  if (t == 0 && tile < n_tiles) {
    tma::mbar_expect_tx(bar0, BYTES);
    tma::load_3d(win0, &tmap, tcx * TX - XO, tcy * TY - 2, a.z_src, bar0);
  }
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const int stage = it & 1;
    const int next = tile + gridDim.x;
    if (t == 0 && next < n_tiles) {
      // the other window was last read in the previous iteration, which ended in a barrier
      tma::fence_proxy_async();
      const uint32_t bar = bar0 + 8u * (stage ^ 1);
      tma::mbar_expect_tx(bar, BYTES);
      tma::load_3d(win0 + (stage ^ 1) * BYTES, &tmap, ncx * TX - XO, ncy * TY - 2, a.z_src, bar);
    }
    // this stage's output tile was last read by the TMA store of two iterations ago
    if (STORE_TMA && t == 0) tma::bulk_wait_read_1();
    const bool ok = tma::mbar_wait(bar0 + 8u * stage, (it >> 1) & 1);
    const T* w = reinterpret_cast<const T*>(win_raw + stage * BYTES);
    const int i0 = tcx * TX, j0 = tcy * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < L.nx && j < L.ny;
    const int gi = i0 + hx, gj = j0 + hy;
    const bool ring = t < NRING && gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny;
    float fw[kQ], fp[kQ], g[kQ];
    if (active) {
      pull_window<T, true>(w, L, i, j, tx + XO, ty + 2, fw, fp, g, a.k.inv_nx);
      s_th[ty + 1][tx + 1] = sum9(g);
      s_rp[ty + 1][tx + 1] = sum9(fp);
    }
    if (ring) {
      float hw[kQ], hp[kQ], hg[kQ];
      pull_window<T, false>(w, L, gi, gj, hx + XO, hy + 2, hw, hp, hg, a.k.inv_nx);
      s_th[hy + 1][hx + 1] = sum9(hg);
      s_rp[hy + 1][hx + 1] = sum9(hp);
    }
    if (!ok) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      if (t == 0) {
        atomicOr(a.err, 1);
        if (STORE_TMA) tma::bulk_wait_all();
        // drain: this tile's copy and, if issued, the next one (bounded waits)
        tma::mbar_wait(bar0 + 8u * stage, (it >> 1) & 1);
        if (next < n_tiles) tma::mbar_wait(bar0 + 8u * (stage ^ 1), ((it + 1) >> 1) & 1);
      }
      return;
    }
    if (active) {
      const float th = s_th[ty + 1][tx + 1], rp = s_rp[ty + 1][tx + 1];
      // theta deviations: the isothermal ghost 2 T_wall - theta is -theta' in deviation form
      const float thW = (i > 0) ? s_th[ty + 1][tx] : -th;
      const float thE = (i + 1 < L.nx) ? s_th[ty + 1][tx + 2] : -th;
      const float thS = (j > 0) ? s_th[ty][tx + 1] : th;
      const float thN = (j + 1 < L.ny) ? s_th[ty + 2][tx + 1] : th;
      const float rpW = (i > 0) ? s_rp[ty + 1][tx] : rp;
      const float rpE = (i + 1 < L.nx) ? s_rp[ty + 1][tx + 2] : rp;
      const float rpS = (j > 0) ? s_rp[ty][tx + 1] : rp;
      const float rpN = (j + 1 < L.ny) ? s_rp[ty + 2][tx + 1] : rp;
      const size_t o = (size_t)j * L.pitch + i;
      const uint32_t seed = SR ? mix32((uint32_t)o ^ sh) : 0u;
      if constexpr (STORE_TMA) {
        T* ob = reinterpret_cast<T*>(win_raw + 2 * BYTES + stage * OUT_BYTES);
        TileSink<T, SR, TX * TY> out{ob + t, seed};
        collide<ALLF>(a.k, L, out, i, j, fw, fp, g, thE, thW, thN, thS, rpE, rpW, rpN, rpS);
      } else {
        StoreSink<T, SR> out{static_cast<T*>(a.dst) + o, L.plane, seed};
        collide<ALLF>(a.k, L, out, i, j, fw, fp, g, thE, thW, thN, thS, rpE, rpW, rpN, rpS);
      }
    }
    if (STORE_TMA) tma::fence_proxy_async();  // generic-proxy writes before the TMA store
    __syncthreads();  // the window and the moment tile are free again
    if (STORE_TMA && t == 0) {
      // nodes outside the cavity fall outside the tensor and are not written
      tma::store_3d(&tmap_out, i0, j0, kPlanes - a.z_src,
                    win0 + 2 * BYTES + stage * OUT_BYTES);
      tma::bulk_commit();
    }
    tcx = ncx;
    tcy = ncy;
    ncx += step_x;
    ncy += step_y;
    if (ncx >= tiles_x) {
      ncx -= tiles_x;
      ++ncy;
    }
  }
  if (STORE_TMA && t == 0) tma::bulk_wait_all();
}

// ---- host-side launch of the step kernels for one storage type ----------------------------
template <class T>
cudaError_t prepare_tma_t(StepConfig* c, const Layout& L) {
  const size_t smem = TmaTile<T>::SMEM;
  const void* fns[4] = {(const void*)step_tma_kernel<T, false, false>,
                        (const void*)step_tma_kernel<T, false, true>,
                        (const void*)step_tma_kernel<T, true, false>,
                        (const void*)step_tma_kernel<T, true, true>};
  cudaError_t e;
  for (const void* fn : fns)
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tma_kernel<T, true, true>,
                                                    kTmaTX * kTmaTY, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm > 2) per_sm = 2;
  const int tiles = ((L.nx + kTmaTX - 1) / kTmaTX) * ((L.ny + kTmaTY - 1) / kTmaTY);
  c->grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  return cudaSuccess;
}

template <class T, bool SR, bool ALLF>
cudaError_t launch_step_t3(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                           cudaLaunchConfig_t& cfg) {
  if (c.variant == 2) {
    if (!map || c.grid < 1) return cudaErrorInvalidValue;
    cfg.gridDim = dim3(c.grid);
    cfg.blockDim = dim3(kTmaTX * kTmaTY);
    cfg.dynamicSmemBytes = TmaTile<T>::SMEM;
    return cudaLaunchKernelEx(&cfg, step_tma_kernel<T, SR, ALLF>, map[0], map[1], a);
  }
  cfg.gridDim = dim3((a.L.nx + 31) / 32, (a.L.ny + 7) / 8);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  return cudaLaunchKernelEx(&cfg, step_tile_kernel<T, SR, ALLF>, a);
}

// Tile and TMA kernels go out with programmatic stream serialization: the kernel itself
// waits on the previous grid (griddepcontrol.wait) before it reads the state.
template <class T>
cudaError_t launch_step_t(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                          cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const bool all = a.k.mask == MCLBM_F_ALL;
  const bool sr = c.sr && Elem<T>::kBytes == 2;
  if (sr)
    return all ? launch_step_t3<T, true, true>(a, c, map, cfg)
               : launch_step_t3<T, true, false>(a, c, map, cfg);
  return all ? launch_step_t3<T, false, true>(a, c, map, cfg)
             : launch_step_t3<T, false, false>(a, c, map, cfg);
}

}  // namespace mcl
