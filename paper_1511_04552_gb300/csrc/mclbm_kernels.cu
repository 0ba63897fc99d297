// CUDA kernels of libmclbm for GB300 (sm_103a).
//
// State: 27 FP32 planes [ny][pitch] per time level (structure of arrays), f^w_0..8, f^p_0..8,
// g_0..8 in the direction order of Eq 21. The planes hold deviations from the initial
// conduction state: f_q - W_q rho_sigma0 and g_q - W_q theta_c(i), theta_c(i) = 1/2 - (i+1/2)/nx,
// so the FP32 mantissa resolves the small departures that carry the flow and the heat.
// Streaming a g deviation across x adds W_q e_qx / nx (the drop of theta_c over one link).
//
// The step is one fused kernel (one launch per time step): pull streaming with the wall rules
// (Eqs 18-19 LHS, 34-36), moments (Eqs 29-32), same-time-level gradients of theta and phi,
// the slip forces of Table 1 (Eqs 4, 6, 20), the exact drag impulse, BGK collision with
// forcing (Eqs 18-19 RHS, 26-28, 24) and the store. Same-time-level gradients need theta and
// rho^p of the neighbours after streaming: a CTA pulls its tile and the ring of nodes around
// it, puts their moments in shared memory, and then finishes its own nodes. Two variants:
// the TMA-staged persistent kernel (default) and a plain tile kernel for small lattices.
// No tensor cores: this is a memory-bound stencil.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

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

__device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }

// Pull streaming of node (i, j). FULL: all 27 populations; otherwise only f^p and g (the
// 18 planes the halo moments need). Wall rules, in absolute values:
//   f^w, f^p: link-wise bounce-back f_q(x) = f*_{-q}(x);
//   g through the hot/cold wall (corners included): g_q(x) = 2 W_q T_wall - g*_{-q}(x);
//   g through the top/bottom wall only: g_q(x) = g*_{mir q}(i - e_qx, j) (specular).
// For the stored g deviations every rule becomes g'_q(x) = W_q e_qx s + (source deviation),
// s = 1/nx: the interior and specular sources by the drop of theta_c over the link, the
// isothermal walls because 2 (T_wall - theta_c) = e_qx s at the outer columns.
template <bool FULL>
__device__ __forceinline__ void pull_node(const float* __restrict__ src, const Layout& L, int i,
                                          int j, float* fw, float* fp, float* g, float s) {
  const size_t self = (size_t)j * L.pitch + i;
  if ((unsigned)(i - 1) < (unsigned)(L.nx - 2) && (unsigned)(j - 1) < (unsigned)(L.ny - 2)) {
    // no link of a node away from the walls leaves the cavity
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const size_t o = self - (size_t)((ptrdiff_t)ey(q) * L.pitch + ex(q));
      if (FULL) fw[q] = ldg(src + (size_t)q * L.plane + o);
      fp[q] = ldg(src + (size_t)(kQ + q) * L.plane + o);
      g[q] = ldg(src + (size_t)(2 * kQ + q) * L.plane + o);
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
      if (FULL) fw[q] = ldg(src + (size_t)q * L.plane + o);
      fp[q] = ldg(src + (size_t)(kQ + q) * L.plane + o);
      g[q] = ldg(src + (size_t)(2 * kQ + q) * L.plane + o);
    } else {
      if (FULL) fw[q] = ldg(src + (size_t)opp(q) * L.plane + self);
      fp[q] = ldg(src + (size_t)(kQ + opp(q)) * L.plane + self);
      if (!inx) {
        g[q] = -ldg(src + (size_t)(2 * kQ + opp(q)) * L.plane + self);
      } else {
        g[q] = ldg(src + (size_t)(2 * kQ + mir(q)) * L.plane + (size_t)j * L.pitch + si);
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
template <bool ALLF>
__device__ __forceinline__ void collide_store(const StepConsts& k, const Layout& L, float* dst,
                                              int i, int j, const float* fw, const float* fp,
                                              const float* g, float thE, float thW, float thN,
                                              float thS, float rpE, float rpW, float rpN,
                                              float rpS) {
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
  const size_t o = (size_t)j * L.pitch + i;
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
    dst[(size_t)q * L.plane + o] = fmaf(fw[q], keep_w, fmaf(om_w, tw + dw, Sw));
    dst[(size_t)qo * L.plane + o] = fmaf(fw[qo], keep_w, fmaf(om_w, tw - dw, -Sw));
    dst[(size_t)(kQ + q) * L.plane + o] = fmaf(fp[q], keep_p, fmaf(om_p, tp + dp, Sp));
    dst[(size_t)(kQ + qo) * L.plane + o] = fmaf(fp[qo], keep_p, fmaf(om_p, tp - dp, -Sp));
    dst[(size_t)(2 * kQ + q) * L.plane + o] = fmaf(g[q], keep_t, om_t * (tg + dg));
    dst[(size_t)(2 * kQ + qo) * L.plane + o] = fmaf(g[qo], keep_t, om_t * (tg - dg));
  }
  // rest populations: equilibrium = zeroth moment minus the moving equilibria
  dst[o] = fmaf(fw[0], keep_w, om_w * (m.rw - 2.0f * sw));
  dst[(size_t)kQ * L.plane + o] = fmaf(fp[0], keep_p, om_p * (m.rp - 2.0f * sp));
  dst[(size_t)(2 * kQ) * L.plane + o] = fmaf(g[0], keep_t, om_t * (m.th - 2.0f * sg));
}

// ---- the fused step, tile variant --------------------------------------------------------------
// One node per thread on a TX x TY tile. Every thread pulls its node's 27 populations; the
// first 2 TX + 2 TY threads also pull the 18 f^p and g populations of one node of the ring
// around the tile, all in the same load phase, so each CTA has all its loads in flight at once
// and the next CTA on the SM overlaps its compute. theta' and rho'^p of the tile and ring go to
// shared memory; one barrier; then every thread finishes its node.
template <int TX, int TY, bool ALLF>
__global__ void __launch_bounds__(TX * TY, 2) step_tile_kernel(const StepArgs a) {
  constexpr int NRING = 2 * TX + 2 * TY;
  static_assert(NRING <= TX * TY, "at most one ring node per thread");
  __shared__ float s_th[TY + 2][TX + 2];
  __shared__ float s_rp[TY + 2][TX + 2];
  const Layout L = a.L;
  const float* __restrict__ src = a.src;
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
  if (active) pull_node<true>(src, L, i, j, fw, fp, g, a.k.inv_nx);
  if (ring) pull_node<false>(src, L, i0 + hx, j0 + hy, hw, hp, hg, a.k.inv_nx);
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
  collide_store<ALLF>(a.k, L, a.dst, i, j, fw, fp, g, thE, thW, thN, thS, rpE, rpW, rpN, rpS);
}

// ---- the fused step, TMA-staged persistent variant -------------------------------------------
// Each persistent CTA walks tiles of 32 x TY nodes. For every tile one TMA tensor load brings
// the tile's window of all 27 planes (columns i0-4 .. i0+35, rows j0-2 .. j0+TY+1; the domain
// outside reads as zeros and is never used) into shared memory, double-buffered: while a tile
// is computed from one buffer the next tile's window streams into the other, so the HBM stays
// busy without the compute warps waiting on their own loads. Completion is tracked by one
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
__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

}  // namespace tma

constexpr int kTmaTX = 32;               // tile width
constexpr int kTmaWX = kTmaTX + 8;       // window width: 4 columns each side (16-byte aligned x)
template <int TY>
struct TmaTile {
  static constexpr int WY = TY + 4;      // window height: 2 rows each side
  static constexpr int WPLANE = kTmaWX * WY;
  static constexpr uint32_t BYTES = (uint32_t)kPlanes * WPLANE * 4u;
  static constexpr size_t SMEM = 2 * (size_t)BYTES;  // dynamic shared memory: two windows
};

// Pull of node (i, j) from a window whose element (wx, wy) of plane p is
// w[p * WPLANE + wy * kTmaWX + wx]; (wx, wy) is the node's own position in the window.
template <bool FULL, int WPLANE>
__device__ __forceinline__ void pull_window(const float* w, const Layout& L, int i, int j, int wx,
                                            int wy, float* fw, float* fp, float* g, float s) {
  const int self = wy * kTmaWX + wx;
  if ((unsigned)(i - 1) < (unsigned)(L.nx - 2) && (unsigned)(j - 1) < (unsigned)(L.ny - 2)) {
    // no link of a node away from the walls leaves the cavity
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int src = self - ey(q) * kTmaWX - ex(q);
      if (FULL) fw[q] = w[q * WPLANE + src];
      fp[q] = w[(kQ + q) * WPLANE + src];
      g[q] = w[(2 * kQ + q) * WPLANE + src];
      if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int si = i - ex(q), sj = j - ey(q);
    const bool inx = (unsigned)si < (unsigned)L.nx;
    const bool iny = (unsigned)sj < (unsigned)L.ny;
    const int src = self - ey(q) * kTmaWX - ex(q);
    if (inx && iny) {
      if (FULL) fw[q] = w[q * WPLANE + src];
      fp[q] = w[(kQ + q) * WPLANE + src];
      g[q] = w[(2 * kQ + q) * WPLANE + src];
    } else {
      if (FULL) fw[q] = w[opp(q) * WPLANE + self];
      fp[q] = w[(kQ + opp(q)) * WPLANE + self];
      if (!inx)
        g[q] = -w[(2 * kQ + opp(q)) * WPLANE + self];
      else
        g[q] = w[(2 * kQ + mir(q)) * WPLANE + self - ex(q)];
    }
    if (ex(q) != 0) g[q] += (float)ex(q) * wq(q) * s;
  }
}

template <int TY, bool ALLF>
__global__ void __launch_bounds__(kTmaTX * TY, (TY <= 8 ? 2 : 1))
    step_tma_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs a) {
  constexpr int TX = kTmaTX;
  constexpr int NRING = 2 * TX + 2 * TY;
  constexpr int WPLANE = TmaTile<TY>::WPLANE;
  constexpr uint32_t BYTES = TmaTile<TY>::BYTES;
  static_assert(NRING <= TX * TY, "at most one ring node per thread");
  static_assert(BYTES % 128 == 0, "second window stays 128-byte aligned");
  extern __shared__ __align__(128) float win_smem[];
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
  const uint32_t win0 = tma::smem_u32(win_smem);

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

  int tile = blockIdx.x;
  if (t == 0 && tile < n_tiles) {
    tma::mbar_expect_tx(bar0, BYTES);
    tma::load_3d(win0, &tmap, (tile % tiles_x) * TX - 4, (tile / tiles_x) * TY - 2, a.z_src, bar0);
  }
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const int stage = it & 1;
    const int next = tile + gridDim.x;
    if (t == 0 && next < n_tiles) {
      // the other window was last read in the previous iteration, which ended in a barrier
      tma::fence_proxy_async();
      const uint32_t bar = bar0 + 8u * (stage ^ 1);
      tma::mbar_expect_tx(bar, BYTES);
      tma::load_3d(win0 + (stage ^ 1) * BYTES, &tmap, (next % tiles_x) * TX - 4,
                   (next / tiles_x) * TY - 2, a.z_src, bar);
    }
    const bool ok = tma::mbar_wait(bar0 + 8u * stage, (it >> 1) & 1);
    const float* w = win_smem + stage * (BYTES / 4);
    const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < L.nx && j < L.ny;
    const int gi = i0 + hx, gj = j0 + hy;
    const bool ring = t < NRING && gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny;
    float fw[kQ], fp[kQ], g[kQ];
    if (active) {
      pull_window<true, WPLANE>(w, L, i, j, tx + 4, ty + 2, fw, fp, g, a.k.inv_nx);
      s_th[ty + 1][tx + 1] = sum9(g);
      s_rp[ty + 1][tx + 1] = sum9(fp);
    }
    if (ring) {
      float hw[kQ], hp[kQ], hg[kQ];
      pull_window<false, WPLANE>(w, L, gi, gj, hx + 4, hy + 2, hw, hp, hg, a.k.inv_nx);
      s_th[hy + 1][hx + 1] = sum9(hg);
      s_rp[hy + 1][hx + 1] = sum9(hp);
    }
    if (!ok) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      if (t == 0) {
        atomicOr(a.err, 1);
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
      collide_store<ALLF>(a.k, L, a.dst, i, j, fw, fp, g, thE, thW, thN, thS, rpE, rpW, rpN,
                          rpS);
    }
    __syncthreads();  // the window and the moment tile are free again
  }
}

// ---- streaming only (test hook) -------------------------------------------------------------
__global__ void stream_only_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                   const Layout L, float s) {
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<true>(src, L, i, j, fw, fp, g, s);
    const size_t o = (size_t)j * L.pitch + i;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      dst[(size_t)q * L.plane + o] = fw[q];
      dst[(size_t)(kQ + q) * L.plane + o] = fp[q];
      dst[(size_t)(2 * kQ + q) * L.plane + o] = g[q];
    }
  }
}

// ---- initial equilibrium (Eqs 26-27) ---------------------------------------------------------
__global__ void init_kernel(float* __restrict__ dst, const Layout L, const StepConsts k,
                            const float* __restrict__ warm) {
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    // FP64 here (once per run) so that the stored FP32 values are correctly rounded
    double ux = 0.0, uy = 0.0, th, drw = 0.0, drp = 0.0;
    if (warm) {
      ux = warm[t];
      uy = warm[n + t];
      th = warm[2 * n + t];
      const double phi = warm[3 * n + t];
      // rho^w = 1 - phi, rho^p = phi rho_p / rho_f, as deviations from the initial values
      drw = (1.0 - phi) - k.rho_w0_d;
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
      dst[(size_t)q * L.plane + o] = (float)(W * (drw + rw * P));
      dst[(size_t)(kQ + q) * L.plane + o] = (float)(W * (drp + rp * P));
      dst[(size_t)(2 * kQ + q) * L.plane + o] = (float)(W * (dth + th * P));
    }
  }
}

// ---- macroscopic fields of the post-stream state ----------------------------------------------
__device__ __forceinline__ void node_fields(const StepConsts& k, const Moments& m, int i,
                                            float* v) {
  const float rw = k.rho_w0 + m.rw, rp = k.rho_p0 + m.rp;
  const float rho = rw + rp;
  v[0] = (m.mwx + m.mpx) / rho;
  v[1] = (m.mwy + m.mpy) / rho;
  v[2] = theta_c(k, i) + m.th;
  v[3] = rp * k.phi_per_rho_p;
  v[4] = rw;
  v[5] = rp;
  const bool has_p = k.has_p && rp > 1e-30f;
  v[6] = has_p ? m.mpx / rp : m.mwx / rw;
  v[7] = has_p ? m.mpy / rp : m.mwy / rw;
}

__global__ void fields_kernel(const float* __restrict__ src, const Layout L, const StepConsts k,
                              uint32_t which, float* __restrict__ out) {
  const int64_t n = (int64_t)L.nx * L.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % L.nx), j = (int)(t / L.nx);
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<true>(src, L, i, j, fw, fp, g, k.inv_nx);
    float v[8];
    node_fields(k, moments_of(fw, fp, g), i, v);
    int slot = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
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

// Wall gradients from the theta deviations: with theta = theta_c + theta',
// (8 T_h - 9 theta_0 + theta_1)/3 = 1/nx + (theta'_1 - 9 theta'_0)/3 and the cold-wall twin
// (9 theta_{n-1} - theta_{n-2} - 8 T_c)/3 = 1/nx + (9 theta'_{n-1} - theta'_{n-2})/3.
__global__ void nusselt_kernel(const float* __restrict__ src, const Layout L, float s,
                               double* __restrict__ red) {
  double acc[2] = {0.0, 0.0};
  for (int j = threadIdx.x; j < L.ny; j += blockDim.x) {
    float fw[kQ], fp[kQ], g[kQ];
    pull_node<false>(src, L, 0, j, fw, fp, g, s);
    const double t0 = sum9(g);
    pull_node<false>(src, L, 1, j, fw, fp, g, s);
    const double t1 = sum9(g);
    pull_node<false>(src, L, L.nx - 1, j, fw, fp, g, s);
    const double c0 = sum9(g);
    pull_node<false>(src, L, L.nx - 2, j, fw, fp, g, s);
    const double c1 = sum9(g);
    const double slope = 1.0 / (double)L.nx;
    acc[0] += slope + (t1 - 9.0 * t0) / 3.0;
    acc[1] += slope + (9.0 * c0 - c1) / 3.0;
  }
  block_reduce_store<2>(acc, red);
}

__global__ void mass_kernel(const float* __restrict__ src, const Layout L,
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
      acc[0] += (double)ldg(src + (size_t)q * L.plane + o);
      acc[1] += (double)ldg(src + (size_t)(kQ + q) * L.plane + o);
    }
  }
  block_reduce_store<kRedWidth>(acc, partials + (size_t)blockIdx.x * kRedWidth);
}

__global__ void residual_kernel(const float* __restrict__ src, const Layout L, const StepConsts k,
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
    pull_node<true>(src, L, i, j, fw, fp, g, k.inv_nx);
    float v[8];
    node_fields(k, moments_of(fw, fp, g), i, v);
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

__global__ void state_copy_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                  const Layout L, int to_packed) {
  const int64_t n = (int64_t)L.nx * L.ny;
  const int64_t total = n * kPlanes;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / n, r = t % n;
    const int i = (int)(r % L.nx), j = (int)(r / L.nx);
    const size_t po = (size_t)p * L.plane + (size_t)j * L.pitch + i;
    if (to_packed)
      dst[t] = src[po];
    else
      dst[po] = src[t];
  }
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

StepConfig choose_step_config(int nx, int ny) {
  StepConfig c;
  // default: TMA-staged tiles for lattices with a few tiles per SM, the plain tile kernel below.
  // MCLBM_STEP_VARIANT = tile | tma overrides (diagnostics and comparisons).
  c.variant = (nx >= 64 && ny >= 32) ? 2 : 0;
  const char* v = std::getenv("MCLBM_STEP_VARIANT");
  if (v && std::strcmp(v, "tile") == 0) c.variant = 0;
  if (v && std::strcmp(v, "tma") == 0) c.variant = 2;
  const char* ty = std::getenv("MCLBM_TMA_TILE_Y");
  c.tma_ty = (ty && std::strcmp(ty, "16") == 0) ? 16 : 8;
  c.grid = 0;
  return c;
}

namespace {
template <int TY>
cudaError_t prepare_tma(StepConfig* c, const Layout& L) {
  const size_t smem = TmaTile<TY>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<TY, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(step_tma_kernel<TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tma_kernel<TY, false>,
                                                    kTmaTX * TY, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int tiles = ((L.nx + kTmaTX - 1) / kTmaTX) * ((L.ny + TY - 1) / TY);
  c->grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  return cudaSuccess;
}
}  // namespace

cudaError_t prepare_step(StepConfig* c, const Layout& L) {
  if (c->variant != 2) return cudaSuccess;
  return c->tma_ty == 16 ? prepare_tma<16>(c, L) : prepare_tma<8>(c, L);
}

cudaError_t make_state_tensor_map(CUtensorMap* map, float* state0, const Layout& L, int tile_ty) {
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
  const cuuint64_t dims[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, (cuuint64_t)(2 * kPlanes)};
  const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * 4u, (cuuint64_t)L.plane * 4u};
  const cuuint32_t box[3] = {(cuuint32_t)kTmaWX, (cuuint32_t)(tile_ty + 4), (cuuint32_t)kPlanes};
  const cuuint32_t elem[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, state0, dims, strides, box, elem,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                        cudaStream_t st) {
  // tile and TMA kernels: programmatic dependent launch (the kernel waits on the previous
  // grid itself with griddepcontrol.wait before it reads the state)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const bool all = a.k.mask == MCLBM_F_ALL;
  if (c.variant == 2) {
    if (!map || c.grid < 1) return cudaErrorInvalidValue;
    cfg.gridDim = dim3(c.grid);
    if (c.tma_ty == 16) {
      cfg.blockDim = dim3(kTmaTX * 16);
      cfg.dynamicSmemBytes = TmaTile<16>::SMEM;
      return all ? cudaLaunchKernelEx(&cfg, step_tma_kernel<16, true>, *map, a)
                 : cudaLaunchKernelEx(&cfg, step_tma_kernel<16, false>, *map, a);
    }
    cfg.blockDim = dim3(kTmaTX * 8);
    cfg.dynamicSmemBytes = TmaTile<8>::SMEM;
    return all ? cudaLaunchKernelEx(&cfg, step_tma_kernel<8, true>, *map, a)
               : cudaLaunchKernelEx(&cfg, step_tma_kernel<8, false>, *map, a);
  }
  constexpr int TX = 32, TY = 8;
  cfg.gridDim = dim3((a.L.nx + TX - 1) / TX, (a.L.ny + TY - 1) / TY);
  cfg.blockDim = dim3(TX * TY);
  return all ? cudaLaunchKernelEx(&cfg, step_tile_kernel<TX, TY, true>, a)
             : cudaLaunchKernelEx(&cfg, step_tile_kernel<TX, TY, false>, a);
}

cudaError_t launch_stream_only(const float* src, float* dst, const Layout& L, const StepConsts& k,
                               cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  stream_only_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(src, dst, L, k.inv_nx);
  return cudaGetLastError();
}

cudaError_t launch_init(float* dst, const Layout& L, const StepConsts& k, const float* warm,
                        cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  init_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(dst, L, k, warm);
  return cudaGetLastError();
}

cudaError_t launch_fields(const float* src, const Layout& L, const StepConsts& k, uint32_t which,
                          float* out, cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  fields_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(src, L, k, which, out);
  return cudaGetLastError();
}

cudaError_t launch_nusselt(const float* src, const Layout& L, const StepConsts& k, double* red,
                           cudaStream_t st) {
  nusselt_kernel<<<1, 256, 0, st>>>(src, L, k.inv_nx, red);
  return cudaGetLastError();
}

cudaError_t launch_mass(const float* src, const Layout& L, double* partials, double* red,
                        cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  const int g = grid_for(n, 256, kMaxRedBlocks);
  mass_kernel<<<g, 256, 0, st>>>(src, L, partials);
  final_reduce_kernel<<<1, 256, 0, st>>>(partials, g, red);
  return cudaGetLastError();
}

cudaError_t launch_residual(const float* src, const Layout& L, const StepConsts& k, float* snap,
                            bool sums, double* partials, double* red, cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny;
  const int g = grid_for(n, 256, kMaxRedBlocks);
  residual_kernel<<<g, 256, 0, st>>>(src, L, k, snap, sums ? 1 : 0, partials);
  if (sums) final_reduce_kernel<<<1, 256, 0, st>>>(partials, g, red);
  return cudaGetLastError();
}

cudaError_t launch_state_copy(const float* src, float* dst, const Layout& L, bool to_packed,
                              cudaStream_t st) {
  const int64_t n = (int64_t)L.nx * L.ny * kPlanes;
  state_copy_kernel<<<grid_for(n, 256, 8192), 256, 0, st>>>(src, dst, L, to_packed ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace mcl
