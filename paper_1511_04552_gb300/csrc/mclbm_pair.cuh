// Node-pair form of the fused MCLBM step: every thread updates two x-adjacent nodes (i, i+1),
// i even, with packed FP32x2 arithmetic (one fma.rn.f32x2 / add / mul instruction serves both
// nodes and rounds each lane exactly like its scalar twin). Used by the tile, TMA-staged and
// batched step kernels, so they give bit-identical states. The arithmetic is the method's
// order (Eqs 29-32 moments, Table 1 forces with Eqs 4, 6, 20, the exact drag impulse, Eqs 18,
// 19, 24, 26-28 collision); the lanes of a pair never mix.
//
// Two nodes per thread halve the arithmetic instructions per node, let the aligned planes
// (e_x = 0) load and every plane store as one 8-byte (FP32) or 4-byte (16-bit) access, and let
// 16-bit storage convert both nodes with one cvt (round to nearest, or the hardware's
// stochastic rounding cvt.rs with random bits from a per-node-pair hash).
#pragma once

#include "mclbm_device.cuh"

namespace mcl {
namespace pair {

// ---- lane vectors: V = 1 (float) or V = 2 (float2, packed FP32x2) -----------------------------
// The same sequence of operations on either type: scalar ops use the _rn intrinsics, which the
// compiler never contracts into an fma, and packed ops the FP32x2 intrinsics; a lane of a
// packed op rounds exactly like its scalar twin, so the V = 1 and V = 2 kernels give
// bit-identical states.
template <int V>
struct VecT;
template <>
struct VecT<1> {
  using type = float;
};
template <>
struct VecT<2> {
  using type = float2;
};
template <int V>
using vec = typename VecT<V>::type;

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float neg(float a) { return -a; }
// a - b as b * (-1) + a (exact product, one rounding), the same form as the packed twin
__device__ __forceinline__ float sub(float a, float b) { return __fmaf_rn(b, -1.0f, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }

template <int V>
__device__ __forceinline__ vec<V> bc(float a);  // broadcast
template <>
__device__ __forceinline__ float bc<1>(float a) { return a; }
template <>
__device__ __forceinline__ float2 bc<2>(float a) { return make_float2(a, a); }
template <int V>
__device__ __forceinline__ vec<V> mk(float a, float b);  // lanes (a, b); V = 1 keeps a
template <>
__device__ __forceinline__ float mk<1>(float a, float) { return a; }
template <>
__device__ __forceinline__ float2 mk<2>(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float ln(float v, int) { return v; }
__device__ __forceinline__ float ln(float2 v, int l) { return l ? v.y : v.x; }

// Reciprocal: hardware approximation refined by one Newton-Raphson step r' = r + r (1 - x r),
// which squares the relative error of the approximation (below 2^-22) to about 2^-44, so the
// result is within rounding of 1/x for the normal, positive x of the step (densities, T/T0,
// relaxation times, drag rates).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp(float x) {
  const float r = rcp_approx(x);
  return fma(r, fma(-x, r, 1.0f), r);
}
__device__ __forceinline__ float2 rcp(float2 x) {
  const float2 r = make_float2(rcp_approx(x.x), rcp_approx(x.y));
  return fma(r, fma(neg(x), r, make_float2(1.0f, 1.0f)), r);
}
__device__ __forceinline__ float lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---- storage: pairs and single elements --------------------------------------------------------
// Loads of stored values as FP32 and stores of one node or a pair (lane x at the lower
// address). 16-bit storage holds S = 2^12 times the deviations; the step works in those scaled
// units throughout (a power-of-two scale commutes exactly with every rounding, so the results
// are those of unscaled arithmetic, bit for bit) and folds 1/S into its constants. 16-bit
// stores convert both lanes with one instruction: round to nearest, or stochastic rounding
// (cvt.rs) driven by 32 random bits, the lower 16 for the lower half, the upper 16 for the
// upper half.
template <class T>
struct St;

template <>
struct St<float> {
  __device__ __forceinline__ static float2 ld2(const float* p) {
    return *reinterpret_cast<const float2*>(p);
  }
  __device__ __forceinline__ static float2 ldg2(const float* p) {
    return __ldg(reinterpret_cast<const float2*>(p));
  }
  __device__ __forceinline__ static float ld1(const float* p) { return *p; }
  __device__ __forceinline__ static float ldg1(const float* p) { return __ldg(p); }
  static constexpr int kLog2S = 0;  // stored = deviation
  template <bool SR>
  __device__ __forceinline__ static void st2(float* p, float2 v, uint32_t) {
    *reinterpret_cast<float2*>(p) = v;
  }
  template <bool SR>
  __device__ __forceinline__ static void st1(float* p, float v, uint32_t) { *p = v; }
};

template <class T>
struct St16 {
  // one cvt for two values; sr: stochastic rounding with the random bits r
  __device__ __forceinline__ static uint32_t pack(float2 v, uint32_t r, bool sr);
  __device__ __forceinline__ static float2 ld2(const T* p) {
    return St16::unpack(*reinterpret_cast<const uint32_t*>(p));
  }
  __device__ __forceinline__ static float2 ldg2(const T* p) {
    return St16::unpack(__ldg(reinterpret_cast<const unsigned int*>(p)));
  }
  __device__ __forceinline__ static float2 unpack(uint32_t u);
  __device__ __forceinline__ static float ld1(const T* p);
  __device__ __forceinline__ static float ldg1(const T* p);
  static constexpr int kLog2S = 12;  // stored = 2^12 x deviation (kStoreScale)
  static_assert(kStoreScale == 4096.0f, "16-bit storage scale is 2^12");
  template <bool SR>
  __device__ __forceinline__ static void st2(T* p, float2 v, uint32_t r) {
    *reinterpret_cast<uint32_t*>(p) = pack(v, r, SR);
  }
  template <bool SR>
  __device__ __forceinline__ static void st1(T* p, float v, uint32_t r) {
    *reinterpret_cast<unsigned short*>(p) = (unsigned short)pack(make_float2(v, 0.0f), r, SR);
  }
};
template <>
__device__ __forceinline__ uint32_t St16<__half>::pack(float2 s, uint32_t r, bool sr) {
  uint32_t d;
  if (sr)
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(s.y), "f"(s.x), "r"(r));
  else
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(s.y), "f"(s.x));
  return d;
}
template <>
__device__ __forceinline__ float2 St16<__half>::unpack(uint32_t u) {
  __half2 h;
  memcpy(&h, &u, 4);
  return __half22float2(h);
}
template <>
__device__ __forceinline__ float St16<__half>::ld1(const __half* p) { return __half2float(*p); }
template <>
__device__ __forceinline__ float St16<__half>::ldg1(const __half* p) {
  return __half2float(__ldg(p));
}
template <>
__device__ __forceinline__ uint32_t St16<__nv_bfloat16>::pack(float2 s, uint32_t r, bool sr) {
  uint32_t d;
  if (sr)
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(s.y), "f"(s.x), "r"(r));
  else
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(s.y), "f"(s.x));
  return d;
}
template <>
__device__ __forceinline__ float2 St16<__nv_bfloat16>::unpack(uint32_t u) {
  // a bf16 is the upper half of an FP32 pattern
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}
template <>
__device__ __forceinline__ float St16<__nv_bfloat16>::ld1(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float St16<__nv_bfloat16>::ldg1(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <>
struct St<__half> : St16<__half> {};
template <>
struct St<__nv_bfloat16> : St16<__nv_bfloat16> {};

// Random bits of output plane p of a node (pair) from its hashed seed in one multiply-add: an
// odd multiplier per plane makes the low 16 bits of the result a bijection of the seed's low
// 16 bits (uniform when they are), and the high 16 bits depend on every bit of the seed.
__device__ __forceinline__ uint32_t rbits(uint32_t seed, int p) {
  return seed * (0x9E3779B9u + 2u * (uint32_t)p * 0x6C8E9CF5u) + (uint32_t)p * 0x85EBCA6Bu;
}

// ---- pull streaming ---------------------------------------------------------------------------
// Acc gives the stored value of plane p at node (i + dx, j + dy) (a1(p, dx, dy)) and the
// aligned pair at (i, j + dy), (i + 1, j + dy) (a2(p, dy)), as FP32 in stored units. The wall rules are those
// of pull_node; the g deviations come WITHOUT the drop of theta_c along the link
// (W_q e_qx / nx), which the collision adds (it cancels in every moment).

// One node, its lane d of the accessor (FULL: all 27 planes, else f^p and g only).
template <bool FULL, class Acc>
__device__ __forceinline__ void pull1(const Acc& acc, const Layout& L, int i, int j, int d,
                                      float* fw, float* fp, float* g) {
  if ((unsigned)(i - 1) < (unsigned)(L.nx - 2) && (unsigned)(j - 1) < (unsigned)(L.ny - 2)) {
#pragma unroll
    for (int q = 0; q < kQ; ++q) {  // no link of a node away from the walls leaves the cavity
      if (FULL) fw[q] = acc.a1(q, d - ex(q), -ey(q));
      fp[q] = acc.a1(kQ + q, d - ex(q), -ey(q));
      g[q] = acc.a1(2 * kQ + q, d - ex(q), -ey(q));
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int si = i - ex(q), sj = j - ey(q);
    const bool inx = (unsigned)si < (unsigned)L.nx;
    const bool iny = (unsigned)sj < (unsigned)L.ny;
    if (inx && iny) {
      if (FULL) fw[q] = acc.a1(q, d - ex(q), -ey(q));
      fp[q] = acc.a1(kQ + q, d - ex(q), -ey(q));
      g[q] = acc.a1(2 * kQ + q, d - ex(q), -ey(q));
    } else {
      if (FULL) fw[q] = acc.a1(opp(q), d, 0);
      fp[q] = acc.a1(kQ + opp(q), d, 0);
      g[q] = inx ? acc.a1(2 * kQ + mir(q), d - ex(q), 0) : -acc.a1(2 * kQ + opp(q), d, 0);
    }
  }
}

// The thermal set whose planes start at `base` (27: g^p of the two-thermal-set state) of one
// node, with the thermal wall rules.
template <class Acc>
__device__ __forceinline__ void pull1_thermal(const Acc& acc, const Layout& L, int i, int j, int d,
                                              int base, float* g) {
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int si = i - ex(q), sj = j - ey(q);
    const bool inx = (unsigned)si < (unsigned)L.nx;
    const bool iny = (unsigned)sj < (unsigned)L.ny;
    if (inx && iny)
      g[q] = acc.a1(base + q, d - ex(q), -ey(q));
    else
      g[q] = inx ? acc.a1(base + mir(q), d - ex(q), 0) : -acc.a1(base + opp(q), d, 0);
  }
}

// V nodes (i, i + V - 1). For V = 2, lane y of a pair whose second node lies outside the cavity
// (i + 1 == nx) repeats lane x.
template <int V, bool FULL, class Acc>
__device__ __forceinline__ void pull(const Acc& acc, const Layout& L, int i, int j, vec<V>* fw,
                                     vec<V>* fp, vec<V>* g) {
  if constexpr (V == 1) {
    pull1<FULL>(acc, L, i, j, 0, fw, fp, g);
  } else {
    const bool two = i + 1 < L.nx;
    if (two && (unsigned)(i - 1) < (unsigned)(L.nx - 3) &&
        (unsigned)(j - 1) < (unsigned)(L.ny - 2)) {
      // both nodes away from the walls: no link leaves the cavity
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        if (ex(q) == 0) {
          if (FULL) fw[q] = acc.a2(q, -ey(q));
          fp[q] = acc.a2(kQ + q, -ey(q));
          g[q] = acc.a2(2 * kQ + q, -ey(q));
        } else {
          if (FULL) fw[q] = make_float2(acc.a1(q, -ex(q), -ey(q)), acc.a1(q, 1 - ex(q), -ey(q)));
          fp[q] = make_float2(acc.a1(kQ + q, -ex(q), -ey(q)), acc.a1(kQ + q, 1 - ex(q), -ey(q)));
          g[q] = make_float2(acc.a1(2 * kQ + q, -ex(q), -ey(q)),
                             acc.a1(2 * kQ + q, 1 - ex(q), -ey(q)));
        }
      }
      return;
    }
    float v[2][3][kQ];
    pull1<FULL>(acc, L, i, j, 0, v[0][0], v[0][1], v[0][2]);
    if (two)
      pull1<FULL>(acc, L, i + 1, j, 1, v[1][0], v[1][1], v[1][2]);
    else
      pull1<FULL>(acc, L, i, j, 0, v[1][0], v[1][1], v[1][2]);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      if (FULL) fw[q] = make_float2(v[0][0][q], v[1][0][q]);
      fp[q] = make_float2(v[0][1][q], v[1][1][q]);
      g[q] = make_float2(v[0][2][q], v[1][2][q]);
    }
  }
}

constexpr int kTY = 8;     // tile height (single cavity and batch)
constexpr int kLowTY = 7;  // low tiles: one node per thread, lattices of 1-2 tiles per SM

// Shared-memory window of a TX x TY tile: all 27 planes with XO columns (16 bytes: TMA's x
// alignment) and 2 rows of halo on each side. PADDED rounds its size up to 128 bytes, where an
// output tile may follow.
template <class T, int TX, int TY = kTY>
struct PairWin {
  static constexpr int XO = 16 / (int)sizeof(T);
  static constexpr int WX = TX + 2 * XO;
  static constexpr int WY = TY + 4;
  static constexpr int WPLANE = WX * WY;
  static constexpr uint32_t BYTES = (uint32_t)kPlanes * WPLANE * sizeof(T);
  static constexpr uint32_t PADDED = (BYTES + 127u) / 128u * 128u;
  static_assert(BYTES % 16 == 0, "TMA transfers of 16-byte multiples");
};

// Accessor of a shared-memory window: element (wx, wy) of plane p at w[p * WPLANE + wy * WX + wx];
// base = the position of node i (lane x).
template <class T, int TX, int TY = kTY>
struct WinAcc {
  const T* base;
  static constexpr int WX = PairWin<T, TX, TY>::WX, WPLANE = PairWin<T, TX, TY>::WPLANE;
  __device__ __forceinline__ float a1(int p, int dx, int dy) const {
    return St<T>::ld1(base + p * WPLANE + dy * WX + dx);
  }
  __device__ __forceinline__ float2 a2(int p, int dy) const {
    return St<T>::ld2(base + p * WPLANE + dy * WX);
  }
};

// Accessor of a state level in global memory (read-only path); base = src + j * pitch + i.
template <class T>
struct GlobAcc {
  const T* base;
  int pitch;
  size_t plane;
  __device__ __forceinline__ float a1(int p, int dx, int dy) const {
    return St<T>::ldg1(base + (size_t)p * plane + (ptrdiff_t)dy * pitch + dx);
  }
  __device__ __forceinline__ float2 a2(int p, int dy) const {
    return St<T>::ldg2(base + (size_t)p * plane + (ptrdiff_t)dy * pitch);
  }
};

template <class X>
__device__ __forceinline__ X sum9(const X* a) {
  return add(add(add(add(a[0], a[1]), add(a[2], a[3])), add(add(a[4], a[5]), add(a[6], a[7]))),
             a[8]);
}
template <class X>
__device__ __forceinline__ X mom_x(const X* a) {
  return add(add(sub(a[1], a[3]), sub(a[5], a[6])), sub(a[8], a[7]));
}
template <class X>
__device__ __forceinline__ X mom_y(const X* a) {
  return add(add(sub(a[2], a[4]), sub(a[5], a[8])), sub(a[6], a[7]));
}

// Eq 33 with two thermal sets: the mixture temperature's deviation from theta_c, in the stored
// units of T, from the sums of the populations of the four sets (srw, srp: f^w, f^p; sw, sp:
// g^w, g^p): the heat-capacity weighted mean (weights rho^w and r rho^p, r = C_p,p / C_p,f).
template <class T>
__device__ __forceinline__ float mixture_s(const StepConsts& k, float srw, float srp, float sw,
                                           float sp) {
  constexpr float iS = 1.0f / (float)(1 << St<T>::kLog2S);
  const float rw = fma(srw, iS, k.rho_w0), rp = fma(srp, iS, k.rho_p0);
  const float cp = mul(k.r_cp, rp);
  return mul(fma(rw, sw, mul(cp, sp)), rcp(add(rw, cp)));
}

// Nearest wall of node (i, j) (ties: left, right, bottom, top): zeta = (2z/H)(0.63 - 2z/H) times
// the inward normal (Table 1 Magnus profile).
__device__ __forceinline__ void magnus_profile(const StepConsts& k, const Layout& L, int i, int j,
                                               float& px, float& py) {
  float z = (float)i + 0.5f, nrx = 1.0f, nry = 0.0f;
  const float dr = (float)(L.nx - i) - 0.5f, db = (float)j + 0.5f;
  const float dt = (float)(L.ny - j) - 0.5f;
  if (dr < z) { z = dr; nrx = -1.0f; nry = 0.0f; }
  if (db < z) { z = db; nrx = 0.0f; nry = 1.0f; }
  if (dt < z) { z = dt; nrx = 0.0f; nry = -1.0f; }
  const float zH = mul(z, k.two_over_ny);
  const float zeta = mul(zH, sub(0.63f, zH));
  px = mul(zeta, nrx);
  py = mul(zeta, nry);
}

// Steps A2-A7 for the V nodes (i, ..., i + V - 1) of row j. Populations, their moments and the
// neighbours' theta and rho^p deviations thE..rpS (ghosts applied by the caller; theta_c's
// slope -1/nx is added to d theta/dx here) are in the stored units of T (S times the
// deviations); out(p, v) receives the 27 post-collision values in the same units. TWO: the
// two-thermal-set state (g = g^w, gp = g^p; theta is the Eq 33 mixture; 36 outputs).
template <int V, bool ALLF, class T, bool TWO, class Sink>
__device__ __forceinline__ void collide(const StepConsts& k, const Layout& L, Sink& out, int i,
                                        int j, const vec<V>* fw, const vec<V>* fp,
                                        const vec<V>* g, const vec<V>* gp, vec<V> thE,
                                        vec<V> thW, vec<V> thN, vec<V> thS, vec<V> rpE,
                                        vec<V> rpW, vec<V> rpN, vec<V> rpS) {
  using X = vec<V>;
  static_assert(!TWO || V == 1, "two thermal sets: one node per thread");
  constexpr float S = (float)(1 << St<T>::kLog2S), iS = 1.0f / S;
  // x / S (exact; no instruction when S = 1)
  auto unscale = [&](X x) {
    if constexpr (St<T>::kLog2S == 0) return x; else return mul(x, bc<V>(iS));
  };
  const uint32_t mask = ALLF ? MCLBM_F_ALL : k.mask;
  const X mrw = sum9(fw), mrp = sum9(fp);
  X mth;
  if constexpr (TWO)
    mth = mixture_s<T>(k, mrw, mrp, sum9(g), sum9(gp));
  else
    mth = sum9(g);
  const X mwx = mom_x(fw), mwy = mom_y(fw), mpx = mom_x(fp), mpy = mom_y(fp);
  // theta_c of each node from its own column (so a lane rounds like the node alone)
  const X thc = mk<V>(fma(-(float)i, k.inv_nx, k.th_c0), fma(-(float)(i + 1), k.inv_nx, k.th_c0));
  const X th = fma(mth, bc<V>(iS), thc);  // absolute temperature
  const X rw = fma(mrw, bc<V>(iS), bc<V>(k.rho_w0));
  const X rp = fma(mrp, bc<V>(iS), bc<V>(k.rho_p0));
  const X rho = add(rw, rp);
  const X inv_rho = rcp(rho);
  const X Yw = mul(rw, inv_rho), Yp = mul(rp, inv_rho);
  const X inv_rho_s = unscale(inv_rho);
  const X ux = mul(add(mwx, mpx), inv_rho_s);  // Eq 32, barycentric
  const X uy = mul(add(mwy, mpy), inv_rho_s);
  const X inv_rw = rcp(rw);
  const X inv_rw_s = unscale(inv_rw);
  const X uwx = mul(mwx, inv_rw_s), uwy = mul(mwy, inv_rw_s);
  // lanes without particles (phi0 = 0, or rho^p <= 1e-30): u^p := u^w, no particle forces
  bool hp[2];
#pragma unroll
  for (int l = 0; l < V; ++l) hp[l] = k.has_p && ln(rp, l) > 1e-30f;
  const bool any_p = V == 1 ? hp[0] : (hp[0] || hp[V - 1]);
  const bool all_p = V == 1 ? hp[0] : (hp[0] && hp[V - 1]);
  const X inv_rp0 = rcp(rp);
  const X inv_rp = mk<V>(hp[0] ? ln(inv_rp0, 0) : 0.0f, hp[V - 1] ? ln(inv_rp0, 1) : 0.0f);
  const X inv_rp_s = unscale(inv_rp);
  const X upx0 = mul(mpx, inv_rp_s), upy0 = mul(mpy, inv_rp_s);
  const X upx = mk<V>(hp[0] ? ln(upx0, 0) : ln(uwx, 0), hp[V - 1] ? ln(upx0, 1) : ln(uwx, 1));
  const X upy = mk<V>(hp[0] ? ln(upy0, 0) : ln(uwy, 0), hp[V - 1] ? ln(upy0, 1) : ln(uwy, 1));

  // external forces: Boussinesq buoyancy on the fluid, gravity pair (Eq 20, Table 1)
  const X Fbuoy = (mask & MCLBM_F_BUOYANCY) ? mul(mul(rho, bc<V>(k.buoy)), th) : bc<V>(0.0f);
  const bool grav = (mask & MCLBM_F_GRAVITY) != 0;
  X Fwx = bc<V>(0.0f), Fwy = bc<V>(0.0f), Fpx = bc<V>(0.0f), Fpy = bc<V>(0.0f);
  if (any_p) {
    // particle-fluid interaction forces on the particle phase (reaction on the fluid)
    X Fix = bc<V>(0.0f), Fiy = bc<V>(0.0f);
    const X TT0 = fma(th, bc<V>(k.t_ratio), bc<V>(1.0f));  // T / T0
    const X wx = sub(uwx, upx), wy = sub(uwy, upy);
    if (mask & MCLBM_F_BROWNIAN) {  // -cB rho^p (T/T0)^2 grad rho^p
      const X c = mul(mul(rp, bc<V>(-0.5f * iS * k.cB)), mul(TT0, TT0));
      Fix = mul(c, sub(rpE, rpW));
      Fiy = mul(c, sub(rpN, rpS));
    }
    if (mask & MCLBM_F_THERMOPHORESIS) {  // -cT rho^p grad theta / (T/T0)
      const X c = mul(mul(rp, bc<V>(-k.cT)), rcp(TT0));
      Fix = fma(c, fma(bc<V>(0.5f * iS), sub(thE, thW), bc<V>(-k.inv_nx)), Fix);
      Fiy = fma(c, mul(bc<V>(0.5f * iS), sub(thN, thS)), Fiy);
    }
    if (mask & MCLBM_F_SAFFMAN) {  // cS rho^p |u^p|^(1/2) R90(u^w - u^p)
      const X q = fma(upx, upx, mul(upy, upy));
      const X q4 = mk<V>(ex2(0.25f * lg2(ln(q, 0))), ex2(0.25f * lg2(ln(q, 1))));
      const X c = mul(mul(rp, bc<V>(k.cS)), q4);
      Fix = fma(c, neg(wy), Fix);
      Fiy = fma(c, wx, Fiy);
    }
    if (mask & MCLBM_F_MAGNUS) {  // cM rho^p |u^w + u^p|^2 zeta(z) n_wall
      float p0x, p0y, p1x = 0.0f, p1y = 0.0f;
      magnus_profile(k, L, i, j, p0x, p0y);
      if (V == 2) magnus_profile(k, L, i + 1, j, p1x, p1y);
      const X sx = add(uwx, upx), sy = add(uwy, upy);
      const X c = mul(mul(rp, bc<V>(k.cM)), fma(sx, sx, mul(sy, sy)));
      Fix = fma(c, mk<V>(p0x, p1x), Fix);
      Fiy = fma(c, mk<V>(p0y, p1y), Fiy);
    }
    // non-drag forces: particles F_int + F_G, fluid F_buoy + F_G0 - F_int
    const X FGp = grav ? mul(rp, bc<V>(-k.gG)) : bc<V>(0.0f);
    const float FG0w = grav ? mul(k.rho_p0, k.gG) : 0.0f;
    const X Fpnx = Fix, Fpny = add(Fiy, FGp);
    const X Fwnx = neg(Fix);
    const X Fwny = sub(add(Fbuoy, bc<V>(FG0w)), Fiy);
    if (mask & MCLBM_F_DRAG) {
      // Exact drag impulse over the step (slip ODE dw/dt = -a w + b from the relaxed slip),
      // rearranged so that the large interaction forces cancel before rounding:
      // F^p = Y_p F_tot + mu_r [(1 - e^-a) w' - ((1 - e^-a)/a) b], F^w = F_tot - F^p.
      // Schiller-Naumann correction 0.15 Re^0.687 = 0.15 2^(0.687 log2 cRe + 0.3435 log2 |w|^2);
      // Re is 1e-8..1e-3 here, so the correction is below 1e-3 of the Stokes rate and the
      // hardware log2 / exp2 suffice (|w| = 0 gives log2 = -inf and exp2 = 0).
      const X w2 = fma(wx, wx, mul(wy, wy));
      const float lc = 0.687f * lg2(k.cRe);
      const X sn = mk<V>(ex2(fma(0.3435f, lg2(ln(w2, 0)), lc)), ex2(fma(0.3435f, lg2(ln(w2, 1)), lc)));
      const X beta = mul(bc<V>(k.beta_dt), fma(bc<V>(0.15f), sn, bc<V>(1.0f)));
      const X a = mul(beta, fma(rp, inv_rw, bc<V>(1.0f)));
      // e^-a is below FP32 resolution of 1 for a > 20 (nanoparticles: a = 1e3..1e7)
      X E = bc<V>(1.0f), Ea = rcp(a);
      if (ln(a, 0) <= 20.0f || ln(a, 1) <= 20.0f) {
        float e[2], r[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const float al = ln(a, l);
          const float El = al > 20.0f ? 1.0f : -expm1f(-al);
          r[l] = (al < 1e-2f) ? 1.0f - al * (0.5f - al * (1.0f / 6.0f - al * (1.0f / 24.0f)))
                              : mul(El, ln(Ea, l));
          e[l] = El;
        }
        E = mk<V>(e[0], e[1]);
        Ea = mk<V>(r[0], r[1]);
      }
      const X mu_r = mul(mul(rw, rp), inv_rho);
      const X relax = fma(Yp, bc<V>(-k.inv_tau_w), fma(Yw, bc<V>(-k.inv_tau_p), bc<V>(1.0f)));
      const X bx = fma(Fwnx, inv_rw, mul(neg(Fpnx), inv_rp));
      const X by = fma(Fwny, inv_rw, mul(neg(Fpny), inv_rp));
      // F_tot: the interaction forces cancel exactly; gravity pair = -(rho^p - rho_p0) gG
      const X Fty = grav ? fma(mrp, bc<V>(-iS * k.gG), Fbuoy) : Fbuoy;
      const X Er = mul(E, relax);
      Fpx = mul(mu_r, fma(Er, wx, mul(neg(Ea), bx)));
      Fpy = fma(Yp, Fty, mul(mu_r, fma(Er, wy, mul(neg(Ea), by))));
      Fwx = neg(Fpx);
      Fwy = sub(Fty, Fpy);
    } else {
      Fpx = Fpnx;
      Fpy = Fpny;
      Fwx = Fwnx;
      Fwy = Fwny;
    }
  }
  if (!all_p) {  // a lane without particles: buoyancy (and the gravity reference) only
    const X Fw0 = add(Fbuoy, bc<V>(grav ? mul(k.rho_p0, k.gG) : 0.0f));
    Fwx = mk<V>(hp[0] ? ln(Fwx, 0) : 0.0f, hp[V - 1] ? ln(Fwx, 1) : 0.0f);
    Fwy = mk<V>(hp[0] ? ln(Fwy, 0) : ln(Fw0, 0), hp[V - 1] ? ln(Fwy, 1) : ln(Fw0, 1));
    Fpx = mk<V>(hp[0] ? ln(Fpx, 0) : 0.0f, hp[V - 1] ? ln(Fpx, 1) : 0.0f);
    Fpy = mk<V>(hp[0] ? ln(Fpy, 0) : 0.0f, hp[V - 1] ? ln(Fpy, 1) : 0.0f);
  }

  // BGK collision with forcing 3 W_q e_q.F on the common velocity (Eqs 18, 26), in deviation
  // form: f' <- (1 - 1/tau) f' + (W_q rho' + rho P_q) / tau + A_q e_q.F; g likewise with theta,
  // plus the drop of theta_c along the link that streaming left out, (1 - 1/tau) W_q e_qx / nx.
  // Opposite directions share the even part of P_q (B (e.u)^2 - C u.u) and negate the odd part
  // (A e.u), the forcing and the theta_c drop, so the loop runs over the four pairs (q, -q).
  // thermal relaxation: one set with tau of Eq 24 at the local fractions, or two sets with
  // their own times (g^w as om_t, g^p as om_t2)
  const X om_t = TWO ? bc<V>(rcp(k.tau_tw))
                     : rcp(fma(Yw, bc<V>(k.tau_tw), mul(Yp, bc<V>(k.tau_tp))));
  const X om_t2 = bc<V>(TWO ? rcp(k.tau_tp) : 0.0f);
  const X keep_t2 = sub(bc<V>(1.0f), om_t2);
  const X om_w = bc<V>(k.inv_tau_w), om_p = bc<V>(k.inv_tau_p);
  const X keep_w = bc<V>(sub(1.0f, k.inv_tau_w)), keep_p = bc<V>(sub(1.0f, k.inv_tau_p));
  const X keep_t = sub(bc<V>(1.0f), om_t);
  const X usq = fma(ux, ux, mul(uy, uy));
  const X ck1 = mul(keep_t, bc<V>(mul(S * wq(1), k.inv_nx)));
  const X ck5 = mul(keep_t, bc<V>(mul(S * wq(5), k.inv_nx)));
  const X ck1b = mul(keep_t2, bc<V>(mul(S * wq(1), k.inv_nx)));
  const X ck5b = mul(keep_t2, bc<V>(mul(S * wq(5), k.inv_nx)));
  X sw = bc<V>(0.0f), sp = bc<V>(0.0f), sg = bc<V>(0.0f);  // half the sum of the moving equilibria
#pragma unroll
  for (int pr = 0; pr < 4; ++pr) {
    const int q = pr == 0 ? 1 : (pr == 1 ? 2 : (pr == 2 ? 5 : 6));
    const int qo = opp(q);
    const X eu = q == 1 ? ux : (q == 2 ? uy : (q == 5 ? add(ux, uy) : sub(uy, ux)));
    // in stored units: the polynomial's coefficients carry S
    const X even = fma(mul(bc<V>(S * bq(q)), eu), eu, mul(bc<V>(-S * cq(q)), usq));
    const X odd = mul(bc<V>(S * aq(q)), eu);
    const X W = bc<V>(wq(q));
    const X tw = fma(rw, even, mul(W, mrw)), dw = mul(rw, odd);
    const X tp = fma(rp, even, mul(W, mrp)), dp = mul(rp, odd);
    const X tg = fma(th, even, mul(W, mth)), dg = mul(th, odd);
    sw = add(sw, tw);
    sp = add(sp, tp);
    sg = add(sg, tg);
    const X efw = q == 1 ? Fwx : (q == 2 ? Fwy : (q == 5 ? add(Fwx, Fwy) : sub(Fwy, Fwx)));
    const X efp = q == 1 ? Fpx : (q == 2 ? Fpy : (q == 5 ? add(Fpx, Fpy) : sub(Fpy, Fpx)));
    const X Sw = mul(bc<V>(S * aq(q)), efw), Sp = mul(bc<V>(S * aq(q)), efp);
    // theta_c drop for q (e_qx = +1 for q = 1, 5; -1 for q = 6; 0 for q = 2) and -q
    const X ck = q == 1 ? ck1 : (q == 5 ? ck5 : (q == 6 ? neg(ck5) : bc<V>(0.0f)));
    out(q, fma(fw[q], keep_w, fma(om_w, add(tw, dw), Sw)));
    out(qo, fma(fw[qo], keep_w, fma(om_w, sub(tw, dw), neg(Sw))));
    out(kQ + q, fma(fp[q], keep_p, fma(om_p, add(tp, dp), Sp)));
    out(kQ + qo, fma(fp[qo], keep_p, fma(om_p, sub(tp, dp), neg(Sp))));
    out(2 * kQ + q, fma(g[q], keep_t, fma(om_t, add(tg, dg), ck)));
    out(2 * kQ + qo, fma(g[qo], keep_t, fma(om_t, sub(tg, dg), neg(ck))));
    if constexpr (TWO) {  // g^p towards the same (mixture) equilibrium
      const X ckb = q == 1 ? ck1b : (q == 5 ? ck5b : (q == 6 ? neg(ck5b) : bc<V>(0.0f)));
      out(3 * kQ + q, fma(gp[q], keep_t2, fma(om_t2, add(tg, dg), ckb)));
      out(3 * kQ + qo, fma(gp[qo], keep_t2, fma(om_t2, sub(tg, dg), neg(ckb))));
    }
  }
  // rest populations: equilibrium = zeroth moment minus the moving equilibria
  out(0, fma(fw[0], keep_w, mul(om_w, fma(bc<V>(-2.0f), sw, mrw))));
  out(kQ, fma(fp[0], keep_p, mul(om_p, fma(bc<V>(-2.0f), sp, mrp))));
  out(2 * kQ, fma(g[0], keep_t, mul(om_t, fma(bc<V>(-2.0f), sg, mth))));
  if constexpr (TWO) out(3 * kQ, fma(gp[0], keep_t2, mul(om_t2, fma(bc<V>(-2.0f), sg, mth))));
}

// ---- output sinks ------------------------------------------------------------------------------
// V nodes to a state level in global memory (tile kernel, FP32 TMA kernel); base = dst + node
// offset of lane x; a pair's lane y is written only when its node is inside the cavity.
template <class T, bool SR, int V>
struct GlobSink {
  T* base;
  size_t plane;
  uint32_t seed;
  bool two;
  __device__ __forceinline__ void operator()(int p, vec<V> v) const {
    const uint32_t r = SR ? rbits(seed, p) : 0u;
    if constexpr (V == 2) {
      if (two) {
        St<T>::template st2<SR>(base + (size_t)p * plane, v, r);
        return;
      }
    }
    St<T>::template st1<SR>(base + (size_t)p * plane, ln(v, 0), r);
  }
};

// V nodes into a [27][TY][TX] shared-memory output tile (TMA-stored afterwards, which clips
// the columns outside the cavity).
template <class T, bool SR, int STRIDE, int V>
struct TileSink {
  T* base;  // tile + ty * TX + column of lane x
  uint32_t seed;
  __device__ __forceinline__ void operator()(int p, vec<V> v) const {
    const uint32_t r = SR ? rbits(seed, p) : 0u;
    if constexpr (V == 2)
      St<T>::template st2<SR>(base + p * STRIDE, v, r);
    else
      St<T>::template st1<SR>(base + p * STRIDE, v, r);
  }
};

// ---- the body of one tile ------------------------------------------------------------------
// Moments of the tile's nodes and of the ring around it (theta' and rho'^p after streaming) in
// shared memory: rows -1..TY, columns -1..TX at [row + 1][col + 2] (pairs 8-byte aligned).
template <int TX, int TY>
struct MomTile {
  static constexpr int W = TX + 4;
  float th[TY + 2][W];
  float rp[TY + 2][W];
};

// Thread t of a TX x TY tile with V nodes per thread: its nodes (V c, row) with c = t % (TX/V).
// Ring tasks: V = 2: t < TX / 2 a pair of the row below, t < TX one of the row above,
// t < TX + TY the left and right ring nodes of row t - TX. V = 1: t < TX the row below,
// t < 2 TX the row above, t < 2 TX + TY the left column, t < 2 TX + 2 TY the right column.
template <int TX, int TY, int V>
struct TileThread {
  static constexpr int NC = TX / V;  // threads per row
  static constexpr int NT = NC * TY;
  static_assert(V == 2 ? TX + TY <= NT : 2 * TX + 2 * TY <= NT, "one ring task per thread");
  int c, ty;
  __device__ __forceinline__ explicit TileThread(int t) : c(t % NC), ty(t / NC) {}
};

template <class X>
__device__ __forceinline__ void put_mom(float* row, int col, X v);
template <>
__device__ __forceinline__ void put_mom<float>(float* row, int col, float v) { row[col] = v; }
template <>
__device__ __forceinline__ void put_mom<float2>(float* row, int col, float2 v) {
  *reinterpret_cast<float2*>(row + col) = v;
}

// Phase 1 of a tile: pulls of the thread's nodes (kept in fw, fp, g and, with two thermal
// sets, gp) and of its ring task; their theta' (the Eq 33 mixture with two sets) and rho'^p go
// to the moment tile. acc_at(dx, dy) returns the accessor of the node at tile position (dx, dy).
template <int TX, int TY, int V, class T, bool TWO, class AccAt>
__device__ __forceinline__ void tile_pull(const AccAt& acc_at, const Layout& L,
                                          const StepConsts& k, int i0, int j0, int t,
                                          MomTile<TX, TY>& mt, vec<V>* fw, vec<V>* fp, vec<V>* g,
                                          vec<V>* gp) {
  static_assert(!TWO || V == 1, "two thermal sets: one node per thread");
  const TileThread<TX, TY, V> tt(t);
  const int i = i0 + V * tt.c, j = j0 + tt.ty;
  if (i < L.nx && j < L.ny) {
    pull<V, true>(acc_at(V * tt.c, tt.ty), L, i, j, fw, fp, g);
    if constexpr (TWO) {
      pull1_thermal(acc_at(tt.c, tt.ty), L, i, j, 0, 3 * kQ, gp);
      put_mom(mt.th[tt.ty + 1], tt.c + 2, mixture_s<T>(k, sum9(fw), sum9(fp), sum9(g), sum9(gp)));
    } else {
      put_mom(mt.th[tt.ty + 1], V * tt.c + 2, sum9(g));
    }
    put_mom(mt.rp[tt.ty + 1], V * tt.c + 2, sum9(fp));
  }
  // a ring node's moments: theta' (or the mixture's) and rho'^p of the pulled node
  auto ring1 = [&](int dx, int dy, int hi, int hj, float& th, float& rp) {
    float hw[kQ], hp[kQ], hg[kQ];
    if constexpr (TWO) {
      float hg2[kQ];
      pull1<true>(acc_at(dx, dy), L, hi, hj, 0, hw, hp, hg);
      pull1_thermal(acc_at(dx, dy), L, hi, hj, 0, 3 * kQ, hg2);
      th = mixture_s<T>(k, sum9(hw), sum9(hp), sum9(hg), sum9(hg2));
    } else {
      pull1<false>(acc_at(dx, dy), L, hi, hj, 0, nullptr, hp, hg);
      th = sum9(hg);
    }
    rp = sum9(hp);
  };
  constexpr int NR = V == 2 ? TX : 2 * TX;  // ring-row tasks
  if (t < NR) {  // ring rows: below and above the tile
    const int hy = t < NR / 2 ? -1 : TY;
    const int hx = V * (t % (NR / 2));
    const int hi = i0 + hx, hj = j0 + hy;
    if (hj >= 0 && hj < L.ny && hi < L.nx) {
      if constexpr (V == 1) {
        float th, rp;
        ring1(hx, hy, hi, hj, th, rp);
        mt.th[hy + 1][hx + 2] = th;
        mt.rp[hy + 1][hx + 2] = rp;
      } else {
        vec<V> hp[kQ], hg[kQ];
        pull<V, false>(acc_at(hx, hy), L, hi, hj, nullptr, hp, hg);
        put_mom(mt.th[hy + 1], hx + 2, sum9(hg));
        put_mom(mt.rp[hy + 1], hx + 2, sum9(hp));
      }
    }
  } else if (t < NR + (V == 2 ? TY : 2 * TY)) {  // ring columns
    const int r = t - NR;
    const int hy = V == 2 ? r : r % TY, hj = j0 + hy;
    // V = 2: both sides in one thread; V = 1: left for r < TY, right otherwise
    const bool left = V == 2 || r < TY, right = V == 2 || r >= TY;
    if (hj < L.ny && left && i0 > 0) ring1(-1, hy, i0 - 1, hj, mt.th[hy + 1][1], mt.rp[hy + 1][1]);
    if (hj < L.ny && right && i0 + TX < L.nx)
      ring1(TX, hy, i0 + TX, hj, mt.th[hy + 1][TX + 2], mt.rp[hy + 1][TX + 2]);
  }
}

// Phase 2 of a tile (after a barrier): neighbours' moments with the wall ghosts, then the
// collision of the thread's nodes into the sink.
template <bool ALLF, int TX, int TY, int V, class T, bool TWO, class Sink>
__device__ __forceinline__ void tile_collide(const StepConsts& k, const Layout& L, int i0, int j0,
                                             int t, const MomTile<TX, TY>& mt, const vec<V>* fw,
                                             const vec<V>* fp, const vec<V>* g, const vec<V>* gp,
                                             Sink& out) {
  using X = vec<V>;
  const TileThread<TX, TY, V> tt(t);
  const int i = i0 + V * tt.c, j = j0 + tt.ty;
  if (!(i < L.nx && j < L.ny)) return;
  const int r = tt.ty + 1, c = V * tt.c + 2;
  X th, rp, thN, thS, rpN, rpS;
  if constexpr (V == 2) {
    th = *reinterpret_cast<const float2*>(&mt.th[r][c]);
    rp = *reinterpret_cast<const float2*>(&mt.rp[r][c]);
    thN = j + 1 < L.ny ? *reinterpret_cast<const float2*>(&mt.th[r + 1][c]) : th;
    thS = j > 0 ? *reinterpret_cast<const float2*>(&mt.th[r - 1][c]) : th;
    rpN = j + 1 < L.ny ? *reinterpret_cast<const float2*>(&mt.rp[r + 1][c]) : rp;
    rpS = j > 0 ? *reinterpret_cast<const float2*>(&mt.rp[r - 1][c]) : rp;
  } else {
    th = mt.th[r][c];
    rp = mt.rp[r][c];
    thN = j + 1 < L.ny ? mt.th[r + 1][c] : th;
    thS = j > 0 ? mt.th[r - 1][c] : th;
    rpN = j + 1 < L.ny ? mt.rp[r + 1][c] : rp;
    rpS = j > 0 ? mt.rp[r - 1][c] : rp;
  }
  // theta deviations: the isothermal ghost 2 T_wall - theta is -theta' in deviation form;
  // adiabatic walls and every wall for rho^p: the ghost is the node's own value
  const float th0 = ln(th, 0), th1 = ln(th, 1), rp0 = ln(rp, 0), rp1 = ln(rp, 1);
  const float thW0 = i > 0 ? mt.th[r][c - 1] : -th0;
  const float rpW0 = i > 0 ? mt.rp[r][c - 1] : rp0;
  const float thE0 = i + 1 < L.nx ? (V == 2 ? th1 : mt.th[r][c + 1]) : -th0;
  const float rpE0 = i + 1 < L.nx ? (V == 2 ? rp1 : mt.rp[r][c + 1]) : rp0;
  const float thE1 = V == 2 && i + 2 < L.nx ? mt.th[r][c + 2] : -th1;
  const float rpE1 = V == 2 && i + 2 < L.nx ? mt.rp[r][c + 2] : rp1;
  collide<V, ALLF, T, TWO>(k, L, out, i, j, fw, fp, g, gp, mk<V>(thE0, thE1), mk<V>(thW0, th0),
                           thN, thS,
                   mk<V>(rpE0, rpE1), mk<V>(rpW0, rp0), rpN, rpS);
}

// ---- kernels ---------------------------------------------------------------------------------
// Tiles of TX x TY nodes with V nodes per thread: TX / V threads per tile row. The
// single-cavity kernels use 32-wide tiles (with two nodes per thread: four CTAs of 128 threads
// per SM, which hide the window loads of each other better than two of 256); the batch uses 64.
// Tiles are 8 rows high, or 7 (one node per thread, 224 threads) on lattices where 32 x 8
// tiles would put a second tile on some SMs and 32 x 7 tiles still fit two per SM.
constexpr int kTileW = 32;  // single-cavity tile width
template <int V, int TX, int TY = kTY>
struct Threads {
  static constexpr int value = TX / V * TY;
};
// resident CTAs per SM the register budget is sized for (at least 128 registers per thread)
template <int V, int TX, int TY = kTY>
struct MinBlocks {
  static constexpr int fit = 65536 / 128 / Threads<V, TX, TY>::value;
  static constexpr int value = fit > 4 ? 4 : (fit < 1 ? 1 : fit);
};

// Plain tile kernel (small lattices): pulls from global memory (L1/L2), one tile per CTA.
template <class T, bool SR, bool ALLF, int V, bool TWO = false>
__global__ void __launch_bounds__(Threads<V, kTileW>::value, MinBlocks<V, kTileW>::value)
    step_pair_tile_kernel(const StepArgs a) {
  constexpr int kTX = kTileW;
  __shared__ __align__(16) MomTile<kTX, kTY> mt;
  const Layout L = a.L;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY;
  vec<V> fw[kQ], fp[kQ], g[kQ], gp[TWO ? kQ : 1];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous step has completed
  auto acc_at = [&](int dx, int dy) {
    return GlobAcc<T>{src + (ptrdiff_t)(j0 + dy) * L.pitch + (i0 + dx), L.pitch, L.plane};
  };
  tile_pull<kTX, kTY, V, T, TWO>(acc_at, L, a.k, i0, j0, t, mt, fw, fp, g, gp);
  __syncthreads();
  const TileThread<kTX, kTY, V> tt(t);
  const int i = i0 + V * tt.c, j = j0 + tt.ty;
  const size_t o = (size_t)j * L.pitch + i;
  GlobSink<T, SR, V> out{static_cast<T*>(a.dst) + o, L.plane,
                         SR ? mix32((uint32_t)o ^ step_hash(a)) : 0u, i + 1 < L.nx};
  tile_collide<ALLF, kTX, kTY, V, T, TWO>(a.k, L, i0, j0, t, mt, fw, fp, g, gp, out);
}

// Shared memory of the TMA-staged kernels: one input window and, where it fits the CTAs per
// SM the kernel runs with, an output tile written back by one TMA store (16-bit storage; FP32
// with one node per thread). FP32 with two nodes per thread (four CTAs per SM) stores each
// pair straight to global memory.
template <class T, int V, int TX_, int TY_ = kTY>
struct TmaPair {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int XO = PairWin<T, TX, TY>::XO;
  static constexpr int WX = PairWin<T, TX, TY>::WX;
  static constexpr uint32_t BYTES = PairWin<T, TX, TY>::BYTES;  // one input window
  static constexpr uint32_t OUT_AT = PairWin<T, TX, TY>::PADDED;  // the output tile's offset
  static constexpr bool STORE_TMA = sizeof(T) == 2 || V == 1;
  static constexpr uint32_t OUT_BYTES = STORE_TMA ? (uint32_t)kPlanes * TX * TY * sizeof(T) : 0;
  static constexpr size_t SMEM = STORE_TMA ? (size_t)OUT_AT + OUT_BYTES : (size_t)BYTES;
};

struct TmaTileDesc {
  const CUtensorMap* map;
  const CUtensorMap* map_out;
  int z, z_out;
  int i0, j0;
  const Layout& L;
  const StepConsts& k;
  void* dst;
  uint32_t hash;
};

// The tile loop of the TMA-staged persistent kernels (single cavity and batch). For every
// tile one TMA tensor load brings the 27-plane window into shared memory; once the pulls have
// read it (first barrier) thread 0 issues the next tile's load into the same buffer, so the
// load overlaps the collision; several CTAs per SM overlap each other. Every mbarrier wait is
// bounded (2 s): on timeout the CTA sets bit 0 of the error word, drains its copies (bounded)
// and returns. tile_of(tile) gives the tile's TmaTileDesc.
template <class T, bool SR, bool ALLF, int V, int TX, int TY, class TileOf>
__device__ __forceinline__ void tma_tile_loop(const TileOf& tile_of, int n_tiles, int* err) {
  using TP = TmaPair<T, V, TX, TY>;
  constexpr int kTX = TX;
  constexpr uint32_t BYTES = TP::BYTES;
  constexpr bool STORE_TMA = TP::STORE_TMA;
  constexpr int XO = TP::XO;
  constexpr int WX = TP::WX;
  extern __shared__ __align__(128) unsigned char win_raw[];
  __shared__ __align__(16) MomTile<kTX, TY> mt;
  __shared__ __align__(8) uint64_t bar_mem;
  __shared__ int s_abort;
  const int t = threadIdx.x;
  const uint32_t bar = tma::smem_u32(&bar_mem);
  const uint32_t win = tma::smem_u32(win_raw);
  const T* w = reinterpret_cast<const T*>(win_raw);
  T* ob = reinterpret_cast<T*>(win_raw + TP::OUT_AT);
  if (t == 0) {
    tma::mbar_init(bar, 1);
    tma::fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (t == 0 && tile < n_tiles) {
    const auto d = tile_of(tile);
    tma::mbar_expect_tx(bar, BYTES);
    tma::load_3d(win, d.map, d.i0 - XO, d.j0 - 2, d.z, bar);
  }
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const auto d = tile_of(tile);
    const Layout& L = d.L;
    const bool ok = tma::mbar_wait(bar, it & 1);
    // the output tile was last read by the previous iteration's TMA store
    if (STORE_TMA && t == 0) tma::bulk_wait_read_0();
    vec<V> fw[kQ], fp[kQ], g[kQ];
    if (ok) {
      auto acc_at = [&](int dx, int dy) {
        return WinAcc<T, kTX, TY>{w + (2 + dy) * WX + (XO + dx)};
      };
      tile_pull<kTX, TY, V, T, false>(acc_at, L, d.k, d.i0, d.j0, t, mt, fw, fp, g, nullptr);
    } else {
      s_abort = 1;
    }
    __syncthreads();  // the window is consumed; the moment tile is complete
    if (s_abort) {
      if (t == 0) {
        atomicOr(err, 1);
        if (STORE_TMA) tma::bulk_wait_all();
        tma::mbar_wait(bar, it & 1);  // drain this tile's copy (bounded)
      }
      return;
    }
    const int next = tile + gridDim.x;
    if (t == 0 && next < n_tiles) {
      const auto dn = tile_of(next);
      tma::fence_proxy_async();  // generic-proxy reads of the window before the async write
      tma::mbar_expect_tx(bar, BYTES);
      tma::load_3d(win, dn.map, dn.i0 - XO, dn.j0 - 2, dn.z, bar);
    }
    const TileThread<kTX, TY, V> tt(t);
    const int i = d.i0 + V * tt.c, j = d.j0 + tt.ty;
    const size_t o = (size_t)j * L.pitch + i;
    const uint32_t seed = SR ? mix32((uint32_t)o ^ d.hash) : 0u;
    if constexpr (STORE_TMA) {
      TileSink<T, SR, kTX * TY, V> out{ob + tt.ty * kTX + V * tt.c, seed};
      tile_collide<ALLF, kTX, TY, V, T, false>(d.k, L, d.i0, d.j0, t, mt, fw, fp, g, nullptr,
                                                out);
      tma::fence_proxy_async();  // generic-proxy writes of the output tile before the TMA store
    } else {
      GlobSink<T, SR, V> out{static_cast<T*>(d.dst) + o, L.plane, seed, i + 1 < L.nx};
      tile_collide<ALLF, kTX, TY, V, T, false>(d.k, L, d.i0, d.j0, t, mt, fw, fp, g, nullptr,
                                                out);
    }
    __syncthreads();  // the moment tile and the output tile are free again
    if (STORE_TMA && t == 0) {
      // nodes outside the cavity fall outside the tensor and are not written
      tma::store_3d(d.map_out, d.i0, d.j0, d.z_out, tma::smem_u32(ob));
      tma::bulk_commit();
    }
  }
  if (STORE_TMA && t == 0) tma::bulk_wait_all();
}

template <class T, bool SR, bool ALLF, int V, int TY = kTY>
__global__ void __launch_bounds__(Threads<V, kTileW, TY>::value, MinBlocks<V, kTileW, TY>::value)
    step_pair_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                         const __grid_constant__ CUtensorMap tmap_out, const StepArgs a) {
  // Programmatic dependent launch: let the next step's CTAs start their prologue while this
  // grid drains, and do not read the state before the previous step has completed.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr int kTX = kTileW;
  const int tiles_x = (a.L.nx + kTX - 1) / kTX;
  const int n_tiles = tiles_x * ((a.L.ny + TY - 1) / TY);
  const uint32_t sh = SR ? step_hash(a) : 0u;
  auto tile_of = [&](int tile) {
    const int ty = tile / tiles_x;
    return TmaTileDesc{&tmap, &tmap_out, a.z_src, kPlanes - a.z_src, (tile - ty * tiles_x) * kTX,
                       ty * TY, a.L, a.k, a.dst, sh};
  };
  tma_tile_loop<T, SR, ALLF, V, kTileW, TY>(tile_of, n_tiles, a.err);
}

// ---- host side ---------------------------------------------------------------------------------
// Nodes per thread: one while a lattice gives every SM at most two tiles (a few hundred nodes
// per SM: the step is latency-bound and needs every warp it can get), two beyond (issue-bound:
// packed arithmetic halves the instructions per node).
inline int nodes_per_thread(const Layout& L, int sms) {
  const int tiles = ((L.nx + 31) / 32) * ((L.ny + kTY - 1) / kTY);  // 32 x 8 tiles
  return tiles <= 2 * sms ? 1 : 2;
}

// Low tiles (32 x 7, one node per thread, two CTAs per SM) when 32 x 8 tiles would put a
// second tile on some SMs and 32 x 7 tiles fit two per SM: the busiest SMs then compute 448
// nodes instead of 512 (measured on the 256 x 256 lattice: 4.65 us per step against 4.87; one
// CTA of 32 x 14 per SM, the same 448 nodes, takes 5.21 us: two CTAs overlap each other's
// barriers and window loads).
inline bool low_tiles_pay(const Layout& L, int sms) {
  const int tx = (L.nx + kTileW - 1) / kTileW;
  return tx * ((L.ny + kTY - 1) / kTY) > sms && tx * ((L.ny + kLowTY - 1) / kLowTY) <= 2 * sms;
}

template <class T, int V, int TY>
cudaError_t prepare_pair_tma_v(StepConfig* c, const Layout& L, int sms) {
  const size_t smem = TmaPair<T, V, kTileW, TY>::SMEM;
  const void* fns[4] = {(const void*)step_pair_tma_kernel<T, false, false, V, TY>,
                        (const void*)step_pair_tma_kernel<T, false, true, V, TY>,
                        (const void*)step_pair_tma_kernel<T, true, false, V, TY>,
                        (const void*)step_pair_tma_kernel<T, true, true, V, TY>};
  cudaError_t e;
  for (const void* fn : fns)
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, step_pair_tma_kernel<T, true, true, V, TY>, Threads<V, kTileW, TY>::value, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm > MinBlocks<V, kTileW, TY>::value) per_sm = MinBlocks<V, kTileW, TY>::value;
  constexpr int kTX = kTileW;
  const int tiles = ((L.nx + kTX - 1) / kTX) * ((L.ny + TY - 1) / TY);
  c->grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  c->vec = V;
  c->th = TY;
  return cudaSuccess;
}

template <class T>
cudaError_t prepare_pair_tma_t(StepConfig* c, const Layout& L) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  int v = nodes_per_thread(L, sms);
  if (c->vec == 1 || c->vec == 2) v = c->vec;  // forced by the caller
  if (v == 2) return prepare_pair_tma_v<T, 2, kTY>(c, L, sms);
  // tile height: forced by the caller (8 or 7), else 7 where low tiles pay
  const bool low = c->th == kLowTY || (c->th != kTY && low_tiles_pay(L, sms));
  return low ? prepare_pair_tma_v<T, 1, kLowTY>(c, L, sms)
             : prepare_pair_tma_v<T, 1, kTY>(c, L, sms);
}

template <class T, bool SR, bool ALLF, int V>
cudaError_t launch_pair_t4(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                           cudaLaunchConfig_t& cfg) {
  constexpr int kTX = kTileW;
  if (a.k.two_sets) {  // two thermal sets: the plain tile kernel, one node per thread
    if (c.variant == 2 || V != 1 || ALLF) return cudaErrorInvalidValue;
    cfg.gridDim = dim3((a.L.nx + kTX - 1) / kTX, (a.L.ny + kTY - 1) / kTY);
    cfg.blockDim = dim3(Threads<1, kTileW>::value);
    cfg.dynamicSmemBytes = 0;
    return cudaLaunchKernelEx(&cfg, step_pair_tile_kernel<T, SR, false, 1, true>, a);
  }
  if (c.variant == 2) {
    if (!map || c.grid < 1) return cudaErrorInvalidValue;
    cfg.gridDim = dim3(c.grid);
    if constexpr (V == 1) {
      if (c.th == kLowTY) {
        cfg.blockDim = dim3(Threads<1, kTileW, kLowTY>::value);
        cfg.dynamicSmemBytes = TmaPair<T, 1, kTileW, kLowTY>::SMEM;
        return cudaLaunchKernelEx(&cfg, step_pair_tma_kernel<T, SR, ALLF, 1, kLowTY>, map[0],
                                  map[1], a);
      }
    }
    if (c.th != kTY) return cudaErrorInvalidValue;
    cfg.blockDim = dim3(Threads<V, kTileW>::value);
    cfg.dynamicSmemBytes = TmaPair<T, V, kTileW>::SMEM;
    return cudaLaunchKernelEx(&cfg, step_pair_tma_kernel<T, SR, ALLF, V>, map[0], map[1], a);
  }
  cfg.gridDim = dim3((a.L.nx + kTX - 1) / kTX, (a.L.ny + kTY - 1) / kTY);
  cfg.blockDim = dim3(Threads<V, kTileW>::value);
  cfg.dynamicSmemBytes = 0;
  return cudaLaunchKernelEx(&cfg, step_pair_tile_kernel<T, SR, ALLF, V>, a);
}

template <class T, bool SR, bool ALLF>
cudaError_t launch_pair_t3(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                           cudaLaunchConfig_t& cfg) {
  return c.vec == 2 ? launch_pair_t4<T, SR, ALLF, 2>(a, c, map, cfg)
                    : launch_pair_t4<T, SR, ALLF, 1>(a, c, map, cfg);
}

// Tile and TMA kernels go out with programmatic stream serialization: the kernel itself
// waits on the previous grid (griddepcontrol.wait) before it reads the state.
template <class T>
cudaError_t launch_pair_t(const StepArgs& a, const StepConfig& c, const CUtensorMap* map,
                          cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const bool all = a.k.mask == MCLBM_F_ALL && !a.k.two_sets;
  const bool sr = c.sr && sizeof(T) == 2;
  if (sr)
    return all ? launch_pair_t3<T, true, true>(a, c, map, cfg)
               : launch_pair_t3<T, true, false>(a, c, map, cfg);
  return all ? launch_pair_t3<T, false, true>(a, c, map, cfg)
             : launch_pair_t3<T, false, false>(a, c, map, cfg);
}

}  // namespace pair
}  // namespace mcl
