// C ABI of the warm-start network (include/mclbm_net.h): workspace planning, the forward and
// backward sequences of launches, Adam, and the exposed tensor-core GEMM. Host code only; the
// kernels are in net_gemm.cu and net_kernels.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/mclbm.h"
#include "../../include/mclbm_net.h"
#include "net_internal.h"
#include "nvtx_range.h"

using namespace mcl::net;

namespace {

constexpr int kNumLayers = 10;
constexpr int kLossBlocks = 1024;
constexpr int kStatBlocks = 256;

struct Layer {
  // definition
  int cu, cs, cout, stride, film, act;
  int src1, src2;  // producing layer of each input source (-1: the geometry input X)
  int up;          // src1 is upsampled by 2
  // shapes
  int H, W, Ho, Wo, kin, Kp, splits;
  int fsplits;  // forward split over K (layers with few output tiles), 1 otherwise
  // input gradient as a convolution of the output gradient (stride 1, 9 cout <= Kp): the
  // flipped, transposed kernel wt [cin][kp2], kp2 = 9 cout rounded up to 8
  int tconv, kp2;
  int64_t w_off, b_off;
  int film_off;  // offset of this layer's (gamma, beta) slice in r, or -1
  // device buffers
  float *pre, *y, *dy;
  __nv_bfloat16 *cols, *wb, *dpre, *wt;
  double* partial;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct mclbm_net {
  mclbm_net_config cfg;
  Layer L[kNumLayers];
  int F = 0;
  int64_t n_params = 0, mlp_off = 0;
  size_t ws_bytes = 0;
  size_t dcols_elems = 0, wpart_elems = 0;
  // bound memory
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  float* norm = nullptr;  // mean[5], scale[5] of the fields' deviations from their rest values
  float* X = nullptr;
  float *dcols = nullptr, *wpart = nullptr;
  float *cond_c = nullptr, *a1 = nullptr, *r = nullptr, *dr = nullptr;
  double *loss_part = nullptr, *loss = nullptr, *stat_part = nullptr;
  int* err = nullptr;
  int adam_t = 0;
  bool bound = false;
  char errmsg[512] = {0};
};

namespace {

int fail(mclbm_net* n, int code, const char* fmt, ...) {
  if (n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(n->errmsg, sizeof(n->errmsg), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(mclbm_net* n, cudaError_t e, const char* what) {
  return fail(n, MCLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool config_valid(const mclbm_net_config* c) {
  return c && c->ny >= 16 && c->nx >= 16 && c->ny <= 4096 && c->nx <= 4096 && c->ny % 16 == 0 &&
         c->nx % 16 == 0 && c->c0 >= 8 && c->c0 <= 64 && c->c0 % 8 == 0 && c->hidden >= 1 &&
         c->hidden <= 256 && c->max_batch >= 1 && c->max_batch <= 256 &&
         (int64_t)c->max_batch * c->ny * c->nx <= (int64_t)1 << 26 &&
         c->max_batch * c->hidden <= 4096;  // the MLP kernels keep [batch][hidden] in shared memory
}

// Layer table, parameter offsets and workspace size (no device work).
void plan(mclbm_net* n) {
  const mclbm_net_config& c = n->cfg;
  const int C0 = c.c0, C1 = 2 * C0, C2 = 4 * C0, C3 = 8 * C0, C4 = 8 * C0;
  // cu, cs, cout, stride, film, act, src1, src2, up
  const int def[kNumLayers][9] = {
      {4, 0, C0, 1, 0, 1, -1, -1, 0},  // e0
      {C0, 0, C1, 2, 0, 1, 0, -1, 0},  // e1
      {C1, 0, C2, 2, 0, 1, 1, -1, 0},  // e2
      {C2, 0, C3, 2, 0, 1, 2, -1, 0},  // e3
      {C3, 0, C4, 2, 1, 1, 3, -1, 0},  // e4
      {C4, C3, C3, 1, 1, 1, 4, 3, 1},  // d3
      {C3, C2, C2, 1, 1, 1, 5, 2, 1},  // d2
      {C2, C1, C1, 1, 1, 1, 6, 1, 1},  // d1
      {C1, C0, C0, 1, 1, 1, 7, 0, 1},  // d0
      {C0, 0, kFields, 1, 0, 0, 8, -1, 0},  // out
  };
  int64_t off = 0;
  int film_off = 0;
  for (int l = 0; l < kNumLayers; ++l) {
    Layer& y = n->L[l];
    std::memset(&y, 0, sizeof(y));
    y.cu = def[l][0];
    y.cs = def[l][1];
    y.cout = def[l][2];
    y.stride = def[l][3];
    y.film = def[l][4];
    y.act = def[l][5];
    y.src1 = def[l][6];
    y.src2 = def[l][7];
    y.up = def[l][8];
    if (y.src1 < 0) {
      y.H = c.ny;
      y.W = c.nx;
    } else {
      const Layer& s = n->L[y.src1];
      y.H = y.up ? 2 * s.Ho : s.Ho;
      y.W = y.up ? 2 * s.Wo : s.Wo;
    }
    y.Ho = y.H / y.stride;
    y.Wo = y.W / y.stride;
    y.kin = 9 * (y.cu + y.cs);
    y.Kp = (y.kin + 7) & ~7;
    y.kp2 = (9 * y.cout + 7) & ~7;
    y.tconv = l > 0 && y.stride == 1 && y.kp2 <= y.Kp;
    y.w_off = off;
    off += (int64_t)y.cout * y.kin;
    y.b_off = off;
    off += y.cout;
    y.film_off = -1;
    if (y.film) {
      y.film_off = film_off;
      film_off += 2 * y.cout;
    }
    const int tiles = ((y.cout + 127) / 128) * ((y.Kp + 127) / 128);
    // weight gradient split over pixels so that its tiles fill one wave of the persistent GEMM
    // (one CTA per SM with an MN-major B; 152 SMs on GB300); it changes only the order in which
    // the FP32 partial sums are added
    y.splits = std::max(1, std::min(64, 152 / tiles));
    // forward GEMMs with fewer output tiles than half a wave are split over K as well (partial
    // sums reduced in a fixed order by the epilogue kernel)
    const int64_t tiles_f = (((int64_t)c.max_batch * y.Ho * y.Wo + 127) / 128) *
                            ((y.cout + 127) / 128);
    const int nks = (y.Kp + 63) / 64;
    y.fsplits = tiles_f >= 76 ? 1 : (int)std::max<int64_t>(
                                        1, std::min<int64_t>({152 / tiles_f, 8, (int64_t)nks}));
  }
  n->F = film_off;
  n->mlp_off = off;
  off += (int64_t)c.hidden * 3 + c.hidden + (int64_t)n->F * c.hidden + n->F;
  n->n_params = off;

  // workspace
  const int64_t B = c.max_batch;
  size_t bytes = 0;
  const size_t np = (size_t)n->n_params;
  bytes += 4 * align256(np * 4);  // params, grads, adam m, v
  bytes += align256(2 * kFields * 4);  // normaliser
  bytes += align256((size_t)4 * B * c.ny * c.nx * 4);  // X
  n->dcols_elems = 0;
  n->wpart_elems = 0;
  for (int l = 0; l < kNumLayers; ++l) {
    const Layer& y = n->L[l];
    const size_t P = (size_t)B * y.Ho * y.Wo;
    bytes += 3 * align256((size_t)y.cout * P * 4);           // pre, y, dy
    bytes += align256(P * y.Kp * 2);                         // cols
    bytes += align256((size_t)y.cout * y.Kp * 2);            // wb
    if (y.tconv) bytes += align256((size_t)(y.cu + y.cs) * y.kp2 * 2);  // wt
    bytes += align256((size_t)y.cout * P * 2);               // dpre
    bytes += align256((size_t)y.cout * B * 3 * 8);           // partial
    if (l > 0) n->dcols_elems = std::max(n->dcols_elems, P * y.Kp);
    n->wpart_elems = std::max(n->wpart_elems, (size_t)y.splits * y.cout * y.Kp);
    if (y.fsplits > 1)
      n->wpart_elems = std::max(n->wpart_elems, (size_t)y.fsplits * y.cout * P);
  }
  bytes += align256(n->dcols_elems * 4);
  bytes += align256(n->wpart_elems * 4);
  bytes += align256((size_t)B * 3 * 4) + align256((size_t)B * c.hidden * 4) +
           2 * align256((size_t)B * n->F * 4);
  bytes += align256(kLossBlocks * 8) + align256(8) + align256(kFields * kStatBlocks * 2 * 8);
  bytes += align256(4);
  n->ws_bytes = bytes;
}

template <typename T>
T* carve(char*& p, size_t count) {
  T* out = reinterpret_cast<T*>(p);
  p += align256(count * sizeof(T));
  return out;
}

void assign(mclbm_net* n) {
  const mclbm_net_config& c = n->cfg;
  const int64_t B = c.max_batch;
  char* p = n->ws;
  const size_t np = (size_t)n->n_params;
  n->params = carve<float>(p, np);
  n->grads = carve<float>(p, np);
  n->adam_m = carve<float>(p, np);
  n->adam_v = carve<float>(p, np);
  n->norm = carve<float>(p, 2 * kFields);
  n->X = carve<float>(p, (size_t)4 * B * c.ny * c.nx);
  for (int l = 0; l < kNumLayers; ++l) {
    Layer& y = n->L[l];
    const size_t P = (size_t)B * y.Ho * y.Wo;
    y.pre = carve<float>(p, (size_t)y.cout * P);
    y.y = carve<float>(p, (size_t)y.cout * P);
    y.dy = carve<float>(p, (size_t)y.cout * P);
    y.cols = carve<__nv_bfloat16>(p, P * y.Kp);
    y.wb = carve<__nv_bfloat16>(p, (size_t)y.cout * y.Kp);
    y.wt = y.tconv ? carve<__nv_bfloat16>(p, (size_t)(y.cu + y.cs) * y.kp2) : nullptr;
    y.dpre = carve<__nv_bfloat16>(p, (size_t)y.cout * P);
    y.partial = carve<double>(p, (size_t)y.cout * B * 3);
  }
  n->dcols = carve<float>(p, n->dcols_elems);
  n->wpart = carve<float>(p, n->wpart_elems);
  n->cond_c = carve<float>(p, (size_t)B * 3);
  n->a1 = carve<float>(p, (size_t)B * c.hidden);
  n->r = carve<float>(p, (size_t)B * n->F);
  n->dr = carve<float>(p, (size_t)B * n->F);
  n->loss_part = carve<double>(p, kLossBlocks);
  n->loss = carve<double>(p, 1);
  n->stat_part = carve<double>(p, kFields * kStatBlocks * 2);
  n->err = carve<int>(p, 1);
}

MlpArgs mlp_args(mclbm_net* n, int batch, const float* cond) {
  MlpArgs a;
  const int64_t o = n->mlp_off;
  const int H = n->cfg.hidden;
  a.cond_raw = cond;
  a.W1 = n->params + o;
  a.b1 = a.W1 + 3 * H;
  a.W2 = a.b1 + H;
  a.b2 = a.W2 + (int64_t)n->F * H;
  a.batch = batch;
  a.H = H;
  a.F = n->F;
  a.c = n->cond_c;
  a.a1 = n->a1;
  a.r = n->r;
  return a;
}

const float* src_tensor(mclbm_net* n, int s) { return s < 0 ? n->X : n->L[s].y; }

cudaError_t refresh_bf16_weights(mclbm_net* n) {
  for (int l = 0; l < kNumLayers; ++l) {
    const Layer& y = n->L[l];
    cudaError_t e = launch_weights_bf16(n->params + y.w_off, y.cout, y.kin, y.Kp, y.wb, n->stream);
    if (e != cudaSuccess) return e;
    if (y.tconv &&
        (e = launch_weights_t_bf16(n->params + y.w_off, y.cout, y.cu + y.cs, y.kp2, y.wt,
                                   n->stream)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

cudaError_t forward(mclbm_net* n, int batch, const float* cond) {
  cudaStream_t st = n->stream;
  cudaError_t e = launch_geometry(n->X, batch, n->cfg.ny, n->cfg.nx, st);
  if (e != cudaSuccess) return e;
  e = launch_mlp_forward(mlp_args(n, batch, cond), st);
  if (e != cudaSuccess) return e;
  for (int l = 0; l < kNumLayers; ++l) {
    Layer& y = n->L[l];
    Im2colArgs ia;
    ia.src1 = src_tensor(n, y.src1);
    ia.src2 = y.src2 >= 0 ? n->L[y.src2].y : nullptr;
    ia.cu = y.cu;
    ia.cs = y.cs;
    ia.up = y.up;
    ia.batch = batch;
    ia.H = y.H;
    ia.W = y.W;
    ia.stride = y.stride;
    ia.Ho = y.Ho;
    ia.Wo = y.Wo;
    ia.Kp = y.Kp;
    ia.cols = y.cols;
    if ((e = launch_im2col(ia, st)) != cudaSuccess) return e;
    const int P = batch * y.Ho * y.Wo;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.a = y.cols;
    g.lda = y.Kp;
    g.a_kmajor = 1;
    g.b = y.wb;
    g.ldb = y.Kp;
    g.b_kmajor = 1;
    g.M = P;
    g.N = y.cout;
    g.K = y.Kp;
    g.ep.bias = n->params + y.b_off;
    g.ep.film = y.film ? n->r : nullptr;
    g.ep.film_stride = n->F;
    g.ep.film_off = y.film_off;
    g.ep.hw = y.Ho * y.Wo;
    g.ep.pre = y.pre;
    g.ep.y = l == kNumLayers - 1 ? nullptr : y.y;
    g.ep.act = y.act;
    g.err = n->err;
    if (y.fsplits > 1) {
      // partial products per K split, column-major [split][cout][P], then the epilogue
      const int nks = (y.Kp + 63) / 64;
      g.k_per_split = (int64_t)((nks + y.fsplits - 1) / y.fsplits) * 64;
      g.mode = kGemmRaw;
      g.d = n->wpart;
      g.ldd = P;
      g.d_trans = 1;
      g.split_stride = (int64_t)y.cout * P;
      if ((e = launch_gemm(g, y.fsplits, st)) != cudaSuccess) return e;
      if ((e = launch_conv_epilogue_splitk(n->wpart, y.fsplits, g.split_stride, P, y.cout, g.ep,
                                           st)) != cudaSuccess)
        return e;
    } else {
      g.k_per_split = ((y.Kp + 63) / 64) * 64;
      g.mode = kGemmConvFwd;
      if ((e = launch_gemm(g, 1, st)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Loss and gradients into n->grads (loss into n->loss on the device).
cudaError_t loss_backward(mclbm_net* n, int batch, const float* cond, const float* target) {
  cudaStream_t st = n->stream;
  const int hw = n->cfg.ny * n->cfg.nx;
  Layer& out = n->L[kNumLayers - 1];
  LossArgs la;
  la.out = out.pre;
  la.target = target;
  la.cond = cond;
  la.norm = n->norm;
  la.batch = batch;
  la.hw = hw;
  la.dout = out.dy;
  la.partial = n->loss_part;
  la.blocks = kLossBlocks;
  cudaError_t e = launch_loss(la, st);
  if (e != cudaSuccess) return e;
  if ((e = launch_sum_partials(n->loss_part, kLossBlocks, n->loss, st)) != cudaSuccess) return e;

  bool written[kNumLayers] = {false};
  for (int l = kNumLayers - 1; l >= 0; --l) {
    Layer& y = n->L[l];
    const int P = batch * y.Ho * y.Wo;
    ActBwdArgs aa;
    aa.dy = y.dy;
    aa.pre = y.pre;
    aa.film = y.film ? n->r : nullptr;
    aa.film_stride = n->F;
    aa.film_off = y.film_off;
    aa.C = y.cout;
    aa.batch = batch;
    aa.hw = y.Ho * y.Wo;
    aa.act = y.act;
    aa.dpre = y.dpre;
    aa.partial = y.partial;
    if ((e = launch_act_backward(aa, st)) != cudaSuccess) return e;
    if ((e = launch_bias_film_grad(y.partial, y.cout, batch, n->grads + y.b_off,
                                   y.film ? n->dr : nullptr, n->F, y.film_off, st)) != cudaSuccess)
      return e;
    // weight gradient: dW[o][k] = sum_p dpre[o][p] cols[p][k], split over p
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.a = y.dpre;
    g.lda = P;
    g.a_kmajor = 1;
    g.b = y.cols;
    g.ldb = y.Kp;
    g.b_kmajor = 0;
    g.M = y.cout;
    g.N = y.Kp;
    g.K = P;
    g.k_per_split = ((((int64_t)P + y.splits - 1) / y.splits + 63) / 64) * 64;
    g.d = n->wpart;
    g.ldd = y.Kp;
    g.split_stride = (int64_t)y.cout * y.Kp;
    g.mode = kGemmRaw;
    g.err = n->err;
    if ((e = launch_gemm(g, y.splits, st)) != cudaSuccess) return e;
    if ((e = launch_splitk_reduce(n->wpart, y.splits, g.split_stride, y.cout, y.kin, y.Kp,
                                  n->grads + y.w_off, st)) != cudaSuccess)
      return e;
    if (l == 0) break;
    if (y.tconv) {
      // input gradient of a stride-1 convolution as the convolution of the output gradient with
      // the flipped, transposed kernel: dX[c][q] = sum_(o, t) wt[c][o 9 + t] cols2[q][o 9 + t],
      // cols2 the im2col rows of dpre (in this layer's cols buffer), then routed to the sources
      Im2colBf16Args ib;
      ib.src = y.dpre;
      ib.C = y.cout;
      ib.batch = batch;
      ib.H = y.Ho;
      ib.W = y.Wo;
      ib.Kp = y.kp2;
      ib.cols = y.cols;
      if ((e = launch_im2col_bf16(ib, st)) != cudaSuccess) return e;
      std::memset(&g, 0, sizeof(g));
      g.a = y.cols;
      g.lda = y.kp2;
      g.a_kmajor = 1;
      g.b = y.wt;
      g.ldb = y.kp2;
      g.b_kmajor = 1;
      g.M = P;
      g.N = y.cu + y.cs;
      g.K = y.kp2;
      g.k_per_split = ((y.kp2 + 63) / 64) * 64;
      g.d = n->dcols;
      g.ldd = P;
      g.d_trans = 1;
      g.mode = kGemmRaw;
      g.err = n->err;
      if ((e = launch_gemm(g, 1, st)) != cudaSuccess) return e;
      RouteArgs ra;
      ra.dx = n->dcols;
      ra.cu = y.cu;
      ra.cs = y.src2 >= 0 ? y.cs : 0;
      ra.up = y.up;
      ra.batch = batch;
      ra.H = y.H;
      ra.W = y.W;
      ra.dsrc1 = n->L[y.src1].dy;
      ra.acc1 = written[y.src1] ? 1 : 0;
      written[y.src1] = true;
      ra.dsrc2 = nullptr;
      ra.acc2 = 0;
      if (y.src2 >= 0) {
        ra.dsrc2 = n->L[y.src2].dy;
        ra.acc2 = written[y.src2] ? 1 : 0;
        written[y.src2] = true;
      }
      if ((e = launch_route_grad(ra, st)) != cudaSuccess) return e;
      continue;
    }
    // input gradient: dcols[k][p] = sum_o dpre[o][p] wb[o][k], stored column-major so that
    // the epilogue's stores and col2im's reads are coalesced over pixels
    std::memset(&g, 0, sizeof(g));
    g.a = y.dpre;
    g.lda = P;
    g.a_kmajor = 0;
    g.b = y.wb;
    g.ldb = y.Kp;
    g.b_kmajor = 0;
    g.M = P;
    g.N = y.Kp;
    g.K = y.cout;
    g.k_per_split = ((y.cout + 63) / 64) * 64;
    g.d = n->dcols;
    g.ldd = P;
    g.d_trans = 1;
    g.mode = kGemmRaw;
    g.err = n->err;
    if ((e = launch_gemm(g, 1, st)) != cudaSuccess) return e;
    for (int s = 0; s < 2; ++s) {
      const int src = s == 0 ? y.src1 : y.src2;
      if (s == 1 && src < 0) break;
      Col2imArgs ca;
      ca.dcols = n->dcols;
      ca.Kp = y.Kp;
      ca.c_lo = s == 0 ? 0 : y.cu;
      ca.C = s == 0 ? y.cu : y.cs;
      ca.up = s == 0 ? y.up : 0;
      ca.batch = batch;
      ca.H = y.H;
      ca.W = y.W;
      ca.stride = y.stride;
      ca.Ho = y.Ho;
      ca.Wo = y.Wo;
      ca.dsrc = n->L[src].dy;
      ca.accumulate = written[src] ? 1 : 0;
      written[src] = true;
      if ((e = launch_col2im(ca, st)) != cudaSuccess) return e;
    }
  }
  const MlpArgs ma = mlp_args(n, batch, nullptr);
  float* gW1 = n->grads + n->mlp_off;
  float* gb1 = gW1 + 3 * n->cfg.hidden;
  float* gW2 = gb1 + n->cfg.hidden;
  float* gb2 = gW2 + (int64_t)n->F * n->cfg.hidden;
  return launch_mlp_backward(ma, n->dr, gW1, gb1, gW2, gb2, st);
}

int check_call(mclbm_net* n, int batch) {
  if (!n) return MCLBM_EINVAL;
  if (!n->bound) return fail(n, MCLBM_ESTATE, "mclbm_net: not bound");
  if (batch < 1 || batch > n->cfg.max_batch)
    return fail(n, MCLBM_EINVAL, "batch %d outside 1..%d", batch, n->cfg.max_batch);
  return MCLBM_OK;
}

// Syncs the stream and reads the error word and the loss.
int finish(mclbm_net* n, double* loss) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream);
  double l = 0.0;
  if (e == cudaSuccess && loss)
    e = cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net sync");
  if (err) return fail(n, MCLBM_ETIMEOUT, "a tensor-core GEMM gave up a bounded wait");
  if (loss) {
    *loss = l;
    if (!std::isfinite(l)) return fail(n, MCLBM_EDIVERGED, "loss is not finite");
  }
  return MCLBM_OK;
}

}  // namespace

extern "C" {

void mclbm_net_config_default(mclbm_net_config* cfg) {
  if (!cfg) return;
  cfg->ny = 256;
  cfg->nx = 256;
  cfg->c0 = 16;
  cfg->hidden = 64;
  cfg->max_batch = 16;
}

int64_t mclbm_net_param_count(const mclbm_net_config* cfg) {
  if (!config_valid(cfg)) return 0;
  mclbm_net n;
  n.cfg = *cfg;
  plan(&n);
  return n.n_params;
}

size_t mclbm_net_workspace_bytes(const mclbm_net_config* cfg) {
  if (!config_valid(cfg)) return 0;
  mclbm_net n;
  n.cfg = *cfg;
  plan(&n);
  return n.ws_bytes;
}

int mclbm_net_create(const mclbm_net_config* cfg, mclbm_net_t** out) {
  if (!out) return MCLBM_EINVAL;
  *out = nullptr;
  if (!config_valid(cfg)) return MCLBM_EINVAL;
  mclbm_net* n = new mclbm_net();
  n->cfg = *cfg;
  plan(n);
  *out = n;
  return MCLBM_OK;
}

void mclbm_net_destroy(mclbm_net_t* net) { delete net; }

const char* mclbm_net_last_error(const mclbm_net_t* net) { return net ? net->errmsg : ""; }

int mclbm_net_bind(mclbm_net_t* n, void* ws, size_t bytes, void* stream) {
  if (!n) return MCLBM_EINVAL;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u))
    return fail(n, MCLBM_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < n->ws_bytes)
    return fail(n, MCLBM_EINVAL, "workspace of %zu bytes, %zu needed", bytes, n->ws_bytes);
  n->ws = static_cast<char*>(ws);
  n->stream = static_cast<cudaStream_t>(stream);
  assign(n);
  cudaStream_t st = n->stream;
  const size_t np = (size_t)n->n_params * 4;
  cudaError_t e = cudaMemsetAsync(n->params, 0, np, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_m, 0, np, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_v, 0, np, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->err, 0, sizeof(int), st);
  float norm[2 * kFields];
  for (int c = 0; c < kFields; ++c) {
    norm[c] = 0.f;
    norm[kFields + c] = 1.f;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->norm, norm, sizeof(norm), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = refresh_bf16_weights(n);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net_bind");
  n->adam_t = 0;
  n->bound = true;
  return MCLBM_OK;
}

int mclbm_net_set_params(mclbm_net_t* n, const float* p) {
  if (!n || !p) return MCLBM_EINVAL;
  if (!n->bound) return fail(n, MCLBM_ESTATE, "mclbm_net: not bound");
  const size_t np = (size_t)n->n_params * 4;
  cudaError_t e = cudaMemcpyAsync(n->params, p, np, cudaMemcpyDeviceToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_m, 0, np, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_v, 0, np, n->stream);
  if (e == cudaSuccess) e = refresh_bf16_weights(n);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net_set_params");
  n->adam_t = 0;
  return MCLBM_OK;
}

int mclbm_net_init_params(mclbm_net_t* n, uint64_t seed) {
  if (!n) return MCLBM_EINVAL;
  if (!n->bound) return fail(n, MCLBM_ESTATE, "mclbm_net: not bound");
  cudaStream_t st = n->stream;
  cudaError_t e = cudaMemsetAsync(n->params, 0, (size_t)n->n_params * 4, st);
  uint32_t stream_id = 0;
  for (int l = 0; l < kNumLayers && e == cudaSuccess; ++l) {
    const Layer& y = n->L[l];
    e = launch_uniform_fill(n->params + y.w_off, (int64_t)y.cout * y.kin,
                            (float)std::sqrt(6.0 / y.kin), seed, stream_id++, st);
  }
  const int H = n->cfg.hidden;
  float* W1 = n->params + n->mlp_off;
  float* W2 = W1 + 3 * H + H;
  if (e == cudaSuccess)
    e = launch_uniform_fill(W1, 3 * H, (float)std::sqrt(6.0 / 3.0), seed, stream_id++, st);
  if (e == cudaSuccess)
    e = launch_uniform_fill(W2, (int64_t)n->F * H, (float)(0.1 * std::sqrt(6.0 / H)), seed,
                            stream_id++, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_m, 0, (size_t)n->n_params * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_v, 0, (size_t)n->n_params * 4, st);
  if (e == cudaSuccess) e = refresh_bf16_weights(n);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net_init_params");
  n->adam_t = 0;
  return MCLBM_OK;
}

int mclbm_net_get_params(mclbm_net_t* n, float* p) {
  if (!n || !p) return MCLBM_EINVAL;
  if (!n->bound) return fail(n, MCLBM_ESTATE, "mclbm_net: not bound");
  cudaError_t e = cudaMemcpyAsync(p, n->params, (size_t)n->n_params * 4, cudaMemcpyDeviceToDevice,
                                  n->stream);
  return e == cudaSuccess ? MCLBM_OK : cuda_fail(n, e, "mclbm_net_get_params");
}

int mclbm_net_set_normalizer(mclbm_net_t* n, const double* mean, const double* scale) {
  if (!n || !mean || !scale) return MCLBM_EINVAL;
  if (!n->bound) return fail(n, MCLBM_ESTATE, "mclbm_net: not bound");
  float v[2 * kFields];
  for (int c = 0; c < kFields; ++c) {
    if (!(scale[c] > 0.0) || !std::isfinite(mean[c]) || !std::isfinite(scale[c]))
      return fail(n, MCLBM_EINVAL, "normaliser channel %d: mean %g scale %g", c, mean[c], scale[c]);
    v[c] = (float)mean[c];
    v[kFields + c] = (float)scale[c];
  }
  // the host array must outlive the copy: synchronous on the stream
  cudaError_t e = cudaMemcpyAsync(n->norm, v, sizeof(v), cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  return e == cudaSuccess ? MCLBM_OK : cuda_fail(n, e, "mclbm_net_set_normalizer");
}

int mclbm_net_field_stats(mclbm_net_t* n, int count, const float* cond, const float* fields,
                          double* mean, double* scale) {
  if (!n || !cond || !fields || !mean || !scale || count < 1) return MCLBM_EINVAL;
  if (!n->bound) return fail(n, MCLBM_ESTATE, "mclbm_net: not bound");
  const int hw = n->cfg.ny * n->cfg.nx;
  cudaError_t e =
      launch_field_moments(fields, cond, count, hw, n->stat_part, kStatBlocks, n->stream);
  std::vector<double> part(kFields * kStatBlocks * 2);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), n->stat_part, part.size() * 8, cudaMemcpyDeviceToHost,
                        n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net_field_stats");
  const double N = (double)count * hw;
  for (int c = 0; c < kFields; ++c) {
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < kStatBlocks; ++b) {
      s += part[(c * kStatBlocks + b) * 2];
      s2 += part[(c * kStatBlocks + b) * 2 + 1];
    }
    const double m = s / N;
    const double var = std::max(0.0, s2 / N - m * m);
    mean[c] = m;
    scale[c] = var > 0.0 ? std::sqrt(var) : 1.0;
  }
  return MCLBM_OK;
}

int mclbm_net_forward(mclbm_net_t* n, int batch, const float* cond, float* fields) {
  mcl::NvtxRange range("mclbm_net_forward");
  int rc = check_call(n, batch);
  if (rc != MCLBM_OK) return rc;
  if (!cond || !fields) return fail(n, MCLBM_EINVAL, "null pointer");
  cudaError_t e = forward(n, batch, cond);
  if (e == cudaSuccess)
    e = launch_denormalize(n->L[kNumLayers - 1].pre, n->norm, cond, batch,
                           n->cfg.ny * n->cfg.nx, fields, n->stream);
  return e == cudaSuccess ? MCLBM_OK : cuda_fail(n, e, "mclbm_net_forward");
}

int mclbm_net_loss_grad(mclbm_net_t* n, int batch, const float* cond, const float* target,
                        float* grad, double* loss) {
  mcl::NvtxRange range("mclbm_net_loss_grad");
  int rc = check_call(n, batch);
  if (rc != MCLBM_OK) return rc;
  if (!cond || !target || !grad || !loss) return fail(n, MCLBM_EINVAL, "null pointer");
  cudaError_t e = forward(n, batch, cond);
  if (e == cudaSuccess) e = loss_backward(n, batch, cond, target);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad, n->grads, (size_t)n->n_params * 4, cudaMemcpyDeviceToDevice,
                        n->stream);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net_loss_grad");
  return finish(n, loss);
}

int mclbm_net_train_step(mclbm_net_t* n, int batch, const float* cond, const float* target,
                         float lr, double* loss) {
  mcl::NvtxRange range("mclbm_net_train_step");
  int rc = check_call(n, batch);
  if (rc != MCLBM_OK) return rc;
  if (!cond || !target || !(lr > 0.f)) return fail(n, MCLBM_EINVAL, "bad argument");
  cudaError_t e = forward(n, batch, cond);
  if (e == cudaSuccess) e = loss_backward(n, batch, cond, target);
  if (e == cudaSuccess) {
    n->adam_t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, n->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, n->adam_t)));
    e = launch_adam(n->params, n->grads, n->adam_m, n->adam_v, n->n_params, lr, (float)b1,
                    (float)b2, 1e-8f, c1, c2, n->stream);
  }
  if (e == cudaSuccess) e = refresh_bf16_weights(n);
  if (e != cudaSuccess) return cuda_fail(n, e, "mclbm_net_train_step");
  return loss ? finish(n, loss) : MCLBM_OK;
}

int mclbm_gemm_bf16(int M, int N, int K, const void* a, int64_t lda, int a_kmajor, const void* b,
                    int64_t ldb, int b_kmajor, float* d, int64_t ldd, int splits,
                    int64_t k_per_split, int64_t split_stride, void* stream) {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.a = static_cast<const __nv_bfloat16*>(a);
  g.lda = lda;
  g.a_kmajor = a_kmajor ? 1 : 0;
  g.b = static_cast<const __nv_bfloat16*>(b);
  g.ldb = ldb;
  g.b_kmajor = b_kmajor ? 1 : 0;
  g.M = M;
  g.N = N;
  g.K = K;
  g.k_per_split = k_per_split;
  g.d = d;
  g.ldd = ldd;
  g.split_stride = split_stride;
  g.mode = kGemmRaw;
  g.err = nullptr;
  if (!gemm_args_valid(g, splits)) return MCLBM_EINVAL;
  return launch_gemm(g, splits, static_cast<cudaStream_t>(stream)) == cudaSuccess ? MCLBM_OK
                                                                                   : MCLBM_ECUDA;
}

}  // extern "C"
