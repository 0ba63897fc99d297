// Internal interfaces of the warm-start network (include/mclbm_net.h): the tensor-core GEMM and
// the CUDA-core kernels around it. Host code in net_abi.cu, kernels in net_gemm.cu and
// net_kernels.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mcl {
namespace net {

// Predicted fields: u_x, u_y, theta, phi, rho^w. Channels 3 and 4 are learned as deviations from
// the sample's rest values phi_0 and 1 - phi_0 (base_fields).
constexpr int kFields = 5;

// Epilogue of the GEMM.
enum GemmMode : int {
  kGemmRaw = 0,      // D(m, n) -> d[z * split_stride + m * ldd + n] (d_trans: + n * ldd + m)
  kGemmConvFwd = 1,  // m = pixel p, n = output channel o (see ConvEpilogue)
};

// Convolution forward epilogue: pre[o][p] = D(p, o) + bias[o];
// z = film ? (1 + film[b][foff + o]) pre + film[b][foff + C + o] : pre, b = p / hw;
// y[o][p] = act ? silu(z) : z (y may be null).
struct ConvEpilogue {
  const float* bias;
  const float* film;  // [batch][film_stride] or null
  int film_stride, film_off, hw;
  float* pre;
  float* y;
  int act;
};

struct GemmArgs {
  const __nv_bfloat16* a;
  int64_t lda;
  int a_kmajor;
  int a_vec;  // set by launch_gemm: 16-byte loads of A
  const __nv_bfloat16* b;
  int64_t ldb;
  int b_kmajor;
  int b_vec;
  int M, N, K;
  int64_t k_per_split;  // multiple of 64
  float* d;
  int64_t ldd, split_stride;
  int d_trans;  // raw epilogue stores D column-major (coalesced when N is small and M large)
  int mode;
  ConvEpilogue ep;
  int* err;  // bit 0 set when a bounded wait gave up (may be null)
  int splits;  // set by launch_gemm: K splits (tiles of D are m x n x split)
};

// Checks the operand requirements and launches a persistent grid over the ceil(M/128) x
// ceil(N/128) x splits tiles of D.
cudaError_t launch_gemm(const GemmArgs& g, int splits, cudaStream_t st);
// True if the arguments satisfy the alignment and extent rules of launch_gemm.
bool gemm_args_valid(const GemmArgs& g, int splits);

// ---- CUDA-core kernels (net_kernels.cu) ---------------------------------------------------
struct Im2colArgs {
  const float* src1;  // [cu][batch * H1 * W1], H1 = up ? H/2 : H
  const float* src2;  // [cs][batch * H * W] or null
  int cu, cs, up;     // channels from each source; up: src1 is upsampled by 2 (nearest)
  int batch, H, W;    // input grid of the convolution (after upsampling and concatenation)
  int stride, Ho, Wo;
  int Kp;             // row stride of cols, >= 9 (cu + cs), multiple of 8
  __nv_bfloat16* cols;  // [batch * Ho * Wo][Kp]
};
cudaError_t launch_im2col(const Im2colArgs& a, cudaStream_t st);

// im2col of a BF16 tensor [C][batch * H * W] for a stride-1 3 x 3 convolution with zero
// padding: cols [batch * H * W][Kp], column c * 9 + tap (tap = 3 ky + kx), zero beyond 9 C.
struct Im2colBf16Args {
  const __nv_bfloat16* src;
  int C, batch, H, W, Kp;
  __nv_bfloat16* cols;
};
cudaError_t launch_im2col_bf16(const Im2colBf16Args& a, cudaStream_t st);

// W [cout][9 cin] FP32 -> the input-gradient operand wt [cin][Kp2] BF16 (round to nearest, as
// wb): wt[c][o 9 + t] = W[o][c 9 + 8 - t], the flipped and transposed kernel; zero beyond 9 cout.
cudaError_t launch_weights_t_bf16(const float* w, int cout, int cin, int Kp2, __nv_bfloat16* wt,
                                  cudaStream_t st);

// dX [cu + cs][P] (P = batch * H * W, the convolution's input grid) to its sources' gradients:
// channels [0, cu) to dsrc1 (summed over each 2 x 2 block, in row order, when src1 was upsampled
// by 2), [cu, cu + cs) to dsrc2; each written (acc = 0) or added to (acc = 1).
struct RouteArgs {
  const float* dx;
  int cu, cs, up, batch, H, W;
  float* dsrc1;
  float* dsrc2;
  int acc1, acc2;
};
cudaError_t launch_route_grad(const RouteArgs& a, cudaStream_t st);

// Gradient with respect to one source of a convolution's input from dcols [Kp][P] (FP32,
// column k = c * 9 + tap of the im2col matrix stored contiguously over the P output pixels):
// channels [c_lo, c_lo + C) of the concatenated input, source grid Hs x Ws (H/2 if up).
struct Col2imArgs {
  const float* dcols;
  int Kp, c_lo, C, up;
  int batch, H, W, stride, Ho, Wo;
  float* dsrc;  // [C][batch * Hs * Ws]
  int accumulate;
};
cudaError_t launch_col2im(const Col2imArgs& a, cudaStream_t st);

// Backward of act(film(pre)) for one layer: dpre (BF16, [C][P]) and per (o, b) partial sums
// {sum dpre, sum dz pre, sum dz} (compensated FP32 per thread, FP64 across the block).
struct ActBwdArgs {
  const float* dy;    // [C][P]
  const float* pre;   // [C][P]
  const float* film;  // [batch][film_stride] or null
  int film_stride, film_off;
  int C, batch, hw, act;
  __nv_bfloat16* dpre;
  double* partial;  // [C][batch][3]
};
cudaError_t launch_act_backward(const ActBwdArgs& a, cudaStream_t st);
// dbias[o] = sum_b partial[o][b][0]; if film: dfilm[b][foff + o] = partial[o][b][1],
// dfilm[b][foff + C + o] = partial[o][b][2].
cudaError_t launch_bias_film_grad(const double* partial, int C, int batch, float* dbias,
                                  float* dfilm, int film_stride, int film_off, cudaStream_t st);

// grad[o][k] = sum_z part[z][o][k] for k < kin (dropping padding columns up to Kp).
cudaError_t launch_splitk_reduce(const float* part, int splits, int64_t split_stride, int C,
                                 int kin, int Kp, float* grad, cudaStream_t st);

// The convolution epilogue after a K-split forward GEMM: part [splits][N][M] (column-major
// partial products, split_stride apart) summed over the splits in order, then bias, FiLM and the
// activation as the GEMM's own epilogue applies them (pre and y [N][M]).
cudaError_t launch_conv_epilogue_splitk(const float* part, int splits, int64_t split_stride,
                                        int M, int N, const ConvEpilogue& e, cudaStream_t st);

// W [C][kin] FP32 -> wb [C][Kp] BF16 (round to nearest, zero padding).
cudaError_t launch_weights_bf16(const float* w, int C, int kin, int Kp, __nv_bfloat16* wb,
                                cudaStream_t st);

// Conditioning MLP. cond_raw [batch][3] (Ra, phi, d_p) -> c [batch][3], a1 [batch][H],
// r [batch][F].
struct MlpArgs {
  const float* cond_raw;
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  int batch, H, F;
  float* c;
  float* a1;
  float* r;
};
cudaError_t launch_mlp_forward(const MlpArgs& a, cudaStream_t st);
// Given dr [batch][F]: gradients of W1, b1, W2, b2 (written, not accumulated).
cudaError_t launch_mlp_backward(const MlpArgs& a, const float* dr, float* gW1, float* gb1,
                                float* gW2, float* gb2, cudaStream_t st);

// Loss against target fields [batch][5][hw]: dout[ch][b*hw + i] = 2 (out - t) / n,
// t = (F - base - mean) / scale; per-block FP64 partial sums of (out - t)^2 into partial[blocks].
struct LossArgs {
  const float* out;     // [5][batch * hw]
  const float* target;  // [batch][5][hw]
  const float* cond;    // [batch][3] raw (Ra, phi, d_p): the base of channels 3 and 4
  const float* norm;    // mean[5], scale[5]
  int batch, hw;
  float* dout;
  double* partial;
  int blocks;
};
cudaError_t launch_loss(const LossArgs& a, cudaStream_t st);
// out[0] = sum of partial[0..n) in a fixed order.
cudaError_t launch_sum_partials(const double* partial, int n, double* out, cudaStream_t st);

// Adam over n parameters; c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t).
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t st);

// p[i] = scale * u_i, u_i uniform in [-1, 1) (splitmix64 of seed, stream and i).
cudaError_t launch_uniform_fill(float* p, int64_t n, float scale, uint64_t seed, uint32_t stream,
                                cudaStream_t st);
// Geometry input X [4][batch * ny * nx].
cudaError_t launch_geometry(float* X, int batch, int ny, int nx, cudaStream_t st);
// fields[b][ch][i] = base[b][ch] + mean[ch] + scale[ch] * out[ch][b*hw + i]; phi (ch 3) and
// rho^w (ch 4) are then shifted so that their means are phi_0 = cond[b][1] and 1 - phi_0.
cudaError_t launch_denormalize(const float* out, const float* norm, const float* cond, int batch,
                               int hw, float* fields, cudaStream_t st);
// Per-channel FP64 sum and sum of squares of fields - base, fields [n][5][hw], cond [n][3], into
// partial[5][blocks][2].
cudaError_t launch_field_moments(const float* fields, const float* cond, int n, int hw,
                                 double* partial, int blocks, cudaStream_t st);

}  // namespace net
}  // namespace mcl
