/*
 * mclbm_net.h -- C ABI of the learned warm start in libmclbm.so: a small conditioned
 * convolutional encoder-decoder that predicts the steady fields (u_x, u_y, theta, phi, rho^w)
 * of a differentially heated cavity from (Ra, phi, d_p), trained and evaluated on the GPU by the
 * library's own BF16 tensor-core kernels (tcgen05 MMA, FP32 accumulation in tensor memory).
 * Its prediction seeds mclbm_init(MCLBM_INIT_WARM_RHO); the plain cold-started solve remains the
 * judge of the steady state. The paper (arXiv:1511.04552) has no learned component: this is
 * an acceleration of its steady-state computation (the results of its Section 3, e.g. Fig. 8,
 * are steady states), and the network below is this library's own design.
 *
 * Network (ny, nx multiples of 16; c0 base channels; C = c0, 2c0, 4c0, 8c0, 8c0):
 *   input X [4][ny][nx]: mask, mask*xi, mask*eta, mask*4*xi*eta, xi = (i+1/2)/nx - 1/2,
 *     eta = (j+1/2)/ny - 1/2;  conditioning c = ((log10 Ra - 4.5)/1.5, (phi - 0.025)/0.025,
 *     (d_p/1nm - 55)/45);  conv = 3x3, zero padding 1;  SiLU activations;
 *   e0 = conv(X, 4->C0), e1..e3 = stride-2 convs, e4 = stride-2 conv + FiLM;
 *   d3, d2, d1, d0 = conv(cat(up2(previous), skip)) + FiLM;  out = conv(d0, C0->5);
 *   FiLM: gamma = 1 + r[a:a+C], beta = r[a+C:a+2C], r = W2 silu(W1 c + b1) + b2, slices in the
 *   order e4, d3, d2, d1, d0;  fields = base + mean + scale * out with base = (0, 0, 0, phi,
 *   1 - phi) (phi and rho^w are learned as deviations from their rest values; per-channel
 *   normaliser of fields - base), then phi and rho^w shifted so that their cavity means are phi
 *   and 1 - phi (the solver conserves both components' masses).
 * Parameters: one flat FP32 vector, per conv layer (e0..e4, d3..d0, out) W[Cout][Cin][3][3]
 *   then b[Cout], then W1[hidden][3], b1[hidden], W2[F][hidden], b2[F], F = 2(C4+C3+C2+C1+C0).
 * Every convolution is an im2col GEMM on the tensor cores with BF16 operands (activations,
 * weights, and in the backward pass the pre-activation gradient, each rounded to nearest) and
 * FP32 accumulation: the forward pass, the weight gradient, and the input gradient (for the
 * stride-1 layers as the convolution of the pre-activation gradient with the flipped,
 * transposed kernel; for the stride-2 layers as a GEMM into the column gradient and its
 * fixed-order gather); everything else (FiLM, SiLU, the conditioning MLP, loss, reductions,
 * Adam) runs in FP32 CUDA-core kernels with fixed-order sums (FP64 across blocks).
 *
 * Conventions: return MCLBM_OK (0) or a negative MCLBM_E* code (mclbm.h); the caller owns all
 * device memory (one workspace handed over by mclbm_net_bind, plus every input and output) and
 * the stream; calls marked "async" only enqueue work, "syncs" wait for the stream.
 * Layouts: cond [batch][3] FP32 (Ra, phi, d_p in metres) on the device; fields
 * [batch][5][ny][nx] FP32 (u_x, u_y, theta, phi, rho^w), per sample the layout
 * mclbm_init(MCLBM_INIT_WARM_RHO) reads and mclbm_fields(UX|UY|THETA|PHI|RHO_W) writes.
 */
#ifndef MCLBM_NET_H
#define MCLBM_NET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mclbm_net mclbm_net_t;

typedef struct mclbm_net_config {
  int32_t ny, nx;     /* output grid; multiples of 16, 16..4096 */
  int32_t c0;         /* base channels; a multiple of 8, 8..64 */
  int32_t hidden;     /* width of the conditioning MLP; 1..256, max_batch * hidden <= 4096 */
  int32_t max_batch;  /* largest batch of any call; 1..256, max_batch * ny * nx <= 2^26 */
} mclbm_net_config;

/* 256 x 256, c0 = 16, hidden = 64, max_batch = 16 (734 293 parameters). */
void mclbm_net_config_default(mclbm_net_config* cfg);
/* Number of FP32 parameters; 0 for an invalid configuration. */
int64_t mclbm_net_param_count(const mclbm_net_config* cfg);
/* Bytes of the device workspace mclbm_net_bind needs (parameters, Adam moments, activations,
 * im2col buffers, gradients); 0 for an invalid configuration. */
size_t mclbm_net_workspace_bytes(const mclbm_net_config* cfg);

/* A network handle for the configuration (copied). Host-only: no device memory until
 * mclbm_net_bind. *out is NULL on failure; EINVAL for a NULL out or an invalid configuration. */
int mclbm_net_create(const mclbm_net_config* cfg, mclbm_net_t** out);
/* Frees the handle (host memory only; the caller's workspace stays the caller's). NULL is a
 * no-op. */
void mclbm_net_destroy(mclbm_net_t* net);
/* Text of the handle's latest error ("" if none or for a NULL handle); owned by the handle,
 * valid until its next call. */
const char* mclbm_net_last_error(const mclbm_net_t* net);

/* Hands over a device workspace of at least mclbm_net_workspace_bytes (256-byte aligned) and
 * the stream of every later call; fills the geometry input. Parameters are zero, the
 * normaliser is mean 0, scale 1 and the Adam step count 0 until set. syncs. */
int mclbm_net_bind(mclbm_net_t* net, void* workspace_dev, size_t bytes, void* cuda_stream);

/* Copies param_count FP32 parameters (device pointer) in or out. set also resets Adam's moments
 * and step count. async. */
int mclbm_net_set_params(mclbm_net_t* net, const float* params_dev);
int mclbm_net_get_params(mclbm_net_t* net, float* params_dev);

/* Seeded initial parameters: every convolution weight and W1, W2 uniform with the variance of
 * He initialisation (bound sqrt(6 / fan_in); W2 scaled by 0.1 so that FiLM starts near the
 * identity), biases zero; resets Adam. async. */
int mclbm_net_init_params(mclbm_net_t* net, uint64_t seed);

/* Per-channel normaliser of fields - base (host arrays of 5; scale > 0). syncs. */
int mclbm_net_set_normalizer(mclbm_net_t* net, const double* mean, const double* scale);
/* Per-channel mean and standard deviation (scale 1 for a constant channel) of fields - base
 * over n samples (cond [n][3], fields [n][5][ny][nx], both on the device), FP64 sums. mean and
 * scale: host arrays of 5. syncs. */
int mclbm_net_field_stats(mclbm_net_t* net, int n, const float* cond_dev, const float* fields_dev,
                          double* mean, double* scale);

/* Predicted fields [batch][5][ny][nx] for cond [batch][3] (see the definition above). async. */
int mclbm_net_forward(mclbm_net_t* net, int batch, const float* cond_dev, float* fields_dev);

/* Loss (mean squared error of the normalised output against the normalised target fields
 * (target - base - mean) / scale, target [batch][5][ny][nx]) and its gradient with respect to
 * the flat parameters (grad_dev, param_count floats). syncs. */
int mclbm_net_loss_grad(mclbm_net_t* net, int batch, const float* cond_dev,
                        const float* target_dev, float* grad_dev, double* loss);

/* One training step: forward, loss, backward and an Adam update (beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr). *loss (may be NULL) receives the loss before the update; with a
 * non-NULL loss the call syncs, otherwise it is async. */
int mclbm_net_train_step(mclbm_net_t* net, int batch, const float* cond_dev,
                         const float* target_dev, float lr, double* loss);

/* The tensor-core GEMM every convolution uses, exposed for tests:
 *   D[z][m][n] = sum over k in split z of A(m, k) B(n, k),   0 <= m < M, 0 <= n < N,
 * A(m, k) = a[m*lda + k] (a_kmajor != 0) or a[k*lda + m]; B(n, k) likewise with b, ldb;
 * BF16 operands, FP32 result d[z*split_stride + m*ldd + n]; K is cut into `splits` ranges of
 * k_per_split (a multiple of 64), splits * k_per_split >= K. When both operands have 16-byte
 * aligned pointers and leading dimensions and contiguous extents in multiples of 8 elements,
 * they are brought in by TMA tensor loads (128-byte swizzle) for a persistent, warp-specialised
 * kernel; otherwise threads stage them (16-byte or element loads). EINVAL for non-positive
 * sizes, null or odd pointers, or a leading dimension below the contiguous extent. async. */
int mclbm_gemm_bf16(int M, int N, int K, const void* a, int64_t lda, int a_kmajor, const void* b,
                    int64_t ldb, int b_kmajor, float* d, int64_t ldd, int splits,
                    int64_t k_per_split, int64_t split_stride, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MCLBM_NET_H */
