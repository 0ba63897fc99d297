// extern "C" entry points of libmclbm (declared in include/mclbm.h): handle life cycle,
// binding of caller memory, graph-captured stepping, reductions and host round trips.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mclbm_internal.h"
#include "nvtx_range.h"

using namespace mcl;

struct mclbm {
  int nx, ny;
  double Ra, Pr, phi, d_p;
  mclbm_props props;
  mclbm_consts c;
  StepConsts k;
  Layout L;
  StepConfig cfg;
  // bound memory
  char* buf = nullptr;
  size_t buf_bytes = 0;
  cudaStream_t stream = nullptr;
  int device = -1;
  char* state[2] = {nullptr, nullptr};  // two time levels, element type of L.storage
  float* snap = nullptr;     // [4][ny][nx]
  float* staging = nullptr;  // [kFields][ny][nx]
  double* partials = nullptr;
  double* red = nullptr;
  int* err_dev = nullptr;       // device error word of the step kernels (bounded waits)
  uint32_t* epoch = nullptr;    // graph replay counter seeding 16-bit stochastic rounding
  CUtensorMap tmap[2];          // two-level state for the TMA step kernel: loads, stores
  CUtensorMap tmap2;            // two-level state for the two-step kernel's window loads
  int cur = 0;
  bool initialised = false;
  bool diverged = false;
  int64_t steps = 0, snap_steps = 0;
  // graph[from][k]: 2^k steps starting from time level 0 or 1 (built on first use)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[2][kGraphLogMax + 1] = {};
  char err[512] = {0};
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int fail(mclbm_t* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(mclbm_t* h, cudaError_t e, const char* where) {
  return fail(h, MCLBM_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(h, expr)                                            \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr);   \
  } while (0)

struct Regions {
  size_t state, snap, staging, partials, red, err, total;
};

Regions regions(const mclbm_t* h) {
  Regions r;
  const size_t n = (size_t)h->nx * h->ny;
  size_t off = 0;
  r.state = off;
  off += align_up(2 * (size_t)h->L.np * h->L.plane * h->L.elem, 256);
  r.snap = off;
  off += align_up(4 * n * sizeof(float), 256);
  r.staging = off;
  off += align_up(kFields * n * sizeof(float), 256);
  r.partials = off;
  off += align_up((size_t)kMaxRedBlocks * kRedWidth * sizeof(double), 256);
  r.red = off;
  off += align_up((size_t)3 * kRedWidth * sizeof(double), 256);  // mclbm_diagnostics: 3 slots
  r.err = off;
  off += 256;
  r.total = off;
  return r;
}

int ready(mclbm_t* h, bool need_init) {
  if (!h) return MCLBM_EINVAL;
  if (!h->buf) return fail(h, MCLBM_ESTATE, "no device buffer bound (call mclbm_bind)");
  if (need_init && !h->initialised)
    return fail(h, MCLBM_ESTATE, "state not initialised (call mclbm_init or mclbm_state_set)");
  int dev = -1;
  CK(h, cudaGetDevice(&dev));
  if (dev != h->device) CK(h, cudaSetDevice(h->device));
  return MCLBM_OK;
}

void drop_graphs(mclbm_t* h) {
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k <= kGraphLogMax; ++k)
      if (h->graph[p][k]) {
        cudaGraphExecDestroy(h->graph[p][k]);
        h->graph[p][k] = nullptr;
      }
}

StepArgs step_args(const mclbm_t* h, int from, uint32_t seed) {
  StepArgs a;
  a.src = h->state[from];
  a.dst = h->state[1 - from];
  a.L = h->L;
  a.seed = seed;
  a.epoch = h->epoch;
  a.z_src = from * kPlanes;
  a.err = h->err_dev;
  a.k = h->k;
  return a;
}

// Captures 2^k (k >= 1) alternating step launches starting from time level `from`.
int build_graph(mclbm_t* h, int from, int k) {
  if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const int n = 1 << k;
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  if (h->cfg.two) {  // pairs of steps: n / 2 launches, the level alternating per pair
    for (int s = 0; s < n / 2 && le == cudaSuccess; ++s)
      le = launch_two_f32(step_args(h, (from + s) & 1, (uint32_t)s), h->cfg, &h->tmap2,
                          h->cap_stream);
  } else {
    for (int s = 0; s < n && le == cudaSuccess; ++s)
      le = launch_step(step_args(h, (from + s) & 1, (uint32_t)s), h->cfg, h->tmap,
                       h->cap_stream);
  }
  // a new stochastic-rounding epoch for the next replay
  if (le == cudaSuccess) le = launch_epoch_advance(h->epoch, h->cap_stream);
  cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, le, "launch_step (capture)");
  }
  if (ee != cudaSuccess) return cuda_fail(h, ee, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(&h->graph[from][k], g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    h->graph[from][k] = nullptr;
    return cuda_fail(h, ie, "cudaGraphInstantiate");
  }
  return MCLBM_OK;
}

// Copies a reduction result to the host and waits; also reports a step kernel that gave up
// a bounded wait since the last init.
int d2h_sync(mclbm_t* h, void* host, const void* dev, size_t bytes) {
  int err = 0;
  CK(h, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaMemcpyAsync(&err, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (err) return fail(h, MCLBM_ETIMEOUT, "a step kernel gave up a bounded wait (error word %d)",
                       err);
  return MCLBM_OK;
}

int snapshot(mclbm_t* h) {
  CK(h, launch_residual(h->state[h->cur], h->L, h->k, h->snap, false, h->partials, h->red,
                        h->stream));
  h->snap_steps = h->steps;
  return MCLBM_OK;
}

}  // namespace

extern "C" {

void mclbm_props_default(mclbm_props* p) {
  if (p) props_default(p);
}

int mclbm_create(int nx, int ny, double Ra, double Pr, double phi, double d_p,
                 const mclbm_props* props, mclbm_t** out) {
  if (!out) return MCLBM_EINVAL;
  *out = nullptr;
  if (nx < 2 || ny < 2 || nx > 32768 || ny > 32768) return MCLBM_EINVAL;
  mclbm_props p;
  if (props)
    p = *props;
  else
    props_default(&p);
  if (!(std::isfinite(Ra) && Ra > 0) || !(std::isfinite(Pr) && Pr > 0) ||
      !(phi >= 0 && phi < 0.2) || !(std::isfinite(d_p) && d_p > 0))
    return MCLBM_EPARAM;
  const double pos[] = {p.rho_f, p.cp_f, p.k_f, p.beta_f, p.mu_f, p.rho_p, p.cp_p,
                        p.k_p,   p.T0_K, p.dT_K, p.g,    p.l_f};
  for (double v : pos)
    if (!(std::isfinite(v) && v > 0)) return MCLBM_EPARAM;
  if (!(p.beta_p >= 0) || !(p.Ma > 0 && p.Ma <= 0.5)) return MCLBM_EPARAM;
  if (p.force_mask & ~MCLBM_F_ALL) return MCLBM_EINVAL;
  if (p.storage != MCLBM_STORE_F32 && p.storage != MCLBM_STORE_F16 &&
      p.storage != MCLBM_STORE_BF16)
    return MCLBM_EINVAL;
  if (p.rounding != MCLBM_ROUND_STOCHASTIC && p.rounding != MCLBM_ROUND_NEAREST)
    return MCLBM_EINVAL;
  if (p.thermal_sets != 1 && p.thermal_sets != 2) return MCLBM_EINVAL;
  mclbm_t* h = new (std::nothrow) mclbm();
  if (!h) return MCLBM_EINVAL;
  h->nx = nx;
  h->ny = ny;
  h->Ra = Ra;
  h->Pr = Pr;
  h->phi = phi;
  h->d_p = d_p;
  h->props = p;
  int rc = derive_consts(nx, ny, Ra, Pr, phi, d_p, p, &h->c);
  if (rc != MCLBM_OK) {
    delete h;
    return rc;
  }
  h->k = fold_step_consts(nx, ny, phi, d_p, p, h->c);
  h->L.nx = nx;
  h->L.ny = ny;
  h->L.storage = p.storage;
  h->L.elem = p.storage == MCLBM_STORE_F32 ? 4 : 2;
  h->L.pitch = (int)align_up((size_t)nx, 128 / h->L.elem);  // 128-byte rows
  h->L.plane = (size_t)h->L.pitch * ny;
  h->L.np = p.thermal_sets == 2 ? kPlanes2 : kPlanes;
  h->cfg = choose_step_config(nx, ny, h->L.np);
  *out = h;
  return MCLBM_OK;
}

void mclbm_destroy(mclbm_t* h) {
  if (!h) return;
  if (h->buf) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != h->device) cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
  }
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

size_t mclbm_buffer_bytes(const mclbm_t* h) { return h ? regions(h).total : 0; }

int mclbm_bind(mclbm_t* h, void* dev_buf, size_t bytes, void* cuda_stream) {
  if (!h) return MCLBM_EINVAL;
  const Regions r = regions(h);
  if (!dev_buf) return fail(h, MCLBM_EINVAL, "device buffer is NULL");
  if (bytes < r.total)
    return fail(h, MCLBM_EINVAL, "buffer of %zu bytes, %zu needed", bytes, r.total);
  if ((reinterpret_cast<uintptr_t>(dev_buf) & 255u) != 0)
    return fail(h, MCLBM_EINVAL, "device buffer not 256-byte aligned");
  cudaPointerAttributes at;
  CK(h, cudaPointerGetAttributes(&at, dev_buf));
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(h, MCLBM_EINVAL, "buffer is not device memory");
  CK(h, cudaSetDevice(at.device));
  drop_graphs(h);
  h->device = at.device;
  h->buf = static_cast<char*>(dev_buf);
  h->buf_bytes = bytes;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->state[0] = h->buf + r.state;
  h->state[1] = h->state[0] + (size_t)h->L.np * h->L.plane * h->L.elem;
  h->snap = reinterpret_cast<float*>(h->buf + r.snap);
  h->staging = reinterpret_cast<float*>(h->buf + r.staging);
  h->partials = reinterpret_cast<double*>(h->buf + r.partials);
  h->red = reinterpret_cast<double*>(h->buf + r.red);
  h->err_dev = reinterpret_cast<int*>(h->buf + r.err);
  h->epoch = reinterpret_cast<uint32_t*>(h->buf + r.err + 4);
  // device-dependent set-up of the step kernel; the TMA variant falls back to the plain tile
  // kernel if the device cannot run it
  h->cfg = choose_step_config(h->nx, h->ny, h->L.np);
  h->cfg.sr = h->props.rounding == MCLBM_ROUND_STOCHASTIC;
  if (h->cfg.variant == 2) {
    if (prepare_step(&h->cfg, h->L) != cudaSuccess ||
        make_state_tensor_map(h->tmap, h->state[0], h->L, step_tile_width(h->cfg), h->cfg.th) !=
            cudaSuccess) {
      cudaGetLastError();
      h->cfg.variant = 0;
    }
  }
  // MCLBM_STEP_VARIANT = two (FP32 lattices of at most one 32 x 16 tile per SM): pairs of steps
  // in one launch, bitwise the same states; not the default, since it is no faster (the first
  // step's 1.7x redundant work outweighs the launch it saves)
  const char* sv = std::getenv("MCLBM_STEP_VARIANT");
  const bool two_asked = sv && std::strcmp(sv, "two") == 0;
  if (two_asked && h->cfg.variant == 2 && h->L.storage == MCLBM_STORE_F32 &&
      h->L.np == kPlanes && h->cfg.vec != 2) {
    if (prepare_two_f32(&h->cfg, h->L) != cudaSuccess ||
        make_two_step_tensor_map(&h->tmap2, h->state[0], h->L) != cudaSuccess) {
      cudaGetLastError();
      h->cfg.two = false;
    }
  }
  CK(h, cudaMemsetAsync(h->err_dev, 0, 2 * sizeof(int), h->stream));
  h->cur = 0;
  h->initialised = false;
  h->diverged = false;
  h->steps = h->snap_steps = 0;
  h->err[0] = 0;
  return MCLBM_OK;
}

int mclbm_init(mclbm_t* h, int mode, const float* warm_dev) {
  int rc = ready(h, false);
  if (rc) return rc;
  if (mode != MCLBM_INIT_REST && mode != MCLBM_INIT_WARM && mode != MCLBM_INIT_WARM_RHO)
    return fail(h, MCLBM_EINVAL, "unknown init mode %d", mode);
  if (mode != MCLBM_INIT_REST && !warm_dev)
    return fail(h, MCLBM_EINVAL, "warm init modes need warm fields");
  h->cur = 0;
  CK(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
  CK(h, launch_init(h->state[0], h->L, h->k, mode == MCLBM_INIT_REST ? nullptr : warm_dev,
                    mode == MCLBM_INIT_WARM_RHO ? 1 : 0, h->stream));
  h->steps = 0;
  h->initialised = true;
  h->diverged = false;
  return snapshot(h);
}

int mclbm_step(mclbm_t* h, int64_t n) {
  mcl::NvtxRange range("mclbm_step");
  int rc = ready(h, true);
  if (rc) return rc;
  if (n < 0) return fail(h, MCLBM_EINVAL, "negative step count");
  // the even part in graphs of 2^k steps, largest first (1000 = 512 + 256 + 128 + 64 + 32 + 8;
  // each graph boundary costs about 4 us of idle GPU), an odd last step as a single launch
  int64_t left = n;
  while (left >= 2) {
    int k = 1;
    while (k < kGraphLogMax && (int64_t(2) << k) <= left) ++k;
    if (!h->graph[h->cur][k]) {
      rc = build_graph(h, h->cur, k);
      if (rc) return rc;
    }
    CK(h, cudaGraphLaunch(h->graph[h->cur][k], h->stream));
    left -= int64_t(1) << k;
    h->steps += int64_t(1) << k;
    // an even number of single steps ends on the level it started from; a pair of steps of
    // the two-step kernel moves to the other level, so 2^(k-1) pairs do so only for k = 1
    if (h->cfg.two && k == 1) h->cur ^= 1;
  }
  for (; left > 0; --left) {
    CK(h, launch_step(step_args(h, h->cur, 0x80000000u ^ (uint32_t)h->steps), h->cfg, h->tmap,
                      h->stream));
    h->cur ^= 1;
    h->steps += 1;
  }
  return MCLBM_OK;
}

int mclbm_stream_only(mclbm_t* h) {
  int rc = ready(h, true);
  if (rc) return rc;
  CK(h, launch_stream_only(h->state[h->cur], h->state[1 - h->cur], h->L, h->k, h->stream));
  h->cur ^= 1;
  return MCLBM_OK;
}

int mclbm_fields(mclbm_t* h, uint32_t which, float* dev_out) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!dev_out || which == 0 || (which & ~kFieldMask))
    return fail(h, MCLBM_EINVAL, "bad field selection 0x%x or NULL output", which);
  CK(h, launch_fields(h->state[h->cur], h->L, h->k, which, dev_out, h->stream));
  return MCLBM_OK;
}

}  // extern "C"

namespace {

// Host halves of the reductions: from the FP64 sums on the device to the reported numbers.
int nusselt_from(mclbm_t* h, const double* s, double* nu_hot, double* nu_cold) {
  const double scale = h->c.k_ratio * (double)h->nx / (double)h->ny;  // L / dT, dT = 1
  *nu_hot = s[0] * scale;
  *nu_cold = s[1] * scale;
  if (!std::isfinite(*nu_hot) || !std::isfinite(*nu_cold)) h->diverged = true;
  if (h->diverged) return fail(h, MCLBM_EDIVERGED, "non-finite Nusselt number");
  return MCLBM_OK;
}

int mass_from(mclbm_t* h, const double* s, double* mass_w, double* mass_p) {
  const double n = (double)h->nx * h->ny;
  *mass_w = s[0] + n * h->c.rho_w0;
  *mass_p = s[1] + n * h->c.rho_p0;
  if (!std::isfinite(*mass_w) || !std::isfinite(*mass_p)) h->diverged = true;
  if (h->diverged) return fail(h, MCLBM_EDIVERGED, "non-finite mass");
  return MCLBM_OK;
}

// K steps since the snapshot; s = the six sums (||q_now - q_then||^2, ||q_now||^2 for u,
// theta, phi), unused when K = 0.
int residual_from(mclbm_t* h, int64_t K, const double* s, double* r) {
  double res = 0.0;
  for (int g = 0; K > 0 && g < 3; ++g) {
    const double num = s[2 * g], den = s[2 * g + 1];
    double term;
    if (num == 0.0)
      term = 0.0;
    else if (den == 0.0)
      term = INFINITY;
    else
      term = std::sqrt(num) / ((double)K * std::sqrt(den));
    if (term > res || std::isnan(term)) res = term;
  }
  *r = res;
  if (std::isnan(res)) h->diverged = true;
  if (h->diverged) return fail(h, MCLBM_EDIVERGED, "non-finite residual");
  return MCLBM_OK;
}

}  // namespace

extern "C" {

int mclbm_nusselt(mclbm_t* h, double* nu_hot, double* nu_cold) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!nu_hot || !nu_cold) return fail(h, MCLBM_EINVAL, "NULL output");
  CK(h, launch_nusselt(h->state[h->cur], h->L, h->k, h->red, h->stream));
  double s[2];
  rc = d2h_sync(h, s, h->red, sizeof(s));
  if (rc) return rc;
  return nusselt_from(h, s, nu_hot, nu_cold);
}

int mclbm_mass(mclbm_t* h, double* mass_w, double* mass_p) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!mass_w || !mass_p) return fail(h, MCLBM_EINVAL, "NULL output");
  CK(h, launch_mass(h->state[h->cur], h->L, h->partials, h->red, h->stream));
  double s[2];
  rc = d2h_sync(h, s, h->red, sizeof(s));
  if (rc) return rc;
  return mass_from(h, s, mass_w, mass_p);
}

int mclbm_residual(mclbm_t* h, double* r) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!r) return fail(h, MCLBM_EINVAL, "NULL output");
  const int64_t K = h->steps - h->snap_steps;
  CK(h, launch_residual(h->state[h->cur], h->L, h->k, h->snap, K > 0, h->partials, h->red,
                        h->stream));
  h->snap_steps = h->steps;
  double s[6] = {0, 0, 0, 0, 0, 0};
  if (K > 0) {
    rc = d2h_sync(h, s, h->red, sizeof(s));
    if (rc) return rc;
  } else {
    CK(h, cudaStreamSynchronize(h->stream));
  }
  return residual_from(h, K, s, r);
}

int mclbm_diagnostics(mclbm_t* h, double* nu_hot, double* nu_cold, double* mass_w,
                      double* mass_p, double* r) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!nu_hot || !nu_cold || !mass_w || !mass_p || !r)
    return fail(h, MCLBM_EINVAL, "NULL output");
  // the three reductions one after another on the stream, each into its own slot of the
  // result area (the partial sums are reused in stream order), then one copy and one wait
  const int64_t K = h->steps - h->snap_steps;
  CK(h, launch_nusselt(h->state[h->cur], h->L, h->k, h->red, h->stream));
  CK(h, launch_mass(h->state[h->cur], h->L, h->partials, h->red + kRedWidth, h->stream));
  CK(h, launch_residual(h->state[h->cur], h->L, h->k, h->snap, K > 0, h->partials,
                        h->red + 2 * kRedWidth, h->stream));
  h->snap_steps = h->steps;
  double s[3 * kRedWidth];
  rc = d2h_sync(h, s, h->red, sizeof(s));
  if (rc) return rc;
  const int r1 = nusselt_from(h, s, nu_hot, nu_cold);
  const int r2 = mass_from(h, s + kRedWidth, mass_w, mass_p);
  const int r3 = residual_from(h, K, s + 2 * kRedWidth, r);
  return r1 ? r1 : (r2 ? r2 : r3);
}

int mclbm_state_get(mclbm_t* h, float* dev_out) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!dev_out) return fail(h, MCLBM_EINVAL, "NULL output");
  CK(h, launch_state_copy(h->state[h->cur], dev_out, h->L, true, h->stream));
  return MCLBM_OK;
}

int mclbm_state_set(mclbm_t* h, const float* dev_in) {
  int rc = ready(h, false);
  if (rc) return rc;
  if (!dev_in) return fail(h, MCLBM_EINVAL, "NULL input");
  h->cur = 0;
  CK(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
  CK(h, launch_state_copy(dev_in, h->state[0], h->L, false, h->stream));
  h->steps = 0;
  h->initialised = true;
  h->diverged = false;
  return snapshot(h);
}

namespace {

// Checkpoint file: this header, then the current time level's population planes exactly as
// stored on the device (27 or 36 planes of pitch x ny elements of the storage type).
struct CheckpointHeader {
  char magic[8];  // "MCLBMCK1"
  uint32_t version;
  int32_t nx, ny, pitch, storage, rounding;
  int64_t steps;
  uint32_t epoch, reserved;
  double Ra, Pr, phi, d_p;
  uint64_t props_hash;
  uint64_t payload_bytes;
};

void fnv1a(uint64_t& x, const void* v, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(v);
  for (size_t i = 0; i < n; ++i) {
    x ^= b[i];
    x *= 1099511628211ull;
  }
}

// FNV-1a over the properties' values, field by field (no padding bytes)
uint64_t props_hash(const mclbm_props& p) {
  uint64_t x = 1469598103934665603ull;
  const double d[14] = {p.rho_f, p.cp_f, p.k_f,  p.beta_f, p.mu_f, p.rho_p, p.cp_p,
                        p.k_p,   p.beta_p, p.T0_K, p.dT_K,   p.g,    p.l_f,  p.Ma};
  fnv1a(x, d, sizeof(d));
  fnv1a(x, &p.force_mask, sizeof(p.force_mask));
  fnv1a(x, &p.storage, sizeof(p.storage));
  fnv1a(x, &p.rounding, sizeof(p.rounding));
  fnv1a(x, &p.thermal_sets, sizeof(p.thermal_sets));
  return x;
}

size_t level_bytes(const mclbm_t* h) { return (size_t)h->L.np * h->L.plane * h->L.elem; }

}  // namespace

int mclbm_save(mclbm_t* h, const char* path) {
  int rc = ready(h, true);
  if (rc) return rc;
  if (!path) return fail(h, MCLBM_EINVAL, "NULL path");
  CheckpointHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "MCLBMCK1", 8);
  hd.version = 1;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.pitch = h->L.pitch;
  hd.storage = h->props.storage;
  hd.rounding = h->props.rounding;
  hd.steps = h->steps;
  hd.Ra = h->Ra;
  hd.Pr = h->Pr;
  hd.phi = h->phi;
  hd.d_p = h->d_p;
  hd.props_hash = props_hash(h->props);
  hd.payload_bytes = level_bytes(h);
  std::vector<char> buf(hd.payload_bytes);
  CK(h, cudaMemcpyAsync(&hd.epoch, h->epoch, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaMemcpyAsync(buf.data(), h->state[h->cur], buf.size(), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, MCLBM_EINVAL, "cannot open %s for writing", path);
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                  std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(h, MCLBM_EINVAL, "writing %s failed", path);
  return MCLBM_OK;
}

int mclbm_load(mclbm_t* h, const char* path) {
  int rc = ready(h, false);
  if (rc) return rc;
  if (!path) return fail(h, MCLBM_EINVAL, "NULL path");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(h, MCLBM_EINVAL, "cannot open %s", path);
  CheckpointHeader hd;
  std::vector<char> buf;
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, "MCLBMCK1", 8) == 0 &&
            hd.version == 1;
  if (ok && (hd.nx != h->nx || hd.ny != h->ny || hd.pitch != h->L.pitch ||
             hd.storage != h->props.storage || hd.payload_bytes != level_bytes(h))) {
    std::fclose(f);
    return fail(h, MCLBM_EINVAL, "%s: lattice or storage differs from the handle's", path);
  }
  if (ok && (hd.Ra != h->Ra || hd.Pr != h->Pr || hd.phi != h->phi || hd.d_p != h->d_p ||
             hd.props_hash != props_hash(h->props))) {
    std::fclose(f);
    return fail(h, MCLBM_EPARAM, "%s: parameters differ from the handle's", path);
  }
  if (ok) {
    buf.resize(hd.payload_bytes);
    ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
  }
  std::fclose(f);
  if (!ok) return fail(h, MCLBM_EINVAL, "%s is not a checkpoint of this library", path);
  h->cur = 0;
  CK(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
  CK(h, cudaMemcpyAsync(h->state[0], buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->epoch, &hd.epoch, sizeof(uint32_t), cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));  // the host buffers go out of scope
  h->steps = hd.steps;
  h->initialised = true;
  h->diverged = false;
  return snapshot(h);
}

int mclbm_run_host(mclbm_t* h, const float* warm_host, int64_t n, uint32_t which,
                   float* fields_host, double* nu_hot, double* nu_cold) {
  int rc = ready(h, false);
  if (rc) return rc;
  if ((which & ~kFieldMask) || (which && !fields_host) || n < 0)
    return fail(h, MCLBM_EINVAL, "bad arguments");
  const size_t nn = (size_t)h->nx * h->ny;
  if (warm_host) {
    CK(h, cudaMemcpyAsync(h->staging, warm_host, 4 * nn * sizeof(float), cudaMemcpyHostToDevice,
                          h->stream));
    rc = mclbm_init(h, MCLBM_INIT_WARM, h->staging);
  } else {
    rc = mclbm_init(h, MCLBM_INIT_REST, nullptr);
  }
  if (rc) return rc;
  rc = mclbm_step(h, n);
  if (rc) return rc;
  if (which) {
    rc = mclbm_fields(h, which, h->staging);
    if (rc) return rc;
    const size_t k = (size_t)__builtin_popcount(which);
    CK(h, cudaMemcpyAsync(fields_host, h->staging, k * nn * sizeof(float),
                          cudaMemcpyDeviceToHost, h->stream));
  }
  if (nu_hot || nu_cold) {
    double a, b;
    rc = mclbm_nusselt(h, &a, &b);
    if (nu_hot) *nu_hot = a;
    if (nu_cold) *nu_cold = b;
    if (rc) return rc;
  } else {
    CK(h, cudaStreamSynchronize(h->stream));
  }
  return MCLBM_OK;
}

int mclbm_get_consts(const mclbm_t* h, mclbm_consts* out) {
  if (!h || !out) return MCLBM_EINVAL;
  *out = h->c;
  return MCLBM_OK;
}

int mclbm_step_kernel(const mclbm_t* h, int* variant, int* nodes_per_thread, int* tile_h,
                      int* grid, int* two) {
  if (!h) return MCLBM_EINVAL;
  if (!h->buf) return MCLBM_ESTATE;
  const bool tma = h->cfg.variant == 2;
  if (variant) *variant = h->cfg.variant;
  if (nodes_per_thread) *nodes_per_thread = h->cfg.vec == 2 ? 2 : 1;
  if (tile_h) *tile_h = tma ? h->cfg.th : 8;
  if (grid) *grid = tma ? h->cfg.grid : 0;
  if (two) *two = h->cfg.two ? 1 : 0;
  return MCLBM_OK;
}

int64_t mclbm_steps_done(const mclbm_t* h) { return h ? h->steps : -1; }

const char* mclbm_last_error(const mclbm_t* h) { return h ? h->err : "NULL handle"; }

const char* mclbm_strerror(int code) {
  switch (code) {
    case MCLBM_OK: return "MCLBM_OK";
    case MCLBM_EINVAL: return "MCLBM_EINVAL";
    case MCLBM_EPARAM: return "MCLBM_EPARAM";
    case MCLBM_ESTATE: return "MCLBM_ESTATE";
    case MCLBM_ECUDA: return "MCLBM_ECUDA";
    case MCLBM_EDIVERGED: return "MCLBM_EDIVERGED";
    case MCLBM_ETOOLARGE: return "MCLBM_ETOOLARGE";
    case MCLBM_ETIMEOUT: return "MCLBM_ETIMEOUT";
    default: return "unknown";
  }
}

}  // extern "C"

// ---- batches -------------------------------------------------------------------------------
struct mclbm_batch {
  std::vector<mclbm_t*> cav;
  std::vector<int> active;
  std::vector<int> nx, ny;
  char* buf = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int device = -1;
  BatchCav* d_cavs = nullptr;
  uint32_t* d_tiles = nullptr;
  double* d_nu = nullptr;
  int* d_err = nullptr;
  uint32_t* d_epoch = nullptr;
  BatchLaunch bl{};
  int per_sm_max = 1, sms = 1, per_sm = 2, order = 0;
  std::vector<uint32_t> table;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t launches = 0;
  char err[512] = {0};
};


namespace mcl {
int batch_size(const mclbm_batch_t* b) { return b ? (int)b->cav.size() : 0; }
}  // namespace mcl

namespace {

int bfail(mclbm_batch_t* b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define BCK(b, expr)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail((b), MCLBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));            \
  } while (0)

struct BatchRegions {
  size_t cavs, tiles, nu, err, total;
};

BatchRegions batch_regions(int n, mclbm_t* const* cavs) {
  BatchRegions r;
  size_t tiles = 0;
  for (int c = 0; c < n; ++c)
    tiles += (size_t)((cavs[c]->nx + 31) / 32) * ((cavs[c]->ny + 7) / 8);
  size_t off = 0;
  r.cavs = off;
  off += align_up((size_t)n * sizeof(BatchCav), 256);
  r.tiles = off;
  off += align_up(tiles * sizeof(uint32_t), 256);
  r.nu = off;
  off += align_up((size_t)n * 2 * sizeof(double), 256);
  r.err = off;
  off += 256;
  r.total = off;
  return r;
}

void batch_drop_graph(mclbm_batch_t* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Uploads the tile table for the current order and active set and sizes the grid.
int batch_retile(mclbm_batch_t* b) {
  build_tile_table(b->nx, b->ny, b->active, b->order, &b->table);
  if (!b->table.empty())
    BCK(b, cudaMemcpyAsync(b->d_tiles, b->table.data(), b->table.size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  b->bl.n_tiles = (int)b->table.size();
  const int slots = b->per_sm * b->sms;
  b->bl.grid = b->bl.n_tiles < slots ? b->bl.n_tiles : slots;
  batch_drop_graph(b);
  return MCLBM_OK;
}

int batch_build_graph(mclbm_batch_t* b) {
  if (!b->cap_stream) BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < kGraphSteps && le == cudaSuccess; ++s)
    le = launch_batch_step(b->bl, s & 1, (uint32_t)s, b->cap_stream);
  if (le == cudaSuccess) le = launch_epoch_advance(b->d_epoch, b->cap_stream);
  cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &g);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, MCLBM_ECUDA, "batch graph capture: %s",
                 cudaGetErrorString(le != cudaSuccess ? le : ee));
  }
  cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, MCLBM_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(ie));
  }
  return MCLBM_OK;
}

}  // namespace

extern "C" {

size_t mclbm_batch_buffer_bytes(int n, mclbm_t* const* cavities) {
  if (n < 1 || n > 1023 || !cavities) return 0;
  for (int c = 0; c < n; ++c)
    if (!cavities[c]) return 0;
  return batch_regions(n, cavities).total;
}

int mclbm_batch_create(int n, mclbm_t* const* cavities, void* dev_buf, size_t bytes,
                       void* cuda_stream, mclbm_batch_t** out) {
  if (!out) return MCLBM_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 1023 || !cavities || !dev_buf) return MCLBM_EINVAL;
  if ((reinterpret_cast<uintptr_t>(dev_buf) & 255u) != 0) return MCLBM_EINVAL;
  for (int c = 0; c < n; ++c) {
    const mclbm_t* h = cavities[c];
    if (!h || !h->buf || !h->initialised) return MCLBM_ESTATE;
    if (h->device != cavities[0]->device || h->L.storage != cavities[0]->L.storage)
      return MCLBM_EINVAL;
    if (h->nx > 65535 || h->ny > 16383) return MCLBM_EINVAL;
    if (h->L.np != kPlanes) return MCLBM_EINVAL;  // one thermal set only
  }
  const BatchRegions r = batch_regions(n, cavities);
  if (bytes < r.total) return MCLBM_EINVAL;
  mclbm_batch_t* b = new (std::nothrow) mclbm_batch();
  if (!b) return MCLBM_EINVAL;
  b->cav.assign(cavities, cavities + n);
  b->active.assign(n, 1);
  for (int c = 0; c < n; ++c) {
    b->nx.push_back(cavities[c]->nx);
    b->ny.push_back(cavities[c]->ny);
  }
  b->buf = static_cast<char*>(dev_buf);
  b->bytes = bytes;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->device = cavities[0]->device;
  int rc = MCLBM_OK;
  auto bail = [&](int code) {
    mclbm_batch_destroy(b);
    return code;
  };
  if (cudaSetDevice(b->device) != cudaSuccess) return bail(MCLBM_ECUDA);
  b->d_cavs = reinterpret_cast<BatchCav*>(b->buf + r.cavs);
  b->d_tiles = reinterpret_cast<uint32_t*>(b->buf + r.tiles);
  b->d_nu = reinterpret_cast<double*>(b->buf + r.nu);
  b->d_err = reinterpret_cast<int*>(b->buf + r.err);
  b->d_epoch = reinterpret_cast<uint32_t*>(b->buf + r.err + 4);
  std::vector<BatchCav> host(n);
  bool all = true;
  for (int c = 0; c < n; ++c) {
    mclbm_t* h = cavities[c];
    std::memset(&host[c], 0, sizeof(BatchCav));
    CUtensorMap maps[2];
    if (make_state_tensor_map(maps, h->state[0], h->L, kBatchTileW, kBatchTileH) != cudaSuccess)
      return bail(MCLBM_ECUDA);
    host[c].map = maps[0];
    host[c].map_out = maps[1];
    host[c].level[0] = h->state[0];
    host[c].level[1] = h->state[1];
    host[c].L = h->L;
    host[c].k = h->k;
    host[c].cur = h->cur;
    all = all && h->k.mask == MCLBM_F_ALL;
  }
  if (cudaMemcpyAsync(b->d_cavs, host.data(), n * sizeof(BatchCav), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_err, 0, 2 * sizeof(int), b->stream) != cudaSuccess)
    return bail(MCLBM_ECUDA);
  if (prepare_batch(cavities[0]->L.storage, &b->per_sm_max) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return bail(MCLBM_ECUDA);
  if (b->per_sm_max < 1) return bail(MCLBM_ECUDA);
  b->per_sm = b->per_sm_max;
  b->bl.cavs = b->d_cavs;
  b->bl.tiles = b->d_tiles;
  b->bl.storage = cavities[0]->L.storage;
  b->bl.sr = cavities[0]->props.rounding == MCLBM_ROUND_STOCHASTIC;
  b->bl.all_forces = all;
  b->bl.epoch = b->d_epoch;
  b->bl.err = b->d_err;
  rc = batch_retile(b);
  if (rc) return bail(rc);
  *out = b;
  return MCLBM_OK;
}

int mclbm_batch_step(mclbm_batch_t* b, int64_t n) {
  mcl::NvtxRange range("mclbm_batch_step");
  if (!b) return MCLBM_EINVAL;
  if (n < 0 || (n & 1)) return bfail(b, MCLBM_EINVAL, "batch step counts must be even");
  BCK(b, cudaSetDevice(b->device));
  int64_t left = n;
  while (left >= kGraphSteps) {
    if (!b->graph) {
      int rc = batch_build_graph(b);
      if (rc) return rc;
    }
    BCK(b, cudaGraphLaunch(b->graph, b->stream));
    left -= kGraphSteps;
  }
  for (; left > 0; --left) {
    BCK(b, launch_batch_step(b->bl, (int)(left & 1), 0x40000000u ^ (uint32_t)b->launches,
                             b->stream));
    ++b->launches;
  }
  for (size_t c = 0; c < b->cav.size(); ++c)
    if (b->active[c]) b->cav[c]->steps += n;
  return MCLBM_OK;
}

int mclbm_batch_nusselt(mclbm_batch_t* b, double* nu_hot, double* nu_cold) {
  if (!b || !nu_hot || !nu_cold) return MCLBM_EINVAL;
  BCK(b, cudaSetDevice(b->device));
  const int n = (int)b->cav.size();
  BCK(b, launch_batch_nusselt(b->bl, n, 0, b->d_nu, b->stream));
  std::vector<double> s(2 * n);
  int err = 0;
  BCK(b, cudaMemcpyAsync(s.data(), b->d_nu, 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                         b->stream));
  BCK(b, cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  if (err) return bfail(b, MCLBM_ETIMEOUT, "a batch step kernel gave up a bounded wait");
  bool finite = true;
  for (int c = 0; c < n; ++c) {
    const mclbm_t* h = b->cav[c];
    const double scale = h->c.k_ratio * (double)h->nx / (double)h->ny;
    nu_hot[c] = s[2 * c] * scale;
    nu_cold[c] = s[2 * c + 1] * scale;
    finite = finite && std::isfinite(nu_hot[c]) && std::isfinite(nu_cold[c]);
  }
  if (!finite) return bfail(b, MCLBM_EDIVERGED, "non-finite Nusselt number in the batch");
  return MCLBM_OK;
}

int mclbm_batch_set_active(mclbm_batch_t* b, const int* active) {
  if (!b || !active) return MCLBM_EINVAL;
  BCK(b, cudaSetDevice(b->device));
  for (size_t c = 0; c < b->cav.size(); ++c) b->active[c] = active[c] ? 1 : 0;
  return batch_retile(b);
}

int mclbm_batch_tune(mclbm_batch_t* b, int64_t steps_per_trial, int* order_out,
                     int* ctas_per_sm_out) {
  if (!b || steps_per_trial < 2 || (steps_per_trial & 1)) return MCLBM_EINVAL;
  BCK(b, cudaSetDevice(b->device));
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_order = b->order, best_per_sm = b->per_sm;
  int rc = MCLBM_OK;
  for (int order = 0; order < 3 && rc == MCLBM_OK; ++order)
    for (int per_sm = 1; per_sm <= b->per_sm_max && rc == MCLBM_OK; ++per_sm) {
      b->order = order;
      b->per_sm = per_sm;
      if ((rc = batch_retile(b))) break;
      if ((rc = mclbm_batch_step(b, steps_per_trial))) break;  // warm-up (builds the graph)
      cudaEventRecord(e0, b->stream);
      if ((rc = mclbm_batch_step(b, steps_per_trial))) break;
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_order = order;
        best_per_sm = per_sm;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->order = best_order;
  b->per_sm = best_per_sm;
  rc = batch_retile(b);
  if (order_out) *order_out = best_order;
  if (ctas_per_sm_out) *ctas_per_sm_out = best_per_sm;
  return rc;
}

const char* mclbm_batch_last_error(const mclbm_batch_t* b) { return b ? b->err : "NULL batch"; }

void mclbm_batch_destroy(mclbm_batch_t* b) {
  if (!b) return;
  if (b->device >= 0) {
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
  }
  batch_drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // extern "C"
