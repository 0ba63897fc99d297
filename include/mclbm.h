/*
 * mclbm.h -- C ABI of libmclbm.so, the GB300 (sm_103a) implementation of one time step of the
 * twin-component lattice Boltzmann model (MCLBM) for buoyancy-driven convection of a
 * nanosuspension in a differentially heated cavity (Savithiri, Dhar, Pattamatta, Das,
 * arXiv:1511.04552). The step streams and collides the base-fluid and particle D2Q9
 * populations f^w, f^p (Eq 18) and the thermal populations g (Eq 19) with the slip forces of
 * Table 1 (Eqs 4, 6, 20) and the cavity walls of Eqs 34-36; reductions give the hot- and
 * cold-wall Nusselt numbers, the component masses and a steady-state residual.
 *
 * Conventions shared by every entry point:
 *  - Return value: MCLBM_OK (0) or a negative MCLBM_E* code. Errors never abort the process;
 *    mclbm_last_error() gives the text of the handle's latest error.
 *  - Units: lattice units (dx = dt = 1) for everything on the lattice, SI for mclbm_props.
 *  - Geometry: nx x ny fluid nodes, node (i, j), i = 0 next to the hot wall (left), j = 0 next
 *    to the bottom wall; walls lie half a link outside the outer nodes. H = ny, L = nx.
 *  - Field and state arrays: row-major [plane][ny][nx], x fastest, FP32, tightly packed.
 *  - Memory ownership: the caller owns all device memory (one buffer handed over by
 *    mclbm_bind, plus every input and output array) and the CUDA stream. A handle owns only
 *    host state, two captured CUDA graphs and one private capture stream; it never allocates
 *    device memory.
 *  - Asynchrony: entry points marked "async" only enqueue work on the bound stream; those
 *    marked "syncs" wait for the bound stream before returning.
 */
#ifndef MCLBM_H
#define MCLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------------- */
#define MCLBM_OK 0
#define MCLBM_EINVAL (-1)    /* bad pointer, size, enum or alignment */
#define MCLBM_EPARAM (-2)    /* physical parameters out of range, or a relaxation time <= 0.501 */
#define MCLBM_ESTATE (-3)    /* call out of order (e.g. step before bind/init) */
#define MCLBM_ECUDA (-4)     /* a CUDA runtime call failed; text in mclbm_last_error */
#define MCLBM_EDIVERGED (-5) /* a reduction saw a non-finite value; sticky until mclbm_init */
#define MCLBM_ETOOLARGE (-6) /* the lattice exceeds the fixed scratch of mclbm_mass_noalloc */
#define MCLBM_ETIMEOUT (-7)  /* a step kernel gave up a bounded device wait (2 s); the state is
                                not valid; reported by the next reduction, cleared by init */

/* ---- slip-mechanism switches (Eq 6 and Table 1; buoyancy of Eq 20) ----------------------- */
#define MCLBM_F_BROWNIAN 1u
#define MCLBM_F_THERMOPHORESIS 2u
#define MCLBM_F_DRAG 4u
#define MCLBM_F_SAFFMAN 8u
#define MCLBM_F_MAGNUS 16u
#define MCLBM_F_GRAVITY 32u
#define MCLBM_F_BUOYANCY 64u
#define MCLBM_F_ALL 127u

/* ---- field selectors (mclbm_fields); outputs follow ascending bit order ------------------ */
#define MCLBM_UX 1u    /* mixture (barycentric) velocity, Eq 32 */
#define MCLBM_UY 2u
#define MCLBM_THETA 4u /* temperature, theta in [-1/2, 1/2], Eq 31 (Eq 33 with two sets) */
#define MCLBM_PHI 8u   /* particle volume fraction rho^p rho_f / rho_p */
#define MCLBM_RHO_W 16u /* base-fluid partial density (normalised by rho_f), Eq 29 */
#define MCLBM_RHO_P 32u /* particle partial density (normalised by rho_f), Eq 29 */
#define MCLBM_UPX 64u  /* particle-component velocity, Eq 30 */
#define MCLBM_UPY 128u
#define MCLBM_THETA_W 256u /* base fluid's thermal set (= MCLBM_THETA with one set), Eq 31 */
#define MCLBM_THETA_P 512u /* particles' thermal set (= MCLBM_THETA with one set), Eq 31 */

/* ---- initial states (mclbm_init) --------------------------------------------------------- */
#define MCLBM_INIT_REST 0 /* rest, uniform phi, theta linear from +1/2 (hot) to -1/2 (cold) */
#define MCLBM_INIT_WARM 2 /* equilibrium of caller fields [4][ny][nx]: ux, uy, theta, phi */
#define MCLBM_INIT_WARM_RHO 3 /* ... [5][ny][nx]: ux, uy, theta, phi, rho^w (MCLBM_RHO_W) */

/* ---- storage of the populations (deviations from the initial conduction state) ----------- */
#define MCLBM_STORE_F32 0  /* 216 bytes per lattice update */
#define MCLBM_STORE_F16 1  /* 2^12 x deviation in FP16, 108 bytes per lattice update */
#define MCLBM_STORE_BF16 2 /* 2^12 x deviation in BF16, 108 bytes per lattice update */
/* rounding of 16-bit stores (arithmetic is FP32 either way) */
#define MCLBM_ROUND_STOCHASTIC 0 /* unbiased random rounding (default) */
#define MCLBM_ROUND_NEAREST 1    /* round to nearest even */

/* Material and model parameters, SI units. mclbm_props_default gives water at 25 C and
 * alumina particles (the paper prints no property values). */
typedef struct mclbm_props {
  double rho_f, cp_f, k_f, beta_f, mu_f; /* base fluid: kg/m^3, J/(kg K), W/(m K), 1/K, Pa s */
  double rho_p, cp_p, k_p, beta_p;       /* particle material */
  double T0_K;                           /* reference temperature (Eq 10b, Table 1 T) */
  double dT_K;                           /* hot minus cold wall temperature */
  double g;                              /* gravity, m/s^2 */
  double l_f;                            /* base-fluid molecular mean free path d_f (Eq 10) */
  double Ma;                             /* lattice buoyancy velocity U0 / c_s, 0 < Ma <= 0.5 */
  uint32_t force_mask;                   /* MCLBM_F_* bits */
  int32_t storage;                       /* MCLBM_STORE_F32, _F16 or _BF16 */
  int32_t rounding;                      /* MCLBM_ROUND_*: 16-bit stores only */
  int32_t thermal_sets;                  /* 1: one thermal set g of the mixture temperature;
                                            2: g^w and g^p (Eq 19 for both components), see
                                            below */
} mclbm_props;

/* Two thermal sets (thermal_sets = 2; the paper's Eq 19 has one thermal population set per
 * component): g^w and g^p stream with the same wall rules and relax, each with its own time
 * (tau_theta^w, and tau_theta^p from Eq 24 at the initial fractions), towards the equilibrium at
 * the mixture temperature of Eq 33, theta^ns = (rho^w theta^w + r rho^p theta^p) /
 * (rho^w + r rho^p), r = C_p,p / C_p,f, as both f^sigma relax at the mixture velocity of Eq 32.
 * theta^ns drives buoyancy, thermophoresis and Nu and is the THETA field; MCLBM_THETA_W and
 * MCLBM_THETA_P select the sets' own temperatures. The state has 36 planes per time level
 * (f^w, f^p, g^w, g^p: 288 bytes per lattice update in FP32); it steps with the plain tile
 * kernel and cannot join a batch. With one set (the default) the state has 27 planes. */

/* Derived create-time constants (FP64), for inspection and tests. Ratios are suspension over
 * base fluid (Eqs 7-11 at the initial phi); tau_* are the BGK relaxation times of Eqs 22-24;
 * rho_w0, rho_p0 the initial partial densities; H_phys, dx, dt the SI cavity height, lattice
 * spacing and time step; C_F converts a force density from N/m^3 to lattice units. */
typedef struct mclbm_consts {
  double U0, nu_w, alpha_w, G_B;
  double rho_ratio, rhocp_ratio, beta_ratio, k_ratio, mu_ratio, Re_T;
  double nu_ns, alpha_ns;
  double rho_w0, rho_p0, Y_w0, Y_p0;
  double tau_w, tau_p, tau_tw, tau_tp;
  double H_phys, dx, dt, C_F, g_lb;
  double mu_ns, rho_ns, k_ns, nu_ns_SI;
  double V_p, A_p, m_p, beta_St, Kn, kstar, K_T;
} mclbm_consts;

typedef struct mclbm mclbm_t; /* opaque handle */

/* Fills *p with the defaults (water / alumina, T0 298.15 K, dT 10 K, g 9.81, l_f 0.17 nm,
 * Ma 0.1, all forces, FP32 storage, stochastic rounding for 16-bit storage). */
void mclbm_props_default(mclbm_props *p);

/* Creates a handle for an nx x ny cavity (2 <= nx, ny <= 32768) at Rayleigh number Ra and
 * Prandtl number Pr of the base fluid, initial particle volume fraction phi in [0, 0.2) and
 * particle diameter d_p (m). props may be NULL (defaults). Host only: derives the constants
 * of Eqs 7-11 and 22-24 and the SI scales, and rejects any relaxation time <= 0.501 with
 * MCLBM_EPARAM. *out receives the handle, or NULL on error. */
int mclbm_create(int nx, int ny, double Ra, double Pr, double phi, double d_p,
                 const mclbm_props *props, mclbm_t **out);

/* Releases the handle's host state, graphs and capture stream; frees no caller memory.
 * Waits for the bound stream first. NULL is ignored. */
void mclbm_destroy(mclbm_t *h);

/* Bytes of device memory the handle needs in mclbm_bind (two time levels of the 27
 * population planes, the residual snapshot, reduction scratch and a staging area). */
size_t mclbm_buffer_bytes(const mclbm_t *h);

/* Hands the handle a caller-owned device buffer (>= mclbm_buffer_bytes, 256-byte aligned)
 * and the CUDA stream (cudaStream_t, may be NULL for the legacy default stream) that every
 * later call enqueues on. The buffer must stay valid until mclbm_destroy or the next bind.
 * Rebinding drops the state: mclbm_init must follow. Selects the current device's context. */
int mclbm_bind(mclbm_t *h, void *dev_buf, size_t bytes, void *cuda_stream);

/* Writes the initial populations (equilibria of Eqs 26-27) as the post-collision state of
 * step 0, resets the step counter, the residual snapshot and the sticky divergence flag.
 * mode MCLBM_INIT_REST ignores warm_dev; MCLBM_INIT_WARM reads warm_dev, a device array
 * [4][ny][nx] FP32 of ux, uy, theta and phi (phi in [0, 1)), and sets rho^w = 1 - phi;
 * MCLBM_INIT_WARM_RHO reads [5][ny][nx] with the base-fluid partial density rho^w (the field
 * MCLBM_RHO_W, normalised by rho_f) as the fifth plane, so that a steady state's pressure field
 * is part of the warm start (without it the buoyancy is out of balance and the start relaxes
 * through pressure waves). Async. */
int mclbm_init(mclbm_t *h, int mode, const float *warm_dev);

/* Advances n >= 0 time steps (Eqs 18-19 with the forces of Table 1 and the walls of
 * Eqs 34-36): the even part in captured CUDA graphs of 2^k steps (2 <= 2^k <= 1024, largest
 * first, built on first use and kept with the handle), an odd last step as a single launch; the
 * stochastic-rounding streams of 16-bit storage follow the graphs' replay count, so a given
 * sequence of calls is reproducible bit for bit. Async. A step kernel
 * that gives up a bounded wait on its own data movement sets an error word instead of
 * hanging; the next mclbm_nusselt, mclbm_mass or mclbm_residual returns MCLBM_ETIMEOUT. */
int mclbm_step(mclbm_t *h, int64_t n);

/* Advances one time step of streaming only (no collision, no forces): a test hook for the
 * wall rules. Async. */
int mclbm_stream_only(mclbm_t *h);

/* Writes the selected moments of the post-stream populations (the macroscopic fields the
 * next step starts from) to dev_out, a device array [popcount(which)][ny][nx] FP32, planes
 * in ascending bit order of which (MCLBM_UX ... MCLBM_THETA_P). Async. */
int mclbm_fields(mclbm_t *h, uint32_t which, float *dev_out);

/* Mean Nusselt numbers of the hot (left) and cold (right) walls: k_ns/k_f times the mean
 * over the wall of the second-order one-sided gradient of theta at the half-way wall,
 * normalised by L = nx and dT. FP64 sums. Syncs. MCLBM_EDIVERGED if non-finite. */
int mclbm_nusselt(mclbm_t *h, double *nu_hot, double *nu_cold);

/* FP64 sums of the base-fluid and particle partial densities over the cavity (Eq 29). These
 * are invariants of the exact method. Syncs. MCLBM_EDIVERGED if non-finite. */
int mclbm_mass(mclbm_t *h, double *mass_w, double *mass_p);

/* Steady-state residual since the previous call (or mclbm_init): K = steps in between,
 * r = max over q in {u, theta, phi} of ||q_now - q_then||_2 / (K ||q_now||_2) (0 when K = 0),
 * FP64 sums. Replaces the snapshot. Syncs. MCLBM_EDIVERGED if non-finite. */
int mclbm_residual(mclbm_t *h, double *r);

/* The three reductions above in one call with one host synchronisation (Sec. 2.d's Nu at the
 * walls, Eq 29's masses, the residual): the same FP64 sums and results as mclbm_nusselt,
 * mclbm_mass and mclbm_residual called in that order (the residual's snapshot is replaced).
 * Syncs once. MCLBM_EINVAL for a NULL output; MCLBM_EDIVERGED if any result is non-finite (every
 * output is still written); MCLBM_ETIMEOUT as the single calls. */
int mclbm_diagnostics(mclbm_t *h, double *nu_hot, double *nu_cold, double *mass_w,
                      double *mass_p, double *r);

/* Copies the population planes [np][ny][nx] FP32 (np = 27: f^w_0..8, f^p_0..8, g_0..8; with
 * two thermal sets np = 36: f^w, f^p, g^w, g^p; directions in the order of Eq 21: rest, +x, +y,
 * -x, -y, (+1,+1), (-1,+1), (-1,-1), (+1,-1)) between the handle's current state and a caller
 * device array. The planes hold deviations from the initial conduction state:
 * f^sigma_q - W_q rho_sigma0 (rho_w0, rho_p0 in mclbm_consts) and g_q - W_q theta_c(i) with
 * theta_c(i) = 1/2 - (i + 1/2)/nx.
 * state_set also makes the state the post-collision state of step 0. Async. */
int mclbm_state_get(mclbm_t *h, float *dev_out);
int mclbm_state_set(mclbm_t *h, const float *dev_in);

/* End-to-end run on host buffers: copies warm_host ([4][ny][nx] FP32 host array, or NULL
 * for the rest state) to the device, initialises, advances n steps, copies the selected
 * fields into fields_host ([popcount(which)][ny][nx], may be NULL when which == 0) and
 * returns both Nusselt numbers (may be NULL). Syncs. */
int mclbm_run_host(mclbm_t *h, const float *warm_host, int64_t n, uint32_t which,
                   float *fields_host, double *nu_hot, double *nu_cold);

/* Component masses for callers that cannot allocate device memory: a host application that
 * hands out all device memory from its own fixed pool and forbids other allocations, or a
 * loop that must not pay for an allocation on every call. Not a method of the paper (it has
 * no counterpart there): the same FP64 sums as mclbm_mass, needing no handle and no buffer.
 *   state_dev: caller-owned device array [27][ny][nx] FP32 in the layout of mclbm_state_get
 *              (deviations from the rest state; only the 18 f planes are read).
 *   rho_w0, rho_p0: the rest-state partial densities (mclbm_consts) added back per node.
 *   mass_w, mass_p: host outputs. cuda_stream: the stream to run on (NULL: legacy default).
 * Its scratch is a static device array of 2 x 8192 + 2 doubles (128 KiB) that every GPU which
 * loads the library holds until the process exits: ny > 8192 or nx > 32768 returns
 * MCLBM_ETOOLARGE. The first call on a device looks the array's device address up (with that
 * device current), so make that first call before any stream capture. Calls that overlap on
 * the GPU share the array and race: serialise them (one stream, or wait in between). Every
 * scratch element a call reads is written earlier by the same call, so a previous call's
 * contents never leak into a result. Calls no cudaMalloc or cudaFree. Host-synchronous: it
 * copies the two totals to host memory and waits for the stream before it returns.
 * It reads a raw state and never sees a handle's error word: after a step kernel gave up a
 * bounded wait (MCLBM_ETIMEOUT from mclbm_mass, mclbm_nusselt or mclbm_residual) the state is
 * partly written, so check the handle's status with one of those before trusting this result.
 * Returns MCLBM_OK, MCLBM_EINVAL, MCLBM_ETOOLARGE, MCLBM_ECUDA or MCLBM_EDIVERGED. */
int mclbm_mass_noalloc(const float *state_dev, int nx, int ny, double rho_w0, double rho_p0,
                       double *mass_w, double *mass_p, void *cuda_stream);

/* ---- batches: many cavities per launch (the parametric sweep) ---------------------------- */
typedef struct mclbm_batch mclbm_batch_t; /* opaque; steps cavities it does not own */

/* Bytes of device memory a batch of the n cavities needs (cavity table, tile table, reduction
 * scratch); 0 for bad arguments (n outside 1..1023, NULL cavity). */
size_t mclbm_batch_buffer_bytes(int n, mclbm_t *const *cavities);

/* Groups n bound and initialised cavities (same device, same storage type; nx <= 65535,
 * ny <= 16383) so that mclbm_batch_step advances all of them with one persistent launch per
 * time step: the 64 x 8 tiles of every active cavity form one table walked by a persistent grid
 * (CTAs per SM chosen by mclbm_batch_tune), each tile streamed into shared memory by TMA and
 * updated two nodes per thread as in the single-cavity step on large lattices
 * (Eqs 18-19 with Table 1 and Eqs 34-36, per cavity with its own parameters). dev_buf: caller
 * device memory (>= mclbm_batch_buffer_bytes, 256-byte aligned), cuda_stream: the stream of
 * every batch call. The cavities stay usable on their own (fields, reductions) between batch
 * calls; do not step them on their own while they are in a batch. */
int mclbm_batch_create(int n, mclbm_t *const *cavities, void *dev_buf, size_t bytes,
                       void *cuda_stream, mclbm_batch_t **out);

/* Advances every active cavity n time steps (n even: each cavity's state returns to the
 * level it started from), in captured graphs of 64 launches. Async. MCLBM_EINVAL for odd n. */
int mclbm_batch_step(mclbm_batch_t *b, int64_t n);

/* Hot- and cold-wall Nusselt numbers of every cavity of the batch (host arrays [n]), as
 * mclbm_nusselt computes them, from one launch. Syncs. */
int mclbm_batch_nusselt(mclbm_batch_t *b, double *nu_hot, double *nu_cold);

/* Selects which cavities mclbm_batch_step advances (active[c] != 0), e.g. to drop cavities that
 * have reached a steady state; rebuilds the tile table. Syncs. */
int mclbm_batch_set_active(mclbm_batch_t *b, const int *active);

/* Autotuner: times steps_per_trial (even) steps for each tile order (0: cavity by cavity,
 * 1: largest first, 2: interleaved) and each CTA count per SM from 1 to the most that fit (at
 * most 4), keeps the fastest and reports it. The trial steps are real steps: every active
 * cavity advances 2 x 3 x (CTA counts tried) x steps_per_trial. */
int mclbm_batch_tune(mclbm_batch_t *b, int64_t steps_per_trial, int *order, int *ctas_per_sm);

/* Text of the batch's latest error. */
const char *mclbm_batch_last_error(const mclbm_batch_t *b);

/* Releases the batch (not the cavities, not the caller's buffer). Waits for its stream. */
void mclbm_batch_destroy(mclbm_batch_t *b);

/* ---- steady state ------------------------------------------------------------------------
 * The paper reports steady states (Sec. 3: the hot-wall Nu of Figs 3, 5-7) without saying when
 * a run is steady. The test here reads "the distance to the steady hot-wall Nu is at most
 * tol |Nu|" on the hot-wall Nusselt numbers of successive, equally spaced checks. For every lag
 * L of lags (in checks) the six values Nu_n, Nu_(n-L), ..., Nu_(n-5L), with the five changes
 * d_0 (latest) ... d_4, must show one of: (a) |d_0| and |d_1| at most 2e-7 L |Nu_n| (round-off
 * at the FP32 fixed point); (b) two or more sign flips among the changes with all six values
 * within tol |Nu_n| / 2 (an oscillation about the limit); (c) the four ratios d_k / d_(k+1) in
 * [0, 0.99) and within 0.05 of each other, and |d_0| r / (1 - r) <= tol |Nu_n| with r the
 * largest ratio (the rest of a geometric tail). Several lags keep a settled fast mode from
 * hiding a slow one that still moves Nu (the particle component's migration). */

/* The test on a history nu_hist[0..n) (oldest first). lags = NULL: {1, 32}; otherwise n_lags
 * (1..8) lags of at least 1. Returns 1 (steady), 0 (not yet, also with fewer than
 * 5 max(lags) + 1 values) or MCLBM_EINVAL (NULL nu_hist with n > 0, tol <= 0, bad lags).
 * Host only: needs no GPU. */
int mclbm_steady_nu_reached(const double *nu_hist, int64_t n, double tol, const int32_t *lags,
                            int n_lags);

/* Steps a bound, initialised cavity check_every (>= 1) steps at a time, taking mclbm_nusselt
 * after each chunk, until the test holds for the hot-wall history of this call or max_steps
 * have been done. Outputs (each may be NULL): steps done by this call, the last Nusselt numbers,
 * converged (1 when the test held). Returns MCLBM_OK, MCLBM_EINVAL for bad arguments, or the
 * first failing mclbm_step / mclbm_nusselt code. Syncs at every check. */
int mclbm_run_to_steady(mclbm_t *h, double tol, int64_t check_every, int64_t max_steps,
                        const int32_t *lags, int n_lags, int64_t *steps, double *nu_hot,
                        double *nu_cold, int *converged);

/* The same for every cavity of a batch (check_every even): a cavity whose history passes the
 * test leaves the tile table (mclbm_batch_set_active) and keeps its state. Host arrays [n] (may
 * be NULL): steps[c] = the batch step count at which cavity c became steady, -1 if it did not
 * within max_steps; nu_hot[c] = its hot-wall Nu at that check (else the last one).
 * *total_steps (may be NULL) = steps the batch ran. Returns as mclbm_run_to_steady, with the
 * batch calls' codes. */
int mclbm_batch_run_to_steady(mclbm_batch_t *b, double tol, int64_t check_every,
                              int64_t max_steps, const int32_t *lags, int n_lags, int64_t *steps,
                              double *nu_hot, int64_t *total_steps);

/* Derived constants of the handle. */
int mclbm_get_consts(const mclbm_t *h, mclbm_consts *out);

/* Checkpoint and resume. mclbm_save writes the current time level exactly as stored (any
 * storage type), the step count and the stochastic-rounding epoch to a file, with the lattice
 * size and a fingerprint of the parameters; mclbm_load restores them into a bound handle
 * created with the same size, storage and parameters (EINVAL for a different lattice or
 * storage or a file that is not a checkpoint, EPARAM for different parameters), so that the
 * continued run is bitwise the uninterrupted one. Both sync. */
int mclbm_save(mclbm_t *h, const char *path);
int mclbm_load(mclbm_t *h, const char *path);

/* Self-test of failure detection, no handle needed: launches one kernel that waits with the
 * step kernels' bounded mbarrier wait on a barrier nothing arrives on; the wait gives up after
 * about 2 s and the kernel returns normally. Returns MCLBM_ETIMEOUT when that happened as
 * designed (the code every stuck step reports), MCLBM_ECUDA otherwise; *seconds (may be NULL)
 * receives the host-measured duration. Syncs the given stream (NULL: legacy default stream). */
int mclbm_selftest_wait_timeout(void *cuda_stream, double *seconds);

/* Time steps done since the last mclbm_init or mclbm_state_set (-1 for a NULL handle). */
int64_t mclbm_steps_done(const mclbm_t *h);

/* Which step kernel the handle launches, as chosen by mclbm_bind from the lattice size, the
 * storage type, the device and the MCLBM_STEP_* environment overrides (no call in the paper: a
 * diagnostic of this implementation). variant: 0 = the plain tile kernel (32 x 8 tiles, one CTA
 * each), 2 = the TMA-staged persistent kernel; nodes_per_thread: 1 or 2; tile_h: the TMA
 * kernel's tile height (8, or 7 where 32 x 8 tiles would give some SMs a second tile and 32 x 7
 * tiles fit two per SM, e.g. 256 x 256 on 152 SMs; 8 for the tile kernel);
 * grid: the TMA kernel's persistent CTAs (0 for the tile kernel); two: 1 when pairs of steps run
 * in the two-step kernel. Outputs may be NULL. Host only, no GPU work. MCLBM_EINVAL for a NULL
 * handle, MCLBM_ESTATE before mclbm_bind. */
int mclbm_step_kernel(const mclbm_t *h, int *variant, int *nodes_per_thread, int *tile_h,
                      int *grid, int *two);

/* Text of the handle's latest error ("" if none); static text for a NULL handle. */
const char *mclbm_last_error(const mclbm_t *h);

/* Short name of a return code. */
const char *mclbm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MCLBM_H */
