/*
 * mclbm_ref.h -- FP64 CPU oracle of the twin-component lattice Boltzmann model (MCLBM) of
 * buoyancy-driven convection of a nanosuspension in a differentially heated cavity
 * (Savithiri, Dhar, Pattamatta, Das, arXiv:1511.04552, Sec. 2.d, Eqs 18-36, Table 1).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load this library. The CUDA library shares no code, header or constant with it.
 *
 * All arrays are row-major [plane][ny][nx], x fastest, j = 0 at the bottom wall, i = 0 at the
 * hot wall. Population planes are ordered f^w_0..8, f^p_0..8, g_0..8 (one thermal set) or
 * f^w_0..8, f^p_0..8, g^w_0..8, g^p_0..8 (two thermal sets) and hold ABSOLUTE values.
 * Every function returns 0 on success or a negative REF_E* code.
 */
#ifndef MCLBM_REF_H
#define MCLBM_REF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REF_OK 0
#define REF_EINVAL (-1)
#define REF_EPARAM (-2)
#define REF_ESTATE (-3)
#define REF_ENOMEM (-4)

/* slip-mechanism switches (Eq 6, Table 1; Eq 20 buoyancy) */
#define REF_F_BROWNIAN 1u
#define REF_F_THERMOPHORESIS 2u
#define REF_F_DRAG 4u
#define REF_F_SAFFMAN 8u
#define REF_F_MAGNUS 16u
#define REF_F_GRAVITY 32u
#define REF_F_BUOYANCY 64u
#define REF_F_ALL 127u

/* field selectors for mclbm_ref_fields; outputs are written in ascending bit order */
#define REF_UX 1u
#define REF_UY 2u
#define REF_THETA 4u
#define REF_PHI 8u
#define REF_RHO_W 16u
#define REF_RHO_P 32u
#define REF_UPX 64u
#define REF_UPY 128u
#define REF_THETA_W 256u /* theta of the base fluid's thermal set (= theta with one set) */
#define REF_THETA_P 512u /* theta of the particles' thermal set (= theta with one set) */

#define REF_INIT_REST 0
#define REF_INIT_WARM 2     /* warm [4][ny][nx]: ux, uy, theta, phi; rho^w = 1 - phi */
#define REF_INIT_WARM_RHO 3 /* warm [5][ny][nx]: ux, uy, theta, phi, rho^w */

typedef struct {
  double rho_f, cp_f, k_f, beta_f, mu_f; /* base fluid, SI */
  double rho_p, cp_p, k_p, beta_p;       /* particle material, SI */
  double T0, dT, g, l_f;                 /* K, K, m/s^2, m */
  double Ma;                             /* lattice buoyancy velocity / c_s */
  uint32_t force_mask;                   /* REF_F_* */
  int periodic_x;                        /* test-only: periodic in x, no side walls */
  double body_fx;                        /* test-only: uniform x force density on f^w (lattice) */
  int thermal_sets;                      /* 1: one set g of the mixture temperature; 2: g^w, g^p */
  double tau_tp_override;                /* test-only: > 0 replaces the particles' thermal tau */
} ref_props;

/* Derived constants (create time, FP64). Ratios are suspension / base fluid. */
typedef struct {
  double U0, nu_w, alpha_w, G_B;
  double rho_ratio, rhocp_ratio, beta_ratio, k_ratio, mu_ratio, Re_T;
  double nu_ns, alpha_ns;
  double rho_w0, rho_p0, Y_w0, Y_p0;
  double tau_w, tau_p, tau_tw, tau_tp;
  double H_phys, dx, dt, C_F, g_lb;
  double mu_ns, rho_ns, k_ns, nu_ns_SI;
  double V_p, A_p, m_p, beta_St, Kn, kstar, K_T;
} ref_consts;

/* Per-node terms of one step (diagnostics for the tests), all in lattice units. */
typedef struct {
  double rho_w, rho_p, theta, phi;
  double u[2], uw[2], up[2];
  double grad_theta[2], grad_phi[2];
  double F_B[2], F_T[2], F_S[2], F_M[2], F_G[2], F_buoy[2], F_G0[2];
  double beta_lb, a, J[2];
  double F_w[2], F_p[2];
  double tau_theta;
} ref_terms;

typedef struct ref_solver ref_t;

void mclbm_ref_props_default(ref_props *p);
int mclbm_ref_create(int nx, int ny, double Ra, double Pr, double phi, double d_p,
                     const ref_props *props, ref_t **out);
void mclbm_ref_destroy(ref_t *h);
int mclbm_ref_consts(const ref_t *h, ref_consts *out);
/* mode REST: rest, uniform phi, linear theta. WARM: warm = [4][ny][nx] (ux, uy, theta, phi). */
int mclbm_ref_init(ref_t *h, int mode, const double *warm);
int mclbm_ref_step(ref_t *h, int64_t n);
/* streaming with wall rules only (no collision); the result becomes the stored state */
int mclbm_ref_stream_only(ref_t *h);
int mclbm_ref_fields(ref_t *h, uint32_t which, double *out);
int mclbm_ref_nusselt(ref_t *h, double *nu_hot, double *nu_cold);
int mclbm_ref_mass(const ref_t *h, double *mass_w, double *mass_p);
int mclbm_ref_residual(ref_t *h, double *r);
int mclbm_ref_get_state(const ref_t *h, double *out);
int mclbm_ref_set_state(ref_t *h, const double *in);
int mclbm_ref_node_terms(ref_t *h, int i, int j, ref_terms *out);
int64_t mclbm_ref_steps_done(const ref_t *h);
void mclbm_ref_equilibrium(double rho, double ux, double uy, double out[9]);
/* exact one-step drag impulse on the particle component (reading of Table 1's drag) */
void mclbm_ref_drag_impulse(double rho_w, double rho_p, const double w_relaxed[2],
                            const double b[2], double a, double J[2]);
void mclbm_ref_set_threads(int n);
int mclbm_ref_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
