/*
 * mclbm_ref.c -- plain, slow FP64 CPU oracle of one time step of the twin-component lattice
 * Boltzmann model (MCLBM) for buoyancy-driven convection of a nanosuspension in a
 * differentially heated cavity (arXiv:1511.04552, Sec. 2.a, 2.b and 2.d).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code with the CUDA library.
 *
 * A step runs the method in the paper's order, one whole-array pass at a time:
 *   1. pull streaming with the wall rules (LHS of Eqs 18-19; Eqs 34-36),
 *   2. moments (Eqs 25, 29-32),
 *   3. same-time-level central gradients of theta and phi,
 *   4. slip forces of Table 1 evaluated in SI units and converted to lattice units (Eqs 4, 6, 20),
 *   5. the drag impulse integrated exactly over the step,
 *   6. BGK collision with forcing (RHS of Eqs 18-19 with Eqs 26-28, 24),
 *   7. store into the other time level.
 *
 * Readings (the paper is silent, ambiguous or garbled at these points):
 *   - one thermal population set g carrying the mixture temperature; its relaxation time is
 *     the mass-fraction average of Eq 24, so Eq 33 is the identity;
 *   - walls half a link outside the outer nodes; f^w and f^p bounce back link-wise (Eq 34,
 *     also the particle wall condition read as zero particle flux); g anti-bounces back at the
 *     isothermal walls (Eq 35) and reflects specularly at the adiabatic walls (Eq 36 is garbled;
 *     specular reflection carries no flux through the wall); a diagonal link that leaves
 *     through a corner takes the isothermal rule;
 *   - lattice scales: U0 = Ma c_s, nu_w = U0 H sqrt(Pr/Ra), alpha_w = nu_w/Pr, G_B = U0^2/H with
 *     Ra and Pr of the base fluid; theta in [-1/2, 1/2];
 *   - f^w and f^p carry partial densities normalised by rho_f; Eq 32 is the barycentric velocity;
 *   - tau_w from Eq 22; tau_p and the particle thermal tau from Eqs 23-24 at the initial mass
 *     fractions with Eqs 7-11 evaluated at the initial phi;
 *   - Eq 10 with d_f = the base-fluid mean free path l_f and T = T0;
 *   - Table 1 forces are per particle; the per-volume force is n_p = phi/V_p times it. Brownian
 *     force points down the phi gradient (factor 2 in D_B as printed). Thermophoresis is the
 *     force whose Stokes terminal drift is v_T (sign hot to cold). Saffman lift with the
 *     square root of rho_ns gamma / mu_ns that a force needs, perpendicular to the slip. Magnus: v_M is a
 *     migration speed along the inward normal of the nearest wall, the speed inside it is
 *     |u^w + u^p|/2, m_dot_p = m_p beta_St. Gravity acts on the particles with its uniform
 *     initial part returned to the fluid (Boussinesq reference). Particle rotation is not a force
 *     and is left out. Every particle-fluid force has its reaction on the fluid (Eq 20 extended);
 *   - drag coefficient beta = 18 mu_ns (1 + 0.15 Re_d^0.687) / (rho_p d_p^2); the drag impulse is
 *     integrated exactly over one step with the other forces frozen;
 *   - Eq 18's forcing term carries the 1/c_s^2 it lost: 3 W_i e_i.F;
 *   - gradients: central differences with ghosts phi_ghost = phi, theta_ghost = 2 T_wall - theta
 *     at the isothermal walls and theta_ghost = theta at the adiabatic walls;
 *   - Nu: mean over the hot wall of the second-order one-sided wall gradient, times k_ns/k_f,
 *     normalised by the hot-cold distance L = nx.
 *   - the two-thermal-set variant (thermal_sets = 2, Eq 19 for both components): g^w and g^p
 *     stream with the same wall rules, each relaxes with its own time (tau_theta^w of Eq 22's
 *     thermal twin, tau_theta^p of Eq 24 at the initial fractions) towards the equilibrium at
 *     the mixture temperature of Eq 33, theta^ns = (rho^w theta^w + r rho^p theta^p) /
 *     (rho^w + r rho^p), r = C_p,p / C_p,f (the garbled weights of Eq 33 read as the
 *     components' heat capacities), just as both f^sigma relax at the mixture velocity of
 *     Eq 32; theta^ns drives buoyancy, the gradients and Nu.
 *
 * Parity pins (tests/test_oracle_*.py): equilibrium moments, streaming permutation and
 * displacement, exact mass conservation, the phi = 0 limit against an independent textbook
 * thermal LBM and against the de Vahl Davis cavity benchmark, the conduction limit, the drag
 * impulse against the two-body ODE, the interaction-force balance, centro-symmetry, the
 * SI-to-lattice constants against an independent derivation, Poiseuille curvature, the
 * thermophoretic terminal drift, the Brownian drift flux, the Saffman lift against Saffman's
 * sphere lift per radius and its scaling exponents, the Magnus migration in SI and its
 * exponents, the gravity (weight less buoyancy) and Boussinesq (Eq 9) force densities in SI
 * through one step's momentum change, the local thermal relaxation time (Eq 24) and the
 * residual recomputed from field snapshots.
 */
#include "mclbm_ref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9
#define T_HOT 0.5
#define T_COLD (-0.5)

/* D2Q9 velocity set (Eq 21): rest, 4 axial at 90 degree steps, 4 diagonal. */
static const int EX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* lattice weights (Eq 28) */
static const double W[NQ] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static const double KB = 1.380649e-23; /* Boltzmann constant, J/K */
static const double PI = 3.14159265358979323846;

/* index of the direction -e_q */
static int opposite(int q) {
  for (int k = 0; k < NQ; ++k)
    if (EX[k] == -EX[q] && EY[k] == -EY[q]) return k;
  return -1;
}
/* index of the direction (e_qx, -e_qy): the mirror image in a horizontal wall */
static int mirror_y(int q) {
  for (int k = 0; k < NQ; ++k)
    if (EX[k] == EX[q] && EY[k] == -EY[q]) return k;
  return -1;
}

/* M_THETA: the (mixture) temperature; M_THW, M_THP: the two sets' own (= M_THETA with one) */
enum { M_RHOW, M_RHOP, M_MWX, M_MWY, M_MPX, M_MPY, M_THETA, M_THW, M_THP, NMOM };

struct ref_solver {
  int nx, ny;
  double Ra, Pr, phi0, d_p;
  ref_props pr;
  ref_consts c;
  int nsets;     /* population sets: 3 (f^w, f^p, g) or 4 (f^w, f^p, g^w, g^p) */
  int np;        /* planes: 9 nsets */
  double *st[2]; /* [np][ny][nx] post-collision populations, two time levels */
  int cur;
  double *post; /* [np][ny][nx] post-stream populations of the step in progress */
  double *mom;  /* [NMOM][ny][nx] moments of the post-stream populations */
  double *snap; /* [4][ny][nx] ux, uy, theta, phi at the last residual check */
  int64_t steps, snap_step;
  int ready;
};

#define AT(arr, plane, i, j) ((arr)[((size_t)(plane) * h->ny + (j)) * h->nx + (i)])

void mclbm_ref_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int mclbm_ref_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Water at 25 C as base fluid and alumina as particle material; the paper prints no values. */
void mclbm_ref_props_default(ref_props *p) {
  memset(p, 0, sizeof(*p));
  p->rho_f = 997.1;
  p->cp_f = 4179.0;
  p->k_f = 0.613;
  p->beta_f = 2.1e-4;
  p->mu_f = 8.9e-4;
  p->rho_p = 3970.0;
  p->cp_p = 765.0;
  p->k_p = 40.0;
  p->beta_p = 0.85e-5;
  p->T0 = 298.15;
  p->dT = 10.0;
  p->g = 9.81;
  p->l_f = 0.17e-9;
  p->Ma = 0.1;
  p->force_mask = REF_F_ALL;
  p->periodic_x = 0;
  p->body_fx = 0.0;
  p->thermal_sets = 1;
  p->tau_tp_override = 0.0;
}

/* Create-time constants: lattice scales, Eqs 7-11 at the initial phi, Eqs 22-24, SI scales. */
static int derive(ref_t *h) {
  const ref_props *p = &h->pr;
  ref_consts *c = &h->c;
  const double phi0 = h->phi0, d = h->d_p;
  const double H = (double)h->ny;
  memset(c, 0, sizeof(*c));
  c->U0 = p->Ma / sqrt(3.0);
  c->nu_w = c->U0 * H * sqrt(h->Pr / h->Ra);
  c->alpha_w = c->nu_w / h->Pr;
  c->G_B = c->U0 * c->U0 / H;
  /* Eqs 7-9: volume-weighted mixing */
  c->rho_ratio = phi0 * p->rho_p / p->rho_f + (1.0 - phi0);
  c->rhocp_ratio = phi0 * (p->rho_p * p->cp_p) / (p->rho_f * p->cp_f) + (1.0 - phi0);
  c->beta_ratio = phi0 * p->beta_p / p->beta_f + (1.0 - phi0);
  /* Eq 10b with d_f = l_f, T = T0; Eq 10a with the exponents as printed */
  c->Re_T = p->rho_f * KB * p->T0 / (3.0 * PI * p->mu_f * p->mu_f * p->l_f);
  c->k_ratio = 1.0 + 64.7 * pow(phi0, 0.764) * pow(p->l_f / d, 0.369) *
                         pow(p->k_f / p->k_p, 0.7476) * pow(h->Pr, 0.995) * pow(c->Re_T, 1.2321);
  /* Eq 11 */
  c->mu_ratio = 1.0 + 4.93 * phi0 + 222.4 * phi0 * phi0;
  c->nu_ns = c->nu_w * c->mu_ratio / c->rho_ratio;
  c->alpha_ns = c->alpha_w * c->k_ratio / c->rhocp_ratio;
  /* partial densities normalised by rho_f; Eq 25 at t = 0 */
  c->rho_w0 = 1.0 - phi0;
  c->rho_p0 = phi0 * p->rho_p / p->rho_f;
  c->Y_w0 = c->rho_w0 / (c->rho_w0 + c->rho_p0);
  c->Y_p0 = c->rho_p0 / (c->rho_w0 + c->rho_p0);
  /* Eq 22 (base fluid), Eq 23 solved for the particle tau, Eq 24 likewise */
  c->tau_w = 3.0 * c->nu_w + 0.5;
  c->tau_tw = 3.0 * c->alpha_w + 0.5;
  if (phi0 > 0.0) {
    c->tau_p = (3.0 * c->nu_ns + 0.5 - c->Y_w0 * c->tau_w) / c->Y_p0;
    c->tau_tp = (3.0 * c->alpha_ns + 0.5 - c->Y_w0 * c->tau_tw) / c->Y_p0;
  } else {
    c->tau_p = c->tau_w;
    c->tau_tp = c->tau_tw;
  }
  if (p->tau_tp_override > 0.0) c->tau_tp = p->tau_tp_override;
  /* SI scales: physical height from Ra of the base fluid, then lattice spacing and time step */
  {
    const double nu_f = p->mu_f / p->rho_f, alpha_f = nu_f / h->Pr;
    c->H_phys = cbrt(h->Ra * nu_f * alpha_f / (p->g * p->beta_f * p->dT));
    c->dx = c->H_phys / H;
    c->dt = c->nu_w * c->dx * c->dx / nu_f;
    c->C_F = c->dt * c->dt / (p->rho_f * c->dx);
    c->g_lb = p->g * c->dt * c->dt / c->dx;
  }
  /* suspension and particle properties used by Table 1 */
  c->mu_ns = p->mu_f * c->mu_ratio;
  c->rho_ns = p->rho_f * c->rho_ratio;
  c->k_ns = p->k_f * c->k_ratio;
  c->nu_ns_SI = c->mu_ns / c->rho_ns;
  c->V_p = PI * d * d * d / 6.0;
  c->A_p = PI * d * d;
  c->m_p = p->rho_p * c->V_p;
  c->beta_St = 18.0 * c->mu_ns / (p->rho_p * d * d);
  c->Kn = p->l_f / d;
  c->kstar = c->k_ns / p->k_p;
  {
    const double Cs = 1.17, Ct = 2.18, Cm = 1.14;
    c->K_T = 6.0 * PI * Cs * (c->kstar + Ct * c->Kn) /
             ((1.0 + 3.0 * Cm * c->Kn) * (1.0 + 2.0 * c->kstar + 2.0 * Ct * c->Kn));
  }
  {
    const double lim = 0.5 + 1e-3;
    if (!(c->tau_w > lim) || !(c->tau_p > lim) || !(c->tau_tw > lim) || !(c->tau_tp > lim))
      return REF_EPARAM;
  }
  return REF_OK;
}

int mclbm_ref_create(int nx, int ny, double Ra, double Pr, double phi, double d_p,
                     const ref_props *props, ref_t **out) {
  if (!out) return REF_EINVAL;
  *out = NULL;
  if (nx < 2 || ny < 2 || nx > 65536 || ny > 65536) return REF_EINVAL;
  if (!(Ra > 0) || !(Pr > 0) || !(phi >= 0 && phi < 0.2) || !(d_p > 0) || !isfinite(Ra))
    return REF_EPARAM;
  ref_props p;
  if (props)
    p = *props;
  else
    mclbm_ref_props_default(&p);
  if (!(p.rho_f > 0) || !(p.cp_f > 0) || !(p.k_f > 0) || !(p.beta_f > 0) || !(p.mu_f > 0) ||
      !(p.rho_p > 0) || !(p.cp_p > 0) || !(p.k_p > 0) || !(p.beta_p >= 0) || !(p.T0 > 0) ||
      !(p.dT > 0) || !(p.g > 0) || !(p.l_f > 0) || !(p.Ma > 0 && p.Ma <= 0.5) ||
      (p.force_mask & ~REF_F_ALL) || (p.thermal_sets != 1 && p.thermal_sets != 2))
    return REF_EPARAM;
  ref_t *h = (ref_t *)calloc(1, sizeof(ref_t));
  if (!h) return REF_ENOMEM;
  h->nx = nx;
  h->ny = ny;
  h->Ra = Ra;
  h->Pr = Pr;
  h->phi0 = phi;
  h->d_p = d_p;
  h->pr = p;
  h->nsets = 2 + p.thermal_sets;
  h->np = NQ * h->nsets;
  int rc = derive(h);
  if (rc) {
    free(h);
    return rc;
  }
  const size_t n = (size_t)nx * ny;
  h->st[0] = (double *)calloc((size_t)h->np * n, sizeof(double));
  h->st[1] = (double *)calloc((size_t)h->np * n, sizeof(double));
  h->post = (double *)calloc((size_t)h->np * n, sizeof(double));
  h->mom = (double *)calloc(NMOM * n, sizeof(double));
  h->snap = (double *)calloc(4 * n, sizeof(double));
  if (!h->st[0] || !h->st[1] || !h->post || !h->mom || !h->snap) {
    mclbm_ref_destroy(h);
    return REF_ENOMEM;
  }
  *out = h;
  return REF_OK;
}

void mclbm_ref_destroy(ref_t *h) {
  if (!h) return;
  free(h->st[0]);
  free(h->st[1]);
  free(h->post);
  free(h->mom);
  free(h->snap);
  free(h);
}

int mclbm_ref_consts(const ref_t *h, ref_consts *out) {
  if (!h || !out) return REF_EINVAL;
  *out = h->c;
  return REF_OK;
}

int64_t mclbm_ref_steps_done(const ref_t *h) { return h ? h->steps : -1; }

/* Second-order equilibrium (Eqs 26-27, c_s^2 = 1/3): W_i rho [1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u]. */
void mclbm_ref_equilibrium(double rho, double ux, double uy, double out[9]) {
  const double uu = ux * ux + uy * uy;
  for (int q = 0; q < NQ; ++q) {
    const double eu = EX[q] * ux + EY[q] * uy;
    out[q] = W[q] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
}

/* Step 1: pull streaming of population (set s, direction q) into node (i, j).
 * Interior: the post-collision value at x - e_q. A link that crosses a wall:
 *   f^w, f^p: link-wise bounce-back f_q(x) = f*_{-q}(x) (Eq 34);
 *   g through the hot or cold wall (corners included): anti-bounce-back
 *     g_q(x) = -g*_{-q}(x) + 2 W_q T_wall, i.e. (g_q + g_{-q}) / (W_q + W_{-q}) = T_wall (Eq 35);
 *   g through an adiabatic wall only: specular reflection, the population that left the
 *     neighbour (i - e_qx, j) with the vertically mirrored velocity (zero wall flux, Eq 36).   */
static double pull(const ref_t *h, const double *st, int s, int q, int i, int j) {
  int si = i - EX[q];
  const int sj = j - EY[q];
  if (h->pr.periodic_x) si = (si + h->nx) % h->nx;
  const int out_x = si < 0 || si >= h->nx;
  const int out_y = sj < 0 || sj >= h->ny;
  if (!out_x && !out_y) return AT(st, s * NQ + q, si, sj);
  if (s < 2) return AT(st, s * NQ + opposite(q), i, j);
  if (out_x) {
    const double Tw = (si < 0) ? T_HOT : T_COLD;
    return -AT(st, s * NQ + opposite(q), i, j) + 2.0 * W[q] * Tw;
  }
  return AT(st, s * NQ + mirror_y(q), si, j);
}

static void stream_all(ref_t *h) {
  const double *st = h->st[h->cur];
#pragma omp parallel for schedule(static)
  for (int j = 0; j < h->ny; ++j)
    for (int i = 0; i < h->nx; ++i)
      for (int s = 0; s < h->nsets; ++s)
        for (int q = 0; q < NQ; ++q) AT(h->post, s * NQ + q, i, j) = pull(h, st, s, q, i, j);
}

/* Eq 33 (two thermal sets): the enthalpy-weighted mixture temperature, with the partial
 * densities (normalised by rho_f) times the specific heats as the components' heat capacities. */
static double mixture_theta(const ref_t *h, double rho_w, double rho_p, double th_w,
                            double th_p) {
  const double r = h->pr.cp_p / h->pr.cp_f;
  return (rho_w * th_w + r * rho_p * th_p) / (rho_w + r * rho_p);
}

/* Step 2: moments of the post-stream populations (Eqs 29-31). */
static void moments_all(ref_t *h) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < h->ny; ++j)
    for (int i = 0; i < h->nx; ++i) {
      double rw = 0, rp = 0, mwx = 0, mwy = 0, mpx = 0, mpy = 0, th = 0, thp = 0;
      for (int q = 0; q < NQ; ++q) {
        const double fw = AT(h->post, q, i, j), fp = AT(h->post, NQ + q, i, j);
        rw += fw;
        rp += fp;
        mwx += fw * EX[q];
        mwy += fw * EY[q];
        mpx += fp * EX[q];
        mpy += fp * EY[q];
        th += AT(h->post, 2 * NQ + q, i, j);
        if (h->nsets == 4) thp += AT(h->post, 3 * NQ + q, i, j);
      }
      AT(h->mom, M_RHOW, i, j) = rw;
      AT(h->mom, M_RHOP, i, j) = rp;
      AT(h->mom, M_MWX, i, j) = mwx;
      AT(h->mom, M_MWY, i, j) = mwy;
      AT(h->mom, M_MPX, i, j) = mpx;
      AT(h->mom, M_MPY, i, j) = mpy;
      AT(h->mom, M_THW, i, j) = th;
      AT(h->mom, M_THP, i, j) = h->nsets == 4 ? thp : th;
      AT(h->mom, M_THETA, i, j) = h->nsets == 4 ? mixture_theta(h, rw, rp, th, thp) : th;
    }
}

/* local volume fraction from the particle partial density (normalised by rho_f) */
static double phi_of(const ref_t *h, double rho_p) { return rho_p * h->pr.rho_f / h->pr.rho_p; }

/* Step 3: central differences of theta and phi at the same time level with wall ghosts. */
static void gradients(const ref_t *h, int i, int j, double gth[2], double gph[2]) {
  const int nx = h->nx, ny = h->ny;
  const double th = AT(h->mom, M_THETA, i, j);
  const double ph = phi_of(h, AT(h->mom, M_RHOP, i, j));
  double thE, thW, phE, phW;
  if (h->pr.periodic_x) {
    thE = AT(h->mom, M_THETA, (i + 1) % nx, j);
    thW = AT(h->mom, M_THETA, (i + nx - 1) % nx, j);
    phE = phi_of(h, AT(h->mom, M_RHOP, (i + 1) % nx, j));
    phW = phi_of(h, AT(h->mom, M_RHOP, (i + nx - 1) % nx, j));
  } else {
    thE = (i + 1 < nx) ? AT(h->mom, M_THETA, i + 1, j) : 2.0 * T_COLD - th;
    thW = (i > 0) ? AT(h->mom, M_THETA, i - 1, j) : 2.0 * T_HOT - th;
    phE = (i + 1 < nx) ? phi_of(h, AT(h->mom, M_RHOP, i + 1, j)) : ph;
    phW = (i > 0) ? phi_of(h, AT(h->mom, M_RHOP, i - 1, j)) : ph;
  }
  const double thN = (j + 1 < ny) ? AT(h->mom, M_THETA, i, j + 1) : th;
  const double thS = (j > 0) ? AT(h->mom, M_THETA, i, j - 1) : th;
  const double phN = (j + 1 < ny) ? phi_of(h, AT(h->mom, M_RHOP, i, j + 1)) : ph;
  const double phS = (j > 0) ? phi_of(h, AT(h->mom, M_RHOP, i, j - 1)) : ph;
  gth[0] = 0.5 * (thE - thW);
  gth[1] = 0.5 * (thN - thS);
  gph[0] = 0.5 * (phE - phW);
  gph[1] = 0.5 * (phN - phS);
}

/* Exact one-step drag impulse J on the particle component. Over the step the slip
 * w = u^w - u^p obeys dw/dt = -a w + b (drag rate a = beta_lb (1 + rho_p/rho_w), other forces
 * frozen in b = F^w_nd/rho_w - F^p_nd/rho_p), starting from the collision-relaxed slip w'.
 * J = mu_r [(1 - e^-a) w' + (1 - (1 - e^-a)/a) b], mu_r = rho_w rho_p / (rho_w + rho_p). */
void mclbm_ref_drag_impulse(double rho_w, double rho_p, const double w_relaxed[2],
                            const double b[2], double a, double J[2]) {
  const double mu_r = rho_w * rho_p / (rho_w + rho_p);
  const double E = -expm1(-a); /* 1 - e^-a */
  /* 1 - E/a; its Taylor series a/2 - a^2/6 + a^3/24 where the difference would cancel */
  const double G = (a < 1e-4) ? a * (0.5 - a * (1.0 / 6.0 - a / 24.0)) : 1.0 - E / a;
  for (int k = 0; k < 2; ++k) J[k] = mu_r * (E * w_relaxed[k] + G * b[k]);
}

/* Steps 2-5 for one node: moments, gradients, slip forces (Table 1, Eqs 4, 6, 20) and the drag
 * impulse. Requires stream_all and moments_all for the current state. */
static void node_terms(const ref_t *h, int i, int j, ref_terms *t) {
  const ref_props *p = &h->pr;
  const ref_consts *c = &h->c;
  const uint32_t mask = p->force_mask;
  memset(t, 0, sizeof(*t));
  const double rw = AT(h->mom, M_RHOW, i, j), rp = AT(h->mom, M_RHOP, i, j);
  const double rho = rw + rp;
  const double Yw = rw / rho, Yp = rp / rho;
  const double mwx = AT(h->mom, M_MWX, i, j), mwy = AT(h->mom, M_MWY, i, j);
  const double mpx = AT(h->mom, M_MPX, i, j), mpy = AT(h->mom, M_MPY, i, j);
  const int has_p = rp > 1e-30;
  t->rho_w = rw;
  t->rho_p = rp;
  t->theta = AT(h->mom, M_THETA, i, j);
  t->phi = phi_of(h, rp);
  /* Eq 32 read as the barycentric velocity; Eq 30 for the component velocities */
  t->u[0] = (mwx + mpx) / rho;
  t->u[1] = (mwy + mpy) / rho;
  t->uw[0] = mwx / rw;
  t->uw[1] = mwy / rw;
  t->up[0] = has_p ? mpx / rp : t->uw[0];
  t->up[1] = has_p ? mpy / rp : t->uw[1];
  t->tau_theta = Yw * c->tau_tw + Yp * c->tau_tp; /* Eq 24 with local mass fractions (Eq 25) */
  gradients(h, i, j, t->grad_theta, t->grad_phi);

  /* fluid-side external forces (lattice units) */
  if (mask & REF_F_BUOYANCY) /* Eq 2 Boussinesq term with beta_ns of Eq 9 */
    t->F_buoy[1] = rho * c->beta_ratio * c->G_B * t->theta;
  t->F_buoy[0] += p->body_fx; /* test-only body force */
  if (mask & REF_F_GRAVITY) {
    const double buoyant = 1.0 - p->rho_f / p->rho_p;
    t->F_G[1] = -rp * buoyant * c->g_lb;        /* Table 1 gravity, per volume */
    t->F_G0[1] = c->rho_p0 * buoyant * c->g_lb; /* uniform part returned to the fluid */
  }

  if (has_p) {
    const double vel = c->dx / c->dt; /* lattice velocity -> m/s */
    const double T_K = p->T0 + t->theta * p->dT;
    const double n_p = t->phi / c->V_p; /* particles per m^3 (Eq 4) */
    const double rho_p_SI = rp * p->rho_f;
    const double d = h->d_p;
    const double w_SI[2] = {(t->uw[0] - t->up[0]) * vel, (t->uw[1] - t->up[1]) * vel};
    const double w_mag = hypot(w_SI[0], w_SI[1]);
    double F_SI[2];
    if (mask & REF_F_BROWNIAN) {
      const double D_B = 2.0 * KB * T_K / (3.0 * PI * c->mu_ns * d);
      const double v_B = 2.0 * KB * T_K / (PI * c->mu_ns * d * d);
      for (int k = 0; k < 2; ++k) {
        const double gphi_SI = t->grad_phi[k] / c->dx;
        F_SI[k] = -n_p * p->rho_p * D_B * gphi_SI * c->A_p * v_B;
        t->F_B[k] = F_SI[k] * c->C_F;
      }
    }
    if (mask & REF_F_THERMOPHORESIS) {
      for (int k = 0; k < 2; ++k) {
        const double gT_SI = p->dT * t->grad_theta[k] / c->dx;
        const double v_T = -c->K_T * c->nu_ns_SI * gT_SI / T_K;
        F_SI[k] = rho_p_SI * c->beta_St * v_T;
        t->F_T[k] = F_SI[k] * c->C_F;
      }
    }
    if (mask & REF_F_SAFFMAN) {
      /* (K_S/4) mu_ns |w| d_p^2 sqrt(rho_ns gamma / mu_ns): the printed form without the
       * square root is not a force; its direction is the slip rotated by +90 degrees */
      const double up_mag = hypot(t->up[0], t->up[1]) * vel;
      const double gamma = 8.0 * up_mag / c->H_phys;
      const double coef =
          n_p * 0.25 * 81.2 * c->mu_ns * d * d * sqrt(c->rho_ns * gamma / c->mu_ns);
      F_SI[0] = -coef * w_SI[1];
      F_SI[1] = coef * w_SI[0];
      t->F_S[0] = F_SI[0] * c->C_F;
      t->F_S[1] = F_SI[1] * c->C_F;
    }
    if (mask & REF_F_MAGNUS) {
      /* nearest wall (ties: left, right, bottom, top) and its inward normal */
      double z = 1e300, nrm[2] = {0, 0};
      if (!p->periodic_x) {
        const double dl = i + 0.5, dr = h->nx - i - 0.5;
        if (dl < z) { z = dl; nrm[0] = 1; nrm[1] = 0; }
        if (dr < z) { z = dr; nrm[0] = -1; nrm[1] = 0; }
      }
      {
        const double db = j + 0.5, dtop = h->ny - j - 0.5;
        if (db < z) { z = db; nrm[0] = 0; nrm[1] = 1; }
        if (dtop < z) { z = dtop; nrm[0] = 0; nrm[1] = -1; }
      }
      const double zH = 2.0 * z * c->dx / c->H_phys;
      const double vbar = 0.5 * hypot(t->uw[0] + t->up[0], t->uw[1] + t->up[1]) * vel;
      const double v_M = 0.34 * (vbar * vbar * c->H_phys / c->nu_ns_SI) *
                         pow(d / c->H_phys, 2.84) * zH * (0.63 - zH);
      for (int k = 0; k < 2; ++k) {
        F_SI[k] = rho_p_SI * c->beta_St * v_M * nrm[k];
        t->F_M[k] = F_SI[k] * c->C_F;
      }
    }
    if (mask & REF_F_DRAG) {
      const double Re_d = p->rho_p * d * w_mag / c->mu_ns;
      const double beta = 18.0 * c->mu_ns * (1.0 + 0.15 * pow(Re_d, 0.687)) / (p->rho_p * d * d);
      t->beta_lb = beta * c->dt;
      t->a = t->beta_lb * (1.0 + rp / rw);
    }
  }
  /* Reactions: every particle-fluid force acts with opposite sign on the fluid (Eq 20). */
  double Fp_nd[2], Fw_nd[2];
  for (int k = 0; k < 2; ++k) {
    const double F_int = t->F_B[k] + t->F_T[k] + t->F_S[k] + t->F_M[k];
    Fp_nd[k] = F_int + t->F_G[k];
    Fw_nd[k] = t->F_buoy[k] + t->F_G0[k] - F_int;
  }
  if (has_p && (mask & REF_F_DRAG)) {
    /* slip after BGK relaxation of both components towards the common velocity */
    const double relax = 1.0 - Yp / c->tau_w - Yw / c->tau_p;
    const double wr[2] = {(t->uw[0] - t->up[0]) * relax, (t->uw[1] - t->up[1]) * relax};
    const double b[2] = {Fw_nd[0] / rw - Fp_nd[0] / rp, Fw_nd[1] / rw - Fp_nd[1] / rp};
    mclbm_ref_drag_impulse(rw, rp, wr, b, t->a, t->J);
  }
  for (int k = 0; k < 2; ++k) {
    t->F_p[k] = Fp_nd[k] + t->J[k];
    t->F_w[k] = Fw_nd[k] - t->J[k];
  }
}

/* Step 6: BGK collision with forcing 3 W_q e_q.F (Eq 18 with its 1/c_s^2), equilibria on the
 * common velocity (Eqs 26-27), thermal relaxation with the local tau of Eq 24 (Eq 19). */
static void collide_node(ref_t *h, const ref_terms *t, int i, int j, double *dst) {
  const ref_consts *c = &h->c;
  double eqw[NQ], eqp[NQ], eqg[NQ];
  mclbm_ref_equilibrium(t->rho_w, t->u[0], t->u[1], eqw);
  mclbm_ref_equilibrium(t->rho_p, t->u[0], t->u[1], eqp);
  mclbm_ref_equilibrium(t->theta, t->u[0], t->u[1], eqg);
  for (int q = 0; q < NQ; ++q) {
    const double fw = AT(h->post, q, i, j), fp = AT(h->post, NQ + q, i, j);
    const double g = AT(h->post, 2 * NQ + q, i, j);
    const double Sw = 3.0 * W[q] * (EX[q] * t->F_w[0] + EY[q] * t->F_w[1]);
    const double Sp = 3.0 * W[q] * (EX[q] * t->F_p[0] + EY[q] * t->F_p[1]);
    AT(dst, q, i, j) = fw - (fw - eqw[q]) / c->tau_w + Sw;
    AT(dst, NQ + q, i, j) = fp - (fp - eqp[q]) / c->tau_p + Sp;
    if (h->nsets == 3) {
      AT(dst, 2 * NQ + q, i, j) = g - (g - eqg[q]) / t->tau_theta;
    } else { /* Eq 19 per component, both towards the mixture temperature (Eqs 27, 33) */
      const double gp = AT(h->post, 3 * NQ + q, i, j);
      AT(dst, 2 * NQ + q, i, j) = g - (g - eqg[q]) / c->tau_tw;
      AT(dst, 3 * NQ + q, i, j) = gp - (gp - eqg[q]) / c->tau_tp;
    }
  }
}

int mclbm_ref_init(ref_t *h, int mode, const double *warm) {
  if (!h) return REF_EINVAL;
  if (mode != REF_INIT_REST && mode != REF_INIT_WARM && mode != REF_INIT_WARM_RHO)
    return REF_EINVAL;
  if (mode != REF_INIT_REST && !warm) return REF_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  double *st = h->st[0];
  for (int j = 0; j < h->ny; ++j)
    for (int i = 0; i < h->nx; ++i) {
      double ux = 0, uy = 0, th, ph, rw;
      if (mode == REF_INIT_REST) {
        th = 0.5 - (i + 0.5) / h->nx; /* linear conduction profile */
        ph = h->phi0;
        rw = 1.0 - ph;
      } else {
        const size_t k = (size_t)j * h->nx + i;
        ux = warm[k];
        uy = warm[n + k];
        th = warm[2 * n + k];
        ph = warm[3 * n + k];
        /* the base-fluid partial density: given (a steady state's pressure field) or 1 - phi */
        rw = mode == REF_INIT_WARM_RHO ? warm[4 * n + k] : 1.0 - ph;
      }
      double e[NQ];
      mclbm_ref_equilibrium(rw, ux, uy, e);
      for (int q = 0; q < NQ; ++q) AT(st, q, i, j) = e[q];
      mclbm_ref_equilibrium(ph * h->pr.rho_p / h->pr.rho_f, ux, uy, e);
      for (int q = 0; q < NQ; ++q) AT(st, NQ + q, i, j) = e[q];
      mclbm_ref_equilibrium(th, ux, uy, e);
      for (int s = 2; s < h->nsets; ++s)
        for (int q = 0; q < NQ; ++q) AT(st, s * NQ + q, i, j) = e[q];
    }
  h->cur = 0;
  h->steps = 0;
  h->ready = 1;
  double r;
  h->snap_step = -1;
  return mclbm_ref_residual(h, &r); /* first snapshot */
}

int mclbm_ref_step(ref_t *h, int64_t n) {
  if (!h || n < 0) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  for (int64_t s = 0; s < n; ++s) {
    stream_all(h);
    moments_all(h);
    double *dst = h->st[1 - h->cur];
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h->ny; ++j)
      for (int i = 0; i < h->nx; ++i) {
        ref_terms t;
        node_terms(h, i, j, &t);
        collide_node(h, &t, i, j, dst);
      }
    h->cur = 1 - h->cur;
    h->steps += 1;
  }
  return REF_OK;
}

int mclbm_ref_stream_only(ref_t *h) {
  if (!h) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  stream_all(h);
  memcpy(h->st[1 - h->cur], h->post, sizeof(double) * h->np * (size_t)h->nx * h->ny);
  h->cur = 1 - h->cur;
  return REF_OK;
}

int mclbm_ref_node_terms(ref_t *h, int i, int j, ref_terms *out) {
  if (!h || !out || i < 0 || j < 0 || i >= h->nx || j >= h->ny) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  stream_all(h);
  moments_all(h);
  node_terms(h, i, j, out);
  return REF_OK;
}

/* Moments of the post-stream state: the fields the next step starts from. */
int mclbm_ref_fields(ref_t *h, uint32_t which, double *out) {
  if (!h || !out || !which || (which & ~0x3FFu)) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  stream_all(h);
  moments_all(h);
  const size_t n = (size_t)h->nx * h->ny;
  double *o = out;
  for (int bit = 0; bit < 10; ++bit) {
    if (!(which & (1u << bit))) continue;
    for (int j = 0; j < h->ny; ++j)
      for (int i = 0; i < h->nx; ++i) {
        const double rw = AT(h->mom, M_RHOW, i, j), rp = AT(h->mom, M_RHOP, i, j);
        const double mwx = AT(h->mom, M_MWX, i, j), mwy = AT(h->mom, M_MWY, i, j);
        const double mpx = AT(h->mom, M_MPX, i, j), mpy = AT(h->mom, M_MPY, i, j);
        double v = 0;
        switch (1u << bit) {
          case REF_UX: v = (mwx + mpx) / (rw + rp); break;
          case REF_UY: v = (mwy + mpy) / (rw + rp); break;
          case REF_THETA: v = AT(h->mom, M_THETA, i, j); break;
          case REF_PHI: v = phi_of(h, rp); break;
          case REF_RHO_W: v = rw; break;
          case REF_RHO_P: v = rp; break;
          case REF_UPX: v = rp > 1e-30 ? mpx / rp : mwx / rw; break;
          case REF_UPY: v = rp > 1e-30 ? mpy / rp : mwy / rw; break;
          case REF_THETA_W: v = AT(h->mom, M_THW, i, j); break;
          case REF_THETA_P: v = AT(h->mom, M_THP, i, j); break;
        }
        o[(size_t)j * h->nx + i] = v;
      }
    o += n;
  }
  return REF_OK;
}

/* Mean Nusselt numbers of the hot and cold walls: k_ns/k_f times L/dT times the mean over the
 * wall of the one-sided second-order gradient at the half-way wall, (8 T_w - 9 th_0 + th_1)/3. */
int mclbm_ref_nusselt(ref_t *h, double *nu_hot, double *nu_cold) {
  if (!h || !nu_hot || !nu_cold) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  stream_all(h);
  moments_all(h);
  const int nx = h->nx;
  double sh = 0, sc = 0;
  for (int j = 0; j < h->ny; ++j) {
    sh += (8.0 * T_HOT - 9.0 * AT(h->mom, M_THETA, 0, j) + AT(h->mom, M_THETA, 1, j)) / 3.0;
    sc += (9.0 * AT(h->mom, M_THETA, nx - 1, j) - AT(h->mom, M_THETA, nx - 2, j) - 8.0 * T_COLD) /
          3.0;
  }
  const double scale = h->c.k_ratio * (double)nx / (T_HOT - T_COLD) / (double)h->ny;
  *nu_hot = sh * scale;
  *nu_cold = sc * scale;
  return REF_OK;
}

int mclbm_ref_mass(const ref_t *h, double *mass_w, double *mass_p) {
  if (!h || !mass_w || !mass_p) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  const double *st = h->st[h->cur];
  const size_t n = (size_t)h->nx * h->ny;
  double mw = 0, mp = 0;
  for (int q = 0; q < NQ; ++q)
    for (size_t k = 0; k < n; ++k) {
      mw += st[q * n + k];
      mp += st[(NQ + q) * n + k];
    }
  *mass_w = mw;
  *mass_p = mp;
  return REF_OK;
}

/* Relative change over the steps since the last check, per step: max over u, theta, phi of
 * ||q_now - q_then||_2 / (K ||q_now||_2). The snapshot is replaced. K = 0 gives 0. */
int mclbm_ref_residual(ref_t *h, double *r) {
  if (!h || !r) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  const size_t n = (size_t)h->nx * h->ny;
  double *now = (double *)malloc(sizeof(double) * 4 * n);
  if (!now) return REF_ENOMEM;
  int rc = mclbm_ref_fields(h, REF_UX | REF_UY | REF_THETA | REF_PHI, now);
  if (rc) {
    free(now);
    return rc;
  }
  const int64_t K = h->snap_step < 0 ? 0 : h->steps - h->snap_step;
  double res = 0.0;
  if (K > 0) {
    double num[3] = {0, 0, 0}, den[3] = {0, 0, 0};
    for (int f = 0; f < 4; ++f) {
      const int grp = f < 2 ? 0 : f - 1;
      for (size_t k = 0; k < n; ++k) {
        const double d = now[f * n + k] - h->snap[f * n + k];
        num[grp] += d * d;
        den[grp] += now[f * n + k] * now[f * n + k];
      }
    }
    for (int g = 0; g < 3; ++g) {
      double term;
      if (num[g] == 0.0)
        term = 0.0;
      else if (den[g] == 0.0)
        term = INFINITY;
      else
        term = sqrt(num[g]) / ((double)K * sqrt(den[g]));
      if (term > res || isnan(term)) res = term;
    }
  }
  memcpy(h->snap, now, sizeof(double) * 4 * n);
  h->snap_step = h->steps;
  free(now);
  *r = res;
  return REF_OK;
}

int mclbm_ref_get_state(const ref_t *h, double *out) {
  if (!h || !out) return REF_EINVAL;
  if (!h->ready) return REF_ESTATE;
  memcpy(out, h->st[h->cur], sizeof(double) * h->np * (size_t)h->nx * h->ny);
  return REF_OK;
}

int mclbm_ref_set_state(ref_t *h, const double *in) {
  if (!h || !in) return REF_EINVAL;
  memcpy(h->st[h->cur], in, sizeof(double) * h->np * (size_t)h->nx * h->ny);
  if (!h->ready) {
    h->ready = 1;
    h->steps = 0;
    h->snap_step = -1;
  }
  return REF_OK;
}
