// Create-time model of libmclbm: material properties of the suspension (Eqs 7-11), lattice
// scales and relaxation times (Eqs 22-24), the SI scale of the cavity, and the FP32 force
// coefficients of Table 1 folded for the step kernel. Host code, FP64.
#include <cmath>
#include <cstring>

#include "mclbm_internal.h"

namespace mcl {

namespace {
constexpr double kBoltzmann = 1.380649e-23;  // J/K
constexpr double kPi = 3.14159265358979323846;
// Table 1 constants
constexpr double kCs = 1.17, kCt = 2.18, kCm = 1.14;  // thermophoresis (Brock form)
constexpr double kKs = 81.2;                          // Saffman lift
constexpr double kMagnus = 0.34, kMagnusExp = 2.84;   // Magnus migration velocity
}  // namespace

void props_default(mclbm_props* p) {
  std::memset(p, 0, sizeof(*p));
  // water at 25 C
  p->rho_f = 997.1;
  p->cp_f = 4179.0;
  p->k_f = 0.613;
  p->beta_f = 2.1e-4;
  p->mu_f = 8.9e-4;
  // alumina
  p->rho_p = 3970.0;
  p->cp_p = 765.0;
  p->k_p = 40.0;
  p->beta_p = 0.85e-5;
  p->T0_K = 298.15;
  p->dT_K = 10.0;
  p->g = 9.81;
  p->l_f = 0.17e-9;
  p->Ma = 0.1;
  p->force_mask = MCLBM_F_ALL;
  p->storage = MCLBM_STORE_F32;
  p->rounding = MCLBM_ROUND_STOCHASTIC;
  p->thermal_sets = 1;
}

int derive_consts(int nx, int ny, double Ra, double Pr, double phi, double d_p,
                  const mclbm_props& p, mclbm_consts* c) {
  (void)nx;
  std::memset(c, 0, sizeof(*c));
  const double H = ny;  // cavity height in lattice units
  const double cs = std::sqrt(1.0 / 3.0);

  // Lattice scales from the base-fluid Ra and Pr: buoyancy velocity U0 = Ma c_s.
  c->U0 = p.Ma * cs;
  c->nu_w = c->U0 * H / std::sqrt(Ra / Pr);
  c->alpha_w = c->nu_w / Pr;
  c->G_B = c->U0 * c->U0 / H;

  // Suspension properties relative to the base fluid, at the initial volume fraction.
  const double rho_ns = (1.0 - phi) * p.rho_f + phi * p.rho_p;                      // Eq 7
  const double rhocp_ns = (1.0 - phi) * p.rho_f * p.cp_f + phi * p.rho_p * p.cp_p;  // Eq 8
  const double beta_ns = (1.0 - phi) * p.beta_f + phi * p.beta_p;                   // Eq 9
  const double mu_ns = p.mu_f * (1.0 + phi * (4.93 + 222.4 * phi));                 // Eq 11
  // Eq 10b with the base-fluid mean free path as d_f, at T0; Eq 10a with printed exponents
  const double Re_T = p.rho_f * kBoltzmann * p.T0_K / (3.0 * kPi * p.mu_f * p.mu_f * p.l_f);
  double k_enh = 0.0;
  if (phi > 0.0)
    k_enh = 64.7 * std::pow(phi, 0.764) * std::pow(p.l_f / d_p, 0.369) *
            std::pow(p.k_f / p.k_p, 0.7476) * std::pow(Pr, 0.995) * std::pow(Re_T, 1.2321);
  const double k_ns = p.k_f * (1.0 + k_enh);
  c->rho_ratio = rho_ns / p.rho_f;
  c->rhocp_ratio = rhocp_ns / (p.rho_f * p.cp_f);
  c->beta_ratio = beta_ns / p.beta_f;
  c->mu_ratio = mu_ns / p.mu_f;
  c->k_ratio = k_ns / p.k_f;
  c->Re_T = Re_T;
  // suspension diffusivities in lattice units
  c->nu_ns = c->nu_w * c->mu_ratio / c->rho_ratio;
  c->alpha_ns = c->alpha_w * c->k_ratio / c->rhocp_ratio;

  // Partial densities (normalised by rho_f) and initial mass fractions (Eq 25).
  c->rho_w0 = 1.0 - phi;
  c->rho_p0 = phi * p.rho_p / p.rho_f;
  const double rho0 = c->rho_w0 + c->rho_p0;
  c->Y_w0 = c->rho_w0 / rho0;
  c->Y_p0 = c->rho_p0 / rho0;

  // Relaxation times: nu = (tau - 1/2)/3 for the base fluid (Eq 22); the mixture values of
  // Eqs 23-24 at the initial mass fractions fix the particle component's taus.
  c->tau_w = 0.5 + 3.0 * c->nu_w;
  c->tau_tw = 0.5 + 3.0 * c->alpha_w;
  if (phi > 0.0) {
    c->tau_p = (0.5 + 3.0 * c->nu_ns - c->Y_w0 * c->tau_w) / c->Y_p0;
    c->tau_tp = (0.5 + 3.0 * c->alpha_ns - c->Y_w0 * c->tau_tw) / c->Y_p0;
  } else {
    c->tau_p = c->tau_w;
    c->tau_tp = c->tau_tw;
  }

  // SI scale: the cavity height that gives Ra for the base fluid, lattice spacing and step.
  const double nu_f = p.mu_f / p.rho_f;
  c->H_phys = std::cbrt(Ra * nu_f * (nu_f / Pr) / (p.g * p.beta_f * p.dT_K));
  c->dx = c->H_phys / H;
  c->dt = c->nu_w * c->dx * c->dx / nu_f;
  c->C_F = c->dt * c->dt / (p.rho_f * c->dx);  // N/m^3 -> lattice force density
  c->g_lb = p.g * c->dt * c->dt / c->dx;

  // Particle and suspension quantities used by Table 1.
  c->mu_ns = mu_ns;
  c->rho_ns = rho_ns;
  c->k_ns = k_ns;
  c->nu_ns_SI = mu_ns / rho_ns;
  c->V_p = kPi * d_p * d_p * d_p / 6.0;
  c->A_p = kPi * d_p * d_p;
  c->m_p = p.rho_p * c->V_p;
  c->beta_St = 18.0 * mu_ns / (p.rho_p * d_p * d_p);
  c->Kn = p.l_f / d_p;
  c->kstar = k_ns / p.k_p;
  const double ck = kCt * c->Kn;
  c->K_T = 6.0 * kPi * kCs * (c->kstar + ck) /
           ((1.0 + 3.0 * kCm * c->Kn) * (1.0 + 2.0 * c->kstar + 2.0 * ck));

  const double lim = 0.501;
  if (!(c->tau_w > lim && c->tau_p > lim && c->tau_tw > lim && c->tau_tp > lim))
    return MCLBM_EPARAM;
  return MCLBM_OK;
}

// Folds Table 1 into per-node lattice coefficients. With rho^p the particle partial density
// (lattice, normalised by rho_f), phi = rho^p rho_f / rho_p, n_p = phi / V_p particles per m^3,
// v_SI = v (dx/dt), grad_SI = grad / dx and F_lattice = C_F F_SI:
//   Brownian   n_p rho_p D_B A_p v_B (-grad phi), D_B, v_B proportional to T
//   thermophoresis  rho_p,SI beta_St v_T, v_T = -K_T nu_ns grad T / T
//   Saffman    n_p (K_S/4) mu_ns |w| d^2 sqrt(rho_ns gamma / mu_ns) along R90(w), gamma = 8|u^p|/H
//   Magnus     rho_p,SI beta_St v_M n, v_M = 0.34 (vbar^2 H/nu_ns)(d/H)^2.84 zeta, vbar = |u^w+u^p|/2
StepConsts fold_step_consts(int nx, int ny, double phi, double d_p, const mclbm_props& p,
                            const mclbm_consts& c) {
  StepConsts k;
  std::memset(&k, 0, sizeof(k));
  const double vel = c.dx / c.dt;
  const double fr = p.rho_f / p.rho_p;
  const double T0 = p.T0_K;
  k.rho_w0 = (float)c.rho_w0;
  k.rho_p0 = (float)c.rho_p0;
  k.inv_tau_w = (float)(1.0 / c.tau_w);
  k.inv_tau_p = (float)(1.0 / c.tau_p);
  k.tau_tw = (float)c.tau_tw;
  k.tau_tp = (float)c.tau_tp;
  k.buoy = (float)(c.beta_ratio * c.G_B);
  k.gG = (float)((1.0 - fr) * c.g_lb);
  k.phi_per_rho_p = (float)fr;
  const double kT0 = kBoltzmann * T0;
  const double D_B0 = 2.0 * kT0 / (3.0 * kPi * c.mu_ns * d_p);
  const double v_B0 = 2.0 * kT0 / (kPi * c.mu_ns * d_p * d_p);
  // n_p = rho^p fr / V_p; grad phi_SI = fr grad rho^p / dx
  k.cB = (float)(c.C_F * (fr / c.V_p) * p.rho_p * D_B0 * c.A_p * v_B0 * fr / c.dx);
  // rho_p,SI = rho^p rho_f; grad T_SI = dT grad theta / dx
  k.cT = (float)(c.C_F * p.rho_f * c.beta_St * c.K_T * c.nu_ns_SI * p.dT_K / (c.dx * T0));
  k.cS = (float)(c.C_F * (fr / c.V_p) * (kKs / 4.0) * c.mu_ns * d_p * d_p *
                 std::sqrt(c.rho_ns * 8.0 * vel / (c.H_phys * c.mu_ns)) * vel);
  k.cM = (float)(c.C_F * p.rho_f * c.beta_St * kMagnus * 0.25 * vel * vel * c.H_phys /
                 c.nu_ns_SI * std::pow(d_p / c.H_phys, kMagnusExp));
  k.t_ratio = (float)(p.dT_K / T0);
  k.beta_dt = (float)(c.beta_St * c.dt);
  k.cRe = (float)(p.rho_p * d_p * vel / c.mu_ns);
  k.two_over_ny = (float)(2.0 / ny);
  k.inv_nx = (float)(1.0 / nx);
  k.th_c0 = (float)(0.5 - 0.5 / nx);
  k.mask = p.force_mask;
  k.has_p = phi > 0.0 ? 1 : 0;
  k.two_sets = p.thermal_sets == 2 ? 1 : 0;
  k.r_cp = (float)(p.cp_p / p.cp_f);
  k.rho_w0_d = c.rho_w0;
  k.rho_p0_d = c.rho_p0;
  k.fr_d = fr;
  return k;
}

}  // namespace mcl
