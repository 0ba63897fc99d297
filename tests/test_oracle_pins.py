"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle by a route other than its own formulas: closed-form moments,
conservation laws, an independent textbook scheme, symmetries, an ODE solved by matrix
exponential, an independent SI derivation and analytic flows.
"""
import math

import numpy as np
import pytest

from tests._textbook_tlbm import TextbookTLBM, E, W

KB = 1.380649e-23


def ref_solver(oracle, nx=32, ny=32, Ra=1e3, Pr=6.2, phi=0.01, d_p=20e-9, **props):
    return oracle.RefSolver(nx, ny, Ra, Pr, phi, d_p, **props)


# ---------------------------------------------------------------- P1: equilibrium moments
@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.97, 0.03, -0.02), (0.04, -0.1, 0.07),
                                       (-0.3, 0.05, 0.01)])
def test_equilibrium_moments(oracle_mod, rho, ux, uy):
    """Eqs 26-28: zeroth, first and second moments of the second-order equilibrium."""
    f = oracle_mod.equilibrium(rho, ux, uy)
    ex, ey = E[:, 0], E[:, 1]
    assert abs(f.sum() - rho) < 1e-15
    assert abs((f * ex).sum() - rho * ux) < 1e-15
    assert abs((f * ey).sum() - rho * uy) < 1e-15
    cs2 = 1.0 / 3.0
    assert abs((f * ex * ex).sum() - rho * (cs2 + ux * ux)) < 1e-15
    assert abs((f * ey * ey).sum() - rho * (cs2 + uy * uy)) < 1e-15
    assert abs((f * ex * ey).sum() - rho * ux * uy) < 1e-15
    # the weights sum to one and are isotropic to second order (Eq 28)
    assert abs(W.sum() - 1) < 1e-16 and abs((W * ex * ex).sum() - cs2) < 1e-16


# ---------------------------------------------------------------- P2: streaming
def _expected_push(st, nx, ny):
    """Forward (push) view of the wall rules, independent of the pull code: every post-collision
    population moves one link; on a wall it comes back to its own node reversed (f), reversed and
    reflected about the wall temperature (g at the side walls), or mirrored in the wall (g at
    the adiabatic walls)."""
    out = np.full_like(st, np.nan)
    opp = {q: int(np.where((E == -E[q]).all(1))[0][0]) for q in range(9)}
    mir = {q: int(np.where((E == E[q] * np.array([1, -1])).all(1))[0][0]) for q in range(9)}
    for s in range(3):
        for q in range(9):
            ex, ey = E[q]
            for j in range(ny):
                for i in range(nx):
                    v = st[9 * s + q, j, i]
                    ti, tj = i + ex, j + ey
                    if 0 <= ti < nx and 0 <= tj < ny:
                        out[9 * s + q, tj, ti] = v
                    elif s < 2:
                        out[9 * s + opp[q], j, i] = v
                    elif not (0 <= ti < nx):
                        Tw = 0.5 if ti < 0 else -0.5
                        out[9 * s + opp[q], j, i] = -v + 2 * W[q] * Tw
                    else:
                        out[9 * s + mir[q], j, ti] = v
    return out


@pytest.mark.parametrize("nx,ny", [(5, 4), (2, 2), (3, 7)])
def test_stream_against_push(oracle_mod, nx, ny):
    rng = np.random.default_rng(11)
    s = ref_solver(oracle_mod, nx, ny).init()
    st = rng.uniform(-1, 1, (27, ny, nx))
    s.set_state(st)
    s.stream_only()
    got = s.get_state()
    exp = _expected_push(st, nx, ny)
    assert not np.isnan(exp).any()
    np.testing.assert_array_equal(got[:18], exp[:18])  # bounce-back: exact permutation
    np.testing.assert_allclose(got[18:], exp[18:], rtol=0, atol=1e-15)
    # f: a permutation inside each set, so every sum is exact
    for s_ in range(2):
        assert np.array_equal(np.sort(got[9 * s_:9 * s_ + 9].ravel()),
                              np.sort(st[9 * s_:9 * s_ + 9].ravel()))


def test_stream_displaces_along_e(oracle_mod):
    """A single interior population moves by +e_q (pull from x - e_q)."""
    nx, ny = 6, 5
    for q in range(9):
        s = ref_solver(oracle_mod, nx, ny).init()
        st = np.zeros((27, ny, nx))
        st[q, 2, 2] = 1.0
        s.set_state(st)
        s.stream_only()
        got = s.get_state()
        assert got[q, 2 + E[q, 1], 2 + E[q, 0]] == 1.0
        assert got[:9].sum() == 1.0


# ---------------------------------------------------------------- P3: mass
def test_mass_conservation_config1(oracle_mod):
    """Bounce-back is a permutation and the collision conserves rho^sigma: both component
    masses are invariant over 2000 steps of the 32x32, Ra 1e3, 1 %, 20 nm cavity."""
    s = ref_solver(oracle_mod).init()
    m0 = s.mass()
    s.step(2000)
    m1 = s.mass()
    for a, b in zip(m0, m1):
        assert abs(b - a) / a < 1e-12
    # and equals the closed form N rho_sigma0
    c = s.consts()
    assert abs(m0[0] - 32 * 32 * c["rho_w0"]) < 1e-12 * m0[0]
    assert abs(m0[1] - 32 * 32 * c["rho_p0"]) < 1e-12 * m0[1]


# ---------------------------------------------------------------- P4: phi = 0 limit
@pytest.mark.parametrize("nx,ny,Ra,Pr", [(16, 12, 1e4, 0.71), (9, 14, 3e3, 6.2)])
def test_phi0_is_textbook_thermal_lbm(oracle_mod, nx, ny, Ra, Pr):
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=0.0).init()
    c = s.consts()
    tb = TextbookTLBM(nx, ny, c["tau_w"], c["tau_tw"], c["G_B"])
    s.step(300)
    tb.step(300)
    fs, gs, rho, ux, uy, th = tb.moments()
    f = s.fields(oracle_mod.UX | oracle_mod.UY | oracle_mod.THETA | oracle_mod.RHO_W |
                 oracle_mod.RHO_P)
    assert np.max(np.abs(f[0] - ux)) < 1e-13
    assert np.max(np.abs(f[1] - uy)) < 1e-13
    assert np.max(np.abs(f[2] - th)) < 1e-13
    assert np.max(np.abs(f[3] - rho)) < 1e-13
    assert np.all(f[4] == 0.0)
    assert abs(s.nusselt()[0] - tb.nusselt_hot()) < 1e-12
    assert np.abs(ux).max() > 1e-4  # the flow is really there


# ---------------------------------------------------------------- P5: conduction limit
@pytest.mark.parametrize("phi", [0.0, 0.02])
def test_conduction_limit(oracle_mod, phi):
    """Without buoyancy, gravity and thermophoresis the fluid stays at rest and the linear
    profile is the exact steady state of the walls' rules: Nu = k_ns/k_f on both walls."""
    mask = oracle_mod.F_DRAG | oracle_mod.F_BROWNIAN | oracle_mod.F_SAFFMAN | oracle_mod.F_MAGNUS
    s = ref_solver(oracle_mod, 12, 9, Ra=1e3, phi=phi, force_mask=mask).init()
    s.step(50)
    k = s.consts()["k_ratio"]
    nh, nc = s.nusselt()
    assert abs(nh - k) < 1e-10 and abs(nc - k) < 1e-10
    th = s.fields(oracle_mod.THETA)[0]
    x = (np.arange(12) + 0.5) / 12
    assert np.max(np.abs(th - (0.5 - x)[None, :])) < 1e-12
    assert np.abs(s.fields(oracle_mod.UX | oracle_mod.UY)).max() < 1e-15
    if phi == 0.0:
        assert k == 1.0


def test_conduction_relaxes_to_linear(oracle_mod):
    """From a uniform temperature the conduction solution is reached; the gradient at the wall
    converges to the exact one (Nu -> k_ns/k_f)."""
    mask = oracle_mod.F_DRAG
    s = ref_solver(oracle_mod, 10, 6, Ra=1e3, Pr=0.71, phi=0.0, force_mask=mask)
    z = np.zeros((6, 10))
    s.init(warm=np.stack([z, z, z, z]))
    s.step(8000)
    nh, nc = s.nusselt()
    assert abs(nh - 1) < 1e-9 and abs(nc - 1) < 1e-9


# ---------------------------------------------------------------- P6: drag impulse
def _two_body(rho_w, rho_p, beta, Fw, Fp, uw0, up0, T=1.0):
    """Exact solution of rho_w du_w/dt = Fw - rho_p beta (u_w - u_p),
    rho_p du_p/dt = Fp + rho_p beta (u_w - u_p) by the matrix exponential."""
    from scipy.linalg import expm
    A = np.array([[-rho_p * beta / rho_w, rho_p * beta / rho_w, Fw / rho_w],
                  [beta, -beta, Fp / rho_p],
                  [0.0, 0.0, 0.0]])
    y = expm(A * T) @ np.array([uw0, up0, 1.0])
    return y[0], y[1]


@pytest.mark.parametrize("beta", [1e-6, 0.3, 2.0, 37.0, 5e4])
def test_drag_impulse_matches_two_body_ode(oracle_mod, beta):
    rho_w, rho_p = 0.97, 0.119
    w0 = np.array([3e-3, -1e-3])
    Fw, Fp = np.array([2e-5, -7e-4]), np.array([-3e-4, 1e-5])
    a = beta * (1 + rho_p / rho_w)
    b = Fw / rho_w - Fp / rho_p
    J = oracle_mod.drag_impulse(rho_w, rho_p, w0, b, a)
    for k in range(2):
        # start both components so that their slip is w0 (the frame does not matter)
        uw1, up1 = _two_body(rho_w, rho_p, beta, Fw[k], Fp[k], w0[k], 0.0)
        J_ode = rho_p * up1 - Fp[k]  # particle momentum change minus the non-drag impulse
        assert abs(J[k] - J_ode) <= 1e-12 * max(1.0, abs(J_ode)) + 1e-17


def test_drag_impulse_limits(oracle_mod):
    rho_w, rho_p = 0.9, 0.2
    w, b = np.array([1e-3, 2e-3]), np.array([0.5, -0.25])
    mu_r = rho_w * rho_p / (rho_w + rho_p)
    # a -> 0: explicit drag rho_p beta w (first order in beta)
    beta = 1e-9
    a = beta * (1 + rho_p / rho_w)
    J = oracle_mod.drag_impulse(rho_w, rho_p, w, b, a)
    np.testing.assert_allclose(J, rho_p * beta * w + mu_r * a / 2 * b, rtol=1e-6)
    # a -> inf: the post-step slip is the Stokesian terminal drift b/a
    a = 1e8
    J = oracle_mod.drag_impulse(rho_w, rho_p, w, b, a)
    w_after = w + b - J / mu_r
    np.testing.assert_allclose(w_after, b / a, rtol=1e-6)


# ---------------------------------------------------------------- P7: force balance
def test_interaction_forces_cancel(oracle_mod):
    """Every particle-fluid force has its reaction: per node F_w + F_p equals the external
    forces alone, and the gravity pair sums to zero over the cavity."""
    s = ref_solver(oracle_mod, 16, 16, Ra=1e4, phi=0.03, d_p=30e-9).init().step(200)
    tot_G = 0.0
    for (i, j) in [(0, 0), (3, 7), (15, 15), (8, 0), (15, 4), (7, 8)]:
        t = s.node_terms(i, j)
        ext = t["F_buoy"] + t["F_G0"] + t["F_G"]
        scale = max(np.abs(t["F_T"]).max(), np.abs(ext).max())
        assert np.max(np.abs(t["F_w"] + t["F_p"] - ext)) < 1e-13 * scale
        assert abs(t["F_G"][0]) == 0 and abs(t["F_buoy"][0]) == 0
    rho_p = s.fields(oracle_mod.RHO_P)[0]
    c = s.consts()
    buoyant = 1 - 997.1 / 3970.0
    tot_G = (-rho_p.sum() + rho_p.size * c["rho_p0"]) * buoyant * c["g_lb"]
    assert abs(tot_G) < 1e-12 * rho_p.size * c["rho_p0"] * c["g_lb"]


# ---------------------------------------------------------------- P8: centro-symmetry
def test_centro_symmetry(oracle_mod):
    """Hot and cold walls are antisymmetric; without the temperature-level dependent forces
    (Brownian, thermophoresis) and gravity the solution is point-symmetric about the centre."""
    mask = oracle_mod.F_DRAG | oracle_mod.F_SAFFMAN | oracle_mod.F_MAGNUS | oracle_mod.F_BUOYANCY
    s = ref_solver(oracle_mod, 14, 10, Ra=2e4, phi=0.02, d_p=30e-9, force_mask=mask).init()
    s.step(400)
    f = s.fields(oracle_mod.UX | oracle_mod.UY | oracle_mod.THETA | oracle_mod.PHI |
                 oracle_mod.UPX | oracle_mod.UPY)
    ux, uy, th, ph, upx, upy = f
    R = lambda a: a[::-1, ::-1]
    assert np.abs(ux).max() > 1e-4
    np.testing.assert_allclose(R(ux), -ux, rtol=0, atol=1e-14)
    np.testing.assert_allclose(R(uy), -uy, rtol=0, atol=1e-14)
    np.testing.assert_allclose(R(th), -th, rtol=0, atol=1e-14)
    np.testing.assert_allclose(R(ph), ph, rtol=0, atol=1e-15)
    np.testing.assert_allclose(R(upx), -upx, rtol=0, atol=1e-14)
    nh, nc = s.nusselt()
    assert abs(nh - nc) < 1e-12


# ---------------------------------------------------------------- P9: constants
def _independent_constants(nx, ny, Ra, Pr, phi, d):
    """Table 1 / Eqs 7-11 / Eqs 22-24 and the SI scale re-derived from the physics."""
    rf, cf, kf, bf, mf = 997.1, 4179.0, 0.613, 2.1e-4, 8.9e-4
    rp, cp, kp, bp = 3970.0, 765.0, 40.0, 0.85e-5
    T0, dT, g, lf, Ma = 298.15, 10.0, 9.81, 0.17e-9, 0.1
    out = {}
    U0 = Ma * math.sqrt(1 / 3)
    nu = U0 * ny / math.sqrt(Ra / Pr)
    out["nu_w"] = nu
    out["tau_w"] = 0.5 + 3 * nu
    out["tau_tw"] = 0.5 + 3 * nu / Pr
    rho_ns = (1 - phi) * rf + phi * rp
    rc_ns = (1 - phi) * rf * cf + phi * rp * cp
    mu_ns = mf * (1 + 4.93 * phi + 222.4 * phi ** 2)
    Re = rf * KB * T0 / (3 * math.pi * mf ** 2 * lf)
    k_ns = kf * (1 + 64.7 * phi ** 0.764 * (lf / d) ** 0.369 * (kf / kp) ** 0.7476
                 * Pr ** 0.995 * Re ** 1.2321)
    out["k_ratio"] = k_ns / kf
    out["mu_ns"], out["rho_ns"] = mu_ns, rho_ns
    nu_ns_lat = nu * (mu_ns / mf) * (rf / rho_ns)
    alpha_ns_lat = (nu / Pr) * (k_ns / kf) * (rf * cf / rc_ns)
    m_w, m_p = 1 - phi, phi * rp / rf
    Yw, Yp = m_w / (m_w + m_p), m_p / (m_w + m_p)
    if phi > 0:
        # Eq 23/24 with the mixture tau equal to the mass-fraction average
        out["tau_p"] = (0.5 + 3 * nu_ns_lat - Yw * out["tau_w"]) / Yp
        out["tau_tp"] = (0.5 + 3 * alpha_ns_lat - Yw * out["tau_tw"]) / Yp
    nu_f = mf / rf
    H = (Ra * nu_f * (nu_f / Pr) / (g * bf * dT)) ** (1 / 3)
    dx = H / ny
    dt = nu * dx * dx / nu_f  # lattice viscosity nu (dx^2/dt) is the physical one
    out["H_phys"], out["dx"], out["dt"] = H, dx, dt
    out["C_F"] = dt * dt / (rf * dx)
    out["g_lb"] = g * dt * dt / dx
    out["beta_St"] = 18 * mu_ns / (rp * d * d)
    kst = k_ns / kp
    Kn = lf / d
    out["K_T"] = (6 * math.pi * 1.17 * (kst + 2.18 * Kn)
                  / ((1 + 3 * 1.14 * Kn) * (1 + 2 * kst + 2 * 2.18 * Kn)))
    return out


@pytest.mark.parametrize("nx,ny,Ra,Pr,phi,d", [(32, 32, 1e3, 6.2, 0.01, 20e-9),
                                               (256, 256, 1e5, 6.2, 0.03, 30e-9),
                                               (40, 20, 1e6, 8.923, 0.04, 33e-9),
                                               (64, 64, 1e4, 6.2, 0.0, 50e-9)])
def test_constants_independent(oracle_mod, nx, ny, Ra, Pr, phi, d):
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=phi, d_p=d)
    c = s.consts()
    ind = _independent_constants(nx, ny, Ra, Pr, phi, d)
    for k, v in ind.items():
        assert abs(c[k] - v) <= 1e-13 * abs(v), k
    # lattice buoyancy of the base fluid equals g beta dT in lattice units
    assert abs(c["g_lb"] * 2.1e-4 * 10.0 - c["G_B"]) < 1e-12 * c["G_B"]
    # Eq 23 read back: the mixture viscosity from the mass-fraction average of tau
    nu_mix = (2 * (c["Y_w0"] * c["tau_w"] + c["Y_p0"] * c["tau_p"]) - 1) / 6
    assert abs(nu_mix - c["nu_ns"]) < 1e-13 * c["nu_ns"]
    # C_F converts a force density: rho_f * g (N/m^3) becomes g_lb in lattice units
    assert abs(997.1 * 9.81 * c["C_F"] - c["g_lb"]) < 1e-13 * c["g_lb"]


def test_invalid_parameters(oracle_mod):
    with pytest.raises(oracle_mod.RefError):
        ref_solver(oracle_mod, 1, 8)
    with pytest.raises(oracle_mod.RefError):
        ref_solver(oracle_mod, phi=0.3)
    with pytest.raises(oracle_mod.RefError):
        ref_solver(oracle_mod, Ra=-1.0)
    with pytest.raises(oracle_mod.RefError):  # Ra 1e8 on 8x8 gives tau_theta <= 0.501
        ref_solver(oracle_mod, 8, 8, Ra=1e8)


# ---------------------------------------------------------------- P10: Poiseuille
def test_poiseuille_curvature(oracle_mod):
    """Periodic channel driven by a uniform force between bounce-back walls: the steady BGK
    profile is a parabola whose curvature is -F/(rho nu) with nu = (tau - 1/2)/3."""
    ny, F = 16, 1e-6
    s = ref_solver(oracle_mod, 4, ny, Ra=1e3, Pr=1.0, phi=0.0, force_mask=0, periodic_x=1,
                   body_fx=F).init()
    s.step(30000)
    c = s.consts()
    ux = s.fields(oracle_mod.UX)[0]
    assert np.abs(ux - ux[:, :1]).max() < 1e-16  # uniform along the channel
    u = ux[:, 0]
    y = np.arange(ny) + 0.5
    p = np.polyfit(y, u, 2)
    assert np.abs(np.polyval(p, y) - u).max() < 1e-9 * u.max()
    nu = (c["tau_w"] - 0.5) / 3
    assert abs(2 * p[0] - (-F / nu)) < 1e-6 * F / nu
    # no-slip near the halfway walls: the parabola's roots sit within O(1e-2) of the walls
    r = np.sort(np.roots(p).real)
    assert abs(r[0]) < 0.05 and abs(r[1] - ny) < 0.05


# ---------------------------------------------------------------- slip-force drifts
def _post_collision_slip(st, i, j):
    fw, fp = st[:9, j, i], st[9:18, j, i]
    uw = (fw[:, None] * E).sum(0) / fw.sum()
    up = (fp[:, None] * E).sum(0) / fp.sum()
    return up - uw


def _one_step_pair(oracle, mask_on, mask_off, warm, nx, ny, **kw):
    out = []
    for m in (mask_on, mask_off):
        s = ref_solver(oracle, nx, ny, force_mask=m, **kw)
        s.init(warm=warm)
        s.step(1)
        out.append((s, s.get_state()))
    return out


def test_thermophoretic_terminal_drift(oracle_mod):
    """With drag, a thermophoretic force on the particle phase makes the particles drift at
    the Brock-type velocity v_T of Table 1 relative to the fluid (hot to cold)."""
    nx, ny, phi, d = 16, 8, 0.01, 20e-9
    base = oracle_mod.F_DRAG
    x = (np.arange(nx) + 0.5) / nx
    z = np.zeros((ny, nx))
    th = np.broadcast_to(0.5 - x[None, :], (ny, nx))
    warm = np.stack([z, z, th, z + phi])
    (s_on, st_on), (s_off, st_off) = _one_step_pair(
        oracle_mod, base | oracle_mod.F_THERMOPHORESIS, base, warm, nx, ny, phi=phi, d_p=d)
    c = s_on.consts()
    i, j = 7, 4
    drift = _post_collision_slip(st_on, i, j) - _post_collision_slip(st_off, i, j)
    # independent Table 1 evaluation: dT/dx = -dT_K / H_x, T at the node
    T = 298.15 + (0.5 - x[i]) * 10.0
    dTdx = -10.0 / (nx * c["dx"])
    v_T = -c["K_T"] * (c["mu_ns"] / c["rho_ns"]) * dTdx / T  # m/s
    v_lb = v_T * c["dt"] / c["dx"]
    assert v_lb > 0  # hot (left) to cold (right)
    assert abs(drift[0] - v_lb) < 1e-4 * v_lb
    assert abs(drift[1]) < 1e-9 * v_lb


def test_brownian_drift_down_gradient(oracle_mod):
    """Brownian force with drag: the particles drift down the concentration gradient at
    rho_p D_B A_p v_B |grad phi| / (m_p beta_St) (Table 1, terminal Stokes drift)."""
    nx, ny, phi, d = 12, 8, 0.02, 10e-9
    base = oracle_mod.F_DRAG
    x = (np.arange(nx) + 0.5) / nx
    z = np.zeros((ny, nx))
    ph = np.broadcast_to(phi * (1 + 0.2 * (x - 0.5))[None, :], (ny, nx))
    warm = np.stack([z, z, z, ph])
    (s_on, st_on), (s_off, st_off) = _one_step_pair(
        oracle_mod, base | oracle_mod.F_BROWNIAN, base, warm, nx, ny, phi=phi, d_p=d)
    c = s_on.consts()
    i, j = 6, 3
    drift = _post_collision_slip(st_on, i, j) - _post_collision_slip(st_off, i, j)
    T = 298.15
    mu = c["mu_ns"]
    D_B = 2 * KB * T / (3 * math.pi * mu * d)
    v_B = 2 * KB * T / (math.pi * mu * d * d)
    gphi = phi * 0.2 / (nx * c["dx"])  # per metre
    m_p = 3970.0 * math.pi * d ** 3 / 6
    v = -3970.0 * D_B * gphi * (math.pi * d * d) * v_B / (m_p * c["beta_St"])
    v_lb = v * c["dt"] / c["dx"]
    assert v_lb < 0
    assert abs(drift[0] - v_lb) < 1e-3 * abs(v_lb)


def test_saffman_and_magnus_invariants(oracle_mod):
    s = ref_solver(oracle_mod, 20, 20, Ra=1e5, phi=0.03, d_p=50e-9).init().step(300)
    seen_magnus_sign = set()
    for i, j in [(2, 9), (9, 2), (17, 11), (11, 17), (5, 5), (9, 10), (1, 15)]:
        t = s.node_terms(i, j)
        w = t["uw"] - t["up"]
        FS = t["F_S"]
        # lift is perpendicular to the slip and turned counter-clockwise from it
        assert abs(FS @ w) <= 1e-12 * np.linalg.norm(FS) * np.linalg.norm(w)
        assert FS[0] * w[1] - FS[1] * w[0] <= 0 or np.linalg.norm(FS) == 0
        # Magnus migration is along the inward normal of the nearest wall
        FM = t["F_M"]
        dists = {"l": i + 0.5, "r": 20 - i - 0.5, "b": j + 0.5, "t": 20 - j - 0.5}
        near = min(dists, key=dists.get)
        nrm = {"l": (1, 0), "r": (-1, 0), "b": (0, 1), "t": (0, -1)}[near]
        assert abs(FM[0] * nrm[1] - FM[1] * nrm[0]) <= 1e-15 * np.linalg.norm(FM) + 1e-300
        zH = 2 * dists[near] / 20
        proj = FM @ np.array(nrm)
        if np.linalg.norm(FM) > 0:
            seen_magnus_sign.add(np.sign(proj) == np.sign(0.63 - zH))
    assert seen_magnus_sign == {True}


def test_warm_init_with_density(oracle_mod):
    """MCLBM_INIT_WARM_RHO: the fluid populations' zeroth moment is the given rho^w, the
    particle and thermal sets are those of the 4-field warm start, and rho^w = 1 - phi gives
    exactly the 4-field state."""
    import numpy as np
    ny, nx = 12, 16
    rng = np.random.default_rng(0)
    w5 = np.stack([rng.normal(size=(ny, nx)) * 1e-3, rng.normal(size=(ny, nx)) * 1e-3,
                   rng.normal(size=(ny, nx)) * 0.1, 0.02 + rng.normal(size=(ny, nx)) * 1e-4,
                   0.98 + rng.normal(size=(ny, nx)) * 1e-3])
    r5 = oracle_mod.RefSolver(nx, ny, 1e4, 6.2, 0.02, 30e-9).init(warm=w5)
    r4 = oracle_mod.RefSolver(nx, ny, 1e4, 6.2, 0.02, 30e-9).init(warm=w5[:4])
    s5, s4 = r5.get_state(), r4.get_state()
    np.testing.assert_allclose(s5[:9].sum(axis=0), w5[4], rtol=1e-14)
    np.testing.assert_array_equal(s5[9:], s4[9:])
    w = w5.copy()
    w[4] = 1.0 - w[3]
    r = oracle_mod.RefSolver(nx, ny, 1e4, 6.2, 0.02, 30e-9).init(warm=w)
    np.testing.assert_array_equal(r.get_state(), s4)


# ---------------------------------------------------------------- Table 1 magnitudes
# A uniform state: every node holds the same equilibrium populations, so the nodes that touch
# no wall see exactly these populations after streaming and every gradient there is zero.
def _uniform_state(nx, ny, rho_w, uw, rho_p, up, theta, u_g=(0.0, 0.0), g_extra=None):
    def feq(rho, u):
        eu = E[:, 0] * u[0] + E[:, 1] * u[1]
        return W * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u[0] ** 2 + u[1] ** 2))
    node = np.concatenate([feq(rho_w, uw), feq(rho_p, up), feq(theta, u_g)])
    if g_extra is not None:
        node[18:] += g_extra
    return np.broadcast_to(node[:, None, None], (27, ny, nx)).copy()


def _set_uniform(s, nx, ny, **kw):
    s.init()
    s.set_state(_uniform_state(nx, ny, **kw))
    return s


def _si_scales(nx, ny, Ra, Pr, phi, d):
    ind = _independent_constants(nx, ny, Ra, Pr, phi, d)
    ind["vel"] = ind["dx"] / ind["dt"]
    return ind


def test_saffman_lift_is_saffmans_sphere_lift(oracle_mod):
    """Table 1 Saffman lift (K_S/4) mu |w| d_p^2 sqrt(rho gamma/mu) with K_S = 81.2 is Saffman's
    lift on a sphere of radius a = d_p/2 in his original form, 81.2 mu a^2 |w| sqrt(gamma/nu):
    the same magnitude written per radius. Per volume it is n_p = phi/V_p times that, with the
    shear rate gamma = 8 |u^p|/H; it points along the slip turned by +90 degrees."""
    nx = ny = 12
    Ra, Pr, phi, d = 1e5, 6.2, 0.03, 30e-9
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=phi, d_p=d,
                   force_mask=oracle_mod.F_SAFFMAN)
    c = s.consts()
    si = _si_scales(nx, ny, Ra, Pr, phi, d)
    rho_w, rho_p = 0.95 * c["rho_w0"], 1.2 * c["rho_p0"]
    uw, up = np.array([2e-3, -1e-3]), np.array([5e-4, 1.5e-3])
    _set_uniform(s, nx, ny, rho_w=rho_w, uw=uw, rho_p=rho_p, up=up, theta=0.1)
    t = s.node_terms(6, 5)
    np.testing.assert_allclose(t["uw"], uw, rtol=1e-12)
    np.testing.assert_allclose(t["up"], up, rtol=1e-12)
    w = (uw - up) * si["vel"]                               # slip, m/s
    gamma = 8 * np.linalg.norm(up) * si["vel"] / si["H_phys"]
    nu_ns = si["mu_ns"] / si["rho_ns"]
    a = d / 2
    lift = 81.2 * si["mu_ns"] * a * a * np.linalg.norm(w) * math.sqrt(gamma / nu_ns)  # N
    n_p = (rho_p * 997.1 / 3970.0) / (math.pi * d ** 3 / 6)
    direction = np.array([-w[1], w[0]]) / np.linalg.norm(w)
    expect = n_p * lift * si["C_F"] * direction
    np.testing.assert_allclose(t["F_S"], expect, rtol=1e-12)


def _saffman_at(oracle_mod, uw, up, d, nx=12, ny=12):
    s = ref_solver(oracle_mod, nx, ny, Ra=1e5, Pr=6.2, phi=0.03, d_p=d,
                   force_mask=oracle_mod.F_SAFFMAN)
    c = s.consts()
    _set_uniform(s, nx, ny, rho_w=c["rho_w0"], uw=np.asarray(uw), rho_p=c["rho_p0"],
                 up=np.asarray(up), theta=0.0)
    return s.node_terms(6, 6)["F_S"]


def test_saffman_scaling_exponents(oracle_mod):
    """The lift is linear in the slip, goes as the square root of the particle speed (through
    the shear rate 8 |u^p|/H), and per unit volume as 1/d_p (n_p d_p^2 ~ d_p^-1)."""
    uw, up, d = np.array([1e-3, 2e-3]), np.array([-4e-4, 7e-4]), 30e-9
    F = _saffman_at(oracle_mod, uw, up, d)
    # slip x 3 at the same particle velocity
    F3 = _saffman_at(oracle_mod, up + 3 * (uw - up), up, d)
    np.testing.assert_allclose(F3, 3 * F, rtol=1e-12)
    # particle velocity x 4 at the same slip: sqrt(4) = 2
    F4 = _saffman_at(oracle_mod, uw + 3 * up, 4 * up, d)
    np.testing.assert_allclose(F4, 2 * F, rtol=1e-12)
    # particle diameter x 2
    F2 = _saffman_at(oracle_mod, uw, up, 2 * d)
    np.testing.assert_allclose(F2, 0.5 * F, rtol=1e-12)


def _magnus_row(oracle_mod, uw, up, d, nx=40, ny=40, j=20, cols=range(1, 15)):
    s = ref_solver(oracle_mod, nx, ny, Ra=1e5, Pr=6.2, phi=0.03, d_p=d,
                   force_mask=oracle_mod.F_MAGNUS)
    c = s.consts()
    _set_uniform(s, nx, ny, rho_w=c["rho_w0"], uw=np.asarray(uw), rho_p=c["rho_p0"],
                 up=np.asarray(up), theta=0.0)
    return np.array([s.node_terms(i, j)["F_M"] for i in cols])


def test_magnus_migration_magnitude(oracle_mod):
    """Table 1 Magnus migration v_M = 0.34 (vbar^2 H/nu)(d_p/H)^2.84 (2z/H)(0.63 - 2z/H) along the
    inward normal of the nearest wall, with vbar = |u^w + u^p|/2 and z the distance to that wall,
    acting through m_dot_p = m_p beta_St: per unit volume phi rho_p beta_St v_M. Evaluated in SI
    with independently derived scales, along a row whose nearest wall is the hot wall."""
    nx = ny = 40
    Ra, Pr, phi, d = 1e5, 6.2, 0.03, 30e-9
    uw, up = np.array([3e-3, -2e-3]), np.array([2.5e-3, -1e-3])
    cols = list(range(1, 15))
    FM = _magnus_row(oracle_mod, uw, up, d, cols=cols)
    si = _si_scales(nx, ny, Ra, Pr, phi, d)
    H = si["H_phys"]
    nu_ns = si["mu_ns"] / si["rho_ns"]
    vbar = 0.5 * np.linalg.norm(uw + up) * si["vel"]
    beta_st = 18 * si["mu_ns"] / (3970.0 * d * d)
    phi_loc = phi  # the node holds the initial partial density
    for k, i in enumerate(cols):
        z = (i + 0.5) * si["dx"]
        zh = 2 * z / H
        v_M = 0.34 * (vbar ** 2 * H / nu_ns) * (d / H) ** 2.84 * zh * (0.63 - zh)
        expect = phi_loc * 3970.0 * beta_st * v_M * si["C_F"]
        assert abs(FM[k][0] - expect) <= 1e-12 * abs(expect) + 1e-30
        assert FM[k][1] == 0.0


def test_magnus_scaling_exponents(oracle_mod):
    """Per unit volume the Magnus force goes as d_p^0.84 (beta_St ~ d_p^-2 times (d_p/H)^2.84),
    as vbar^2, and along the wall normal as the profile (2z/H)(0.63 - 2z/H)."""
    uw, up, d = np.array([3e-3, -2e-3]), np.array([2.5e-3, -1e-3]), 30e-9
    cols = list(range(1, 15))
    F = _magnus_row(oracle_mod, uw, up, d, cols=cols)[:, 0]
    F2 = _magnus_row(oracle_mod, uw, up, 2 * d, cols=cols)[:, 0]
    np.testing.assert_allclose(F2, 2 ** 0.84 * F, rtol=1e-12)
    Fv = _magnus_row(oracle_mod, 2 * uw, 2 * up, d, cols=cols)[:, 0]
    np.testing.assert_allclose(Fv, 4 * F, rtol=1e-12)
    zh = 2 * (np.array(cols) + 0.5) / 40
    prof = zh * (0.63 - zh)
    ratio = F / prof
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-12)
    assert np.all(np.sign(F) == np.sign(prof))


def test_gravity_is_table1_weight_less_buoyancy(oracle_mod):
    """Table 1 gravity -V_p (rho_p - rho_f) g per particle, n_p = phi/V_p per volume: with only
    gravity on, one step changes the particle momentum at a node by exactly that force density
    (converted with an independently derived force scale), downward, and the fluid's by the
    uniform part phi_0 (rho_p - rho_f) g upward (the Boussinesq reference), so a node's total is
    the weight of its particle excess only."""
    nx = ny = 10
    Ra, Pr, phi, d = 1e4, 6.2, 0.02, 40e-9
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=phi, d_p=d,
                   force_mask=oracle_mod.F_GRAVITY)
    c = s.consts()
    si = _si_scales(nx, ny, Ra, Pr, phi, d)
    rho_p = 1.25 * c["rho_p0"]
    z2 = np.zeros(2)
    _set_uniform(s, nx, ny, rho_w=c["rho_w0"], uw=z2, rho_p=rho_p, up=z2, theta=0.0)
    s.step(1)
    st = s.get_state()
    i, j = 4, 5
    dmp = (st[9:18, j, i][:, None] * E).sum(0)   # particle momentum after one step (it was 0)
    dmw = (st[0:9, j, i][:, None] * E).sum(0)
    phi_loc = rho_p * 997.1 / 3970.0
    g = 9.81
    Fp = -phi_loc * (3970.0 - 997.1) * g * si["C_F"]
    Fw = phi * (3970.0 - 997.1) * g * si["C_F"]
    assert Fp < 0 < Fw
    assert abs(dmp[1] - Fp) <= 1e-12 * abs(Fp) and abs(dmp[0]) < 1e-16
    assert abs(dmw[1] - Fw) <= 1e-12 * abs(Fw) and abs(dmw[0]) < 1e-16
    assert abs((dmp + dmw)[1] + 0.25 * Fw) <= 1e-11 * abs(Fw)


def test_buoyancy_uses_eq9_expansion(oracle_mod):
    """Eq 2's Boussinesq force rho_ns beta_ns g (T - T_ref) with the volume-weighted expansion
    coefficient of Eq 9, evaluated in SI (T - T_ref = theta dT) and converted with an
    independently derived force scale."""
    nx = ny = 10
    Ra, Pr, phi, d = 1e4, 6.2, 0.04, 40e-9
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=phi, d_p=d,
                   force_mask=oracle_mod.F_BUOYANCY)
    c = s.consts()
    si = _si_scales(nx, ny, Ra, Pr, phi, d)
    beta_ns = phi * 0.85e-5 + (1 - phi) * 2.1e-4       # Eq 9 as printed
    assert abs(c["beta_ratio"] - beta_ns / 2.1e-4) <= 1e-14
    rho_w, rho_p, theta = 0.97 * c["rho_w0"], 1.1 * c["rho_p0"], 0.3
    z2 = np.zeros(2)
    _set_uniform(s, nx, ny, rho_w=rho_w, uw=z2, rho_p=rho_p, up=z2, theta=theta)
    t = s.node_terms(5, 4)
    assert abs(t["theta"] - theta) < 1e-15
    rho_si = (rho_w + rho_p) * 997.1
    expect = rho_si * beta_ns * 9.81 * theta * 10.0 * si["C_F"]
    assert abs(t["F_buoy"][1] - expect) <= 1e-12 * expect and t["F_buoy"][0] == 0.0


@pytest.mark.parametrize("scale_p", [0.5, 2.0])
def test_thermal_relaxation_uses_local_mass_fractions(oracle_mod, scale_p):
    """Eq 24 with the local mass fractions of Eq 25: a node whose particle partial density differs
    from the initial one relaxes g towards its equilibrium at tau_theta = Y_w tau_theta^w +
    Y_p tau_theta^p of its own fractions (not of the initial ones)."""
    nx = ny = 8
    Ra, Pr, phi, d = 1e4, 6.2, 0.04, 30e-9
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=phi, d_p=d, force_mask=0)
    c = s.consts()
    ind = _independent_constants(nx, ny, Ra, Pr, phi, d)
    rho_w, rho_p, theta = c["rho_w0"], scale_p * c["rho_p0"], 0.2
    # a non-equilibrium part with zero sum (theta unchanged) and a heat flux
    delta = np.array([0.0, 1.0, -0.5, -1.0, 0.5, 0.25, -0.25, -0.25, 0.25]) * 1e-3
    delta[0] = -delta[1:].sum()
    z2 = np.zeros(2)
    _set_uniform(s, nx, ny, rho_w=rho_w, uw=z2, rho_p=rho_p, up=z2, theta=theta,
                 g_extra=delta)
    s.step(1)
    g_after = s.get_state()[18:, 4, 3]
    d_after = g_after - W * theta
    tau = delta[1:] / (delta[1:] - d_after[1:])
    Yw, Yp = rho_w / (rho_w + rho_p), rho_p / (rho_w + rho_p)
    expect = Yw * ind["tau_tw"] + Yp * ind["tau_tp"]
    np.testing.assert_allclose(tau, expect, rtol=1e-10)
    # the initial fractions' tau differs by far more than the 1e-10 this test resolves
    at_initial = ind["tau_tw"] * c["Y_w0"] + ind["tau_tp"] * c["Y_p0"]
    assert abs(expect - at_initial) > 1e-5 * at_initial


def test_residual_from_field_snapshots(oracle_mod):
    """The steady-state residual: max over u, theta and phi of ||q_now - q_then||_2 /
    (K ||q_now||_2), K the steps between the two snapshots, recomputed from the fields."""
    s = ref_solver(oracle_mod, 20, 16, Ra=1e4, phi=0.02, d_p=30e-9).init()
    s.step(150)
    s.residual()  # snapshot at step 150
    which = oracle_mod.UX | oracle_mod.UY | oracle_mod.THETA | oracle_mod.PHI
    then = s.fields(which)
    s.step(70)
    now = s.fields(which)
    r = s.residual()
    K = 70
    terms = []
    for sel in ([0, 1], [2], [3]):
        num = np.sqrt(((now[sel] - then[sel]) ** 2).sum())
        den = np.sqrt((now[sel] ** 2).sum())
        terms.append(num / (K * den))
    assert r > 0 and abs(r - max(terms)) <= 1e-12 * r


# ---------------------------------------------------------------- two thermal sets (Eq 19 x 2)
def _two_set_uniform(nx, ny, rho_w, rho_p, th_w, th_p):
    """Rest state, uniform partial densities and set temperatures (absolute populations)."""
    node = np.concatenate([W * rho_w, W * rho_p, W * th_w, W * th_p])
    return np.broadcast_to(node[:, None, None], (36, ny, nx)).copy()


def test_two_sets_reduce_to_one_set(oracle_mod):
    """With equal thermal relaxation times and equal initial sets, the two-set model (g^w, g^p
    relaxing to the mixture temperature of Eq 33) stays with g^w = g^p and is the one-set model:
    the same fields and Nusselt numbers (to rounding: the mixture weights and the local tau of
    Eq 24 sum to one only to an ulp)."""
    nx, ny, Ra, phi, d = 24, 20, 2e4, 0.03, 30e-9
    tau = ref_solver(oracle_mod, nx, ny, Ra=Ra, phi=phi, d_p=d).consts()["tau_tw"]
    one = ref_solver(oracle_mod, nx, ny, Ra=Ra, phi=phi, d_p=d, tau_tp_override=tau).init()
    two = ref_solver(oracle_mod, nx, ny, Ra=Ra, phi=phi, d_p=d, tau_tp_override=tau,
                     thermal_sets=2).init()
    one.step(400)
    two.step(400)
    st = two.get_state()
    assert st.shape[0] == 36
    np.testing.assert_allclose(st[27:36], st[18:27], rtol=0, atol=1e-14)
    which = (oracle_mod.UX | oracle_mod.UY | oracle_mod.THETA | oracle_mod.PHI | oracle_mod.RHO_W
             | oracle_mod.UPX | oracle_mod.UPY)
    a, b = one.fields(which), two.fields(which)
    assert np.abs(a[0]).max() > 1e-4  # the flow is there
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(two.nusselt(), one.nusselt(), rtol=1e-12)


def test_two_sets_conduction_limit(oracle_mod):
    """No buoyancy, gravity or thermophoresis: both sets and the mixture settle on the exact
    linear conduction profile, Nu = k_ns/k_f, whatever their relaxation times."""
    mask = oracle_mod.F_DRAG | oracle_mod.F_BROWNIAN | oracle_mod.F_SAFFMAN | oracle_mod.F_MAGNUS
    s = ref_solver(oracle_mod, 12, 9, Ra=1e3, phi=0.02, force_mask=mask, thermal_sets=2).init()
    c = s.consts()
    assert abs(c["tau_tw"] - c["tau_tp"]) > 1e-3  # distinct relaxation times
    s.step(50)
    nh, nc = s.nusselt()
    assert abs(nh - c["k_ratio"]) < 1e-10 and abs(nc - c["k_ratio"]) < 1e-10
    x = (np.arange(12) + 0.5) / 12
    for f in s.fields(oracle_mod.THETA | oracle_mod.THETA_W | oracle_mod.THETA_P):
        assert np.max(np.abs(f - (0.5 - x)[None, :])) < 1e-12


def test_two_sets_equilibrate_at_mixture_temperature(oracle_mod):
    """One step from rest with uniform but different set temperatures (periodic in x, no
    forces): each set relaxes by 1/tau_theta^sigma towards the mixture temperature
    (rho^w theta^w + r rho^p theta^p) / (rho^w + r rho^p), r = C_p,p / C_p,f (Eq 33 with the
    components' heat capacities), tau_theta^w from the base fluid's diffusivity and tau_theta^p
    from Eq 24 at the initial fractions (both derived independently)."""
    nx, ny, Ra, Pr, phi, d = 6, 8, 1e4, 6.2, 0.04, 30e-9
    s = ref_solver(oracle_mod, nx, ny, Ra=Ra, Pr=Pr, phi=phi, d_p=d, force_mask=0, periodic_x=1,
                   thermal_sets=2)
    c = s.consts()
    ind = _independent_constants(nx, ny, Ra, Pr, phi, d)
    rho_w, rho_p, th_w, th_p = c["rho_w0"], 1.3 * c["rho_p0"], 0.3, -0.2
    s.init()
    s.set_state(_two_set_uniform(nx, ny, rho_w, rho_p, th_w, th_p))
    s.step(1)
    th = s.fields(oracle_mod.THETA_W | oracle_mod.THETA_P)
    r = 765.0 / 4179.0
    th_ns = (rho_w * th_w + r * rho_p * th_p) / (rho_w + r * rho_p)
    exp_w = th_w - (th_w - th_ns) / ind["tau_tw"]
    exp_p = th_p - (th_p - th_ns) / ind["tau_tp"]
    np.testing.assert_allclose(th[0], exp_w, rtol=1e-12)
    np.testing.assert_allclose(th[1], exp_p, rtol=1e-12)
    # the mixture temperature the fields report after the step is Eq 33 of the new set values
    mix = s.fields(oracle_mod.THETA)[0]
    np.testing.assert_allclose(mix, (rho_w * exp_w + r * rho_p * exp_p) / (rho_w + r * rho_p),
                               rtol=1e-12)


def test_two_sets_conserve_enthalpy_at_equal_tau(oracle_mod):
    """Closed box (periodic in x, adiabatic top and bottom), fluid at rest, no forces, equal
    relaxation times: streaming and the relaxation towards the Eq 33 mixture temperature
    conserve the total enthalpy sum(rho^w theta^w + r rho^p theta^p) from nonuniform set
    temperatures."""
    nx, ny = 10, 12
    tau = ref_solver(oracle_mod, nx, ny, Ra=1e4, phi=0.03, d_p=30e-9).consts()["tau_tw"]
    s = ref_solver(oracle_mod, nx, ny, Ra=1e4, phi=0.03, d_p=30e-9, force_mask=0, periodic_x=1,
                   thermal_sets=2, tau_tp_override=tau)
    c = s.consts()
    rng = np.random.default_rng(7)
    st = _two_set_uniform(nx, ny, c["rho_w0"], c["rho_p0"], 0.0, 0.0)
    thw = rng.uniform(-0.5, 0.5, (ny, nx))
    thp = rng.uniform(-0.5, 0.5, (ny, nx))
    st[18:27] = W[:, None, None] * thw[None]
    st[27:36] = W[:, None, None] * thp[None]
    s.init()
    s.set_state(st)
    r = 765.0 / 4179.0

    def enthalpy():
        f = s.fields(oracle_mod.RHO_W | oracle_mod.RHO_P | oracle_mod.THETA_W | oracle_mod.THETA_P)
        return (f[0] * f[2] + r * f[1] * f[3]).sum()
    h0 = enthalpy()
    s.step(200)
    f = s.fields(oracle_mod.THETA_W | oracle_mod.THETA_P)
    assert np.abs(f[0] - f[1]).max() < 0.5 * np.abs(thw - thp).max()  # the sets exchanged heat
    assert abs(enthalpy() - h0) <= 1e-12 * np.abs(thw).sum()
