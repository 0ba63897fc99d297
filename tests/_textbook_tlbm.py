"""Independent textbook thermal D2Q9 BGK lattice Boltzmann scheme (single component).

This is the classical Boussinesq double-population scheme: one BGK set f for the flow with
the simple forcing term 3 W_q e_q.F and one BGK set g for the temperature, both advected
with u = sum(f e)/sum(f), walls half a link outside the outer nodes (bounce-back for f,
anti-bounce-back for g at the isothermal side walls, mirror reflection of g at the adiabatic
top and bottom walls, corners take the side-wall rule).

It is written in vectorised numpy, push-free and shift-based, with no code shared with the
oracle, and is the reference the oracle must reproduce when the particle fraction is zero.
"""
import numpy as np

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = [int(np.where((E == -E[q]).all(1))[0][0]) for q in range(9)]
MIR = [int(np.where((E == E[q] * np.array([1, -1])).all(1))[0][0]) for q in range(9)]


def equilibrium(rho, ux, uy):
    eu = E[:, 0, None, None] * ux + E[:, 1, None, None] * uy
    usq = ux * ux + uy * uy
    return W[:, None, None] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * usq)


def _shifted(a, ex, ey):
    """out[j, i] = a[j - ey, i - ex] where that index exists, NaN elsewhere."""
    ny, nx = a.shape
    out = np.full_like(a, np.nan)
    out[max(ey, 0):ny + min(ey, 0), max(ex, 0):nx + min(ex, 0)] = \
        a[max(-ey, 0):ny + min(-ey, 0), max(-ex, 0):nx + min(-ex, 0)]
    return out


class TextbookTLBM:
    def __init__(self, nx, ny, tau, tau_t, G, T_hot=0.5, T_cold=-0.5):
        self.nx, self.ny = nx, ny
        self.tau, self.tau_t, self.G = tau, tau_t, G
        self.Th, self.Tc = T_hot, T_cold
        x = np.arange(nx)
        self.i = np.broadcast_to(x[None, :], (ny, nx))
        th = np.broadcast_to(0.5 - (x[None, :] + 0.5) / nx, (ny, nx)).copy()
        z = np.zeros((ny, nx))
        self.f = equilibrium(np.ones((ny, nx)), z, z)
        self.g = equilibrium(th, z, z)

    def _stream(self):
        f, g = self.f, self.g
        fs, gs = np.empty_like(f), np.empty_like(g)
        for q in range(9):
            ex, ey = E[q]
            a = _shifted(f[q], ex, ey)
            fs[q] = np.where(np.isnan(a), f[OPP[q]], a)
            b = _shifted(g[q], ex, ey)
            src_i = self.i - ex
            side = (src_i < 0) | (src_i >= self.nx)
            Tw = np.where(src_i < 0, self.Th, self.Tc)
            anti = -g[OPP[q]] + 2 * W[q] * Tw
            # mirror: population that left (i - ex, j) with velocity (ex, -ey)
            mir = _shifted(g[MIR[q]], ex, 0)
            gs[q] = np.where(np.isnan(b), np.where(side, anti, mir), b)
        return fs, gs

    def moments(self):
        fs, gs = self._stream()
        rho = fs.sum(0)
        ux = (fs * E[:, 0, None, None]).sum(0) / rho
        uy = (fs * E[:, 1, None, None]).sum(0) / rho
        return fs, gs, rho, ux, uy, gs.sum(0)

    def step(self, n=1):
        for _ in range(n):
            fs, gs, rho, ux, uy, th = self.moments()
            Fy = rho * self.G * th
            force = 3 * W[:, None, None] * (E[:, 1, None, None] * Fy)
            self.f = fs - (fs - equilibrium(rho, ux, uy)) / self.tau + force
            self.g = gs - (gs - equilibrium(th, ux, uy)) / self.tau_t
        return self

    def nusselt_hot(self):
        th = self.moments()[5]
        grad = (8 * self.Th - 9 * th[:, 0] + th[:, 1]) / 3
        return grad.mean() * self.nx / (self.Th - self.Tc)
