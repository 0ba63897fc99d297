"""ctypes wrapper of the FP64 CPU oracle (oracle/mclbm_ref.c).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU-baseline leg use
it. It shares no code with the CUDA library and never imports it.
"""
import ctypes as C

import numpy as np

from . import build as _build

F_BROWNIAN, F_THERMOPHORESIS, F_DRAG, F_SAFFMAN, F_MAGNUS, F_GRAVITY, F_BUOYANCY = (
    1, 2, 4, 8, 16, 32, 64)
F_ALL = 127
UX, UY, THETA, PHI, RHO_W, RHO_P, UPX, UPY = 1, 2, 4, 8, 16, 32, 64, 128
THETA_W, THETA_P = 256, 512  # the thermal sets' own temperatures (= THETA with one set)
INIT_REST, INIT_WARM, INIT_WARM_RHO = 0, 2, 3


class RefProps(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "rho_f", "cp_f", "k_f", "beta_f", "mu_f", "rho_p", "cp_p", "k_p", "beta_p",
        "T0", "dT", "g", "l_f", "Ma")] + [
        ("force_mask", C.c_uint32), ("periodic_x", C.c_int), ("body_fx", C.c_double),
        ("thermal_sets", C.c_int), ("tau_tp_override", C.c_double)]


CONST_NAMES = (
    "U0", "nu_w", "alpha_w", "G_B",
    "rho_ratio", "rhocp_ratio", "beta_ratio", "k_ratio", "mu_ratio", "Re_T",
    "nu_ns", "alpha_ns",
    "rho_w0", "rho_p0", "Y_w0", "Y_p0",
    "tau_w", "tau_p", "tau_tw", "tau_tp",
    "H_phys", "dx", "dt", "C_F", "g_lb",
    "mu_ns", "rho_ns", "k_ns", "nu_ns_SI",
    "V_p", "A_p", "m_p", "beta_St", "Kn", "kstar", "K_T")


class RefConsts(C.Structure):
    _fields_ = [(n, C.c_double) for n in CONST_NAMES]


_V2 = C.c_double * 2
TERM_FIELDS = [("rho_w", C.c_double), ("rho_p", C.c_double), ("theta", C.c_double),
               ("phi", C.c_double), ("u", _V2), ("uw", _V2), ("up", _V2),
               ("grad_theta", _V2), ("grad_phi", _V2), ("F_B", _V2), ("F_T", _V2),
               ("F_S", _V2), ("F_M", _V2), ("F_G", _V2), ("F_buoy", _V2), ("F_G0", _V2),
               ("beta_lb", C.c_double), ("a", C.c_double), ("J", _V2), ("F_w", _V2),
               ("F_p", _V2), ("tau_theta", C.c_double)]


class RefTerms(C.Structure):
    _fields_ = TERM_FIELDS


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.mclbm_ref_props_default.argtypes = [C.POINTER(RefProps)]
        L.mclbm_ref_props_default.restype = None
        L.mclbm_ref_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.POINTER(RefProps), C.POINTER(C.c_void_p)]
        L.mclbm_ref_destroy.argtypes = [C.c_void_p]
        L.mclbm_ref_destroy.restype = None
        L.mclbm_ref_consts.argtypes = [C.c_void_p, C.POINTER(RefConsts)]
        L.mclbm_ref_init.argtypes = [C.c_void_p, C.c_int, dp]
        L.mclbm_ref_step.argtypes = [C.c_void_p, C.c_int64]
        L.mclbm_ref_stream_only.argtypes = [C.c_void_p]
        L.mclbm_ref_fields.argtypes = [C.c_void_p, C.c_uint32, dp]
        L.mclbm_ref_nusselt.argtypes = [C.c_void_p, dp, dp]
        L.mclbm_ref_mass.argtypes = [C.c_void_p, dp, dp]
        L.mclbm_ref_residual.argtypes = [C.c_void_p, dp]
        L.mclbm_ref_get_state.argtypes = [C.c_void_p, dp]
        L.mclbm_ref_set_state.argtypes = [C.c_void_p, dp]
        L.mclbm_ref_node_terms.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(RefTerms)]
        L.mclbm_ref_steps_done.argtypes = [C.c_void_p]
        L.mclbm_ref_steps_done.restype = C.c_int64
        L.mclbm_ref_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.mclbm_ref_equilibrium.restype = None
        L.mclbm_ref_drag_impulse.argtypes = [C.c_double, C.c_double, dp, dp, C.c_double, dp]
        L.mclbm_ref_drag_impulse.restype = None
        L.mclbm_ref_set_threads.argtypes = [C.c_int]
        L.mclbm_ref_set_threads.restype = None
        L.mclbm_ref_get_threads.argtypes = []
        L.mclbm_ref_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class RefError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with code %d" % (what, code))
        self.code = code


def _check(rc, what):
    if rc != 0:
        raise RefError(rc, what)


def default_props(**overrides) -> RefProps:
    p = RefProps()
    lib().mclbm_ref_props_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def set_threads(n: int) -> None:
    lib().mclbm_ref_set_threads(int(n))


def get_threads() -> int:
    return int(lib().mclbm_ref_get_threads())


def equilibrium(rho, ux, uy):
    out = np.zeros(9)
    lib().mclbm_ref_equilibrium(rho, ux, uy, _dp(out))
    return out


def drag_impulse(rho_w, rho_p, w_relaxed, b, a):
    w = np.ascontiguousarray(w_relaxed, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    J = np.zeros(2)
    lib().mclbm_ref_drag_impulse(rho_w, rho_p, _dp(w), _dp(bb), a, _dp(J))
    return J


class RefSolver:
    """One cavity solved by the oracle. Arrays are [plane][ny][nx] float64."""

    def __init__(self, nx, ny, Ra, Pr, phi, d_p, props=None, **overrides):
        self.nx, self.ny = int(nx), int(ny)
        p = props if props is not None else default_props()
        for k, v in overrides.items():
            setattr(p, k, v)
        self.props = p
        self.np = 9 * (2 + p.thermal_sets)  # population planes
        h = C.c_void_p()
        _check(lib().mclbm_ref_create(self.nx, self.ny, Ra, Pr, phi, d_p, C.byref(p),
                                      C.byref(h)), "mclbm_ref_create")
        self._h = h

    def close(self):
        if self._h:
            lib().mclbm_ref_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def consts(self) -> dict:
        c = RefConsts()
        _check(lib().mclbm_ref_consts(self._h, C.byref(c)), "mclbm_ref_consts")
        return {n: getattr(c, n) for n in CONST_NAMES}

    def init(self, mode=INIT_REST, warm=None):
        if warm is not None:
            w = np.ascontiguousarray(warm, dtype=np.float64)
            assert w.shape[1:] == (self.ny, self.nx) and w.shape[0] in (4, 5)
            _check(lib().mclbm_ref_init(self._h, INIT_WARM if w.shape[0] == 4 else INIT_WARM_RHO,
                                        _dp(w)), "mclbm_ref_init")
        else:
            _check(lib().mclbm_ref_init(self._h, mode, None), "mclbm_ref_init")
        return self

    def step(self, n=1):
        _check(lib().mclbm_ref_step(self._h, int(n)), "mclbm_ref_step")
        return self

    def stream_only(self):
        _check(lib().mclbm_ref_stream_only(self._h), "mclbm_ref_stream_only")
        return self

    def steps_done(self) -> int:
        return int(lib().mclbm_ref_steps_done(self._h))

    def fields(self, which):
        k = bin(which).count("1")
        out = np.zeros((k, self.ny, self.nx))
        _check(lib().mclbm_ref_fields(self._h, which, _dp(out)), "mclbm_ref_fields")
        return out

    def nusselt(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().mclbm_ref_nusselt(self._h, C.byref(a), C.byref(b)), "mclbm_ref_nusselt")
        return a.value, b.value

    def mass(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().mclbm_ref_mass(self._h, C.byref(a), C.byref(b)), "mclbm_ref_mass")
        return a.value, b.value

    def residual(self):
        r = C.c_double()
        _check(lib().mclbm_ref_residual(self._h, C.byref(r)), "mclbm_ref_residual")
        return r.value

    def get_state(self):
        out = np.zeros((self.np, self.ny, self.nx))
        _check(lib().mclbm_ref_get_state(self._h, _dp(out)), "mclbm_ref_get_state")
        return out

    def set_state(self, st):
        s = np.ascontiguousarray(st, dtype=np.float64)
        assert s.shape == (self.np, self.ny, self.nx)
        _check(lib().mclbm_ref_set_state(self._h, _dp(s)), "mclbm_ref_set_state")
        return self

    def node_terms(self, i, j) -> dict:
        t = RefTerms()
        _check(lib().mclbm_ref_node_terms(self._h, i, j, C.byref(t)), "mclbm_ref_node_terms")
        out = {}
        for name, typ in TERM_FIELDS:
            v = getattr(t, name)
            out[name] = np.array([v[0], v[1]]) if typ is _V2 else float(v)
        return out
