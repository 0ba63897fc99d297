"""Thin Python binding of libmclbm (include/mclbm.h): argument marshalling only.

Every step of the method runs in the CUDA library. PyTorch is used for device memory and
streams. There is no CPU fallback: if libmclbm.so is missing or cannot load, the calls raise.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmclbm.so")

OK, EINVAL, EPARAM, ESTATE, ECUDA, EDIVERGED, ETOOLARGE, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
F_BROWNIAN, F_THERMOPHORESIS, F_DRAG, F_SAFFMAN, F_MAGNUS, F_GRAVITY, F_BUOYANCY = (
    1, 2, 4, 8, 16, 32, 64)
F_ALL = 127
UX, UY, THETA, PHI, RHO_W, RHO_P, UPX, UPY = 1, 2, 4, 8, 16, 32, 64, 128
THETA_W, THETA_P = 256, 512  # the thermal sets' own temperatures (= THETA with one set)
INIT_REST, INIT_WARM, INIT_WARM_RHO = 0, 2, 3
STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2
ROUND_STOCHASTIC, ROUND_NEAREST = 0, 1

# every entry point declared in include/mclbm.h
EXPORTS = ("mclbm_props_default", "mclbm_create", "mclbm_destroy", "mclbm_buffer_bytes",
           "mclbm_bind", "mclbm_init", "mclbm_step", "mclbm_stream_only", "mclbm_fields",
           "mclbm_nusselt", "mclbm_mass", "mclbm_residual", "mclbm_diagnostics",
           "mclbm_state_get", "mclbm_state_set", "mclbm_run_host", "mclbm_get_consts",
           "mclbm_steps_done", "mclbm_step_kernel", "mclbm_last_error", "mclbm_strerror",
           "mclbm_mass_noalloc", "mclbm_save", "mclbm_load", "mclbm_selftest_wait_timeout",
           "mclbm_batch_buffer_bytes", "mclbm_batch_create", "mclbm_batch_step",
           "mclbm_batch_nusselt", "mclbm_batch_set_active", "mclbm_batch_tune",
           "mclbm_batch_last_error", "mclbm_batch_destroy",
           # include/mclbm_net.h
           "mclbm_net_config_default", "mclbm_net_param_count", "mclbm_net_workspace_bytes",
           "mclbm_net_create", "mclbm_net_destroy", "mclbm_net_last_error", "mclbm_net_bind",
           "mclbm_net_init_params", "mclbm_net_set_params", "mclbm_net_get_params",
           "mclbm_net_set_normalizer", "mclbm_net_field_stats", "mclbm_net_forward",
           "mclbm_net_loss_grad", "mclbm_net_train_step", "mclbm_gemm_bf16")


class NetConfig(C.Structure):
    """mclbm_net_config (include/mclbm_net.h): grid, base channels, MLP width, largest batch."""
    _fields_ = [("ny", C.c_int32), ("nx", C.c_int32), ("c0", C.c_int32), ("hidden", C.c_int32),
                ("max_batch", C.c_int32)]


class Props(C.Structure):
    """mclbm_props: material and scale properties, force mask, storage, rounding, thermal
    sets (field meanings and defaults in include/mclbm.h)."""
    _fields_ = [(n, C.c_double) for n in (
        "rho_f", "cp_f", "k_f", "beta_f", "mu_f", "rho_p", "cp_p", "k_p", "beta_p",
        "T0_K", "dT_K", "g", "l_f", "Ma")] + [("force_mask", C.c_uint32),
                                              ("storage", C.c_int32), ("rounding", C.c_int32),
                                              ("thermal_sets", C.c_int32)]


CONST_NAMES = (
    "U0", "nu_w", "alpha_w", "G_B",
    "rho_ratio", "rhocp_ratio", "beta_ratio", "k_ratio", "mu_ratio", "Re_T",
    "nu_ns", "alpha_ns",
    "rho_w0", "rho_p0", "Y_w0", "Y_p0",
    "tau_w", "tau_p", "tau_tw", "tau_tp",
    "H_phys", "dx", "dt", "C_F", "g_lb",
    "mu_ns", "rho_ns", "k_ns", "nu_ns_SI",
    "V_p", "A_p", "m_p", "beta_St", "Kn", "kstar", "K_T")


class Consts(C.Structure):
    """mclbm_consts: the derived constants of a handle (CONST_NAMES, in order)."""
    _fields_ = [(n, C.c_double) for n in CONST_NAMES]


class MclbmError(RuntimeError):
    """A libmclbm call returned an error code (.code); the message names the call, the code and
    the handle's last error text."""

    def __init__(self, code, what, detail=""):
        super().__init__("%s returned %d (%s)%s" % (
            what, code, _strerror(code), (": " + detail) if detail else ""))
        self.code = code


_lib = None


def lib():
    """Loads libmclbm.so from the package directory; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libmclbm.so is not built (run paper_1511_04552_gb300.build.build() or "
                "__graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)
        L.mclbm_props_default.argtypes = [C.POINTER(Props)]
        L.mclbm_props_default.restype = None
        L.mclbm_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.POINTER(Props), C.POINTER(vp)]
        L.mclbm_destroy.argtypes = [vp]
        L.mclbm_destroy.restype = None
        L.mclbm_buffer_bytes.argtypes = [vp]
        L.mclbm_buffer_bytes.restype = C.c_size_t
        L.mclbm_bind.argtypes = [vp, vp, C.c_size_t, vp]
        L.mclbm_init.argtypes = [vp, C.c_int, vp]
        L.mclbm_step.argtypes = [vp, C.c_int64]
        L.mclbm_stream_only.argtypes = [vp]
        L.mclbm_fields.argtypes = [vp, C.c_uint32, vp]
        L.mclbm_nusselt.argtypes = [vp, dp, dp]
        L.mclbm_mass.argtypes = [vp, dp, dp]
        L.mclbm_residual.argtypes = [vp, dp]
        L.mclbm_diagnostics.argtypes = [vp, dp, dp, dp, dp, dp]
        L.mclbm_state_get.argtypes = [vp, vp]
        L.mclbm_state_set.argtypes = [vp, vp]
        L.mclbm_run_host.argtypes = [vp, fp, C.c_int64, C.c_uint32, fp, dp, dp]
        L.mclbm_get_consts.argtypes = [vp, C.POINTER(Consts)]
        L.mclbm_selftest_wait_timeout.argtypes = [vp, dp]
        L.mclbm_selftest_wait_timeout.restype = C.c_int
        L.mclbm_save.argtypes = [vp, C.c_char_p]
        L.mclbm_load.argtypes = [vp, C.c_char_p]
        L.mclbm_save.restype = C.c_int
        L.mclbm_load.restype = C.c_int
        L.mclbm_steps_done.argtypes = [vp]
        L.mclbm_steps_done.restype = C.c_int64
        ip = C.POINTER(C.c_int)
        L.mclbm_step_kernel.argtypes = [vp, ip, ip, ip, ip, ip]
        L.mclbm_step_kernel.restype = C.c_int
        L.mclbm_last_error.argtypes = [vp]
        L.mclbm_last_error.restype = C.c_char_p
        L.mclbm_strerror.argtypes = [C.c_int]
        L.mclbm_strerror.restype = C.c_char_p
        L.mclbm_mass_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp, vp]
        L.mclbm_mass_noalloc.restype = C.c_int
        L.mclbm_batch_buffer_bytes.argtypes = [C.c_int, C.POINTER(vp)]
        L.mclbm_batch_buffer_bytes.restype = C.c_size_t
        L.mclbm_batch_create.argtypes = [C.c_int, C.POINTER(vp), vp, C.c_size_t, vp,
                                         C.POINTER(vp)]
        L.mclbm_batch_step.argtypes = [vp, C.c_int64]
        L.mclbm_batch_nusselt.argtypes = [vp, dp, dp]
        L.mclbm_batch_set_active.argtypes = [vp, C.POINTER(C.c_int)]
        L.mclbm_batch_tune.argtypes = [vp, C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.mclbm_batch_last_error.argtypes = [vp]
        L.mclbm_batch_last_error.restype = C.c_char_p
        L.mclbm_batch_destroy.argtypes = [vp]
        L.mclbm_batch_destroy.restype = None
        ip, i64p = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        L.mclbm_steady_nu_reached.argtypes = [dp, C.c_int64, C.c_double, ip, C.c_int]
        L.mclbm_steady_nu_reached.restype = C.c_int
        L.mclbm_run_to_steady.argtypes = [vp, C.c_double, C.c_int64, C.c_int64, ip, C.c_int,
                                          i64p, dp, dp, C.POINTER(C.c_int)]
        L.mclbm_run_to_steady.restype = C.c_int
        L.mclbm_batch_run_to_steady.argtypes = [vp, C.c_double, C.c_int64, C.c_int64, ip,
                                                C.c_int, i64p, dp, i64p]
        L.mclbm_batch_run_to_steady.restype = C.c_int
        for name in ("mclbm_batch_create", "mclbm_batch_step", "mclbm_batch_nusselt",
                     "mclbm_batch_set_active", "mclbm_batch_tune"):
            getattr(L, name).restype = C.c_int
        ncp = C.POINTER(NetConfig)
        L.mclbm_net_config_default.argtypes = [ncp]
        L.mclbm_net_config_default.restype = None
        L.mclbm_net_param_count.argtypes = [ncp]
        L.mclbm_net_param_count.restype = C.c_int64
        L.mclbm_net_workspace_bytes.argtypes = [ncp]
        L.mclbm_net_workspace_bytes.restype = C.c_size_t
        L.mclbm_net_create.argtypes = [ncp, C.POINTER(vp)]
        L.mclbm_net_destroy.argtypes = [vp]
        L.mclbm_net_destroy.restype = None
        L.mclbm_net_last_error.argtypes = [vp]
        L.mclbm_net_last_error.restype = C.c_char_p
        L.mclbm_net_bind.argtypes = [vp, vp, C.c_size_t, vp]
        L.mclbm_net_init_params.argtypes = [vp, C.c_uint64]
        L.mclbm_net_set_params.argtypes = [vp, vp]
        L.mclbm_net_get_params.argtypes = [vp, vp]
        L.mclbm_net_set_normalizer.argtypes = [vp, dp, dp]
        L.mclbm_net_field_stats.argtypes = [vp, C.c_int, vp, vp, dp, dp]
        L.mclbm_net_forward.argtypes = [vp, C.c_int, vp, vp]
        L.mclbm_net_loss_grad.argtypes = [vp, C.c_int, vp, vp, vp, dp]
        L.mclbm_net_train_step.argtypes = [vp, C.c_int, vp, vp, C.c_float, dp]
        L.mclbm_gemm_bf16.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.c_int64, C.c_int, vp,
                                      C.c_int64, C.c_int, vp, C.c_int64, C.c_int, C.c_int64,
                                      C.c_int64, vp]
        for name in ("mclbm_net_create", "mclbm_net_bind", "mclbm_net_init_params",
                     "mclbm_net_set_params", "mclbm_net_get_params", "mclbm_net_set_normalizer",
                     "mclbm_net_field_stats", "mclbm_net_forward", "mclbm_net_loss_grad",
                     "mclbm_net_train_step", "mclbm_gemm_bf16"):
            getattr(L, name).restype = C.c_int
        for name in ("mclbm_create", "mclbm_bind", "mclbm_init", "mclbm_step",
                     "mclbm_stream_only", "mclbm_fields", "mclbm_nusselt", "mclbm_mass",
                     "mclbm_residual", "mclbm_diagnostics", "mclbm_state_get",
                     "mclbm_state_set", "mclbm_run_host", "mclbm_get_consts"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _strerror(code):
    try:
        return lib().mclbm_strerror(code).decode()
    except Exception:
        return "?"


def props_default(**overrides) -> Props:
    """mclbm_props_default, then the given fields overridden."""
    p = Props()
    lib().mclbm_props_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def create(nx, ny, Ra, Pr, phi, d_p, props=None):
    """mclbm_create: returns an opaque handle (c_void_p)."""
    h = C.c_void_p()
    rc = lib().mclbm_create(int(nx), int(ny), float(Ra), float(Pr), float(phi), float(d_p),
                            C.byref(props) if props is not None else None, C.byref(h))
    if rc != OK:
        raise MclbmError(rc, "mclbm_create")
    return h


def get_consts(h) -> dict:
    """mclbm_get_consts of a handle, as a dict keyed by CONST_NAMES."""
    c = Consts()
    rc = lib().mclbm_get_consts(h, C.byref(c))
    if rc != OK:
        raise MclbmError(rc, "mclbm_get_consts")
    return {n: getattr(c, n) for n in CONST_NAMES}


def _nfields(which):
    return bin(int(which)).count("1")


class Cavity:
    """One cavity on one GPU: a libmclbm handle bound to a torch-owned device buffer and a
    torch stream. Methods mirror the C entry points."""

    def __init__(self, nx, ny, Ra, Pr, phi, d_p, props=None, device=None, stream=None,
                 **prop_overrides):
        import torch
        self.torch = torch
        self.nx, self.ny = int(nx), int(ny)
        self.params = dict(Ra=Ra, Pr=Pr, phi=phi, d_p=d_p)
        p = props if props is not None else props_default()
        for k, v in prop_overrides.items():
            setattr(p, k, v)
        self.props = p
        self.np = 9 * (2 + p.thermal_sets)  # population planes per time level
        self.device = torch.device(device if device is not None else "cuda")
        self._h = create(nx, ny, Ra, Pr, phi, d_p, p)
        nbytes = int(lib().mclbm_buffer_bytes(self._h))
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(lib().mclbm_bind(self._h, C.c_void_p(self.buffer.data_ptr()), nbytes,
                                     C.c_void_p(self.stream.cuda_stream)), "mclbm_bind")

    # -- plumbing
    def _check(self, rc, what):
        if rc != OK:
            detail = lib().mclbm_last_error(self._h).decode(errors="replace")
            raise MclbmError(rc, what, detail)

    def close(self):
        """mclbm_destroy (idempotent); the device buffer goes with the object."""
        if getattr(self, "_h", None):
            lib().mclbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        """The opaque mclbm_t handle (c_void_p)."""
        return self._h

    def consts(self) -> dict:
        """mclbm_get_consts as a dict."""
        return get_consts(self._h)

    def steps_done(self) -> int:
        """mclbm_steps_done: time steps since the last init or state_set."""
        return int(lib().mclbm_steps_done(self._h))

    def step_kernel(self) -> dict:
        """mclbm_step_kernel: the step kernel this cavity launches (variant, nodes per thread,
        tile height, persistent CTAs, two-step pairs)."""
        v = [C.c_int(0) for _ in range(5)]
        rc = lib().mclbm_step_kernel(self._h, *[C.byref(x) for x in v])
        if rc != 0:
            raise MclbmError(rc, "mclbm_step_kernel")
        return dict(zip(("variant", "nodes_per_thread", "tile_h", "grid", "two"),
                        (x.value for x in v)))

    # -- the C entry points
    def init(self, mode=INIT_REST, warm=None):
        """mclbm_init. warm: device float32 tensor [4, ny, nx] (ux, uy, theta, phi) or
        [5, ny, nx] (+ rho^w, mode MCLBM_INIT_WARM_RHO)."""
        if warm is not None:
            assert warm.dtype == self.torch.float32 and warm.is_cuda
            assert tuple(warm.shape[1:]) == (self.ny, self.nx) and warm.is_contiguous()
            assert warm.shape[0] in (4, 5)
            self._warm_keepalive = warm
            rc = lib().mclbm_init(self._h, INIT_WARM if warm.shape[0] == 4 else INIT_WARM_RHO,
                                  C.c_void_p(warm.data_ptr()))
        else:
            rc = lib().mclbm_init(self._h, mode, None)
        self._check(rc, "mclbm_init")
        return self

    def step(self, n=1):
        """mclbm_step: n time steps (async)."""
        self._check(lib().mclbm_step(self._h, int(n)), "mclbm_step")
        return self

    def stream_only(self):
        """mclbm_stream_only: one step of streaming alone (a test hook)."""
        self._check(lib().mclbm_stream_only(self._h), "mclbm_stream_only")
        return self

    def fields(self, which, out=None):
        """mclbm_fields: the selected macroscopic fields (mask of UX, UY, THETA, PHI, ...) as a
        device float32 tensor [fields][ny][nx], in the order of the mask's bits."""
        k = _nfields(which)
        if out is None:
            out = self.torch.empty((k, self.ny, self.nx), dtype=self.torch.float32,
                                   device=self.device)
        self._check(lib().mclbm_fields(self._h, int(which), C.c_void_p(out.data_ptr())),
                    "mclbm_fields")
        return out

    def save(self, path):
        """mclbm_save: checkpoint of the current state (syncs)."""
        self._check(lib().mclbm_save(self._h, os.fsencode(path)), "mclbm_save")
        return self

    def load(self, path):
        """mclbm_load: resume from a checkpoint of a cavity with the same size and parameters."""
        self._check(lib().mclbm_load(self._h, os.fsencode(path)), "mclbm_load")
        return self

    def nusselt(self):
        """mclbm_nusselt: (hot-wall, cold-wall) mean Nusselt numbers (syncs)."""
        a, b = C.c_double(), C.c_double()
        self._check(lib().mclbm_nusselt(self._h, C.byref(a), C.byref(b)), "mclbm_nusselt")
        return a.value, b.value

    def mass(self):
        """mclbm_mass: (base fluid, particle) masses (syncs)."""
        a, b = C.c_double(), C.c_double()
        self._check(lib().mclbm_mass(self._h, C.byref(a), C.byref(b)), "mclbm_mass")
        return a.value, b.value

    def residual(self):
        """mclbm_residual: steady-state residual since the previous call (syncs)."""
        r = C.c_double()
        self._check(lib().mclbm_residual(self._h, C.byref(r)), "mclbm_residual")
        return r.value

    def diagnostics(self) -> dict:
        """mclbm_diagnostics: Nusselt numbers, masses and residual with one synchronisation."""
        v = [C.c_double() for _ in range(5)]
        self._check(lib().mclbm_diagnostics(self._h, *[C.byref(x) for x in v]),
                    "mclbm_diagnostics")
        return dict(zip(("nu_hot", "nu_cold", "mass_w", "mass_p", "residual"),
                        (x.value for x in v)))

    def state_get(self, out=None):
        """mclbm_state_get: the population planes [np][ny][nx] (deviations) as float32."""
        if out is None:
            out = self.torch.empty((self.np, self.ny, self.nx), dtype=self.torch.float32,
                                   device=self.device)
        self._check(lib().mclbm_state_get(self._h, C.c_void_p(out.data_ptr())),
                    "mclbm_state_get")
        return out

    def state_set(self, st):
        """mclbm_state_set: replace the state by the planes of st (layout of state_get)."""
        assert st.dtype == self.torch.float32 and st.is_cuda and st.is_contiguous()
        assert tuple(st.shape) == (self.np, self.ny, self.nx)
        self._check(lib().mclbm_state_set(self._h, C.c_void_p(st.data_ptr())), "mclbm_state_set")
        return self

    def run_host(self, warm_host, n, which=0, fields_out=None):
        """mclbm_run_host on host arrays: returns (fields or None, nu_hot, nu_cold)."""
        fptr = C.POINTER(C.c_float)
        w = None
        if warm_host is not None:
            w = self._host_f32(warm_host)
            assert w.numel() == 4 * self.nx * self.ny
        out = None
        if which:
            out = fields_out if fields_out is not None else self.torch.empty(
                (_nfields(which), self.ny, self.nx), dtype=self.torch.float32)
        a, b = C.c_double(), C.c_double()
        rc = lib().mclbm_run_host(
            self._h, C.cast(w.data_ptr(), fptr) if w is not None else None, int(n), int(which),
            C.cast(out.data_ptr(), fptr) if out is not None else None, C.byref(a), C.byref(b))
        self._check(rc, "mclbm_run_host")
        return out, a.value, b.value

    def _host_f32(self, arr):
        t = arr if isinstance(arr, self.torch.Tensor) else self.torch.from_numpy(
            np.ascontiguousarray(arr, dtype=np.float32))
        assert t.device.type == "cpu" and t.dtype == self.torch.float32 and t.is_contiguous()
        return t


STRICT_LAGS = (1, 32)


def _lags(lags):
    arr = (C.c_int32 * len(lags))(*[int(x) for x in lags])
    return arr, len(lags)


def steady_nu_reached(hist, tol=1e-4, lags=STRICT_LAGS):
    """mclbm_steady_nu_reached: is the hot-wall Nusselt history (oldest first, equally spaced
    checks) steady to tol on every lag (in checks)? The test is stated in include/mclbm.h."""
    h = np.ascontiguousarray(np.asarray(hist, dtype=np.float64))
    arr, n_lags = _lags(lags)
    rc = lib().mclbm_steady_nu_reached(h.ctypes.data_as(C.POINTER(C.c_double)), h.size,
                                       float(tol), arr, n_lags)
    if rc < 0:
        raise MclbmError(rc, "mclbm_steady_nu_reached")
    return rc == 1


def run_to_steady(cav: Cavity, tol=1e-4, check_every=1000, max_steps=3_000_000,
                  lags=STRICT_LAGS):
    """mclbm_run_to_steady: advances until the hot-wall Nusselt number is steady to tol (checks
    `check_every` steps apart). Returns the step count, the final Nusselt numbers and whether the
    test held."""
    arr, n_lags = _lags(lags)
    steps, nh, nc, conv = C.c_int64(), C.c_double(), C.c_double(), C.c_int()
    cav._check(lib().mclbm_run_to_steady(cav.handle, float(tol), int(check_every),
                                         int(max_steps), arr, n_lags, C.byref(steps),
                                         C.byref(nh), C.byref(nc), C.byref(conv)),
               "mclbm_run_to_steady")
    return dict(steps=steps.value, nu_hot=nh.value, nu_cold=nc.value, converged=bool(conv.value))


class Batch:
    """Several Cavity objects stepped together, one persistent launch per time step
    (mclbm_batch_*). Keeps references to its cavities; do not step them alone meanwhile."""

    def __init__(self, cavities, stream=None):
        import torch
        self.torch = torch
        self.cavities = list(cavities)
        n = len(self.cavities)
        self._hs = (C.c_void_p * n)(*[c.handle.value for c in self.cavities])
        nbytes = int(lib().mclbm_batch_buffer_bytes(n, self._hs))
        if nbytes == 0:
            raise MclbmError(EINVAL, "mclbm_batch_buffer_bytes")
        dev = self.cavities[0].device
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = C.c_void_p()
        rc = lib().mclbm_batch_create(n, self._hs, C.c_void_p(self.buffer.data_ptr()), nbytes,
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != OK:
            raise MclbmError(rc, "mclbm_batch_create")
        self._h = h

    def _check(self, rc, what):
        if rc != OK:
            raise MclbmError(rc, what, lib().mclbm_batch_last_error(self._h).decode())

    def step(self, n):
        """mclbm_batch_step: n (even) time steps of every active cavity (async)."""
        self._check(lib().mclbm_batch_step(self._h, int(n)), "mclbm_batch_step")
        return self

    def nusselt(self):
        """mclbm_batch_nusselt: hot- and cold-wall Nusselt numbers of every cavity (syncs)."""
        n = len(self.cavities)
        a, b = np.zeros(n), np.zeros(n)
        dp = C.POINTER(C.c_double)
        self._check(lib().mclbm_batch_nusselt(self._h, a.ctypes.data_as(dp), b.ctypes.data_as(dp)),
                    "mclbm_batch_nusselt")
        return a, b

    def set_active(self, active):
        """mclbm_batch_set_active: only the cavities flagged true keep stepping."""
        arr = (C.c_int * len(self.cavities))(*[1 if x else 0 for x in active])
        self._check(lib().mclbm_batch_set_active(self._h, arr), "mclbm_batch_set_active")
        return self

    def tune(self, steps_per_trial=200):
        """mclbm_batch_tune: times each tile order x CTAs per SM and keeps the fastest;
        returns (tile order, CTAs per SM)."""
        o, p = C.c_int(), C.c_int()
        self._check(lib().mclbm_batch_tune(self._h, int(steps_per_trial), C.byref(o), C.byref(p)),
                    "mclbm_batch_tune")
        return o.value, p.value

    def close(self):
        """mclbm_batch_destroy (idempotent); the cavities stay usable."""
        if getattr(self, "_h", None):
            lib().mclbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_to_steady(batch: Batch, tol=1e-4, check_every=1000, max_steps=3_000_000,
                    lags=STRICT_LAGS):
    """mclbm_batch_run_to_steady: runs every cavity of a batch until its hot-wall Nusselt number
    is steady to tol; converged cavities leave the tile table. Returns per-cavity step counts
    (None where the test did not hold) and Nusselt numbers."""
    n = len(batch.cavities)
    arr, n_lags = _lags(lags)
    steps = np.zeros(n, dtype=np.int64)
    nu = np.zeros(n)
    total = C.c_int64()
    batch._check(lib().mclbm_batch_run_to_steady(
        batch._h, float(tol), int(check_every), int(max_steps), arr, n_lags,
        steps.ctypes.data_as(C.POINTER(C.c_int64)), nu.ctypes.data_as(C.POINTER(C.c_double)),
        C.byref(total)), "mclbm_batch_run_to_steady")
    done = [int(x) if x >= 0 else None for x in steps]
    return dict(steps=done, nu_hot=nu, total_steps=total.value,
                converged=all(d is not None for d in done))
