"""Helpers shared by the GPU parity tests: running the same seeded inputs through the CUDA
library (via its C ABI binding) and through the FP64 oracle, and comparing the results."""
import os

import numpy as np

import workloads

ALL_FIELDS = 0xFF  # ux, uy, theta, phi, rho_w, rho_p, upx, upy
FIELD_NAMES = ("ux", "uy", "theta", "phi", "rho_w", "rho_p", "upx", "upy")
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

# FP32 path against the FP64 oracle: relative L2 per field and relative Nusselt number
FIELD_RTOL = 1e-5
NU_RTOL = 1e-5


def ensure_built():
    from paper_1511_04552_gb300 import build
    build.build()
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    if den == 0.0:
        return num
    return num / den


def make_pair(nx, ny, Ra, Pr, phi, d_p, seed=None, amp=1e-3, **props):
    """A GPU cavity and an oracle cavity with identical parameters and initial state."""
    import torch

    import oracle
    import paper_1511_04552_gb300 as m
    gpu = m.Cavity(nx, ny, Ra, Pr, phi, d_p, **props)
    ref = oracle.RefSolver(nx, ny, Ra, Pr, phi, d_p, **props)
    if seed is None:
        gpu.init()
        ref.init()
    else:
        warm = workloads.perturbed_rest_fields(nx, ny, phi, seed=seed, amp=amp)
        gpu.init(warm=torch.from_numpy(warm).cuda())
        ref.init(warm=warm.astype(np.float64))
    return gpu, ref


def compare_fields(gpu, ref, rtol=FIELD_RTOL):
    g = gpu.fields(ALL_FIELDS).cpu().numpy()
    r = ref.fields(ALL_FIELDS)
    errs = {}
    for k, name in enumerate(FIELD_NAMES):
        errs[name] = rel_l2(g[k], r[k])
    bad = {k: v for k, v in errs.items() if not v <= rtol}
    return errs, bad


def _offsets(consts, np_, nx, ny):
    """Per-plane offsets of the stored deviations: W_q rho_sigma0 for f, W_q theta_c(i) for each
    thermal set (np_ = 27 or 36 planes)."""
    off = np.zeros((np_, ny, nx))
    off[:9] = (W * consts["rho_w0"])[:, None, None]
    off[9:18] = (W * consts["rho_p0"])[:, None, None]
    th_c = 0.5 - (np.arange(nx) + 0.5) / nx
    for b in range(18, np_, 9):
        off[b:b + 9] = W[:, None, None] * th_c[None, None, :]
    return off


def dev_to_abs(dev, consts):
    dev = np.asarray(dev, dtype=np.float64)
    return dev + _offsets(consts, dev.shape[0], dev.shape[2], dev.shape[1])


def abs_to_dev(st_abs, consts):
    st_abs = np.asarray(st_abs, dtype=np.float64)
    return st_abs - _offsets(consts, st_abs.shape[0], st_abs.shape[2], st_abs.shape[1])


def gpu_state_abs(gpu):
    """The GPU state as absolute FP64 populations [27 or 36][ny][nx]."""
    return dev_to_abs(gpu.state_get().cpu().numpy(), gpu.consts())
