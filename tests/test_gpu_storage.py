"""16-bit population storage (FP16 / BF16 holding 2^12 x the deviations, FP32 arithmetic):
exact round trips, identical results from both step kernels, and accuracy against the FP64
oracle within the reduced-storage target (mean Nusselt number within 0.5 %)."""
import os

import numpy as np
import pytest

import workloads
from tests import _parity as P

pytestmark = pytest.mark.gpu

STORE = {"f16": 1, "bf16": 2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.ensure_built()


def _cav(nx, ny, Ra, phi, d_p, storage, rounding=0, **kw):
    import paper_1511_04552_gb300 as m
    return m.Cavity(nx, ny, Ra, 6.2, phi, d_p, storage=STORE[storage], rounding=rounding, **kw)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_state_round_trip_is_the_16_bit_grid(storage):
    import torch
    cav = _cav(70, 40, 1e4, 0.02, 30e-9, storage).init()
    dev = workloads.random_state(70, 40, seed=4, amp=0.05)
    cav.state_set(torch.from_numpy(dev).cuda())
    got = cav.state_get().cpu()
    scaled = torch.from_numpy(dev) * 4096.0
    dt = torch.float16 if storage == "f16" else torch.bfloat16
    exp = scaled.to(dt).to(torch.float32) / 4096.0
    assert torch.equal(got, exp)


@pytest.mark.parametrize("storage,rounding", [("f16", 0), ("f16", 1), ("bf16", 0), ("bf16", 1)])
def test_tile_and_tma_kernels_agree_bitwise(storage, rounding, monkeypatch):
    import torch
    out = []
    for variant in ("tile", "tma"):
        monkeypatch.setenv("MCLBM_STEP_VARIANT", variant)
        cav = _cav(130, 67, 1e5, 0.03, 30e-9, storage, rounding).init()
        cav.step(200)
        out.append(cav.state_get())
        cav.nusselt()
    assert torch.equal(out[0], out[1])


# FP16 meets the reduced-storage target (mean Nu within 0.5 %); BF16 (8-bit mantissa) does not:
# measured on GB300 after 20 000 steps, Nu 0.9 %, velocity 1.4 %, theta 1.0 %. Its bounds are
# the measured errors with margin, so a regression still fails.
@pytest.mark.parametrize("storage,nu_tol,u_tol,th_tol", [("f16", 5e-3, 1e-2, 5e-3),
                                                         ("bf16", 2e-2, 3e-2, 2e-2)])
def test_accuracy_against_fp64_oracle(storage, nu_tol, u_tol, th_tol):
    """64 x 64, Ra 1e5, 3 %, 30 nm, 20 000 steps with stochastic rounding: the errors per result
    of an FP32-arithmetic step that stores 16 bits, against the FP64 oracle."""
    import oracle
    n, Ra, phi, d = 64, 1e5, 0.03, 30e-9
    cav = _cav(n, n, Ra, phi, d, storage).init()
    ref = oracle.RefSolver(n, n, Ra, 6.2, phi, d).init()
    cav.step(20000)
    ref.step(20000)
    g = cav.fields(0xFF).cpu().numpy()
    r = ref.fields(0xFF)
    e = {name: P.rel_l2(g[k], r[k]) for k, name in enumerate(P.FIELD_NAMES)}
    nu_g, nu_r = cav.nusselt()[0], ref.nusselt()[0]
    print(storage, "Nu rel %.2e" % (abs(nu_g - nu_r) / nu_r), e)
    assert abs(nu_g - nu_r) <= nu_tol * nu_r
    assert e["ux"] <= u_tol and e["uy"] <= u_tol
    assert e["theta"] <= th_tol
    assert e["phi"] <= 1e-3
    mw, mp = cav.mass()
    rw, rp = ref.mass()
    assert abs(mw - rw) <= 1e-4 * rw and abs(mp - rp) <= 1e-3 * rp


GOLDEN_1024 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "oracle_cavity1024_20000.npz")


# Measured on GB300 (per result: Nu, max |u|, phi - phi0, velocity fields):
#   FP32 3.9e-7, 2.0e-5, 1.8e-4, 2.2e-5; FP16 2.1e-4, 2.8e-4, 7.5e-3, 2.8e-4;
#   BF16 9.0e-4, 5.5e-3, 6.2e-2, 2.3e-3.
# FP32: Nu within the parity bar, the velocities at 2e-5 (FP32 rounding accumulated over 20 000
# steps of a 1024^2 lattice; the 32^2 and 64^2 parity cases stay below 1e-5), and phi - phi0 has
# an RMS of 5e-4 of phi0 here, which a float32 phi (the fields' and the stored sample's type)
# resolves only to about 2e-4. FP16 meets the
# reduced-storage target (mean Nu within 0.5 %); BF16 its measured errors with margin.
@pytest.mark.parametrize("storage,nu_tol,u_tol,phi_tol", [("f32", 1e-5, 5e-5, 5e-4),
                                                          ("f16", 5e-3, 1e-2, 5e-2),
                                                          ("bf16", 3e-2, 5e-2, 3e-1)])
def test_per_result_error_at_1024(storage, nu_tol, u_tol, phi_tol):
    """The precision configuration: 1024^2, Ra 1e6, phi 2 %, 50 nm, 20 000 steps from rest, each
    storage type against the FP64 oracle's run of the same case (stored by
    tests/golden/make_oracle_runs.py, which calls only the oracle). Errors per result: the mean
    hot-wall Nusselt number, the maximum speed |u|, and the relative L2 of the concentration's
    deviation from its initial value phi - phi0 (on every 4th row and column, the oracle's stored
    sample), with the velocity fields on the same sample."""
    import paper_1511_04552_gb300 as m
    ref = np.load(GOLDEN_1024)
    w = workloads.CAVITY_1024
    assert str(ref["workload"]) == w["name"] and int(ref["steps"]) == 20000
    store = {"f32": 0, "f16": 1, "bf16": 2}[storage]
    cav = m.Cavity(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"], storage=store)
    cav.init().step(20000)
    f = cav.fields(m.UX | m.UY | m.PHI).cpu().numpy().astype(np.float64)
    nu = cav.nusselt()[0]
    k = int(ref["sample"])
    ux, uy, phi = f[0][::k, ::k], f[1][::k, ::k], f[2][::k, ::k]
    e_nu = abs(nu - float(ref["nu_hot"])) / float(ref["nu_hot"])
    umax = float(np.sqrt(f[0] ** 2 + f[1] ** 2).max())
    e_u = abs(umax - float(ref["umax"])) / float(ref["umax"])
    dphi_ref = ref["phi"].astype(np.float64) - w["phi"]
    e_phi = P.rel_l2(phi - w["phi"], dphi_ref)
    e_ux, e_uy = P.rel_l2(ux, ref["ux"]), P.rel_l2(uy, ref["uy"])
    print("%s at 1024^2 against FP64: Nu %.2e, max|u| %.2e, phi deviation L2 %.2e, ux %.2e, uy %.2e"
          % (storage, e_nu, e_u, e_phi, e_ux, e_uy))
    assert e_nu <= nu_tol
    assert e_u <= u_tol and e_ux <= u_tol and e_uy <= u_tol
    assert e_phi <= phi_tol
