"""Two thermal population sets on the GPU (g^w for the base fluid, g^p for the particles, each
relaxing with its own time toward the equilibrium at the Eq 33 mixture temperature), called
through the C ABI, against the FP64 oracle's two-set model on the same seeded inputs: every
field, both sets' temperatures and the Nusselt numbers to the FP32 parity bar (1e-5 relative)."""
import numpy as np
import pytest

import workloads
from tests import _parity as P

pytestmark = pytest.mark.gpu

TWO_FIELDS = 256 | 512  # theta^w, theta^p


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.ensure_built()


def _pair(steps, **kw):
    gpu, ref = P.make_pair(thermal_sets=2, **kw)
    gpu.step(steps)
    ref.step(steps)
    return gpu, ref


def _assert_parity(gpu, ref, rtol=P.FIELD_RTOL, nu_rtol=P.NU_RTOL):
    errs, bad = P.compare_fields(gpu, ref, rtol)
    g = gpu.fields(TWO_FIELDS).cpu().numpy()
    r = ref.fields(TWO_FIELDS)
    for k, name in enumerate(("theta_w", "theta_p")):
        errs[name] = P.rel_l2(g[k], r[k])
        if not errs[name] <= rtol:
            bad[name] = errs[name]
    assert not bad, errs
    gh, gc = gpu.nusselt()
    rh, rc = ref.nusselt()
    assert abs(gh - rh) <= nu_rtol * abs(rh), (gh, rh)
    assert abs(gc - rc) <= nu_rtol * abs(rc), (gc, rc)
    return errs


@pytest.mark.parametrize("seed", [None, 1])
def test_cavity32_2000_steps(seed):
    w = workloads.CAVITY_32
    gpu, ref = _pair(w["steps"], nx=w["nx"], ny=w["ny"], Ra=w["Ra"], Pr=w["Pr"], phi=w["phi"],
                     d_p=w["d_p"], seed=seed)
    print("two sets, cavity32 seed", seed, _assert_parity(gpu, ref))


@pytest.mark.parametrize("nx,ny,Ra,phi,d_p,steps,mask", [
    (37, 29, 1e4, 0.02, 30e-9, 500, 127),     # ragged against the 32 x 8 tiles
    (130, 7, 1e3, 0.01, 20e-9, 300, 127),     # five column tiles, a ragged one, few rows
    (2, 2, 1e3, 0.01, 20e-9, 200, 127),       # every node touches two walls
    (200, 67, 1e5, 0.03, 30e-9, 400, 127),    # several tiles, ragged both ways
    (48, 40, 1e5, 0.0, 30e-9, 600, 127),      # pure fluid: the mixture is theta^w
    (40, 40, 1e5, 0.03, 30e-9, 400, 4 | 8 | 16 | 64),   # no Brownian, thermophoresis, gravity
    (33, 65, 1e4, 0.19, 100e-9, 300, 127),    # dense suspension, large particles
])
def test_ragged_and_masked(nx, ny, Ra, phi, d_p, steps, mask):
    gpu, ref = _pair(steps, nx=nx, ny=ny, Ra=Ra, Pr=6.2, phi=phi, d_p=d_p, seed=3,
                     force_mask=mask)
    _assert_parity(gpu, ref)


def test_cavity64_5000_steps():
    gpu, ref = _pair(5000, nx=64, ny=64, Ra=1e5, Pr=6.2, phi=0.03, d_p=30e-9, seed=2)
    print("two sets, cavity64", _assert_parity(gpu, ref))


def test_state_holds_36_planes_and_matches_the_oracle():
    """state_get returns f^w, f^p, g^w, g^p; after 100 steps every plane agrees with the
    oracle's populations (absolute, relative L2 per plane)."""
    gpu, ref = _pair(100, nx=45, ny=30, Ra=1e4, Pr=6.2, phi=0.02, d_p=30e-9, seed=5)
    st = P.gpu_state_abs(gpu)
    assert st.shape == (36, 30, 45)
    r = ref.get_state()
    errs = [P.rel_l2(st[p], r[p]) for p in range(36)]
    assert max(errs) <= 1e-6, errs


def test_sets_start_equal_and_separate():
    """From a warm start both sets hold the same temperature (theta^w = theta^p = theta, up to
    the order in which the field kernel sums each set); where the sets relax at different rates
    they drift apart under convection."""
    gpu, ref = P.make_pair(40, 40, 1e5, 6.2, 0.03, 30e-9, seed=4, thermal_sets=2)
    g = gpu.fields(TWO_FIELDS | 4).cpu().numpy()
    assert np.allclose(g[1], g[0], rtol=0, atol=1e-6)
    assert np.allclose(g[2], g[0], rtol=0, atol=1e-6)
    gpu.step(300)
    g = gpu.fields(TWO_FIELDS).cpu().numpy()
    c = gpu.consts()
    if abs(c["tau_tw"] - c["tau_tp"]) > 1e-3:
        assert np.abs(g[0] - g[1]).max() > 0.0


def test_dispatch_ignores_tma_and_two_node_overrides(monkeypatch):
    """Two thermal sets always run the plain tile kernel with one node per thread: forcing the
    TMA variant or two nodes per thread gives the same bits."""
    import torch
    import paper_1511_04552_gb300 as m
    a = m.Cavity(130, 67, 1e5, 6.2, 0.03, 30e-9, thermal_sets=2).init()
    a.step(50)
    monkeypatch.setenv("MCLBM_STEP_VARIANT", "tma")
    monkeypatch.setenv("MCLBM_STEP_VEC", "2")
    b = m.Cavity(130, 67, 1e5, 6.2, 0.03, 30e-9, thermal_sets=2).init()
    b.step(50)
    assert torch.equal(a.state_get(), b.state_get())


@pytest.mark.parametrize("storage,rtol,nu_rtol", [("f16", 5e-3, 5e-3), ("bf16", 5e-2, 3e-2)])
def test_16_bit_storage(storage, rtol, nu_rtol):
    """16-bit storage of all 36 planes with stochastic rounding: 64 x 64, Ra 1e5, 5000 steps;
    bounds those of the one-set model at the same storage."""
    import paper_1511_04552_gb300 as m
    st = {"f16": m.STORE_F16, "bf16": m.STORE_BF16}[storage]
    gpu, ref = P.make_pair(64, 64, 1e5, 6.2, 0.03, 30e-9, seed=2, thermal_sets=2, storage=st)
    gpu.step(5000)
    ref.step(5000)
    g = gpu.fields(1 | 2 | 4 | TWO_FIELDS).cpu().numpy()
    r = ref.fields(1 | 2 | 4 | TWO_FIELDS)
    errs = {n: P.rel_l2(g[k], r[k]) for k, n in enumerate(("ux", "uy", "theta", "theta_w",
                                                             "theta_p"))}
    nh, _ = gpu.nusselt()
    rh, _ = ref.nusselt()
    print(storage, "two sets: Nu rel %.2e" % (abs(nh - rh) / rh), errs)
    assert abs(nh - rh) <= nu_rtol * rh
    assert max(errs.values()) <= rtol, errs


def test_batch_rejects_two_sets():
    import paper_1511_04552_gb300 as m
    a = m.Cavity(64, 64, 1e5, 6.2, 0.03, 30e-9, thermal_sets=2).init()
    with pytest.raises(m.MclbmError):
        m.Batch([a])


def test_checkpoint_resume_is_bitwise(tmp_path):
    import torch
    import paper_1511_04552_gb300 as m
    a = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9, thermal_sets=2).init()
    a.step(300)
    path = str(tmp_path / "ck2.bin")
    a.save(path)
    a.step(200)
    b = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9, thermal_sets=2).load(path)
    b.step(200)
    assert torch.equal(a.state_get(), b.state_get())
    c = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9).init()  # one set: a different state size
    with pytest.raises(m.MclbmError):
        c.load(path)
