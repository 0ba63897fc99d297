"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle on the same
seeded inputs. Fields must agree to a relative L2 of 1e-5 and the Nusselt numbers to 1e-5
relative (FP32 arithmetic against FP64)."""
import numpy as np
import pytest

import workloads
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.ensure_built()


def _run_pair(steps, **kw):
    gpu, ref = P.make_pair(**kw)
    gpu.step(steps)
    ref.step(steps)
    return gpu, ref


def _assert_parity(gpu, ref, rtol=P.FIELD_RTOL, nu_rtol=P.NU_RTOL):
    errs, bad = P.compare_fields(gpu, ref, rtol)
    assert not bad, errs
    gh, gc = gpu.nusselt()
    rh, rc = ref.nusselt()
    assert abs(gh - rh) <= nu_rtol * abs(rh), (gh, rh)
    assert abs(gc - rc) <= nu_rtol * abs(rc), (gc, rc)
    return errs


@pytest.mark.parametrize("seed", [None, 1])
def test_cavity32_2000_steps(seed):
    """32 x 32, Ra 1e3, Pr 6.2, 1 % alumina 20 nm, all slip forces, 2000 steps."""
    w = workloads.CAVITY_32
    gpu, ref = _run_pair(w["steps"], nx=w["nx"], ny=w["ny"], Ra=w["Ra"], Pr=w["Pr"], phi=w["phi"],
                         d_p=w["d_p"], seed=seed)
    errs = _assert_parity(gpu, ref)
    print("cavity32 seed", seed, errs)


@pytest.mark.parametrize("nx,ny,Ra,phi,d_p,steps,mask", [
    (37, 29, 1e4, 0.02, 30e-9, 500, 127),     # ragged against 64-column tiles and strips
    (130, 7, 1e3, 0.01, 20e-9, 300, 127),     # two column tiles, a ragged one, few rows
    (2, 2, 1e3, 0.01, 20e-9, 200, 127),       # every node touches two walls
    (3, 5, 1e3, 0.04, 50e-9, 200, 127),
    (200, 67, 1e5, 0.03, 30e-9, 400, 127),    # several tiles and strips, ragged both ways
    (48, 40, 1e5, 0.0, 30e-9, 600, 127),      # pure fluid
    (40, 40, 1e5, 0.03, 30e-9, 400, 4 | 8 | 16 | 64),   # no B, T, G
    # no drag: explicit forces only (thermophoresis and gravity without drag are unstable
    # by construction: beta dt is 1e3-1e7, which is why the drag impulse is integrated exactly)
    # (Saffman lift without drag grows the slip without bound too)
    (40, 40, 1e5, 0.03, 30e-9, 400, 1 | 16 | 64),
    (33, 65, 1e4, 0.19, 100e-9, 300, 127),    # dense suspension, large particles
])
def test_ragged_and_masked(nx, ny, Ra, phi, d_p, steps, mask):
    gpu, ref = _run_pair(steps, nx=nx, ny=ny, Ra=Ra, Pr=6.2, phi=phi, d_p=d_p, seed=3,
                         force_mask=mask)
    _assert_parity(gpu, ref)


def test_low_tiles_lattice_2000_steps():
    """A lattice ragged both ways on which the handle picks the 32 x 7 tiles by itself (9 x 28
    tiles of 32 x 8 would give some of 152 SMs a second tile; 9 x 32 of 32 x 7 fit two per
    SM): 2000 steps against the oracle."""
    import torch
    gpu, ref = _run_pair(2000, nx=280, ny=220, Ra=1e5, Pr=6.2, phi=0.03, d_p=30e-9, seed=5)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if 252 > sms and 288 <= 2 * sms:
        k = gpu.step_kernel()
        assert (k["variant"], k["nodes_per_thread"], k["tile_h"]) == (2, 1, 7), k
    errs = _assert_parity(gpu, ref)
    print("low tiles 280 x 220", errs)


def test_cavity64_20000_steps():
    gpu, ref = _run_pair(20000, nx=64, ny=64, Ra=1e5, Pr=6.2, phi=0.03, d_p=30e-9, seed=2)
    errs = _assert_parity(gpu, ref)
    print("cavity64", errs)


def test_stream_only_matches_oracle_pull():
    """Streaming with the wall rules on a random state: a permutation for f (bit-exact), and
    g exact up to the rounding of the added conduction-profile drop."""
    import torch
    for nx, ny in [(5, 4), (67, 33), (130, 9), (2, 2)]:
        gpu, ref = P.make_pair(nx, ny, 1e3, 6.2, 0.01, 20e-9)
        c = gpu.consts()
        dev = workloads.random_state(nx, ny, seed=nx * 100 + ny)
        gpu.state_set(torch.from_numpy(dev).cuda())
        ref.set_state(P.dev_to_abs(dev, c))
        gpu.stream_only()
        ref.stream_only()
        g = gpu.state_get().cpu().numpy()
        r = P.abs_to_dev(ref.get_state(), c)
        np.testing.assert_array_equal(g[:18], r[:18].astype(np.float32))
        np.testing.assert_allclose(g[18:], r[18:], rtol=0, atol=2.5e-7)


LARGE = dict(nx=4096, ny=2048, Ra=1e6, Pr=6.2, phi=0.02, d_p=50e-9)  # 8.4 M nodes, 1.8 GB


@pytest.mark.parametrize("w,pre", [(workloads.CAVITY_256, 3000), (workloads.CAVITY_1024, 200),
                                   (LARGE, 64)])
def test_one_step_full_size(w, pre):
    """At the benchmark sizes (and a 4096 x 2048 lattice, 32 times the 1024^2 one, with two
    nodes per thread over 32 768 tiles): evolve on the GPU (graph-captured launches, as timed),
    then one more step on both sides from the identical exported state, compared plane by
    plane."""
    import torch
    import oracle
    import paper_1511_04552_gb300 as m
    gpu = m.Cavity(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"])
    gpu.init()
    gpu.step(pre)
    st_abs = P.gpu_state_abs(gpu)
    dev_before = gpu.state_get().clone()
    gpu.step(1)
    after = P.gpu_state_abs(gpu)
    ref = oracle.RefSolver(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"])
    ref.set_state(st_abs)
    ref.step(1)
    r = ref.get_state()
    c = gpu.consts()
    dev_ref = P.abs_to_dev(r, c)
    dev_gpu = P.abs_to_dev(after, c)
    for q in range(27):
        e = P.rel_l2(dev_gpu[q], dev_ref[q])
        assert e < 1e-5, (q, e)
    # the input state itself survived the export unchanged
    gpu.state_set(dev_before)
    assert torch.equal(gpu.state_get(), dev_before)


def test_mass_conservation_gpu():
    w = workloads.CAVITY_32
    gpu, ref = P.make_pair(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"], seed=1)
    m0 = gpu.mass()
    r0 = ref.mass()
    assert abs(m0[0] - r0[0]) < 1e-9 * r0[0] and abs(m0[1] - r0[1]) < 1e-7 * r0[1]
    gpu.step(2000)
    m1 = gpu.mass()
    assert abs(m1[0] - m0[0]) < 1e-6 * m0[0]
    assert abs(m1[1] - m0[1]) < 1e-6 * m0[1]


def test_conduction_limit_gpu():
    mask = 4 | 1 | 8 | 16
    gpu, ref = P.make_pair(24, 16, 1e3, 6.2, 0.02, 20e-9, force_mask=mask)
    gpu.step(300)
    k = gpu.consts()["k_ratio"]
    nh, nc = gpu.nusselt()
    assert abs(nh - k) < 2e-6 * k and abs(nc - k) < 2e-6 * k
    u = gpu.fields(1 | 2).abs().max().item()
    assert u < 1e-7


def test_residual_matches_oracle():
    gpu, ref = _run_pair(1000, nx=40, ny=40, Ra=1e4, Pr=6.2, phi=0.02, d_p=30e-9, seed=4)
    rg, rr = gpu.residual(), ref.residual()
    assert abs(rg - rr) < 1e-3 * rr, (rg, rr)
    gpu.step(500)
    ref.step(500)
    rg, rr = gpu.residual(), ref.residual()
    assert abs(rg - rr) < 1e-3 * rr, (rg, rr)
    assert gpu.residual() == 0.0  # no steps since the last check


def test_diagnostics_equal_the_single_reductions():
    """mclbm_diagnostics (three reductions, one synchronisation) returns exactly what
    mclbm_nusselt, mclbm_mass and mclbm_residual return on an identical cavity, including the
    residual's snapshot handling (0 right after a call)."""
    import paper_1511_04552_gb300 as m
    a = m.Cavity(70, 45, 1e5, 6.2, 0.03, 30e-9).init()
    b = m.Cavity(70, 45, 1e5, 6.2, 0.03, 30e-9).init()
    for n in (500, 333):
        a.step(n)
        b.step(n)
        nu, ms, r = a.nusselt(), a.mass(), a.residual()
        d = b.diagnostics()
        assert (d["nu_hot"], d["nu_cold"]) == nu
        assert (d["mass_w"], d["mass_p"]) == ms
        assert d["residual"] == r and r > 0
    assert b.diagnostics()["residual"] == 0.0 == a.residual()


def test_graph_and_single_launches_agree_bitwise():
    import torch
    import paper_1511_04552_gb300 as m
    a = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9).init()
    b = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9).init()
    a.step(64 * 2 + 7)
    for _ in range(64 * 2 + 7):
        b.step(1)
    assert a.steps_done() == b.steps_done() == 135
    assert torch.equal(a.state_get(), b.state_get())


def test_run_host_matches_device_path():
    import torch
    import paper_1511_04552_gb300 as m
    warm = workloads.perturbed_rest_fields(48, 32, 0.02, seed=9)
    a = m.Cavity(48, 32, 1e4, 6.2, 0.02, 30e-9)
    f_host, nh, nc = a.run_host(warm, 777, P.ALL_FIELDS)
    b = m.Cavity(48, 32, 1e4, 6.2, 0.02, 30e-9)
    b.init(warm=torch.from_numpy(warm).cuda()).step(777)
    assert torch.equal(f_host, b.fields(P.ALL_FIELDS).cpu())
    assert (nh, nc) == b.nusselt()


def test_nan_state_reports_divergence():
    """A non-finite population makes the reductions that read it fail with MCLBM_EDIVERGED,
    and the flag stays set (sticky) until the next init."""
    import paper_1511_04552_gb300 as m
    cav = m.Cavity(16, 16, 1e3, 6.2, 0.01, 20e-9).init()
    for plane, (j, i), call in [(20, (5, 7), "residual"), (3, (2, 0), "mass"),
                                (19, (9, 0), "nusselt")]:
        cav.init()
        cav.step(2)
        st = cav.state_get()
        st[plane, j, i] = float("nan")
        cav.state_set(st)
        cav.step(1)
        with pytest.raises(m.MclbmError) as e:
            getattr(cav, call)()
        assert e.value.code == -5
        with pytest.raises(m.MclbmError):  # sticky
            cav.nusselt()
    cav.init()  # clears the flag
    assert np.isfinite(cav.nusselt()[0])


def test_errors_with_device():
    import torch
    import paper_1511_04552_gb300 as m
    cav = m.Cavity(16, 16, 1e3, 6.2, 0.01, 20e-9)
    L = m.lib()
    assert L.mclbm_init(cav.handle, 2, None) == -1  # warm mode without fields
    assert L.mclbm_step(cav.handle, 1) == -3        # not initialised
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    assert L.mclbm_bind(cav.handle, small.data_ptr(), 1024, None) == -1
    cav.init()
    assert L.mclbm_fields(cav.handle, 0, cav.buffer.data_ptr()) == -1
    assert L.mclbm_step(cav.handle, -1) == -1
    cav.step(3)
    assert cav.steps_done() == 3


def test_determinism():
    import torch
    import paper_1511_04552_gb300 as m
    outs = []
    for _ in range(2):
        cav = m.Cavity(96, 80, 1e5, 6.2, 0.03, 30e-9).init()
        cav.step(300)
        outs.append((cav.state_get(), cav.nusselt(), cav.mass(), cav.residual()))
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


@pytest.mark.parametrize("nx,ny", [(64, 32), (130, 35), (200, 67), (100, 100), (37, 29)])
@pytest.mark.parametrize("storage", [0, 1])
def test_step_variants_bitwise_identical(nx, ny, storage, monkeypatch):
    """The tile kernel and the TMA-staged persistent kernel organise the same per-node
    arithmetic differently; with the same number of nodes per thread their states after 300
    steps are identical bit for bit (16-bit storage with round to nearest, so that the random
    rounding streams do not enter). One node per thread against two (packed FP32x2
    arithmetic): the all-forces build rounds a few operations differently on odd-width
    lattices (a 1-ulp difference first seen in the drag's frozen-force term at the centre
    column), so there the two widths agree to a relative L2 of 1e-6 per plane group in FP32,
    and to 1e-3 with 16-bit storage, where one FP32 ulp can flip a stored rounding."""
    import torch
    import paper_1511_04552_gb300 as m
    states = {}
    for name in ("tile", "tma"):
        for vec in ("1", "2"):
            monkeypatch.setenv("MCLBM_STEP_VARIANT", name)
            monkeypatch.setenv("MCLBM_STEP_VEC", vec)
            cav = m.Cavity(nx, ny, 1e5, 6.2, 0.03, 30e-9, storage=storage, rounding=1).init()
            cav.step(300)
            states[name + vec] = cav.state_get()
            cav.nusselt()  # raises MCLBM_ETIMEOUT if a bounded wait gave up
    assert torch.equal(states["tma1"], states["tile1"])
    assert torch.equal(states["tma2"], states["tile2"])
    a, b = states["tile1"].double(), states["tile2"].double()
    for g in range(3):  # f^w, f^p, g deviations
        den = a[9 * g:9 * g + 9].norm()
        tol = 1e-6 if storage == 0 else 1e-3
        assert (a[9 * g:9 * g + 9] - b[9 * g:9 * g + 9]).norm() <= tol * den, g


@pytest.mark.parametrize("nx,ny,mask,steps", [
    (64, 32, 127, 131),     # graphs of 128 and 2 steps (as pairs) and an odd last step
    (256, 256, 127, 67),    # the benchmark lattice: 128 tiles of 32 x 16
    (130, 35, 127, 64),     # ragged tiles both ways
    (200, 67, 4 | 8 | 16 | 64, 66),  # masked forces (the general build)
    (100, 100, 127, 2),     # one pair
])
def test_two_step_kernel_equals_single_steps(nx, ny, mask, steps, monkeypatch):
    """The two-step kernel (MCLBM_STEP_VARIANT=two; FP32 lattices of at most one 32 x 16 tile
    per SM) runs pairs of steps in one launch, the first step on the tile's 36 x 20
    surroundings kept in shared memory; the states equal those of single steps with one node
    per thread bit for bit."""
    import torch
    import paper_1511_04552_gb300 as m
    monkeypatch.setenv("MCLBM_STEP_VARIANT", "two")
    monkeypatch.delenv("MCLBM_STEP_VEC", raising=False)
    two = m.Cavity(nx, ny, 1e5, 6.2, 0.03, 30e-9, force_mask=mask).init()
    two.step(steps)
    monkeypatch.setenv("MCLBM_STEP_VARIANT", "tma")
    monkeypatch.setenv("MCLBM_STEP_VEC", "1")
    one = m.Cavity(nx, ny, 1e5, 6.2, 0.03, 30e-9, force_mask=mask).init()
    one.step(steps)
    assert two.steps_done() == one.steps_done() == steps
    assert torch.equal(two.state_get(), one.state_get())
    assert two.nusselt() == one.nusselt()


@pytest.mark.parametrize("nx,ny,storage,rounding", [
    (64, 32, 0, 1),     # 32 rows: tile rows of 7, 7, 7, 7 and 4
    (130, 35, 0, 1),    # ragged tiles in x; 35 = 5 x 7
    (200, 67, 1, 1),    # FP16, round to nearest
    (200, 67, 1, 0),    # FP16, stochastic rounding (per-node streams do not depend on tiles)
    (96, 90, 2, 0),     # BF16
])
def test_tile_heights_bitwise_identical(nx, ny, storage, rounding, monkeypatch):
    """The TMA kernel with 32 x 7 tiles and with 32 x 8 tiles (one node per thread) gives the
    same states bit for bit after 300 steps: the tile height changes which CTA computes a node,
    not its arithmetic. The handle reports the kernel it launches."""
    import torch
    import paper_1511_04552_gb300 as m
    monkeypatch.setenv("MCLBM_STEP_VARIANT", "tma")
    monkeypatch.setenv("MCLBM_STEP_VEC", "1")
    states, nus = {}, {}
    for th in ("7", "8"):
        monkeypatch.setenv("MCLBM_STEP_TILE_H", th)
        cav = m.Cavity(nx, ny, 1e5, 6.2, 0.03, 30e-9, storage=storage, rounding=rounding).init()
        k = cav.step_kernel()
        assert (k["variant"], k["nodes_per_thread"], k["tile_h"]) == (2, 1, int(th)), k
        tiles = -(-nx // 32) * -(-ny // int(th))
        assert 1 <= k["grid"] <= tiles
        cav.step(300)
        states[th] = cav.state_get()
        nus[th] = cav.nusselt()
    assert torch.equal(states["7"], states["8"])
    assert nus["7"] == nus["8"]


def test_benchmark_lattice_uses_low_tiles():
    """On the 256 x 256 benchmark lattice 32 x 8 tiles (256) would put a second tile on 104 of
    the 152 SMs; 32 x 7 tiles (8 x 37 = 296) fit two per SM, so the handle picks them (the
    busiest SMs compute 448 nodes instead of 512), and one step from an evolved state still
    equals the oracle's."""
    import paper_1511_04552_gb300 as m
    import torch
    import oracle
    w = workloads.CAVITY_256
    gpu = m.Cavity(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"]).init()
    k = gpu.step_kernel()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if not (256 > sms and 296 <= 2 * sms):
        pytest.skip("the low-tile rule applies for 148 to 255 SMs")
    assert (k["variant"], k["nodes_per_thread"], k["tile_h"], k["grid"]) == (2, 1, 7, 296), k
    gpu.step(500)
    st_abs = P.gpu_state_abs(gpu)
    gpu.step(1)
    after = P.gpu_state_abs(gpu)
    ref = oracle.RefSolver(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"])
    ref.set_state(st_abs)
    ref.step(1)
    c = gpu.consts()
    dev_ref = P.abs_to_dev(ref.get_state(), c)
    dev_gpu = P.abs_to_dev(after, c)
    for q in range(27):
        e = P.rel_l2(dev_gpu[q], dev_ref[q])
        assert e < 1e-5, (q, e)


def test_warm_init_with_density_matches_oracle():
    """MCLBM_INIT_WARM_RHO (ux, uy, theta, phi, rho^w) against the oracle's same init, then 500
    steps."""
    import torch
    nx, ny = 40, 32
    warm = workloads.perturbed_rest_fields(nx, ny, 0.02, seed=5, amp=1e-3).astype(np.float64)
    rng = np.random.default_rng(5)
    rho_w = (1.0 - warm[3]) + 1e-3 * rng.standard_normal((ny, nx))
    w5 = np.concatenate([warm, rho_w[None]]).astype(np.float32)
    import paper_1511_04552_gb300 as m
    import oracle
    gpu = m.Cavity(nx, ny, 1e4, 6.2, 0.02, 30e-9).init(warm=torch.from_numpy(w5).cuda())
    ref = oracle.RefSolver(nx, ny, 1e4, 6.2, 0.02, 30e-9).init(warm=w5.astype(np.float64))
    gpu.step(500)
    ref.step(500)
    _assert_parity(gpu, ref)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_checkpoint_resume_is_bitwise(storage, tmp_path):
    """save after 300 steps, run 200 more; a fresh handle loads the file and runs 200: the same
    state bit for bit (stochastic rounding included) and the same step count."""
    import torch
    import paper_1511_04552_gb300 as m
    st = {"f32": m.STORE_F32, "bf16": m.STORE_BF16}[storage]
    a = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9, storage=st).init()
    a.step(300)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(200)
    b = m.Cavity(70, 50, 1e5, 6.2, 0.03, 30e-9, storage=st).load(path)
    assert b.steps_done() == 300
    b.step(200)
    assert torch.equal(a.state_get(), b.state_get())
    assert a.nusselt() == b.nusselt()
    c = m.Cavity(70, 50, 2e5, 6.2, 0.03, 30e-9, storage=st)
    with pytest.raises(m.MclbmError) as e:
        c.load(path)
    assert e.value.code == m.binding.EPARAM
    d = m.Cavity(72, 50, 1e5, 6.2, 0.03, 30e-9, storage=st)
    with pytest.raises(m.MclbmError) as e:
        d.load(path)
    assert e.value.code == m.binding.EINVAL


def test_bounded_wait_gives_up_and_reports():
    """Failure detection without a fault: the step kernels' bounded mbarrier wait, on a barrier
    that nothing arrives on, gives up after about 2 s and reports MCLBM_ETIMEOUT; the context
    stays usable (a cavity steps afterwards)."""
    import ctypes as C
    import torch
    import paper_1511_04552_gb300 as m
    secs = C.c_double()
    st = torch.cuda.current_stream()
    rc = m.lib().mclbm_selftest_wait_timeout(C.c_void_p(st.cuda_stream), C.byref(secs))
    assert rc == m.binding.ETIMEOUT
    assert 0.1 < secs.value < 10.0, secs.value
    cav = m.Cavity(32, 32, 1e3, 6.2, 0.01, 20e-9).init()
    cav.step(10)
    assert np.isfinite(cav.nusselt()[0])
