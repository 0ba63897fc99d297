"""The seeded input generators shared by the CUDA path and the oracle (no GPU): splitmix64 pinned
to its published output sequence, and the workloads' shapes, ranges and determinism."""
import numpy as np

import workloads as W


def test_splitmix64_matches_the_published_sequence():
    """splitmix64 started from state 0 (Steele, Lea and Flood 2014; the generator used to seed
    xoshiro): its first five outputs."""
    out = W.splitmix64(np.arange(5, dtype=np.uint64))
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                                     0xF88BB8A8724C81EC, 0x1B39896A51A8749B]


def test_uniform_draws_are_in_range_and_counter_based():
    u = W.uniform_pm1(3, 2, 100000)
    assert u.dtype == np.float64 and u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
    # counter based: a prefix is the shorter draw; other streams and seeds differ
    np.testing.assert_array_equal(W.uniform_pm1(3, 2, 10), u[:10])
    assert not np.array_equal(W.uniform_pm1(3, 1, 10), u[:10])
    assert not np.array_equal(W.uniform_pm1(4, 2, 10), u[:10])


def test_perturbed_rest_fields():
    nx, ny, phi0, amp = 40, 24, 0.03, 1e-3
    f = W.perturbed_rest_fields(nx, ny, phi0, seed=5, amp=amp)
    assert f.shape == (4, ny, nx) and f.dtype == np.float32
    assert np.abs(f[0]).max() <= amp and np.abs(f[1]).max() <= amp
    theta0 = 0.5 - (np.arange(nx) + 0.5) / nx
    assert np.abs(f[2] - theta0[None, :]).max() <= amp * (1 + 1e-6)
    assert np.abs(f[3] / phi0 - 1.0).max() <= amp * (1 + 1e-5)
    np.testing.assert_array_equal(f, W.perturbed_rest_fields(nx, ny, phi0, seed=5, amp=amp))


def test_sweep80_is_the_full_grid_with_every_size():
    sw = W.sweep80()
    assert len(sw) == 80
    assert {(c["Ra"], c["phi"], c["d_p"]) for c in sw} == {
        (r, p, d) for r in W.SWEEP_RA for p in W.SWEEP_PHI for d in W.SWEEP_DP}
    sizes = [c["nx"] for c in sw]
    assert set(sizes) == set(W.SWEEP_SIZES) and all(c["nx"] == c["ny"] for c in sw)
    assert sum(n * n for n in sizes) == 7761920  # the 7.76 M nodes of the benchmark's sweep
    assert W.sweep80() == sw


def test_random_conditions_ranges():
    c = W.random_conditions(1000, seed=3)
    assert c.shape == (1000, 3)
    assert 1e3 <= c[:, 0].min() and c[:, 0].max() < 1e6
    assert 0.0 <= c[:, 1].min() and c[:, 1].max() < 0.05
    assert 10e-9 <= c[:, 2].min() and c[:, 2].max() < 100e-9
    np.testing.assert_array_equal(c, W.random_conditions(1000, seed=3))
