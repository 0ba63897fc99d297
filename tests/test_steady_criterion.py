"""The steady-Nusselt test (mclbm_steady_nu_reached in the C library, called through the
binding) on synthetic histories; no GPU needed."""
import numpy as np

from paper_1511_04552_gb300.binding import steady_nu_reached


def _first_stop(seq, tol=1e-4, lags=(1, 32)):
    for n in range(1, len(seq) + 1):
        if steady_nu_reached(list(seq[:n]), tol, lags):
            return n
    return None


def test_geometric_approach_stops_within_tolerance():
    """Nu_n = Nu_inf + A r^n from either side: the check stops once the true distance to the
    limit is at most about tol, never earlier than that by more than the estimate's slack."""
    for A in (1.0, -0.5, 3.0):
        for r in (0.5, 0.9, 0.98):
            seq = 4.0 + A * r ** np.arange(2000)
            n = _first_stop(seq)
            assert n is not None
            dist = abs(seq[n - 1] - 4.0) / 4.0
            assert dist <= 1.0001e-4, (A, r, dist)
            if n > 161:  # not long after either (161 checks: the history the lags need)
                assert abs(seq[n - 2] - 4.0) / 4.0 > 0.5e-4 * r


def test_extremum_of_the_transient_does_not_stop():
    """An overshoot: Nu rises, peaks and relaxes; near the peak successive changes are small
    (a plain change test stops there), but they change sign."""
    t = np.arange(400) * 1000.0
    seq = 3.0 - 2.0 * np.exp(-t / 2e4) + 1.5 * (t / 2e4) * np.exp(-t / 2e4)
    n = _first_stop(seq)
    assert n is not None
    peak = int(np.argmax(seq))
    assert n > peak + 3
    assert abs(seq[n - 1] - 3.0) <= 1.5e-4 * 3.0


def test_damped_oscillation_waits_for_the_floor_or_a_monotone_tail():
    t = np.arange(3000)
    seq = 5.0 + 0.1 * np.cos(t * 0.7) * np.exp(-t / 200.0)
    n = _first_stop(seq)
    assert n is not None and abs(seq[n - 1] - 5.0) <= 1e-4 * 5.0


def test_fixed_point_noise_stops_on_the_floor():
    r = np.random.default_rng(0)
    seq = 2.0 + 1e-8 * r.standard_normal(400)
    assert _first_stop(seq) == 161  # the first six values 32 checks apart
    assert _first_stop(seq, lags=(1,)) == 6
    assert not steady_nu_reached([1.0, 1.1, 1.2, 1.25, 1.27], lags=(1,))  # too short


def test_small_persistent_wobble_counts_as_steady():
    """A neutral oscillation of relative amplitude 1e-5 about the limit (e.g. a weakly damped
    acoustic mode) is steady to 1e-4; one of amplitude 1e-3 is not."""
    t = np.arange(400)
    assert _first_stop(3.0 + 3e-5 * np.sin(1.3 * t)) == 161
    assert _first_stop(3.0 + 3e-3 * np.sin(1.3 * t)) is None


def test_slow_mode_behind_a_fast_one():
    """Nu = 3 + 0.5 e^(-t/3) + 2e-3 e^(-t/300) (checks as time unit): the two-lag test stops
    within the tolerance of the limit."""
    t = np.arange(6000)
    seq = 3.0 + 0.5 * np.exp(-t / 3.0) + 2e-3 * np.exp(-t / 300.0)
    n = _first_stop(seq)
    assert n is not None and abs(seq[n - 1] - 3.0) <= 1e-4 * 3.0


def test_ablation_cases_keep_drag_and_buoyancy():
    from paper_1511_04552_gb300 import binding as B
    from paper_1511_04552_gb300.studies import ABLATION
    masks = [m for _, m in ABLATION]
    assert len(set(masks)) == len(masks) and masks[0] == B.F_ALL
    for m in masks:
        assert m & B.F_DRAG and m & B.F_BUOYANCY and 0 < m <= B.F_ALL
    assert sorted(bin(B.F_ALL ^ m).count("1") for m in masks) == [0, 1, 1, 1, 1, 1]


def _restated(hist, tol, lags, floor=2e-7, spread=0.05):
    """The steadiness test restated from its definition (include/mclbm.h), independently of the
    library's code: for every lag, the six values 0, L, ..., 5L checks back."""
    if len(hist) < 5 * max(lags) + 1:
        return False
    for L in lags:
        p = [hist[-1 - k * L] for k in range(6)]
        d = [p[k] - p[k + 1] for k in range(5)]
        nu = abs(p[0])
        if abs(d[0]) <= floor * L * nu and abs(d[1]) <= floor * L * nu:
            continue
        flips = sum(d[k] * d[k + 1] < 0 for k in range(4))
        if flips >= 2 and max(p) - min(p) <= 0.5 * tol * nu:
            continue
        if any(x == 0.0 for x in d[1:]):
            return False
        r = [d[k] / d[k + 1] for k in range(4)]
        if min(r) < 0.0 or max(r) >= 0.99 or max(r) - min(r) > spread:
            return False
        if abs(d[0]) * max(r) / (1.0 - max(r)) > tol * nu:
            return False
    return True


def test_library_test_matches_its_definition_on_random_histories():
    """mclbm_steady_nu_reached against the restated definition on every prefix of random
    histories: relaxations with one or two modes, noise at and above the round-off floor,
    damped and persistent oscillations, several tolerances and lag sets."""
    rng = np.random.default_rng(11)
    t = np.arange(260, dtype=np.float64)
    for case in range(60):
        kind = case % 4
        nu0 = rng.uniform(1.0, 8.0)
        if kind == 0:
            seq = nu0 + rng.uniform(-1, 1) * rng.uniform(0.8, 0.99) ** t
        elif kind == 1:
            seq = (nu0 + rng.uniform(-1, 1) * np.exp(-t / rng.uniform(2, 10))
                   + rng.uniform(-3e-3, 3e-3) * np.exp(-t / rng.uniform(50, 400)))
        elif kind == 2:
            seq = nu0 + rng.uniform(1e-9, 1e-5) * rng.standard_normal(t.size) * nu0
        else:
            seq = nu0 + rng.uniform(1e-6, 1e-3) * np.sin(rng.uniform(0.3, 2.5) * t) * \
                np.exp(-t / rng.uniform(50, 5000)) * nu0
        tol = [1e-4, 1e-3, 1e-5][case % 3]
        lags = [(1, 32), (1,), (1, 4, 16)][(case // 3) % 3]
        for n in range(1, t.size + 1):
            h = list(seq[:n])
            assert steady_nu_reached(h, tol, lags) == _restated(h, tol, lags), (case, n)


def test_bad_arguments_are_refused():
    from paper_1511_04552_gb300.binding import MclbmError
    for kw in (dict(tol=0.0), dict(tol=-1.0), dict(lags=()), dict(lags=(0,)), dict(lags=(1,) * 9)):
        try:
            steady_nu_reached([1.0] * 10, **kw)
        except MclbmError as e:
            assert e.code == -1
        else:
            raise AssertionError(kw)
