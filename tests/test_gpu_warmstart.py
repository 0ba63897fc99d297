"""The learned warm start against cold starts, judged by the cold solve (both run to the two-lag
steady-Nu test): the trained network shipped with the package, on seeded held-out parameter
points that were not in its training draw, and the warm-start mechanism itself from exact
steady fields."""
import os

import numpy as np
import pytest

import workloads
from tests import _parity as P

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1511_04552_gb300", "weights", "warmnet_256.npz")


@pytest.fixture(scope="module", autouse=True)
def _built():
    P.ensure_built()


# How unique the steady hot-wall Nu is, measured on GB300 (`python -m
# paper_1511_04552_gb300.warmstart --spread 4 --starts 6`): four held-out points, each solved
# from rest and from six rest states perturbed by seeded noise of amplitude 1e-3, all to the
# same two-lag steadiness test, settle (max - min) / median = 5.4e-5, 2.3e-4, 2.7e-4 and 7.7e-4
# apart. The particle component's slow migration leaves each path's phi pattern in place, so
# "the same steady Nu" holds only to that spread; the same cold starts stepped with one node per
# thread instead of two (rounding differences of one ulp) differ by up to 1.0e-4 over 100
# points. The bound is that measured spread, rounded up.
COLD_START_SPREAD = 1e-3
# Of these four points, one lands within 1e-4 of its cold solve (the 100-point evaluation: 19 %,
# all within 7.6e-4); the count guards against a regression toward larger differences.
MIN_WITHIN_1E4 = 1


def test_trained_network_shortens_the_steady_solve():
    """Four held-out points at 256^2: the warm starts need fewer steps in total than the cold
    starts and reach the cold solve's steady Nu within the model's measured cold-start spread."""
    from paper_1511_04552_gb300 import warmstart as W
    assert os.path.exists(WEIGHTS), "the trained network must ship with the package"
    net = W.WarmNet.load(WEIGHTS)
    conds = workloads.random_conditions(4, seed=3)
    ev = W.evaluate(net, conds, group=4)
    within = int(np.sum(ev["nu_rel_diff"] <= 1e-4))
    print("cold steps", ev["cold_steps"], "warm steps", ev["warm_steps"], "Nu rel diff",
          ev["nu_rel_diff"], "within 1e-4: %d of %d" % (within, len(conds)))
    assert ev["warm_steps"].sum() < ev["cold_steps"].sum()
    assert np.all(ev["nu_rel_diff"] <= COLD_START_SPREAD)
    assert within >= MIN_WITHIN_1E4


def test_warm_start_from_exact_steady_fields():
    """The mechanism without the network: seeding a cavity with its own steady (u, theta, phi,
    rho^w) must return to the same steady Nu within the steadiness tolerance, faster than the
    cold start."""
    import paper_1511_04552_gb300 as m
    from paper_1511_04552_gb300.warmstart import FIELD_MASK
    Ra, phi, dp = 3e4, 0.02, 40e-9
    cold = m.Cavity(128, 128, Ra, 6.2, phi, dp).init()
    rc = m.run_to_steady(cold)
    f = cold.fields(FIELD_MASK).clone()
    warm = m.Cavity(128, 128, Ra, 6.2, phi, dp).init(warm=f)
    rw = m.run_to_steady(warm)
    print("cold", rc["steps"], rc["nu_hot"], "warm", rw["steps"], rw["nu_hot"])
    assert rc["converged"] and rw["converged"]
    assert abs(rw["nu_hot"] - rc["nu_hot"]) <= 1e-4 * rc["nu_hot"]
    assert rw["steps"] < rc["steps"]
