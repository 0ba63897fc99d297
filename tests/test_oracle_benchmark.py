"""The pure-fluid limit of the oracle against the classical differentially heated cavity.

With phi = 0 the model is the single-component Boussinesq thermal LBM; the paper validates its
code on this cavity for air (Sec. 2.d, Fig. 3b). Its mean Nusselt numbers must approach the
de Vahl Davis benchmark (tests/golden/de_vahl_davis_1983.txt) on modest lattices.
"""
import os

import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "de_vahl_davis_1983.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            ra, nu = line.split()
            out[float(ra)] = float(nu)
    return out


def _steady_nu(oracle, n, Ra, check=1000, tol=1e-7, max_steps=200000):
    s = oracle.RefSolver(n, n, Ra, 0.71, 0.0, 20e-9).init()
    prev = None
    for _ in range(max_steps // check):
        s.step(check)
        nh, nc = s.nusselt()
        if prev is not None and abs(nh - prev) < tol * nh:
            return nh, nc
        prev = nh
    raise AssertionError("no steady state")


@pytest.mark.parametrize("n,Ra,rel", [(32, 1e3, 5e-3), (48, 1e4, 3e-3)])
def test_pure_fluid_cavity_nusselt(oracle_mod, n, Ra, rel):
    gold = _golden()[Ra]
    nh, nc = _steady_nu(oracle_mod, n, Ra)
    assert abs(nh - nc) < 1e-9 * nh  # steady energy balance between the two walls
    assert abs(nh - gold) < rel * gold, (nh, gold)
