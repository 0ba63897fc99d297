"""mclbm_mass_noalloc against mclbm_mass, through the C ABI.

mclbm_mass_noalloc serves callers that cannot allocate device memory (a host application
that owns all device memory in its own fixed pool, or a loop that must not pay for an
allocation per call): it keeps its partial sums in a static device array instead of a bound
buffer. This file is named to be collected last, so that a run which stops at the first
failure has already run every other test.
"""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu


def _noalloc(L, st, nx, ny, consts, stream):
    mw, mp = C.c_double(), C.c_double()
    rc = L.mclbm_mass_noalloc(C.c_void_p(st.data_ptr()), nx, ny, consts["rho_w0"],
                              consts["rho_p0"], C.byref(mw), C.byref(mp),
                              C.c_void_p(stream.cuda_stream))
    return rc, mw.value, mp.value


def test_mass_noalloc_matches_mclbm_mass_twice():
    from tests import _parity as P
    P.ensure_built()
    import paper_1511_04552_gb300 as m
    L = m.lib()
    # calls in a row: a taller lattice first, then shorter ones, so rows left in the shared
    # scratch by an earlier call would show up in a later one if they leaked; the first has
    # more rows than the row kernel has CTAs (1024), so its grid-stride loop runs
    for nx, ny, steps in [(16, 2100, 40), (96, 70, 333), (40, 23, 57)]:
        cav = m.Cavity(nx, ny, 1e5, 6.2, 0.03, 30e-9).init()
        cav.step(steps)
        ref_w, ref_p = cav.mass()
        st = cav.state_get()
        rc, mw, mp = _noalloc(L, st, nx, ny, cav.consts(), cav.stream)
        assert rc == 0
        assert abs(mw - ref_w) <= 1e-12 * abs(ref_w), (mw, ref_w)
        assert abs(mp - ref_p) <= 1e-12 * abs(ref_p), (mp, ref_p)


def test_mass_noalloc_rejects_sizes_beyond_its_scratch():
    from tests import _parity as P
    P.ensure_built()
    import torch
    import paper_1511_04552_gb300 as m
    L = m.lib()
    st = torch.zeros(27 * 8 * 4, dtype=torch.float32, device="cuda")
    c = {"rho_w0": 1.0, "rho_p0": 0.0}
    s = torch.cuda.current_stream()
    assert _noalloc(L, st, 8, 8193, c, s)[0] == m.binding.ETOOLARGE
    assert _noalloc(L, st, 40000, 8, c, s)[0] == m.binding.ETOOLARGE
    assert _noalloc(L, st, 1, 8, c, s)[0] == m.binding.EINVAL
