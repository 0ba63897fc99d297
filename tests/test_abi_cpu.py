"""C-ABI checks that need no GPU: the library loads, exports every entry point declared in
include/mclbm.h, validates its arguments, and derives the create-time constants (Eqs 7-11,
22-24, SI scales) independently of the oracle yet to the same values."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1511_04552_gb300 import build
    build.build()
    import paper_1511_04552_gb300 as m
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mclbm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(pkg):
    L = pkg.lib()
    decl = _declared()
    assert len(decl) >= 19
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert set(pkg.EXPORTS) <= decl


def test_every_declaration_is_documented():
    """Each entry point in include/*.h sits under a comment that states what it does (several
    declarations of one family may share the comment directly above them)."""
    undocumented = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", fn)).read().split("\n")
        for k, line in enumerate(lines):
            m = re.match(r"^[A-Za-z_][\w\s\*]*?\b(mclbm_\w+)\s*\(", line)
            if not m or line.startswith(("typedef", "#")):
                continue
            j = k - 1
            # skip earlier declarations of the same group (and their continuation lines)
            while j >= 0 and lines[j].strip() and not lines[j].rstrip().endswith("*/"):
                j -= 1
            if j < 0 or not lines[j].rstrip().endswith("*/"):
                undocumented.append("%s: %s" % (fn, m.group(1)))
    assert not undocumented, undocumented


def test_props_default(pkg):
    p = pkg.props_default()
    assert p.rho_f == 997.1 and p.rho_p == 3970.0 and p.force_mask == pkg.F_ALL
    assert p.Ma == 0.1 and p.storage == 0


@pytest.mark.parametrize("args", [(32, 32, 1e3, 6.2, 0.01, 20e-9), (256, 256, 1e5, 6.2, 0.03, 30e-9),
                                  (1024, 1024, 1e6, 6.2, 0.02, 50e-9), (40, 20, 1e6, 8.923, 0.04, 33e-9),
                                  (64, 64, 1e4, 0.71, 0.0, 10e-9), (17, 9, 3e3, 6.2, 0.19, 100e-9)])
def test_consts_match_oracle(pkg, oracle_mod, args):
    h = pkg.create(*args)
    try:
        c = pkg.get_consts(h)
    finally:
        pkg.lib().mclbm_destroy(h)
    r = oracle_mod.RefSolver(*args).consts()
    assert set(c) == set(r)
    for k in c:
        assert abs(c[k] - r[k]) <= 4e-15 * abs(r[k]), (k, c[k], r[k])


@pytest.mark.parametrize("args,code", [((1, 8, 1e3, 6.2, 0.01, 2e-8), -1),
                                       ((8, 40000, 1e3, 6.2, 0.01, 2e-8), -1),
                                       ((8, 8, -1.0, 6.2, 0.01, 2e-8), -2),
                                       ((8, 8, 1e3, 0.0, 0.01, 2e-8), -2),
                                       ((8, 8, 1e3, 6.2, 0.25, 2e-8), -2),
                                       ((8, 8, 1e3, 6.2, -0.01, 2e-8), -2),
                                       ((8, 8, 1e3, 6.2, 0.01, 0.0), -2),
                                       ((8, 8, 1e8, 6.2, 0.01, 2e-8), -2),
                                       ((8, 8, float("nan"), 6.2, 0.01, 2e-8), -2)])
def test_create_rejects(pkg, args, code):
    with pytest.raises(pkg.MclbmError) as e:
        pkg.create(*args)
    assert e.value.code == code


def test_create_rejects_bad_props(pkg):
    for field, val, code in [("Ma", 0.0, -2), ("Ma", 0.7, -2), ("rho_p", -1.0, -2),
                             ("force_mask", 1024, -1), ("storage", 3, -1), ("mu_f", 0.0, -2),
                             ("rounding", 2, -1), ("rounding", -1, -1)]:
        p = pkg.props_default(**{field: val})
        with pytest.raises(pkg.MclbmError) as e:
            pkg.create(16, 16, 1e3, 6.2, 0.01, 2e-8, p)
        assert e.value.code == code, field


def test_unbound_handle_is_refused_without_device_work(pkg):
    L = pkg.lib()
    h = pkg.create(16, 12, 1e3, 6.2, 0.01, 2e-8)
    try:
        assert L.mclbm_step(h, 1) == pkg.binding.ESTATE
        assert L.mclbm_init(h, 0, None) == pkg.binding.ESTATE
        a, b = C.c_double(), C.c_double()
        assert L.mclbm_nusselt(h, C.byref(a), C.byref(b)) == pkg.binding.ESTATE
        assert b"mclbm_bind" in L.mclbm_last_error(h)
        assert L.mclbm_steps_done(h) == 0
        d = [C.c_double() for _ in range(5)]
        assert L.mclbm_diagnostics(h, *[C.byref(x) for x in d]) == pkg.binding.ESTATE
        v = C.c_int(-7)
        assert L.mclbm_step_kernel(h, C.byref(v), None, None, None, None) == pkg.binding.ESTATE
        assert v.value == -7
        n = L.mclbm_buffer_bytes(h)
        assert n >= 2 * 27 * 32 * 12 * 4 + 12 * 16 * 4 * 12
        assert L.mclbm_bind(h, None, n, None) == pkg.binding.EINVAL
        assert L.mclbm_bind(h, C.c_void_p(256), 16, None) == pkg.binding.EINVAL
    finally:
        L.mclbm_destroy(h)
    assert L.mclbm_steps_done(None) == -1
    assert L.mclbm_step_kernel(None, None, None, None, None, None) == pkg.binding.EINVAL
    assert L.mclbm_diagnostics(None, None, None, None, None, None) == pkg.binding.EINVAL
    assert L.mclbm_last_error(None) == b"NULL handle"
    L.mclbm_destroy(None)
    assert L.mclbm_strerror(-5) == b"MCLBM_EDIVERGED"


def test_steady_drivers_refuse_bad_arguments_without_device_work(pkg):
    """mclbm_run_to_steady and mclbm_batch_run_to_steady check their arguments before any
    device call; an unbound handle reports MCLBM_ESTATE from its first step."""
    L = pkg.lib()
    i64, dbl, cint = C.c_int64(), C.c_double(), C.c_int()
    EINVAL, ESTATE = pkg.binding.EINVAL, pkg.binding.ESTATE
    assert L.mclbm_run_to_steady(None, 1e-4, 1000, 10000, None, 0, C.byref(i64), C.byref(dbl),
                                 C.byref(dbl), C.byref(cint)) == EINVAL
    assert L.mclbm_batch_run_to_steady(None, 1e-4, 1000, 10000, None, 0, None, None,
                                       C.byref(i64)) == EINVAL
    h = pkg.create(16, 12, 1e3, 6.2, 0.01, 2e-8)
    try:
        for tol, every, lags, n_lags in ((0.0, 1000, None, 0), (1e-4, 0, None, 0),
                                         (1e-4, 1000, (C.c_int32 * 1)(0), 1)):
            assert L.mclbm_run_to_steady(h, tol, every, 10000, lags, n_lags, None, None, None,
                                         None) == EINVAL
        assert L.mclbm_run_to_steady(h, 1e-4, 1000, 10000, None, 0, None, None, None,
                                     None) == ESTATE
    finally:
        L.mclbm_destroy(h)


def test_storage_types_size_the_buffer(pkg):
    """16-bit storage halves the population planes of the bound buffer."""
    sizes = {}
    for storage in (0, 1, 2):
        h = pkg.create(256, 100, 1e5, 6.2, 0.03, 30e-9, pkg.props_default(storage=storage))
        try:
            sizes[storage] = pkg.lib().mclbm_buffer_bytes(h)
        finally:
            pkg.lib().mclbm_destroy(h)
    planes32 = 2 * 27 * 256 * 100 * 4
    assert sizes[0] - sizes[1] == planes32 // 2 and sizes[1] == sizes[2]


def test_net_config_and_param_count_match_oracle(pkg):
    """The network's parameter count and layout size from the library (host-only calls) against
    the oracle's statement of the same network."""
    import ctypes as C
    from oracle import warmnet as WN
    L = pkg.lib()
    cfg = pkg.binding.NetConfig()
    L.mclbm_net_config_default(C.byref(cfg))
    assert (cfg.ny, cfg.nx, cfg.c0, cfg.hidden, cfg.max_batch) == (256, 256, 16, 64, 16)
    assert L.mclbm_net_param_count(C.byref(cfg)) == WN.param_count(16, 64) == 734293
    for c0, hid in [(8, 16), (24, 5), (64, 1)]:
        c = pkg.binding.NetConfig(32, 48, c0, hid, 2)
        assert L.mclbm_net_param_count(C.byref(c)) == WN.param_count(c0, hid)
        assert L.mclbm_net_workspace_bytes(C.byref(c)) > 0
    for bad in [(20, 32, 16, 64, 4), (32, 32, 12, 64, 4), (32, 32, 16, 0, 4), (32, 32, 16, 64, 0),
                (32, 32, 16, 256, 32), (4096, 4096, 16, 8, 8)]:
        c = pkg.binding.NetConfig(*bad)
        assert L.mclbm_net_param_count(C.byref(c)) == 0
        h = C.c_void_p()
        assert L.mclbm_net_create(C.byref(c), C.byref(h)) == -1
    h = C.c_void_p()
    assert L.mclbm_net_create(C.byref(cfg), C.byref(h)) == 0
    # no workspace bound: every compute call is refused without touching a device
    assert L.mclbm_net_forward(h, 1, None, None) == -3
    assert L.mclbm_net_bind(h, C.c_void_p(256), 16, None) == -1  # too small
    L.mclbm_net_destroy(h)
    # the GEMM validates its operands on the host
    args = lambda **kw: [kw.get(k, v) for k, v in (  # noqa: E731
        ("M", 128), ("N", 128), ("K", 64), ("a", C.c_void_p(256)), ("lda", 64), ("akm", 1),
        ("b", C.c_void_p(256)), ("ldb", 64), ("bkm", 1), ("d", C.c_void_p(256)), ("ldd", 128),
        ("splits", 1), ("kps", 64), ("ss", 0), ("st", None))]
    assert L.mclbm_gemm_bf16(*args(lda=32)) == -1              # leading dimension below K
    assert L.mclbm_gemm_bf16(*args(a=C.c_void_p(257))) == -1   # odd address
    assert L.mclbm_gemm_bf16(*args(kps=96)) == -1              # split not a multiple of 64
    assert L.mclbm_gemm_bf16(*args(K=200, kps=64, splits=3)) == -1  # splits do not cover K
    assert L.mclbm_gemm_bf16(*args(M=0)) == -1
    assert L.mclbm_gemm_bf16(*args(akm=0, lda=100)) == -1      # MN-major: lda below M
