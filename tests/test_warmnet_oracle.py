"""Pins of the FP64 warm-start network oracle (oracle/warmnet.py) against things other than
itself: scipy's 2-D correlation, adjoint identities, central finite differences of the loss,
torch's float32 -> bfloat16 conversion, closed forms of Adam's first step and of the loss of a
constant output, and the parameter count worked out by hand."""
import numpy as np
import pytest

import workloads
from oracle import warmnet as WN


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_matches_scipy_correlate(stride):
    from scipy.signal import correlate2d
    r = _rng(1)
    x = r.normal(size=(2, 3, 8, 10))
    W = r.normal(size=(4, 3, 3, 3))
    b = r.normal(size=4)
    out = WN.conv3x3(x, W, b, stride)
    for bi in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[bi, i], W[o, i], mode="same") for i in range(3)) + b[o]
            np.testing.assert_allclose(out[bi, o], ref[::stride, ::stride], rtol=1e-13, atol=1e-13)


def test_conv_backward_is_adjoint():
    """<conv(x) - b, y> = <x, dX(y)> and the weight gradient is d<conv(x), y>/dW (linearity)."""
    r = _rng(2)
    for stride in (1, 2):
        x = r.normal(size=(2, 3, 8, 8))
        W = r.normal(size=(5, 3, 3, 3))
        y = r.normal(size=(2, 5, 8 // stride, 8 // stride))
        z = np.zeros(5)
        dx, dW, db = WN.conv3x3_backward(x, W, y, stride)
        lhs = np.sum(WN.conv3x3(x, W, z, stride) * y)
        assert np.isclose(lhs, np.sum(x * dx), rtol=1e-12)
        assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)
        np.testing.assert_allclose(db, y.sum(axis=(0, 2, 3)))


def test_upsample_adjoint():
    r = _rng(3)
    x = r.normal(size=(2, 3, 4, 5))
    y = r.normal(size=(2, 3, 8, 10))
    assert np.isclose(np.sum(WN.up2(x) * y), np.sum(x * WN.up2_backward(y)), rtol=1e-13)
    assert WN.up2(x)[1, 2, 7, 9] == x[1, 2, 3, 4]


def test_param_count_by_hand():
    # conv weights 685 584 (the 5-channel head has 16*5*9 = 720), conv biases 613, conditioning
    # MLP 3*64 + 64 + 736*64 + 736 = 48 096
    assert WN.param_count(16, 64) == 734293
    segs = WN.param_segments(16, 64)
    assert sum(s for _, s, _ in segs) == 734293
    assert [n for n, _, _ in segs][:2] == ["e0.W", "e0.b"] and segs[-1][0] == "b2"


def test_bf16_round_matches_torch():
    import torch
    r = _rng(4)
    x = np.concatenate([r.normal(size=4000) * 10.0 ** r.integers(-8, 8, 4000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.5 - 2.0 ** -8, 0.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(WN.bf16_round(x), ref)
    assert WN.bf16_round(1.0 + 2.0 ** -8) == 1.0            # tie to even
    assert WN.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.015625  # tie to even (upwards)


def test_adam_first_step_closed_form():
    """After one step from zero moments, m/(1-b1) = g and v/(1-b2) = g^2, so every parameter
    moves by lr * g / (|g| + eps)."""
    g = np.array([1e-3, -2.0, 5.0, 0.0])
    p0 = np.array([0.1, 0.2, -0.3, 0.4])
    p1, m, v = WN.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=1e-2)
    np.testing.assert_allclose(p1, p0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def _tiny(seed=0):
    c0, hid, n = 2, 4, 16
    p = workloads.random_net_params(WN.param_segments(c0, hid), seed=seed).astype(np.float64)
    cond = WN.condition([2e3, 3e5], [0.01, 0.04], [20e-9, 90e-9])
    r = _rng(5 + seed)
    fields = r.normal(size=(2, 5, n, n))
    mean, scale = np.array([0.1, -0.2, 0.0, 0.3, 0.05]), np.array([2.0, 0.5, 1.0, 3.0, 0.7])
    return c0, hid, n, p, cond, fields, mean, scale


PHI = np.array([0.01, 0.04])


def test_loss_of_constant_output():
    """All weights zero and the output bias b: every output equals b, so the loss is the mean of
    (b_ch - (F - mean_ch)/scale_ch)^2."""
    c0, hid, n, p, cond, fields, mean, scale = _tiny()
    p = np.zeros_like(p)
    lay, _ = WN.param_layout(c0, hid)
    o, _ = lay["out.b"]
    b = np.array([0.3, -0.1, 0.2, 0.05, -0.4])
    p[o:o + 5] = b
    loss, g = WN.loss_and_grad(p, cond, fields, mean, scale, n, n, c0, hid, phi=PHI)
    base = np.zeros((2, 5))
    base[:, 3], base[:, 4] = PHI, 1.0 - PHI
    t = (fields - base[:, :, None, None] - mean[None, :, None, None]) / scale[None, :, None, None]
    assert np.isclose(loss, np.mean((b[None, :, None, None] - t) ** 2), rtol=1e-14)
    np.testing.assert_allclose(g[o:o + 5], 2.0 * np.mean(b[None, :, None, None] - t, axis=(0, 2, 3)) / 5,
                               rtol=1e-12)


def test_gradient_matches_central_differences():
    """dL/dp from backward() against (L(p + h e_k) - L(p - h e_k)) / 2h for a few parameters of
    every tensor (FP64, no rounding)."""
    c0, hid, n, p, cond, fields, mean, scale = _tiny()
    loss, g = WN.loss_and_grad(p, cond, fields, mean, scale, n, n, c0, hid, phi=PHI)
    lay, _ = WN.param_layout(c0, hid)
    r = _rng(9)
    worst = 0.0
    for name, (o, s) in lay.items():
        size = int(np.prod(s))
        for k in r.choice(size, size=min(3, size), replace=False):
            h = 1e-5
            pp, pm = p.copy(), p.copy()
            pp[o + k] += h
            pm[o + k] -= h
            lp = WN.loss_and_grad(pp, cond, fields, mean, scale, n, n, c0, hid, phi=PHI)[0]
            lm = WN.loss_and_grad(pm, cond, fields, mean, scale, n, n, c0, hid, phi=PHI)[0]
            fd = (lp - lm) / (2 * h)
            err = abs(fd - g[o + k]) / max(abs(fd), 1e-4 * abs(loss))
            worst = max(worst, err)
            assert err < 1e-5, (name, k, fd, g[o + k])
    print("worst FD relative error", worst)


def test_bf16_mode_stays_close_to_fp64():
    """Rounding the convolution operands to bfloat16 changes the loss and gradient by about the
    bfloat16 unit roundoff (2^-8), not more."""
    c0, hid, n, p, cond, fields, mean, scale = _tiny(1)
    l64, g64 = WN.loss_and_grad(p, cond, fields, mean, scale, n, n, c0, hid, phi=PHI)
    l16, g16 = WN.loss_and_grad(p, cond, fields, mean, scale, n, n, c0, hid, bf16=True, phi=PHI)
    assert abs(l16 - l64) < 2e-2 * l64
    assert np.linalg.norm(g16 - g64) < 5e-2 * np.linalg.norm(g64)
    assert l16 != l64


def test_field_stats():
    r = _rng(6)
    phi = np.array([0.0, 0.02, 0.05])
    f = r.normal(size=(3, 5, 5, 6)) * np.array([1, 2, 3, 0, 1])[None, :, None, None] + 7.0
    f[:, 3] = phi[:, None, None]  # phi equal to its rest value: a constant deviation
    mean, scale = WN.field_stats(f, phi)
    assert scale[3] == 1.0 and mean[3] == 0.0  # a constant channel keeps unit scale
    np.testing.assert_allclose(mean[:3], [f[:, c].mean() for c in range(3)])
    np.testing.assert_allclose(mean[4], (f[:, 4] - (1.0 - phi)[:, None, None]).mean())


def test_predicted_masses_are_the_cold_starts():
    """phi and rho^w means are phi_0 and 1 - phi_0; the other channels are base + mean +
    scale * out, and phi, rho^w differ from that by a constant per sample."""
    c0, hid, n, p, cond, fields, mean, scale = _tiny()
    f = WN.predict_fields(p, cond, mean, scale, n, n, c0, hid, phi=PHI)
    np.testing.assert_allclose(f[:, 3].mean(axis=(1, 2)), PHI, rtol=1e-13)
    np.testing.assert_allclose(f[:, 4].mean(axis=(1, 2)), 1.0 - PHI, rtol=1e-13)
    out, _ = WN.forward(p, cond, n, n, c0, hid)
    raw = mean[None, :, None, None] + scale[None, :, None, None] * out
    np.testing.assert_allclose(f[:, :3], raw[:, :3], rtol=1e-14)
    for ch in (3, 4):
        d = f[:, ch] - raw[:, ch]
        assert np.ptp(d[0]) < 1e-14 and np.ptp(d[1]) < 1e-14


def test_conv_flop_count_matches_the_network_definition():
    """warmstart.conv_flops (the training benchmark's FLOP count) against a count taken from
    the oracle's layer list: 2 multiply-adds per weight per output pixel."""
    from paper_1511_04552_gb300.warmstart import conv_flops, sample_conditions
    c0, ny, nx, batch = 16, 256, 256, 3
    grid = {"e0": 1, "e1": 2, "e2": 4, "e3": 8, "e4": 16, "d3": 8, "d2": 4, "d1": 2, "d0": 1,
            "out": 1}
    ref = 0.0
    for name, cu, cs, co, _, _, _ in WN.layers(c0):
        s = grid[name]
        ref += 2.0 * batch * (ny // s) * (nx // s) * co * 9 * (cu + cs)
    assert conv_flops(ny, nx, c0, batch) == ref
    c = sample_conditions(500, 4)
    assert np.all((c[:, 0] >= 1e3) & (c[:, 0] <= 1e6))
    assert np.all((c[:, 1] >= 0.0) & (c[:, 1] <= 0.05))
    assert np.all((c[:, 2] >= 10e-9) & (c[:, 2] <= 100e-9))
