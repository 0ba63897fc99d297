"""FP64 CPU restatement of the warm-start network: a conditioned convolutional encoder-decoder
that maps the cavity parameters (Ra, phi, d_p) and a geometry encoding to the steady fields
u_x, u_y, theta, phi and rho^w (the base-fluid partial density, i.e. the pressure), used to
seed the MCLBM solver.

TEST INFRASTRUCTURE. Only tests/ (and the smoke check) use this module; the CUDA library never
imports it and shares no code with it. It is deliberately plain: every convolution is the sum of
nine shifted channel contractions (one numpy matmul per tap), nothing is fused or reordered.

The paper has no learned component; the network is this project's design, and the definition
below is the one the CUDA path implements independently:

* Geometry input X (4 channels, ny x nx): mask m (1 inside the cavity), m*xi, m*eta, m*4*xi*eta
  with xi = (i + 1/2)/nx - 1/2 and eta = (j + 1/2)/ny - 1/2.
* Conditioning c = ((log10 Ra - 4.5)/1.5, (phi - 0.025)/0.025, (d_p/1 nm - 55)/45).
* conv(x; W, b, s): 3x3, zero padding 1, stride s; out[o, y, x] = b[o] +
  sum_{i,ky,kx} W[o, i, ky, kx] in[i, s*y + ky - 1, s*x + kx - 1].
* SiLU(z) = z / (1 + exp(-z)).  up(x): nearest-neighbour upsampling by 2.  cat: channel concat.
* Channels C = (c0, 2c0, 4c0, 8c0, 8c0). Layers, in parameter order:
    e0 = silu(conv(X, 4 -> C0, 1))
    e1 = silu(conv(e0, C0 -> C1, 2)); e2 = silu(conv(e1, C1 -> C2, 2)); e3 = silu(conv(e2, C2 -> C3, 2))
    e4 = silu(film(conv(e3, C3 -> C4, 2)))
    d3 = silu(film(conv(cat(up(e4), e3), C4 + C3 -> C3, 1)))
    d2 = silu(film(conv(cat(up(d3), e2), C3 + C2 -> C2, 1)))
    d1 = silu(film(conv(cat(up(d2), e1), C2 + C1 -> C1, 1)))
    d0 = silu(film(conv(cat(up(d1), e0), C1 + C0 -> C0, 1)))
    out = conv(d0, C0 -> 5, 1)
  film(p) = gamma * p + beta per sample and channel, gamma = 1 + r[a : a + C], beta = r[a + C : a + 2C],
  with r = W2 silu(W1 c + b1) + b2 and the FiLM layers e4, d3, d2, d1, d0 taking consecutive
  slices of r in that order.
* Parameters, one flat FP32 vector: for each conv layer in the order above W [Cout][Cin][3][3]
  then b [Cout]; then W1 [hidden][3], b1 [hidden], W2 [F][hidden], b2 [F], F = 2 (C4+C3+C2+C1+C0).
* Fields F = (u_x, u_y, theta, phi, rho^w). Channels 3 and 4 are learned as deviations from the
  sample's rest values, base = (0, 0, 0, phi_0, 1 - phi_0): F_ch = base_ch + mean_ch +
  scale_ch * out_ch (per-channel normaliser of F - base, not trained). For a warm start phi and
  rho^w are then shifted by a constant each so that their cavity means are phi_0 and 1 - phi_0:
  the solver conserves both components' masses, so the steady state has the cold start's.
  Loss = mean over samples, channels and nodes of (out - (F_target - base - mean)/scale)^2.
* Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

With bf16=True every operand of a convolution (its input values, its weights, and in the
backward pass the gradient with respect to its pre-activation) is rounded to bfloat16 (round to
nearest even) before the FP64 arithmetic, which is what a BF16 tensor-core GEMM with exact
accumulation computes; with bf16=False the network is evaluated in plain FP64.
"""
import numpy as np

N_IN = 4
N_OUT = 5
FILM_LAYERS = ("e4", "d3", "d2", "d1", "d0")


def channels(c0):
    return (c0, 2 * c0, 4 * c0, 8 * c0, 8 * c0)


def layers(c0):
    """(name, cin_up, cin_skip, cout, stride, film, act) in parameter order. cin_up channels come
    from the upsampled (or plain, for the encoder) source, cin_skip from the skip source."""
    C = channels(c0)
    return [
        ("e0", N_IN, 0, C[0], 1, False, True),
        ("e1", C[0], 0, C[1], 2, False, True),
        ("e2", C[1], 0, C[2], 2, False, True),
        ("e3", C[2], 0, C[3], 2, False, True),
        ("e4", C[3], 0, C[4], 2, True, True),
        ("d3", C[4], C[3], C[3], 1, True, True),
        ("d2", C[3], C[2], C[2], 1, True, True),
        ("d1", C[2], C[1], C[1], 1, True, True),
        ("d0", C[1], C[0], C[0], 1, True, True),
        ("out", C[0], 0, N_OUT, 1, False, False),
    ]


def film_width(c0):
    C = channels(c0)
    return 2 * (C[4] + C[3] + C[2] + C[1] + C[0])


def param_layout(c0, hidden):
    """name -> (offset, shape) in the flat parameter vector."""
    lay = {}
    off = 0
    for name, cu, cs, co, _, _, _ in layers(c0):
        cin = cu + cs
        lay[name + ".W"] = (off, (co, cin, 3, 3))
        off += co * cin * 9
        lay[name + ".b"] = (off, (co,))
        off += co
    F = film_width(c0)
    for name, shape in (("W1", (hidden, 3)), ("b1", (hidden,)), ("W2", (F, hidden)), ("b2", (F,))):
        lay[name] = (off, shape)
        off += int(np.prod(shape))
    return lay, off


def param_count(c0, hidden):
    return param_layout(c0, hidden)[1]


def unpack(params, c0, hidden):
    lay, n = param_layout(c0, hidden)
    assert params.size == n
    return {k: params[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in lay.items()}


def pack(d, c0, hidden):
    lay, n = param_layout(c0, hidden)
    out = np.zeros(n)
    for k, (o, s) in lay.items():
        out[o:o + int(np.prod(s))] = np.asarray(d[k], dtype=np.float64).ravel()
    return out


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64. The value is first
    rounded to float32 (as the CUDA path holds it) and then to 8 mantissa bits."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def geometry(ny, nx):
    """The 4 input channels [4][ny][nx] of a full square-cavity mask."""
    xi = (np.arange(nx) + 0.5) / nx - 0.5
    eta = (np.arange(ny) + 0.5) / ny - 0.5
    XI, ETA = np.meshgrid(xi, eta)
    m = np.ones((ny, nx))
    return np.stack([m, m * XI, m * ETA, m * 4.0 * XI * ETA])


def condition(Ra, phi, d_p):
    """Normalised conditioning vector(s), shape [..., 3]."""
    Ra, phi, d_p = (np.asarray(v, dtype=np.float64) for v in (Ra, phi, d_p))
    return np.stack([(np.log10(Ra) - 4.5) / 1.5, (phi - 0.025) / 0.025,
                     (d_p * 1e9 - 55.0) / 45.0], axis=-1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def pad1(x):
    return np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))


def conv3x3(x, W, b, stride):
    """x [B][Cin][H][W], W [Cout][Cin][3][3] -> [B][Cout][H/s][W/s]: one matmul per tap."""
    B, Cin, H, Wd = x.shape
    Ho, Wo = H // stride, Wd // stride
    xp = pad1(x)
    out = np.zeros((B, W.shape[0], Ho, Wo))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride]
            out += np.einsum("oi,bihw->bohw", W[:, :, ky, kx], patch)
    return out + b[None, :, None, None]


def conv3x3_backward(x, W, dpre, stride):
    """Gradients of conv3x3 with respect to x, W and b, given dL/d(output)."""
    B, Cin, H, Wd = x.shape
    Ho, Wo = dpre.shape[2], dpre.shape[3]
    xp = pad1(x)
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(None), slice(ky, ky + stride * Ho, stride),
                  slice(kx, kx + stride * Wo, stride))
            dW[:, :, ky, kx] = np.einsum("bohw,bihw->oi", dpre, xp[sl])
            dxp[sl] += np.einsum("oi,bohw->bihw", W[:, :, ky, kx], dpre)
    db = dpre.sum(axis=(0, 2, 3))
    return dxp[:, :, 1:-1, 1:-1], dW, db


def up2(x):
    return x.repeat(2, axis=2).repeat(2, axis=3)


def up2_backward(d):
    B, C, H, W = d.shape
    return d.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(params, cond, ny, nx, c0=16, hidden=64, geom=None, bf16=False):
    """Network output (normalised fields) [B][5][ny][nx] and the cache for backward().
    cond: [B][3] normalised conditioning (see condition())."""
    P = unpack(np.asarray(params, dtype=np.float64), c0, hidden)
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    cond = np.asarray(cond, dtype=np.float64).reshape(-1, 3)
    B = cond.shape[0]
    if geom is None:
        geom = geometry(ny, nx)
    X = np.broadcast_to(geom, (B,) + geom.shape).astype(np.float64)
    a1 = cond @ P["W1"].T + P["b1"]
    h = silu(a1)
    r = h @ P["W2"].T + P["b2"]
    film = {}
    off = 0
    C = channels(c0)
    for name, width in zip(FILM_LAYERS, (C[4], C[3], C[2], C[1], C[0])):
        film[name] = (1.0 + r[:, off:off + width], r[:, off + width:off + 2 * width])
        off += 2 * width
    acts = {"X": X}
    cache = {"cond": cond, "a1": a1, "h": h, "film": film, "layers": {}}
    src = {"e0": ("X", None), "e1": ("e0", None), "e2": ("e1", None), "e3": ("e2", None),
           "e4": ("e3", None), "d3": ("e4", "e3"), "d2": ("d3", "e2"), "d1": ("d2", "e1"),
           "d0": ("d1", "e0"), "out": ("d0", None)}
    for name, cu, cs, co, stride, has_film, act in layers(c0):
        s1, s2 = src[name]
        xin = up2(acts[s1]) if s2 is not None else acts[s1]
        if s2 is not None:
            xin = np.concatenate([xin, acts[s2]], axis=1)
        xq, Wq = q(xin), q(P[name + ".W"])
        pre = conv3x3(xq, Wq, P[name + ".b"], stride)
        if has_film:
            g, bt = film[name]
            z = g[:, :, None, None] * pre + bt[:, :, None, None]
        else:
            z = pre
        y = silu(z) if act else z
        acts[name] = y
        cache["layers"][name] = dict(xq=xq, Wq=Wq, pre=pre, z=z, stride=stride, cu=cu, cs=cs)
    cache["acts"] = acts
    return acts["out"], cache


def backward(params, cache, dout, c0=16, hidden=64, bf16=False):
    """dL/dparams (flat, FP64) given dL/d(output) [B][5][ny][nx]."""
    P = unpack(np.asarray(params, dtype=np.float64), c0, hidden)
    q = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    grads = {k: np.zeros_like(v) for k, v in P.items()}
    dfilm = {}
    dacts = {"out": np.asarray(dout, dtype=np.float64)}
    src = {"e0": ("X", None), "e1": ("e0", None), "e2": ("e1", None), "e3": ("e2", None),
           "e4": ("e3", None), "d3": ("e4", "e3"), "d2": ("d3", "e2"), "d1": ("d2", "e1"),
           "d0": ("d1", "e0"), "out": ("d0", None)}

    def add(name, g):
        dacts[name] = dacts[name] + g if name in dacts else g

    for name, cu, cs, co, stride, has_film, act in reversed(layers(c0)):
        L = cache["layers"][name]
        dy = dacts[name]
        dz = dy * dsilu(L["z"]) if act else dy
        if has_film:
            g, _ = cache["film"][name]
            dgam = (dz * L["pre"]).sum(axis=(2, 3))
            dbet = dz.sum(axis=(2, 3))
            dfilm[name] = (dgam, dbet)
            dpre = dz * g[:, :, None, None]
        else:
            dpre = dz
        # the weight and input gradients contract rounded operands; the bias gradient sums the
        # unrounded pre-activation gradient
        dxq, dW, _ = conv3x3_backward(L["xq"], L["Wq"], q(dpre), stride)
        grads[name + ".W"] = dW
        grads[name + ".b"] = dpre.sum(axis=(0, 2, 3))
        if name == "e0":
            continue
        s1, s2 = src[name]
        if s2 is None:
            add(s1, dxq)
        else:
            add(s1, up2_backward(dxq[:, :cu]))
            add(s2, dxq[:, cu:])
    # conditioning MLP
    C = channels(c0)
    parts = []
    for name, width in zip(FILM_LAYERS, (C[4], C[3], C[2], C[1], C[0])):
        parts += [dfilm[name][0], dfilm[name][1]]
    dr = np.concatenate(parts, axis=1)
    grads["W2"] = dr.T @ cache["h"]
    grads["b2"] = dr.sum(axis=0)
    dh = dr @ P["W2"]
    da1 = dh * dsilu(cache["a1"])
    grads["W1"] = da1.T @ cache["cond"]
    grads["b1"] = da1.sum(axis=0)
    return pack(grads, c0, hidden)


def base_fields(phi):
    """Per-sample rest values [B][5] of the five fields for volume fractions phi [B]."""
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    z = np.zeros_like(phi)
    return np.stack([z, z, z, phi, 1.0 - phi], axis=1)


def normalised_target(fields, mean, scale, phi):
    fields = np.asarray(fields, dtype=np.float64) - base_fields(phi)[:, :, None, None]
    return (fields - np.asarray(mean)[None, :, None, None]) / np.asarray(scale)[None, :, None, None]


def loss_and_grad(params, cond, fields, mean, scale, ny, nx, c0=16, hidden=64, bf16=False,
                  phi=None):
    """Mean squared error of the normalised output against the normalised target fields
    [B][5][ny][nx] (phi: the samples' volume fractions, [B]), and its gradient with respect to
    the flat parameters."""
    out, cache = forward(params, cond, ny, nx, c0, hidden, bf16=bf16)
    t = normalised_target(fields, mean, scale, phi)
    diff = out - t
    loss = float(np.mean(diff * diff))
    dout = 2.0 * diff / diff.size
    return loss, backward(params, cache, dout, c0, hidden, bf16=bf16)


def predict_fields(params, cond, mean, scale, ny, nx, c0=16, hidden=64, bf16=False, phi=None):
    """base + mean + scale * output for the samples' volume fractions phi [B]; phi and rho^w are
    then shifted by a constant per sample so that their cavity means are phi and 1 - phi."""
    out, _ = forward(params, cond, ny, nx, c0, hidden, bf16=bf16)
    base = base_fields(phi)
    f = (base[:, :, None, None] + np.asarray(mean)[None, :, None, None] +
         np.asarray(scale)[None, :, None, None] * out)
    for ch in (3, 4):
        f[:, ch] += (base[:, ch] - f[:, ch].mean(axis=(1, 2)))[:, None, None]
    return f


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def field_stats(fields, phi):
    """Per-channel mean and standard deviation over samples and nodes of fields - base:
    [B][5][ny][nx]."""
    f = np.asarray(fields, dtype=np.float64) - base_fields(phi)[:, :, None, None]
    mean = f.mean(axis=(0, 2, 3))
    std = f.std(axis=(0, 2, 3))
    return mean, np.where(std > 0, std, 1.0)


def param_segments(c0, hidden):
    """(name, size, fan_in) of every parameter tensor in flat order; fan_in is 0 for biases.
    Test inputs draw parameters segment by segment from these (workloads.random_net_params)."""
    lay, _ = param_layout(c0, hidden)
    out = []
    for k, (o, s) in sorted(lay.items(), key=lambda kv: kv[1][0]):
        size = int(np.prod(s))
        fan_in = s[1] * 9 if k.endswith(".W") else (s[1] if k in ("W1", "W2") else 0)
        out.append((k, size, fan_in))
    return out
