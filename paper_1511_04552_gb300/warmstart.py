"""Learned warm start (include/mclbm_net.h): a conditioned convolutional encoder-decoder that
predicts the steady fields (u_x, u_y, theta, phi, rho^w) of a cavity from (Ra, phi, d_p),
trained on steady solutions that the batched MCLBM solver computes, and used to seed
mclbm_init(MCLBM_INIT_WARM_RHO). The cold-started solve stays the judge: a warm-started run must
reach the same steady Nusselt number.

Argument marshalling only: the network's forward, backward and optimiser run in libmclbm's
kernels; PyTorch holds device memory and picks minibatches.

    python -m paper_1511_04552_gb300.warmstart --train 2000 --held-out 100 --out warmnet.npz
"""
import argparse
import ctypes as C
import json
import time

import numpy as np

from . import binding as B

N_FIELDS = 5
FIELD_MASK = B.UX | B.UY | B.THETA | B.PHI | B.RHO_W  # the order of the network's fields


class WarmNet:
    """The network bound to a torch-owned workspace on one GPU."""

    def __init__(self, ny=256, nx=256, c0=16, hidden=64, max_batch=16, device=None, stream=None):
        import torch
        self.torch = torch
        L = B.lib()
        self.cfg = B.NetConfig(int(ny), int(nx), int(c0), int(hidden), int(max_batch))
        self.n_params = int(L.mclbm_net_param_count(C.byref(self.cfg)))
        nbytes = int(L.mclbm_net_workspace_bytes(C.byref(self.cfg)))
        if self.n_params == 0 or nbytes == 0:
            raise B.MclbmError(B.EINVAL, "mclbm_net_param_count")
        self.device = torch.device(device if device is not None else "cuda")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        rc = L.mclbm_net_create(C.byref(self.cfg), C.byref(h))
        if rc != B.OK:
            raise B.MclbmError(rc, "mclbm_net_create")
        self.handle = h
        self._check(L.mclbm_net_bind(h, C.c_void_p(self.workspace.data_ptr()), nbytes,
                                     C.c_void_p(self.stream.cuda_stream)), "mclbm_net_bind")
        self.mean = np.zeros(N_FIELDS)
        self.scale = np.ones(N_FIELDS)

    @property
    def ny(self):
        return self.cfg.ny

    @property
    def nx(self):
        return self.cfg.nx

    def _check(self, rc, what):
        if rc != B.OK:
            raise B.MclbmError(rc, what, B.lib().mclbm_net_last_error(self.handle).decode())

    def _dev(self, t, dtype=None):
        t = t.to(self.device, dtype=dtype or self.torch.float32)
        return t.contiguous()

    def init_params(self, seed=0):
        self._check(B.lib().mclbm_net_init_params(self.handle, int(seed)), "mclbm_net_init_params")
        return self

    def set_params(self, params):
        p = self._dev(self.torch.as_tensor(params))
        if p.numel() != self.n_params:
            raise ValueError("expected %d parameters, got %d" % (self.n_params, p.numel()))
        self._check(B.lib().mclbm_net_set_params(self.handle, C.c_void_p(p.data_ptr())),
                    "mclbm_net_set_params")
        self.stream.synchronize()
        return self

    def get_params(self):
        p = self.torch.empty(self.n_params, dtype=self.torch.float32, device=self.device)
        self._check(B.lib().mclbm_net_get_params(self.handle, C.c_void_p(p.data_ptr())),
                    "mclbm_net_get_params")
        self.stream.synchronize()
        return p

    def set_normalizer(self, mean, scale):
        m = (C.c_double * N_FIELDS)(*[float(v) for v in mean])
        s = (C.c_double * N_FIELDS)(*[float(v) for v in scale])
        self._check(B.lib().mclbm_net_set_normalizer(self.handle, m, s), "mclbm_net_set_normalizer")
        self.mean, self.scale = np.array(mean, dtype=float), np.array(scale, dtype=float)
        return self

    def field_stats(self, cond, fields):
        """Normaliser statistics of fields [n][5][ny][nx] for conditions cond [n][3]."""
        c, f = self._dev(self.torch.as_tensor(cond)), self._dev(fields)
        m, s = (C.c_double * N_FIELDS)(), (C.c_double * N_FIELDS)()
        self._check(B.lib().mclbm_net_field_stats(self.handle, int(f.shape[0]),
                                                  C.c_void_p(c.data_ptr()),
                                                  C.c_void_p(f.data_ptr()), m, s),
                    "mclbm_net_field_stats")
        return np.array(m[:]), np.array(s[:])

    def forward(self, cond, out=None):
        """cond [b][3] (Ra, phi, d_p) -> fields [b][5][ny][nx] on the device."""
        c = self._dev(self.torch.as_tensor(cond))
        b = int(c.shape[0])
        if out is None:
            out = self.torch.empty((b, N_FIELDS, self.ny, self.nx), dtype=self.torch.float32,
                                   device=self.device)
        self._check(B.lib().mclbm_net_forward(self.handle, b, C.c_void_p(c.data_ptr()),
                                              C.c_void_p(out.data_ptr())), "mclbm_net_forward")
        return out

    def predict(self, cond, chunk=None):
        """Forward in chunks of at most max_batch."""
        c = self.torch.as_tensor(cond)
        chunk = chunk or self.cfg.max_batch
        return self.torch.cat([self.forward(c[i:i + chunk]) for i in range(0, c.shape[0], chunk)])

    def loss_grad(self, cond, target):
        c, t = self._dev(self.torch.as_tensor(cond)), self._dev(target)
        g = self.torch.empty(self.n_params, dtype=self.torch.float32, device=self.device)
        loss = C.c_double()
        self._check(B.lib().mclbm_net_loss_grad(self.handle, int(c.shape[0]),
                                                C.c_void_p(c.data_ptr()),
                                                C.c_void_p(t.data_ptr()), C.c_void_p(g.data_ptr()),
                                                C.byref(loss)), "mclbm_net_loss_grad")
        return loss.value, g

    def train_step(self, cond, target, lr, want_loss=True):
        c, t = self._dev(self.torch.as_tensor(cond)), self._dev(target)
        loss = C.c_double()
        self._check(B.lib().mclbm_net_train_step(self.handle, int(c.shape[0]),
                                                 C.c_void_p(c.data_ptr()),
                                                 C.c_void_p(t.data_ptr()), float(lr),
                                                 C.byref(loss) if want_loss else None),
                    "mclbm_net_train_step")
        return loss.value if want_loss else None

    def save(self, path):
        np.savez(path, params=self.get_params().cpu().numpy(), mean=self.mean, scale=self.scale,
                 config=np.array([self.cfg.ny, self.cfg.nx, self.cfg.c0, self.cfg.hidden]))

    @classmethod
    def load(cls, path, max_batch=16, device=None):
        d = np.load(path)
        ny, nx, c0, hidden = (int(v) for v in d["config"])
        net = cls(ny, nx, c0, hidden, max_batch=max_batch, device=device)
        net.set_params(d["params"])
        net.set_normalizer(d["mean"], d["scale"])
        return net

    def close(self):
        if getattr(self, "handle", None):
            B.lib().mclbm_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_bf16(a, b, a_kmajor=True, b_kmajor=True, splits=1, k_per_split=None, stream=None):
    """D = A B^T through the library's tensor-core GEMM (mclbm_gemm_bf16). a, b: BF16 CUDA
    tensors, [M][K] / [N][K] if K-major else [K][M] / [K][N]. Returns FP32 D[splits][M][N]."""
    import torch
    M, K = (a.shape[0], a.shape[1]) if a_kmajor else (a.shape[1], a.shape[0])
    N = b.shape[0] if b_kmajor else b.shape[1]
    if k_per_split is None:
        k_per_split = ((K + splits - 1) // splits + 63) // 64 * 64
    d = torch.empty((splits, M, N), dtype=torch.float32, device=a.device)
    st = stream if stream is not None else torch.cuda.current_stream(a.device)
    rc = B.lib().mclbm_gemm_bf16(int(M), int(N), int(K), C.c_void_p(a.data_ptr()),
                                 int(a.stride(0)), int(bool(a_kmajor)), C.c_void_p(b.data_ptr()),
                                 int(b.stride(0)), int(bool(b_kmajor)), C.c_void_p(d.data_ptr()),
                                 int(N), int(splits), int(k_per_split), int(M * N),
                                 C.c_void_p(st.cuda_stream))
    if rc != B.OK:
        raise B.MclbmError(rc, "mclbm_gemm_bf16")
    return d


def conv_flops(ny=256, nx=256, c0=16, batch=1):
    """Multiply-add FLOPs (2 per MAC) of the network's convolutions for one forward pass of a
    batch (the backward pass does twice as many: input and weight gradients)."""
    C = (c0, 2 * c0, 4 * c0, 8 * c0, 8 * c0)
    # (cin, cout, output grid divisor) per layer, in the order of include/mclbm_net.h
    layers = [(4, C[0], 1), (C[0], C[1], 2), (C[1], C[2], 4), (C[2], C[3], 8), (C[3], C[4], 16),
              (C[4] + C[3], C[3], 8), (C[3] + C[2], C[2], 4), (C[2] + C[1], C[1], 2),
              (C[1] + C[0], C[0], 1), (C[0], N_FIELDS, 1)]
    return sum(2.0 * batch * (ny // s) * (nx // s) * co * 9 * ci for ci, co, s in layers)


def bench_train(steps=20, batch=16, ny=256, nx=256, seed=0):
    """Times training steps of the network on synthetic targets (CUDA events on the bound
    stream): ms per step and the convolution FLOP rate (forward + backward = 3x forward)."""
    import torch
    net = WarmNet(ny, nx, max_batch=batch).init_params(seed)
    r = np.random.default_rng(seed)
    cond = torch.as_tensor(sample_conditions(batch, seed).astype(np.float32)).cuda()
    tgt = torch.as_tensor(r.standard_normal((batch, N_FIELDS, ny, nx)).astype(np.float32)).cuda()
    net.set_normalizer(*net.field_stats(cond, tgt))
    for _ in range(3):
        net.train_step(cond, tgt, 1e-4, want_loss=False)
    st = net.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        net.train_step(cond, tgt, 1e-4, want_loss=False)
    b.record(st)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    flops = 3.0 * conv_flops(ny, nx, net.cfg.c0, batch)
    return {"ms_per_step": ms, "batch": batch, "conv_tflops_per_s": flops / (ms * 1e-3) / 1e12,
            "conv_gflop_per_step": flops / 1e9}


GEMM_SHAPES = ((8192, 8192, 8192), (4096, 4096, 4096), (65536, 128, 1152), (16384, 64, 576))


def bench_gemm(shapes=GEMM_SHAPES, reps=10, seed=0):
    """The library's tensor-core GEMM (mclbm_gemm_bf16, K-major BF16 operands, FP32 result)
    against torch.matmul on BF16 (cuBLAS) for shapes (M, N, K): best and median TFLOP/s of each
    (2 M N K flops per product; CUDA events, 3 untimed calls first) and the relative error of the
    library's product against an FP32 product of the same BF16 operands."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e-3)
        ts.sort()
        return ts[0], ts[len(ts) // 2]

    out = []
    for M, N, K in shapes:
        A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
        Bm = torch.randn(N, K, device="cuda", generator=g).bfloat16()
        ref = A.float() @ Bm.float().T
        err = float((gemm_bf16(A, Bm)[0] - ref).norm() / ref.norm())
        del ref
        fl = 2.0 * M * N * K
        ours = timed(lambda: gemm_bf16(A, Bm))
        lib = timed(lambda: A @ Bm.T)
        out.append({"M": M, "N": N, "K": K, "rel_err": err,
                    "tflops": fl / ours[0] / 1e12, "tflops_median": fl / ours[1] / 1e12,
                    "cublas_tflops": fl / lib[0] / 1e12, "cublas_tflops_median": fl / lib[1] / 1e12})
        del A, Bm
        torch.cuda.empty_cache()
    return out


# ---- data, training and evaluation drivers ----------------------------------------------------

def sample_conditions(n, seed):
    """n points [n][3]: log10 Ra uniform in [3, 6], phi uniform in [0, 5 %], d_p uniform in
    [10, 100] nm."""
    r = np.random.default_rng(seed)
    return np.stack([10.0 ** r.uniform(3.0, 6.0, n), r.uniform(0.0, 0.05, n),
                     r.uniform(10e-9, 100e-9, n)], axis=1)


def solve_steady(conds, ny=256, nx=256, warm=None, group=64, tol=1e-4, check_every=1000,
                 max_steps=3_000_000, want_fields=False, Pr=6.2, lags=B.STRICT_LAGS):
    """Runs every cavity of conds [n][3] to a steady hot-wall Nusselt number with the batched
    solver (groups of `group` cavities per persistent launch). warm: optional device fields
    [n][5][ny][nx] for mclbm_init(WARM_RHO). Returns per-cavity steps and Nu, the total wall
    time and, if asked, the steady fields [n][5][ny][nx] (device)."""
    import torch
    n = len(conds)
    steps = np.zeros(n, dtype=np.int64)
    nu = np.zeros(n)
    fields = (torch.empty((n, N_FIELDS, ny, nx), dtype=torch.float32, device="cuda")
              if want_fields else None)
    # cavities of similar Ra converge after similar step counts: group them so that a batch does
    # not run on with a few slow cavities left
    order = np.argsort(np.asarray(conds, dtype=np.float64)[:, 0], kind="stable")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g0 in range(0, n, group):
        idx = [int(i) for i in order[g0:g0 + group]]
        cavs = []
        for i in idx:
            Ra, phi, dp = (float(v) for v in conds[i])
            cav = B.Cavity(nx, ny, Ra, Pr, phi, dp)
            cav.init(warm=warm[i] if warm is not None else None)
            cavs.append(cav)
        batch = B.Batch(cavs)
        res = B.sweep_to_steady(batch, tol=tol, check_every=check_every, max_steps=max_steps,
                                lags=lags)
        for k, i in enumerate(idx):
            steps[i] = res["steps"][k] if res["steps"][k] is not None else res["total_steps"]
            nu[i] = res["nu_hot"][k]
            if want_fields:
                fields[i] = cavs[k].fields(FIELD_MASK)
        batch.close()
        del cavs
    torch.cuda.synchronize()
    return dict(steps=steps, nu=nu, wall_s=time.perf_counter() - t0, fields=fields)


def train(net, conds, fields, epochs=100, batch=16, lr=2e-3, lr_final=1e-4, seed=0, log=None):
    """Adam on random minibatches, learning rate decaying geometrically from lr to lr_final.
    conds [n][3] (host or device), fields [n][5][ny][nx] (device). Returns the loss history."""
    import torch
    n = len(conds)
    c_all = torch.as_tensor(np.asarray(conds, dtype=np.float32)).cuda()
    mean, scale = net.field_stats(c_all, fields)
    net.set_normalizer(mean, scale)
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    hist = []
    k = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        acc = 0.0
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            rate = lr * (lr_final / lr) ** (k / max(1, total - 1))
            acc += net.train_step(c_all[idx], fields[idx], rate)
            k += 1
        hist.append(acc / steps_per_epoch)
        if log:
            log("epoch %d loss %.4e (%.1f s)" % (ep, hist[-1], time.perf_counter() - t0))
    return hist


def solve_plain(conds, ny=256, nx=256, tol=1e-4, Pr=6.2):
    """Each point solved cold on its own (one cavity's launches, run_to_steady), one after
    another: the plain method without batching or a learned start."""
    import torch
    steps, nu = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in conds:
        Ra, phi, dp = (float(v) for v in c)
        r = B.run_to_steady(B.Cavity(nx, ny, Ra, Pr, phi, dp).init(), tol=tol)
        steps.append(r["steps"])
        nu.append(r["nu_hot"])
    torch.cuda.synchronize()
    return dict(steps=np.array(steps), nu=np.array(nu), wall_s=time.perf_counter() - t0)


def evaluate(net, conds, group=64, tol=1e-4, ny=256, nx=256, plain=False):
    """Cold against warm-started steady solves of the same points, both batched: steps, wall time
    (the warm side includes the network's inference) and the steady Nusselt numbers. With plain,
    also each point solved cold on its own, one after another (solve_plain), and the speedup of
    the warm-started batched sweep over those plain solves."""
    import torch
    cold = solve_steady(conds, ny, nx, group=group, tol=tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pred = net.predict(np.asarray(conds, dtype=np.float32))
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    warm = solve_steady(conds, ny, nx, warm=pred, group=group, tol=tol)
    rel = np.abs(warm["nu"] - cold["nu"]) / np.abs(cold["nu"])
    out = dict(n=len(conds), cold_steps=cold["steps"], warm_steps=warm["steps"],
               cold_wall_s=cold["wall_s"], warm_wall_s=warm["wall_s"] + t_inf,
               inference_s=t_inf, nu_cold=cold["nu"], nu_warm=warm["nu"], nu_rel_diff=rel,
               speedup_wall=cold["wall_s"] / (warm["wall_s"] + t_inf),
               speedup_steps=float(cold["steps"].sum()) / float(warm["steps"].sum()))
    if plain:
        pl = solve_plain(conds, ny, nx, tol=tol)
        out.update(plain_steps=pl["steps"], plain_wall_s=pl["wall_s"], nu_plain=pl["nu"],
                   speedup_vs_plain=pl["wall_s"] / (warm["wall_s"] + t_inf),
                   nu_rel_diff_plain=np.abs(warm["nu"] - pl["nu"]) / np.abs(pl["nu"]))
    return out


def perturbed_rest(nx, ny, phi, seed, amp=1e-3):
    """(u_x, u_y, theta, phi) [4][ny][nx] float32: rest, the conduction profile and phi, plus
    seeded uniform noise of amplitude amp (amp * phi on phi) from numpy's PCG64 stream."""
    r = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    out = np.empty((4, ny, nx), dtype=np.float32)
    out[0] = amp * r.uniform(-1.0, 1.0, (ny, nx))
    out[1] = amp * r.uniform(-1.0, 1.0, (ny, nx))
    out[2] = (0.5 - x)[None, :] + amp * r.uniform(-1.0, 1.0, (ny, nx))
    out[3] = phi * (1.0 + amp * r.uniform(-1.0, 1.0, (ny, nx)))
    return out


def cold_start_spread(conds, n_starts=6, amp=1e-3, ny=256, nx=256, tol=1e-4, seed=0):
    """How unique the steady hot-wall Nu is: every point of conds [n][3] solved from rest and
    from n_starts seeded perturbed rest states (perturbed_rest, amplitude amp), all to the same
    steadiness test. Returns the steady Nu [n][1 + n_starts] (column 0 from rest), the steps,
    and per point the relative spread (max - min) / median."""
    import torch
    n = len(conds)
    rest = solve_steady(conds, ny, nx, group=n, tol=tol)
    reps = np.repeat(np.asarray(conds, dtype=np.float64), n_starts, axis=0)
    warm = [torch.from_numpy(perturbed_rest(nx, ny, float(c[1]), seed * 7919 + k, amp)).cuda()
            for k, c in enumerate(reps)]
    pert = solve_steady(reps, ny, nx, warm=warm, group=len(reps), tol=tol)
    nu = np.concatenate([rest["nu"][:, None], pert["nu"].reshape(n, n_starts)], axis=1)
    steps = np.concatenate([rest["steps"][:, None], pert["steps"].reshape(n, n_starts)], axis=1)
    spread = (nu.max(axis=1) - nu.min(axis=1)) / np.median(nu, axis=1)
    return dict(nu=nu, steps=steps, spread=spread,
                wall_s=rest["wall_s"] + pert["wall_s"])


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", type=int, default=2000, help="training points")
    ap.add_argument("--held-out", type=int, default=100)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--group", type=int, default=100, help="cavities per batched launch")
    ap.add_argument("--tol", type=float, default=1e-4, help="steady Nu tolerance of the judged solves")
    ap.add_argument("--data-tol", type=float, default=1e-3,
                    help="steady Nu tolerance of the training solves (the network's own error is "
                         "larger than this)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default="warmnet.npz")
    ap.add_argument("--report", default=None, help="JSON file for the evaluation")
    ap.add_argument("--init", default=None, help="start from these weights (a saved network)")
    ap.add_argument("--data-strict", action="store_true",
                    help="training solves to the judged steadiness (both lags, --tol): targets at "
                         "the end of each cold path instead of a point on it")
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--bench-train", type=int, default=0,
                    help="only time this many training steps on synthetic targets and exit")
    ap.add_argument("--bench-gemm", action="store_true",
                    help="only time the library GEMM against cuBLAS on a few shapes and exit")
    ap.add_argument("--evaluate", default=None,
                    help="only evaluate these weights on --held-out points (seed --seed + 1)")
    ap.add_argument("--plain", action="store_true",
                    help="with --evaluate: also solve every point cold on its own")
    ap.add_argument("--spread", type=int, default=0,
                    help="only measure the cold-start spread of the steady Nu on this many "
                         "held-out points (seed --seed + 1), --starts perturbed starts each")
    ap.add_argument("--starts", type=int, default=6)
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)  # noqa: E731
    if a.spread:
        held = sample_conditions(a.spread, a.seed + 1)
        sp = cold_start_spread(held, a.starts, ny=a.size, nx=a.size, tol=a.tol)
        summary = dict(conds=held.tolist(), **{k: (v.tolist() if isinstance(v, np.ndarray)
                                                    else v) for k, v in sp.items()})
        log(json.dumps(summary))
        if a.report:
            with open(a.report, "w") as f:
                json.dump(summary, f)
        return
    if a.bench_train:
        log(json.dumps(bench_train(a.bench_train, ny=a.size, nx=a.size)))
        return
    if a.bench_gemm:
        for r in bench_gemm():
            log(json.dumps(r))
        return
    if a.evaluate:
        net = WarmNet.load(a.evaluate)
        held = sample_conditions(a.held_out, a.seed + 1)
        ev = evaluate(net, held, group=a.group, tol=a.tol, ny=net.ny, nx=net.nx, plain=a.plain)
        summary = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in ev.items()}
        log(json.dumps({k: summary[k] for k in ("n", "cold_wall_s", "warm_wall_s", "speedup_wall",
                                                "speedup_steps", "plain_wall_s",
                                                "speedup_vs_plain") if k in summary}))
        if a.report:
            with open(a.report, "w") as f:
                json.dump(summary, f)
        return
    conds = sample_conditions(a.train, a.seed)
    t0 = time.perf_counter()
    # training targets: points on each cold path near its quasi-steady state (one lag, looser
    # tolerance); a warm start that reproduces such a point follows the cold path from there
    if a.data_strict:
        data = solve_steady(conds, a.size, a.size, group=a.group, tol=a.tol, want_fields=True)
    else:
        data = solve_steady(conds, a.size, a.size, group=a.group, tol=a.data_tol,
                            want_fields=True, lags=(1,))
    log("generated %d steady solutions in %.1f s (mean %.0f steps)" % (
        a.train, time.perf_counter() - t0, data["steps"].mean()))
    if a.init:
        net = WarmNet.load(a.init)
    else:
        net = WarmNet(a.size, a.size).init_params(a.seed)
    t0 = time.perf_counter()
    hist = train(net, conds, data["fields"], epochs=a.epochs, lr=a.lr, log=log)
    log("trained %d epochs in %.1f s, final loss %.3e" % (a.epochs, time.perf_counter() - t0,
                                                          hist[-1]))
    net.save(a.out)
    held = sample_conditions(a.held_out, a.seed + 1)
    ev = evaluate(net, held, group=a.group, tol=a.tol, ny=a.size, nx=a.size)
    summary = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in ev.items()}
    summary["train_loss"] = hist
    summary["train_steps_mean"] = float(data["steps"].mean())
    summary["train_gen_s"] = data["wall_s"]
    log(json.dumps({k: summary[k] for k in ("n", "cold_wall_s", "warm_wall_s", "speedup_wall",
                                            "speedup_steps")}))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(summary, f)


if __name__ == "__main__":
    main()
