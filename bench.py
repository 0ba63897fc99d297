"""Benchmark of the MCLBM step on GB300: MLUPS and HBM roofline fraction.

Workload (default): the 256 x 256 cavity at Ra 1e5, Pr 6.2, 3 % alumina of 30 nm, all slip
forces, cold start. One benchmark step is one pass of the whole hot path: 1000 time steps
(stream, moments, gradients, slip forces, drag, collision, store; graph-captured launches)
followed by the reductions (hot/cold Nusselt numbers, component masses, residual). L2 is
flushed (a 256 MiB write) between benchmark steps. The 256^2 state (14 MB) is L2-resident
inside a step, so the HBM roofline is also measured on the 1024 x 1024 cavity (Ra 1e6, 2 %,
50 nm, 226 MB of state) and reported under "hbm_case".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): independent replicas, one cavity per GPU, no data-path collective; the
value is the sum of all ranks' lattice updates over the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "MLUPS & HBM GB/s fraction per MCLBM step; wall time to steady Nu (1e-4)"
UNIT = "MLUPS"
BYTES_PER_LU = 216  # 27 FP32 populations read + 27 written per lattice-node update
STORAGE = {"f32": (0, 216), "f16": (1, 108), "bf16": (2, 108)}  # (code, bytes per update)
CHUNK = 1000        # time steps per benchmark step (one residual / Nusselt check interval)
OUR_KERNELS_PER_REDUCTION = 5  # nusselt, residual + final, mass + final
WORKLOADS = {"cavity256": workloads.CAVITY_256, "cavity1024": workloads.CAVITY_1024}
STEP_SOURCES = ("mclbm_device.cuh", "mclbm_pair.cuh")  # the step kernels' source


def step_launches(n):
    """Kernel launches of mclbm_step(n) on one cavity (the library's decomposition): the even
    part in graphs of 2^k <= 1024 steps, largest first, each graph one step kernel per step and
    one epoch kernel; an odd last step as a single launch."""
    launches, left = 0, n
    while left >= 2:
        k = 1
        while k < 10 and (2 << k) <= left:
            k += 1
        launches += (1 << k) + 1
        left -= 1 << k
    return launches + left


def nodes_per_thread(nx, ny, sms):
    """The step kernel's nodes per thread (the library's rule): one while the lattice gives
    every SM at most two 32 x 8 tiles, two beyond."""
    tiles = ((nx + 31) // 32) * ((ny + 7) // 8)
    return 1 if tiles <= 2 * sms else 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity256", choices=sorted(WORKLOADS))
    ap.add_argument("--chunk", type=int, default=CHUNK,
                    help="time steps per benchmark step (default: one 1000-step check interval)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage (16-bit: stochastic rounding, FP32 arithmetic)")
    ap.add_argument("--sweep-to-steady", action="store_true",
                    help="only run the 80-cavity sweep to steady Nu, batched and cavity by cavity, "
                         "and print that comparison (minutes)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 1024^2 roofline case, the steady-Nu run and the CPU baseline")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group). Used for the job time:
    the slowest rank decides."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world_size, slowest_seconds):
    """Independent replicas: every rank processes the same number of lattice updates; the job's
    rate (MLUPS) is all ranks' updates over the slowest rank's time."""
    return units_per_rank * world_size / slowest_seconds / 1e6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region: the sampler starts before
    the region (nvidia-smi takes a moment to print its first line), every sample carries its
    timestamp, and only the samples inside the region (host clock, +-60 ms) are summarised."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, interval_ms=50):
        self.gpu = gpu_index
        self.interval = interval_ms
        self.proc = None
        self.t0 = self.t1 = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", str(self.interval)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)
        except Exception:
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        import datetime
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if self.t0 is not None and not (self.t0 - 0.06 <= ts <= self.t1 + 0.06):
                    continue
                sm.append(float(p[2]))
                mx.append(float(p[3]))
            except ValueError:
                continue
            for n, v in zip(names, p[6:10]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "window_s": round(self.t1 - self.t0, 3)}


def reference_arm(args, ws, rank):
    """The FP64 oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    w = workloads.CAVITY_256
    s = oracle.RefSolver(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"]).init()
    n_nodes = w["nx"] * w["ny"]
    t0 = time.perf_counter()
    s.step(5)
    per = (time.perf_counter() - t0) / 5
    chunk = max(2, min(200, int(3.0 / max(per, 1e-6))))  # about 3 s of CPU work per step
    for _ in range(args.warmup):
        s.step(chunk)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(chunk)
        s.nusselt()
    dt = time.perf_counter() - t0
    mlups = n_nodes * chunk * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "nx": w["nx"], "ny": w["ny"],
                                        "time_steps_per_bench_step": chunk},
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": oracle.get_threads(),
                         "kind": "oracle",
                         "sample": "%d bench steps of %d time steps of the %s cavity" % (
                             args.steps, chunk, w["name"])},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(seconds=10.0):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    w = workloads.CAVITY_256
    s = oracle.RefSolver(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"]).init()
    t0 = time.perf_counter()
    s.step(5)
    per = (time.perf_counter() - t0) / 5
    n = max(5, int(seconds / max(per, 1e-6)))
    t0 = time.perf_counter()
    s.step(n)
    dt = time.perf_counter() - t0
    return {"value": w["nx"] * w["ny"] * n / dt / 1e6, "unit": UNIT,
            "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "%d time steps of the %s cavity from rest (%.1f s)" % (n, w["name"], dt)}


def ncu_traffic(workload_name):
    """DRAM bytes per step launch (FP32 storage) from the committed ncu summary, if it was
    taken on the current step-kernel source (else None)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1511_04552_gb300", "csrc")
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    try:
        h = hashlib.sha256()
        for name in STEP_SOURCES:
            h.update(open(os.path.join(csrc, name), "rb").read())
        sha = h.hexdigest()[:16]
        vals = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != sha:
            return None
        return float(vals["%s_dram_bytes_per_launch" % workload_name.split("_")[0]])
    except Exception:
        return None


def sweep_measure(m, torch, steps=1000, tune_steps=64):
    """The 80-cavity parametric sweep (sizes 64^2..512^2, Ra x phi x d_p): aggregate MLUPS of
    one batched persistent launch per time step (autotuned) against stepping each cavity with
    its own launches one after another, for the same number of steps."""
    sw = workloads.sweep80()
    nodes = sum(c["nx"] * c["ny"] for c in sw)
    cavs = [m.Cavity(c["nx"], c["ny"], c["Ra"], c["Pr"], c["phi"], c["d_p"]).init() for c in sw]
    batch = m.Batch(cavs)
    order, per_sm = batch.tune(tune_steps)
    batch.step(steps)  # warm-up
    torch.cuda.synchronize()
    st = batch.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    batch.step(steps)
    b.record(st)
    b.synchronize()
    t_batch = a.elapsed_time(b) / 1e3
    batch.close()
    for c in cavs:
        c.step(steps)  # warm-up (captures each cavity's graphs)
    torch.cuda.synchronize()
    a.record(st)
    for c in cavs:
        c.step(steps)
    b.record(st)
    b.synchronize()
    t_seq = a.elapsed_time(b) / 1e3
    return {"workload": "sweep80: %d cavities, %.2f M nodes, sizes 64^2..512^2" % (len(sw), nodes / 1e6),
            "time_steps": steps, "batched_mlups": nodes * steps / t_batch / 1e6,
            "sequential_mlups": nodes * steps / t_seq / 1e6, "speedup": t_seq / t_batch,
            "autotuned": {"tile_order": order, "ctas_per_sm": per_sm}}


def sweep_to_steady_measure(m, torch, tol=1e-4, check_every=1000, max_steps=3_000_000):
    """The 80-cavity parametric sweep run to the steady hot-wall Nu (tol, two-lag test), once
    batched (autotuned persistent launches, converged cavities leaving the tile table) and once
    cavity by cavity with their own launches, one after another. Lattice updates counted per
    cavity up to its own steady step; wall time on the host around each whole solve."""
    sw = workloads.sweep80()
    nodes = np.array([c["nx"] * c["ny"] for c in sw], dtype=np.float64)
    cavs = [m.Cavity(c["nx"], c["ny"], c["Ra"], c["Pr"], c["phi"], c["d_p"]).init() for c in sw]
    batch = m.Batch(cavs)
    order, per_sm = batch.tune(2)
    for c in cavs:  # the tuner's trial steps are real steps: start again from rest
        c.init()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rb = m.sweep_to_steady(batch, tol=tol, check_every=check_every, max_steps=max_steps)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    batch.close()
    steps_b = np.array([s if s is not None else rb["total_steps"] for s in rb["steps"]], float)
    t0 = time.perf_counter()
    rs = [m.run_to_steady(c.init(), tol=tol, check_every=check_every, max_steps=max_steps)
          for c in cavs]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    steps_s = np.array([r["steps"] for r in rs], float)
    nu_b, nu_s = np.asarray(rb["nu_hot"]), np.array([r["nu_hot"] for r in rs])
    return {"workload": "sweep80 to steady Nu (%g, two-lag test, checks every %d steps)" % (
                tol, check_every),
            "cavities": len(sw), "nodes": int(nodes.sum()),
            "autotuned": {"tile_order": order, "ctas_per_sm": per_sm},
            "batched": {"wall_s": t_batch, "mlups": float((nodes * steps_b).sum() / t_batch / 1e6),
                        "converged": rb["converged"], "total_steps": rb["total_steps"]},
            "sequential": {"wall_s": t_seq, "mlups": float((nodes * steps_s).sum() / t_seq / 1e6),
                           "converged": all(r["converged"] for r in rs)},
            "speedup_wall": t_seq / t_batch,
            "steps_mean": {"batched": float(steps_b.mean()), "sequential": float(steps_s.mean())},
            "nu_rel_diff_max": float(np.max(np.abs(nu_b - nu_s) / np.abs(nu_s)))}


WARMNET = os.path.join(ROOT, "paper_1511_04552_gb300", "weights", "warmnet_256.npz")


def warm_start_measure(m, torch, n_points=12):
    """Learned warm start against cold starts on held-out parameter points (256^2, steady Nu to
    1e-4): warm and cold solved with the batched solver (the warm side's wall time includes the
    network's inference), and the plain method: each point solved cold on its own."""
    if not os.path.exists(WARMNET):
        return {"unavailable": "no trained network weights in the package"}
    from paper_1511_04552_gb300 import warmstart as W
    net = W.WarmNet.load(WARMNET)
    conds = workloads.random_conditions(n_points, seed=2)
    ev = W.evaluate(net, conds, group=n_points, plain=True)
    return {"workload": "%d held-out points, 256^2, log-uniform Ra 1e3..1e6, phi 0..5 %%, "
                        "d_p 10..100 nm" % n_points,
            "cold_wall_s": ev["cold_wall_s"], "warm_wall_s": ev["warm_wall_s"],
            "speedup_wall": ev["speedup_wall"], "speedup_steps": ev["speedup_steps"],
            "cold_steps_mean": float(ev["cold_steps"].mean()),
            "warm_steps_mean": float(ev["warm_steps"].mean()),
            "max_nu_rel_diff": float(ev["nu_rel_diff"].max()),
            "inference_s": ev["inference_s"],
            # the same points solved cold one by one with each cavity's own launches
            "plain_wall_s": ev["plain_wall_s"],
            "speedup_vs_plain": ev["speedup_vs_plain"],
            "max_nu_rel_diff_vs_plain": float(ev["nu_rel_diff_plain"].max())}


def time_steps_only(cav, torch, nsteps):
    """Average duration of one step launch: events around back-to-back graph replays."""
    st = cav.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cav.step(nsteps)  # warm
    st.synchronize()
    a.record(st)
    cav.step(nsteps)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / 1e3 / nsteps


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return
    import torch
    import paper_1511_04552_gb300 as m
    from paper_1511_04552_gb300 import build as pkg_build

    pkg_build.build()
    torch.cuda.set_device(local)
    if args.sweep_to_steady:
        if rank == 0:
            print(json.dumps(sweep_to_steady_measure(m, torch)), flush=True)
        return
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod

    def barrier():
        if dist is not None:
            dist.barrier()

    w = WORKLOADS[args.workload]
    CH = args.chunk
    nx, ny = w["nx"], w["ny"]
    store, bytes_lu = STORAGE[args.storage]
    cav = m.Cavity(nx, ny, w["Ra"], w["Pr"], w["phi"], w["d_p"], storage=store)
    cav.init()
    st = cav.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def bench_step(ev=None):
        if ev is not None:
            ev[0].record(st)
        cav.step(CH)
        if ev is not None:
            ev[1].record(st)
        cav.diagnostics()  # Nu, masses and residual: one synchronisation
        flush.zero_()

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(st)
        for k in range(args.steps):
            bench_step(evs[k])
        t_end.record(st)
        torch.cuda.synchronize()
    barrier()
    elapsed = max_over_ranks(t_start.elapsed_time(t_end) / 1e3, dist, "cuda")
    step_time = sum(a.elapsed_time(b) for a, b in evs) / 1e3 / (args.steps * CH)
    lu = nx * ny * CH * args.steps
    value = whole_job_rate(lu, ws, elapsed)
    hbm_peak, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    achieved = bytes_lu * nx * ny / step_time / 1e9

    # end to end through the C ABI with host buffers: H2D warm fields, init, 1000 steps,
    # all 8 fields and the Nusselt numbers back to the host
    warm = torch.from_numpy(workloads.perturbed_rest_fields(nx, ny, w["phi"], seed=1)).pin_memory()
    fields_host = torch.empty((8, ny, nx), dtype=torch.float32).pin_memory()
    e2e_cav = m.Cavity(nx, ny, w["Ra"], w["Pr"], w["phi"], w["d_p"], storage=store)
    for _ in range(max(1, args.warmup)):
        e2e_cav.run_host(warm, CH, 0xFF, fields_host)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_cav.run_host(warm, CH, 0xFF, fields_host)
    e2e_time = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = whole_job_rate(nx * ny * CH * args.steps, ws, e2e_time)

    extras = {}
    if not args.no_extras and rank == 0 and ws == 1:  # the scaling runs report the main line
        # HBM case: 1024^2, state larger than L2
        w4 = workloads.CAVITY_1024
        big = m.Cavity(w4["nx"], w4["ny"], w4["Ra"], w4["Pr"], w4["phi"], w4["d_p"])
        big.init()
        t_big = time_steps_only(big, torch, 640)
        ach_big = BYTES_PER_LU * w4["nx"] * w4["ny"] / t_big / 1e9
        extras["hbm_case"] = {
            "workload": w4["name"], "mlups": w4["nx"] * w4["ny"] / t_big / 1e6,
            "roofline": {"bound": "hbm", "achieved": ach_big, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ach_big / hbm_peak, "traffic": ncu_traffic(w4["name"]),
                         "peak_kind": peak_kind, "kernel": "step_pair_tma_kernel",
                         "nodes_per_thread": nodes_per_thread(w4["nx"], w4["ny"], sms),
                         "bytes_per_launch": BYTES_PER_LU * w4["nx"] * w4["ny"],
                         "launch_us": t_big * 1e6}}
        del big
        torch.cuda.empty_cache()
        extras["sweep"] = sweep_measure(m, torch)
        torch.cuda.empty_cache()
        extras["warm_start"] = warm_start_measure(m, torch)
        torch.cuda.empty_cache()
        # cold start to steady Nu (estimated distance to the steady value <= 1e-4, checks every
        # 1000 steps; mclbm_run_to_steady)
        w2 = workloads.CAVITY_256
        sc = m.Cavity(w2["nx"], w2["ny"], w2["Ra"], w2["Pr"], w2["phi"], w2["d_p"]).init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = m.run_to_steady(sc, tol=1e-4, check_every=1000, max_steps=3000000)
        extras["steady_nu"] = {"wall_s": time.perf_counter() - t0, "steps": res["steps"],
                               "converged": res["converged"], "nu_hot": res["nu_hot"],
                               "nu_cold": res["nu_cold"], "workload": w2["name"]}
        if ws == 1:
            extras["cpu_baseline"] = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "storage": args.storage,
            "data": "synthetic",
            "config": {"workload": w["name"], "nx": nx, "ny": ny, "Ra": w["Ra"], "Pr": w["Pr"],
                       "phi": w["phi"], "d_p": w["d_p"], "time_steps_per_bench_step": CH,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed between bench steps (256 MiB write); state %.0f MB" % (
                           2 * 27 * 4 * nx * ny / 1e6)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": ncu_traffic(w["name"]) if args.storage == "f32" else None,
                         "peak_kind": peak_kind,
                         "kernel": "step_pair_tma_kernel",
                         "nodes_per_thread": nodes_per_thread(nx, ny, sms),
                         "bytes_per_launch": bytes_lu * nx * ny,
                         "launch_us": step_time * 1e6},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 4 * nx * ny * 4,
                    "d2h_bytes_per_step": 8 * nx * ny * 4 + 16},
            "gpu_launches": args.steps * (step_launches(CH) + OUR_KERNELS_PER_REDUCTION),
            "clocks": clk.summary(),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
