"""Writes the stored FP64 oracle results that the long GPU parity tests compare against.

Calls only the oracle (oracle/) and the seeded workload definitions (workloads.py); nothing
here comes from the CUDA path. Each run is long on CPU cores, so it checkpoints its state to a
working directory and resumes from there.

  python tests/golden/make_oracle_runs.py cavity256 [--work DIR] [--threads N]
      256 x 256, Ra 1e5, Pr 6.2, 3 % alumina of 30 nm, all slip forces, from rest, until the
      steady-state residual (max over u, theta, phi of ||q_n - q_(n-K)|| / (K ||q_n||),
      K = 1000 steps) first falls below 1e-8. Stores the step count, the Nusselt history
      (every 1000 steps) and the final ux, uy, theta, phi, rho_w (float32).
  python tests/golden/make_oracle_runs.py cavity1024 [--work DIR] [--threads N]
      1024 x 1024, Ra 1e6, 2 %, 50 nm, from rest, 20 000 steps. Stores the Nusselt numbers,
      the maximum speed |u|, the full-field L2 norm of phi - phi0, and ux, uy, phi on every
      4th row and column (float32).
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

K = 1000
RES_TOL = 1e-8
MAX_STEPS = 2_000_000
STEPS_1024 = 20000
SAMPLE = 4


def _solver(w):
    return oracle.RefSolver(w["nx"], w["ny"], w["Ra"], w["Pr"], w["phi"], w["d_p"])


def _resume(s, ckpt):
    """Initialise from rest, or from the checkpoint (state and histories) if there is one."""
    s.init()
    if not os.path.exists(ckpt):
        return 0, [], []
    d = np.load(ckpt)
    s.set_state(d["state"])
    s.residual()  # a fresh snapshot at the resumed state
    return int(d["steps"]), list(d["nu_hist"]), list(d["res_hist"])


def cavity256(work):
    w = workloads.CAVITY_256
    s = _solver(w)
    ckpt = os.path.join(work, "oracle_cavity256.ckpt.npz")
    steps, nu_hist, res_hist = _resume(s, ckpt)
    if steps == 0:
        s.residual()
    t0 = time.time()
    while steps < MAX_STEPS:
        s.step(K)
        steps += K
        nu_hist.append(s.nusselt())
        r = s.residual()
        res_hist.append(r)
        if steps % 20000 == 0:
            np.savez(ckpt, state=s.get_state(), steps=steps, nu_hist=np.array(nu_hist),
                     res_hist=np.array(res_hist))
            print("step %d  Nu %.8f  residual %.3e  (%.0f s)" % (steps, nu_hist[-1][0], r,
                                                                 time.time() - t0), flush=True)
        if r < RES_TOL and len(res_hist) > 1:
            break
    f = s.fields(oracle.UX | oracle.UY | oracle.THETA | oracle.PHI | oracle.RHO_W)
    nh, nc = s.nusselt()
    out = os.path.join(HERE, "oracle_cavity256_steady.npz")
    np.savez_compressed(out, steps=steps, nu_hot=nh, nu_cold=nc, residual=res_hist[-1],
                        nu_hist=np.array(nu_hist), res_hist=np.array(res_hist),
                        fields=f.astype(np.float32), check_every=K, res_tol=RES_TOL,
                        workload=w["name"])
    print("wrote", out, "steps", steps, "Nu", nh, nc)


def cavity1024(work):
    w = workloads.CAVITY_1024
    s = _solver(w)
    ckpt = os.path.join(work, "oracle_cavity1024.ckpt.npz")
    steps, _, _ = _resume(s, ckpt)
    t0 = time.time()
    while steps < STEPS_1024:
        n = min(2000, STEPS_1024 - steps)
        s.step(n)
        steps += n
        np.savez(ckpt, state=s.get_state(), steps=steps, nu_hist=np.zeros(0),
                 res_hist=np.zeros(0))
        print("step %d (%.0f s)" % (steps, time.time() - t0), flush=True)
    ux, uy, phi = s.fields(oracle.UX | oracle.UY | oracle.PHI)
    nh, nc = s.nusselt()
    out = os.path.join(HERE, "oracle_cavity1024_20000.npz")
    sl = (slice(0, None, SAMPLE), slice(0, None, SAMPLE))
    np.savez_compressed(out, steps=steps, nu_hot=nh, nu_cold=nc,
                        umax=float(np.sqrt(ux ** 2 + uy ** 2).max()),
                        dphi_l2=float(np.linalg.norm((phi - w["phi"]).ravel())),
                        sample=SAMPLE, ux=ux[sl].astype(np.float32),
                        uy=uy[sl].astype(np.float32), phi=phi[sl].astype(np.float32),
                        workload=w["name"])
    print("wrote", out, "Nu", nh, nc)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("run", choices=["cavity256", "cavity1024"])
    ap.add_argument("--work", default=os.path.join(ROOT, "_work"))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    os.makedirs(a.work, exist_ok=True)
    oracle.build()
    oracle.set_threads(a.threads)
    {"cavity256": cavity256, "cavity1024": cavity1024}[a.run](a.work)


if __name__ == "__main__":
    main()
