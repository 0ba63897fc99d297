"""Parametric studies of the paper's Section 3 run with the library's batched solver: grid
independence (the paper settles on 160 x 160 before its runs), the aspect ratio of the cavity
(Section 3.e) and the slip-mechanism ablation (each force of Table 1 switched off in turn, the
drag always on: without it the explicit forcing of the interaction is unstable at these drag
rates). Every point is run to the steady hot-wall Nusselt number (mclbm_batch_run_to_steady).

    python -m paper_1511_04552_gb300.studies [--only grid|aspect|ablation] [--out studies.json]
"""
import argparse
import json
import time

from . import binding as B

BASE = dict(Ra=1e5, Pr=6.2, phi=0.03, d_p=30e-9)
ABLATION = (("all forces", B.F_ALL),
            ("no Brownian", B.F_ALL & ~B.F_BROWNIAN),
            ("no thermophoresis", B.F_ALL & ~B.F_THERMOPHORESIS),
            ("no Saffman", B.F_ALL & ~B.F_SAFFMAN),
            ("no Magnus", B.F_ALL & ~B.F_MAGNUS),
            ("no gravity", B.F_ALL & ~B.F_GRAVITY))


def _steady(specs, tol=1e-4):
    """specs: list of (label, nx, ny, props overrides). One batched solve; per point the steady
    hot- and cold-wall Nusselt numbers and the steps taken."""
    import torch
    cavs = [B.Cavity(nx, ny, BASE["Ra"], BASE["Pr"], BASE["phi"], BASE["d_p"], **kw).init()
            for _, nx, ny, kw in specs]
    batch = B.Batch(cavs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = B.sweep_to_steady(batch, tol=tol)
    wall = time.perf_counter() - t0
    out = []
    for k, (label, nx, ny, _) in enumerate(specs):
        nh, nc = cavs[k].nusselt()
        out.append({"case": label, "nx": nx, "ny": ny, "steps": res["steps"][k],
                    "nu_hot": nh, "nu_cold": nc})
    batch.close()
    return {"points": out, "wall_s": wall, "converged": res["converged"]}


def grid_independence(sizes=(64, 128, 256, 512)):
    """The benchmark cavity (Ra 1e5, 3 %, 30 nm) on square lattices of increasing size."""
    return _steady([("%d^2" % n, n, n, {}) for n in sizes])


def aspect_ratio(h=128, ratios=(0.5, 1.0, 2.0)):
    """Cavities of height H = h nodes (Ra is based on H) and width H / AR."""
    return _steady([("AR %g" % r, int(round(h / r)), h, {}) for r in ratios])


def ablation(n=128):
    """Each slip mechanism of Table 1 switched off in turn (drag and buoyancy always on)."""
    return _steady([(label, n, n, {"force_mask": mask}) for label, mask in ABLATION])


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--only", choices=("grid", "aspect", "ablation"), default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    runs = {"grid": grid_independence, "aspect": aspect_ratio, "ablation": ablation}
    out = {}
    for name, fn in runs.items():
        if a.only and name != a.only:
            continue
        out[name] = fn()
        print(json.dumps({name: out[name]}), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f)


if __name__ == "__main__":
    main()
