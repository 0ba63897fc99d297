"""Parametric studies of the paper's Section 3 run with the library's batched solver: grid
independence (the paper settles on 160 x 160 before its runs), the aspect ratio of the cavity
(Section 3.e), the slip-mechanism ablation (each force of Table 1 switched off in turn, the
drag always on: without it the explicit forcing of the interaction is unstable at these drag
rates) and the materials (the particle material and the base fluid of Section 3's Figs 9-10;
the paper prints no property values, so handbook values near 25 C are used). Every point is run
to the steady hot-wall Nusselt number (mclbm_batch_run_to_steady).

    python -m paper_1511_04552_gb300.studies [--only grid|aspect|ablation|materials]
        [--out studies.json]
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
# particle materials (SI: density, specific heat, conductivity, expansion coefficient)
PARTICLES = (("Al2O3", dict(rho_p=3970.0, cp_p=765.0, k_p=40.0, beta_p=0.85e-5)),
             ("SiO2", dict(rho_p=2220.0, cp_p=745.0, k_p=1.38, beta_p=0.55e-6)),
             ("CuO", dict(rho_p=6500.0, cp_p=535.6, k_p=20.0, beta_p=0.85e-5)),
             ("Cu", dict(rho_p=8933.0, cp_p=385.0, k_p=401.0, beta_p=1.67e-5)))
# base fluids (+ dynamic viscosity); Pr = mu cp / k of each
FLUIDS = (("water", dict(rho_f=997.1, cp_f=4179.0, k_f=0.613, beta_f=2.1e-4, mu_f=8.9e-4)),
          ("ethylene glycol", dict(rho_f=1111.4, cp_f=2415.0, k_f=0.252, beta_f=6.5e-4,
                                   mu_f=1.57e-2)),
          ("EG-water 50/50", dict(rho_f=1063.0, cp_f=3300.0, k_f=0.38, beta_f=5.8e-4,
                                  mu_f=3.4e-3)))


def _steady(specs, tol=1e-4):
    """specs: list of (label, nx, ny, props overrides). One batched solve; per point the steady
    hot- and cold-wall Nusselt numbers and the steps taken."""
    import torch
    cavs = []
    for _, nx, ny, kw in specs:
        kw = dict(kw)
        pr = kw.pop("Pr", BASE["Pr"])
        cavs.append(B.Cavity(nx, ny, BASE["Ra"], pr, BASE["phi"], BASE["d_p"], **kw).init())
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


def materials(n=128):
    """Each particle material in water (Pr of the benchmark), and alumina in each base fluid
    (Pr = mu cp / k of the fluid)."""
    specs = [("%s in water" % name, n, n, dict(props)) for name, props in PARTICLES]
    al2o3 = dict(PARTICLES[0][1])
    for name, props in FLUIDS[1:]:
        kw = dict(al2o3, **props)
        kw["Pr"] = props["mu_f"] * props["cp_f"] / props["k_f"]
        specs.append(("Al2O3 in %s (Pr %.1f)" % (name, kw["Pr"]), n, n, kw))
    return _steady(specs)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--only", choices=("grid", "aspect", "ablation", "materials"), default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    runs = {"grid": grid_independence, "aspect": aspect_ratio, "ablation": ablation,
            "materials": materials}
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
