"""FP64 central differences of the differentiable column's loss, from the oracle.

Writes tests/golden/diff_column_fd.json, the expected gradients of the
differentiable-column test (262,144 particles, Drucker-Prager phi = 30 deg,
E = 5e6 Pa, 400 steps of dt = 2e-4 s on a Coulomb floor with gravity).  The
loss is the squared error of the front runout and of the particle-mean
position after 400 steps against a target run at phi = 34 deg:

    L(phi, E) = (R(x) - R*)^2 + |mean(x) - m*|^2,
    R(x) = (mean_p r_p^8)^(1/8),  r_p = horizontal distance of particle p
           from the column's initial axis (mean initial x, y),

the smooth runout measure of the differentiable column.  The runout and mean
position of every trajectory are stored as well.  Every trajectory,
the target's included, is the serial FP64 oracle's; nothing here comes from
the CUDA library.  The derivatives are central differences at three step
sizes each, so that their agreement (the step-size study) shows whether the
loss is smooth at this point.

    python tests/golden/make_diff_column_fd.py [--procs 7]

Runs 14 trajectories of 400 oracle steps (about 5 minutes each on one core).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "diff_column_fd.json")

PHI0, E0, PHI_TARGET = 30.0, 5e6, 34.0
PHI_STEPS = (1e-2, 1e-3, 1e-4)        # degrees
E_STEPS = (1e-3, 1e-4, 1e-5)          # relative


def _workload():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2605_28525_b300 import workloads as W
    return W.diff_column()


def _final_x(args):
    phi, E = args
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    wl = _workload()
    o = oracle.Oracle(lo=wl.lo, hi=wl.hi, h=wl.dx, dt=wl.dt, g=wl.gravity, B=4, material=wl.material, E=E,
                      nu=wl.nu, rho=wl.rho, phi_deg=phi, ppc=wl.ppc, floor_kind=wl.floor_kind,
                      floor_z=wl.floor_z, floor_mu=wl.floor_mu, wall_layers=wl.wall_layers)
    t0 = time.perf_counter()
    x, _, _, _ = o.run(wl.x.astype(np.float64), None, None, None, None, nsteps=wl.steps)
    return (phi, E), x, time.perf_counter() - t0


def runout(x, axis, p=8.0):
    d = x[:, :2] - np.asarray(axis)
    r = np.sqrt((d * d).sum(1) + 1e-12)
    return float(np.mean(r ** p) ** (1.0 / p))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=7)
    a = ap.parse_args()
    wl = _workload()
    axis = (float(wl.x[:, 0].mean()), float(wl.x[:, 1].mean()))
    runs = [(PHI_TARGET, E0), (PHI0, E0)]
    runs += [(PHI0 + s * h, E0) for h in PHI_STEPS for s in (1, -1)]
    runs += [(PHI0, E0 * (1 + s * h)) for h in E_STEPS for s in (1, -1)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = {k: (x, t) for k, x, t in pool.imap_unordered(_final_x, runs)}
    xt = res[(PHI_TARGET, E0)][0]
    target_R, target_m = runout(xt, axis), xt.mean(0)

    def L(key):
        x = res[key][0]
        return (runout(x, axis) - target_R) ** 2 + float(((x.mean(0) - target_m) ** 2).sum())

    out = {
        "what": "FP64 oracle central differences of the differentiable column's loss "
                "(written by tests/golden/make_diff_column_fd.py; oracle trajectories only)",
        "citation": "Sec. 4.1 (the explicit step), Drucker-Prager return map of Klar et al. 2016; "
                    "loss: squared error of front runout and mean position against a phi = 34 deg run",
        "config": {"workload": wl.name, "particles": wl.n, "steps": wl.steps, "dt": wl.dt, "dx": wl.dx,
                   "phi_deg": PHI0, "E": E0, "target_phi_deg": PHI_TARGET, "floor_mu": wl.floor_mu,
                   "runout_p": 8.0, "axis": axis},
        "target": {"runout": target_R, "mean": [float(v) for v in target_m]},
        "loss": L((PHI0, E0)),
        "dL_dphi_per_deg": {"%g" % h: (L((PHI0 + h, E0)) - L((PHI0 - h, E0))) / (2 * h) for h in PHI_STEPS},
        "dL_dE": {"%g" % h: (L((PHI0, E0 * (1 + h))) - L((PHI0, E0 * (1 - h)))) / (2 * h * E0) for h in E_STEPS},
        # the runout and mean position of every trajectory, so that the
        # derivatives of other functionals of them can be formed too
        "runs": [{"phi_deg": k[0], "E": k[1], "runout": runout(x, axis), "mean": [float(v) for v in x.mean(0)]}
                 for k, (x, _) in sorted(res.items())],
        "oracle_seconds_per_run": float(np.mean([t for _, t in res.values()])),
        "wall_seconds": time.perf_counter() - t0,
    }
    json.dump(out, open(OUT, "w"), indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
