"""Writes the oracle's SIMP trajectories of the full-size workloads under
tests/golden/, from oracle/ only (no GPU code is imported or run).

  python tests/golden/make_trajectories.py cantilever2d    # 600 x 200, 3 cases, 50 iterations, SuperLU
  python tests/golden/make_trajectories.py cantilever3d    # 120 x 40 x 40, 30 iterations, Jacobi-CG
  python tests/golden/make_trajectories.py cantilever3d_large  # 240 x 80 x 80, one iteration, Jacobi-CG
  python tests/golden/make_trajectories.py cg_count        # 240 x 80 x 80: CG iterations to 1e-6

Each iteration follows the paper's main loop (Section 4: solve, objective and
sensitivities, the sensitivity filter of Eq. "filter_mat", the OC update of
Eq. "update" with bisection on lambda) from the uniform start rho = volfrac.
The 2D solve is the paper's direct factorisation (SuperLU).  A direct solve of
the 3D grids does not fit (the factorisation of the 120 x 40 x 40 operator ran
for half an hour and more than 11 GB before it was stopped), so they use the
oracle's SciPy Jacobi-CG, warm started from the previous iteration's
displacement, to relative residual 1e-12 (1e-11 where that floor is not
reached; the file records the tolerance of every iteration).

Stored per iteration: compliance c, the bisection multiplier lambda, the
exact root of the volume constraint, volume and change.  At the snapshot
iterations k the input density rho_k and the output rho_{k+1} are stored
whole (2D, 120 x 40 x 40); at 240 x 80 x 80 only c, the multipliers, volume,
change and rho_1 at 65,536 seeded sample indices.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import fem, filt, oc, sens  # noqa: E402

SPECS = {
    "cantilever2d": dict(make=W.cantilever2d, n_iter=50, snaps=(0, 10, 30, 49), method="lu",
                         out="traj_cantilever2d_600x200.npz"),
    "cantilever3d": dict(make=W.cantilever3d, n_iter=30, snaps=(0, 10, 29), method="cg",
                         out="traj_cantilever3d_120x40x40.npz"),
    "cantilever3d_large": dict(make=W.cantilever3d_large, n_iter=1, snaps=(0,), method="cg",
                               out="traj_cantilever3d_240x80x80.npz", sample=65536),
}


def solve(w, rho, method, U_prev):
    if method == "lu":
        return fem.solve(w, rho, method="lu"), 0.0
    K = fem.assemble(w, rho)
    for rtol in (1e-12, 1e-11):
        try:
            return fem.solve(w, rho, method="cg", rtol=rtol, K=K, x0=U_prev, maxiter=400000), rtol
        except RuntimeError:
            continue
    raise RuntimeError("the oracle CG reached neither 1e-12 nor 1e-11")


def main(name):
    spec = SPECS[name]
    w = spec["make"]()
    Wm = filt.sparse_weights(w)
    rho = w.initial_density()
    U = None
    hist = {k: [] for k in ("c", "lam", "lam_exact", "vol", "change", "rtol", "seconds")}
    snaps = {}
    for it in range(spec["n_iter"]):
        t0 = time.perf_counter()
        U, rtol = solve(w, rho, spec["method"], U)
        c, ce, dc = sens.sensitivities(w, rho, U)
        dcf = filt.sensitivity_filter(Wm, rho, dc)
        rho_new, lam, vol, change, _ = oc.bisect(rho, dcf, w.volfrac, w.move, w.dmin, w.passive)
        lam_exact = oc.exact_lambda(rho, dcf, w.volfrac, w.move, w.dmin, w.passive)
        for k, v in (("c", c), ("lam", lam), ("lam_exact", lam_exact), ("vol", vol), ("change", change),
                     ("rtol", rtol), ("seconds", time.perf_counter() - t0)):
            hist[k].append(v)
        if it in spec["snaps"]:
            snaps[it] = (rho.copy(), rho_new.copy())
        print(f"{name} it {it}: c {c:.12g} lam {lam:.12g} change {change:.4f} rtol {rtol} "
              f"{hist['seconds'][-1]:.1f} s", flush=True)
        rho = rho_new
    out = {k: np.array(v) for k, v in hist.items()}
    ks = sorted(snaps)
    out["snap_it"] = np.array(ks)
    if "sample" in spec:
        idx = np.sort(np.random.default_rng(2026).choice(w.n_el, size=spec["sample"], replace=False))
        out["sample_idx"] = idx
        out["rho_out_sample"] = np.stack([snaps[k][1][idx] for k in ks])
    else:
        out["rho_in"] = np.stack([snaps[k][0] for k in ks])
        out["rho_out"] = np.stack([snaps[k][1] for k in ks])
    np.savez_compressed(os.path.join(HERE, spec["out"]), **out)


def cg_count(out="cg_iterations_cantilever3d_240x80x80.json"):
    """The oracle's Jacobi-CG iteration count to relative residual 1e-6 on the
    240 x 80 x 80 cantilever at the uniform start (the solve of its first SIMP
    iteration at the workload's tolerance), with the time per iteration here."""
    import json
    w = W.cantilever3d_large()
    K = fem.assemble(w, w.initial_density())
    n = [0]
    t0 = time.perf_counter()
    fem.solve(w, w.initial_density(), method="cg", rtol=w.tol, K=K,
              callback=lambda xk: n.__setitem__(0, n[0] + 1))
    dt = time.perf_counter() - t0
    with open(os.path.join(HERE, out), "w") as f:
        json.dump({"workload": "cantilever3d_240x80x80", "rho": "uniform volfrac", "rtol": w.tol,
                   "iterations": n[0], "seconds_here": round(dt, 1),
                   "how": "oracle.fem.solve(method='cg'), SciPy Jacobi-preconditioned CG from u = 0"}, f, indent=1)
    print("iterations", n[0], "seconds", dt)


if __name__ == "__main__":
    if sys.argv[1] == "cg_count":
        cg_count()
    else:
        main(sys.argv[1])
