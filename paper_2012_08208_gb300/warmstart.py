"""Training and evaluation of the learned PCG warm start (3D problems).

Data: seeded SIMP trajectories of `workloads.warmstart3d` problems at
48 x 16 x 16 and 96 x 32 x 32 elements, solved by the library's own PCG (mixed
precision, true relative residual <= tol).  At each of the first `snapshots`
OC iterations the network input (tpnn_features) and the normalised element-mean
displacement (tpnn_targets) of the current density are stored on the device
in bf16.  The network is trained on the GPU by the library's own forward,
backward and Adam kernels (tpnn_train_step) with an MSE loss.

Evaluation: time to a true relative residual `tol` of the same problem and
density by plain FP64 Jacobi-PCG from u = 0, by mixed-precision PCG from
u = 0, and by mixed-precision PCG from the learned start (network time
included).

    python -m paper_2012_08208_gb300.warmstart train --out weights.npz
    python -m paper_2012_08208_gb300.warmstart evaluate --weights weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import topo

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_unet_16-32-64-64.npz")
WIDTHS = (16, 32, 64, 64)
SIZES = ((48, 16, 16, 48), (96, 32, 32, 32))  # (nelx, nely, nelz, trajectories)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the warm-start training and evaluation run on a CUDA device")
    return torch


class Dataset:
    """Samples of one grid size: X [N, 8, D, H, W] and T [N, 3, D, H, W] (bf16),
    R [N, n_el] densities (FP64), comp [N] compliances, traj [N] index of the
    trajectory problem (kept alive: its loads and supports define K and f)."""

    def __init__(self, X, T, R, comp, traj, problems):
        self.X, self.T, self.R, self.comp, self.traj, self.problems = X, T, R, comp, traj, problems

    def __len__(self):
        return self.X.shape[0]


def generate(sizes=SIZES, snapshots=25, seed0=1000, tol=1e-7, log=print):
    """Returns {(nelz, nely, nelx): Dataset}; samples are stored in a seeded
    random order of slots."""
    torch = _torch()
    import workloads as W
    out = {}
    opts = topo.solve_opts(tol=tol, max_it=200000, precision=topo.TP_PREC_MIXED,
                           warm_start=topo.TP_WARM_PREVIOUS, update_drop=0.1)
    seed = seed0
    for (nx, ny, nz, ntraj) in sizes:
        N = ntraj * snapshots
        ne = nx * ny * nz
        X = torch.empty((N, topo.TPNN_FEATURES, nz, ny, nx), dtype=torch.bfloat16, device="cuda")
        T = torch.empty((N, 3, nz, ny, nx), dtype=torch.bfloat16, device="cuda")
        R = torch.empty((N, ne), dtype=torch.float64, device="cuda")
        comp = np.zeros(N)
        traj = np.zeros(N, dtype=np.int64)
        slots = np.random.default_rng(seed0 + nx).permutation(N)
        problems = []
        t0 = time.time()
        k = 0
        for tr in range(ntraj):
            w = W.warmstart3d(nx, ny, nz, seed)
            seed += 1
            p = topo.Problem.from_workload(w)
            problems.append(p)
            for it in range(snapshots):
                info = p.solve(opts, check=False)
                if info.status not in (topo.TP_OK, topo.TP_ERR_NOT_CONVERGED):
                    raise topo.TopoError(info.status, p.last_error())
                sl = int(slots[k])
                p.features(X[sl:sl + 1])
                p.targets(T[sl:sl + 1])
                p.get(topo.TP_RHO, out=R[sl])
                comp[sl] = p.sensitivities()
                traj[sl] = tr
                k += 1
                p.filter()
                p.oc_update()
        torch.cuda.synchronize()
        log(f"generated {N} samples at {nx}x{ny}x{nz} in {time.time() - t0:.1f} s")
        out[(nz, ny, nx)] = Dataset(X, T, R, comp, traj, problems)
    return out


def _batches(data, steps, batch, seed):
    """(key, start, size) per step: groups drawn in proportion to their sizes,
    contiguous windows of the (already shuffled) slots."""
    keys = sorted(data)
    counts = np.array([len(data[k]) for k in keys], float)
    rng = np.random.default_rng(seed)
    pos = {k: 0 for k in keys}
    for _ in range(steps):
        k = keys[rng.choice(len(keys), p=counts / counts.sum())]
        b = batch.get(k[0], 2)
        if pos[k] + b > len(data[k]):
            pos[k] = int(rng.integers(0, b))  # new pass with a shifted window
        yield k, pos[k], b
        pos[k] += b


def _lr(s, steps, lr, lr_min):
    return lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * s / max(1, steps - 1)))


def train(net, data, steps=3000, batch=None, lr=2e-3, lr_min=1e-4, seed=0, log=print, log_every=250):
    """Pre-training: MSE of the element-mean targets.  Adam on minibatches,
    cosine learning-rate decay.  Returns the loss per step."""
    batch = batch or {16: 8, 32: 2}
    hist = []
    t0 = time.time()
    for s, (k, i, b) in enumerate(_batches(data, steps, batch, seed)):
        d = data[k]
        cur = _lr(s, steps, lr, lr_min)
        hist.append(net.train_step(d.X[i:i + b], d.T[i:i + b], cur))
        if log and (s % log_every == 0 or s == steps - 1):
            log(f"mse step {s:5d} lr {cur:.2e} loss {np.mean(hist[-log_every:]):.5f} ({time.time() - t0:.1f} s)")
    return hist


def train_energy(net, data, steps=3000, batch=None, lr=5e-4, lr_min=1e-5, seed=1, log=print, log_every=250):
    """Fine-tuning on the quantity the solver gains from: the relative energy
    error of the best multiple of the node-averaged prediction (tpnn_energy_grad
    on each sample's own operator).  Returns the mean loss per step."""
    torch = _torch()
    batch = batch or {16: 8, 32: 2}
    bufs = {}
    hist = []
    t0 = time.time()
    for s, (k, i, b) in enumerate(_batches(data, steps, batch, seed)):
        d = data[k]
        if (k, b) not in bufs:
            bufs[(k, b)] = (torch.empty((b, 3) + k, device="cuda"), torch.empty((b, 3) + k, device="cuda"))
        Y, GY = bufs[(k, b)]
        net.zero_grad()
        net.forward(d.X[i:i + b], Y)
        ls = []
        for j in range(b):
            p = d.problems[int(d.traj[i + j])]
            p.set_density(d.R[i + j])
            ls.append(float(p.energy_grad(Y[j:j + 1], d.comp[i + j], GY[j:j + 1])[0]))
        net.backward(GY)
        net.adam(_lr(s, steps, lr, lr_min))
        hist.append(float(np.mean(ls)))
        if log and (s % log_every == 0 or s == steps - 1):
            log(f"energy step {s:5d} loss {np.mean(hist[-log_every:]):.4f} ({time.time() - t0:.1f} s)")
    return hist


def energy_error(p, net, comp):
    """Relative energy-norm error of the learned start for problem p (whose
    compliance at the current density is comp)."""
    torch = _torch()
    pr = p.params
    shape = (pr.nelz, pr.nely, pr.nelx)
    X = torch.empty((p.n_cases, topo.TPNN_FEATURES) + shape, dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((p.n_cases, 3) + shape, device="cuda")
    GY = torch.empty_like(Y)
    p.features(X)
    net.forward(X, Y)
    return float(np.sqrt(max(p.energy_grad(Y, comp, GY)[0], 0.0)))


def time_to_tol(p, kind, tol=1e-6, net=None, max_it=400000, drop=0.1, warm_max_rel=0.0):
    """Solve the problem's current state equation from scratch to `tol`:
    kind 'f64' (plain FP64 PCG, u = 0), 'mixed' (u = 0), 'learned' (mixed
    PCG from the network's start, dropped for u = 0 when its true relative
    residual exceeds warm_max_rel, 0 meaning 1), 'mg' (multigrid-preconditioned
    CG from u = 0) or 'mg_learned' (the same from the network's start).  Returns a dict of the device
    time (ms, network included), CG iterations, initial and final true
    residuals."""
    ws_ms = 0.0
    alpha = None
    # the same density again: every arm pays its setup (moduli, diagonals, and
    # the multigrid hierarchy) inside its timed solve
    p.set_density(p.get(topo.TP_RHO))
    if kind == "f64":
        o = topo.solve_opts(tol=tol, max_it=max_it, precision=topo.TP_PREC_F64, warm_start=topo.TP_WARM_ZERO)
    elif kind == "mixed":
        o = topo.solve_opts(tol=tol, max_it=max_it, precision=topo.TP_PREC_MIXED, warm_start=topo.TP_WARM_ZERO,
                            update_drop=drop)
    elif kind == "learned":
        a, ws_ms = p.warm_start_nn(net)
        alpha = float(a[0])
        o = topo.solve_opts(tol=tol, max_it=max_it, precision=topo.TP_PREC_MIXED, warm_start=topo.TP_WARM_USER,
                            update_drop=drop, warm_max_rel=warm_max_rel)
    elif kind == "mg":
        o = topo.solve_opts(tol=tol, max_it=max_it, precision=topo.TP_PREC_MIXED, warm_start=topo.TP_WARM_ZERO,
                            precond=topo.TP_PRECOND_MG)
    elif kind == "mg_learned":
        a, ws_ms = p.warm_start_nn(net)
        alpha = float(a[0])
        o = topo.solve_opts(tol=tol, max_it=max_it, precision=topo.TP_PREC_MIXED, warm_start=topo.TP_WARM_USER,
                            warm_max_rel=warm_max_rel, precond=topo.TP_PRECOND_MG)
    else:
        raise ValueError(kind)
    info = p.solve(o, check=False)
    return {"kind": kind, "ms": info.ms + ws_ms, "solve_ms": info.ms, "warm_ms": ws_ms, "iters": info.iters,
            "rel_res": info.rel_res[0], "rel_res_init": info.rel_res_init[0], "converged": info.converged,
            "fallback": info.warm_fallback, "alpha": alpha}


def density_after(w, n_oc, tol=1e-6):
    """Problem object of workload `w` advanced by n_oc SIMP iterations (mixed PCG
    to tol, previous displacement as start)."""
    p = topo.Problem.from_workload(w)
    o = topo.solve_opts(tol=tol, max_it=400000, precision=topo.TP_PREC_MIXED, warm_start=topo.TP_WARM_PREVIOUS,
                        update_drop=0.1)
    for _ in range(n_oc):
        p.simp_step(o, check=False)
    return p


def evaluate(w, net, n_oc=(0, 5), tol=1e-6, kinds=("f64", "mixed", "learned"), warm_max_rel=0.0, log=print):
    out = []
    for k in n_oc:
        p = density_after(w, k, tol)
        p.solve(topo.solve_opts(tol=1e-9, max_it=400000, precision=topo.TP_PREC_MIXED, update_drop=0.1),
                check=False)
        err = energy_error(p, net, p.sensitivities())
        if log:
            log(json.dumps({"oc_iter": k, "learned_energy_err": err}))
        for kind in kinds:
            r = time_to_tol(p, kind, tol, net, warm_max_rel=warm_max_rel)
            r["oc_iter"] = k
            out.append(r)
            if log:
                log(json.dumps(r))
        p.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", default=WEIGHTS)
    t.add_argument("--steps", type=int, default=3000)
    t.add_argument("--energy-steps", type=int, default=3000)
    t.add_argument("--init", default=None, help="start from these weights (skips the MSE stage)")
    t.add_argument("--snapshots", type=int, default=25)
    t.add_argument("--scale", type=float, default=1.0, help="fraction of the trajectories to generate")
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=0)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=WEIGHTS)
    e.add_argument("--size", default="240x80x80")
    e.add_argument("--oc", default="0,5")
    e.add_argument("--kinds", default="f64,mixed,learned")
    e.add_argument("--warm-max-rel", type=float, default=0.0)
    a = ap.parse_args(argv)
    import workloads as W
    torch = _torch()
    if a.cmd == "train":
        sizes = tuple((nx, ny, nz, max(1, int(round(n * a.scale)))) for (nx, ny, nz, n) in SIZES)
        data = generate(sizes, snapshots=a.snapshots)
        hist = [float("nan")]
        if a.init:
            net = topo.Net.load(a.init)
        else:
            rng = np.random.default_rng(a.seed)
            net = topo.Net(topo.TPNN_FEATURES, WIDTHS)
            params = []
            for co, ci in net.shapes:
                params.append((rng.normal(0.0, math.sqrt(2.0 / (27 * ci)), size=(co, ci, 27)), np.zeros(co)))
            net.set_params(params)
            hist = train(net, data, steps=a.steps, lr=a.lr, seed=a.seed)
        if a.energy_steps > 0:
            hist = train_energy(net, data, steps=a.energy_steps, seed=a.seed + 1)
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        net.save(a.out)
        print(json.dumps({"saved": a.out, "final_loss": float(np.mean(hist[-100:])), "steps": a.steps}))
    else:
        nx, ny, nz = (int(v) for v in a.size.split("x"))
        w = W.cantilever3d_large() if (nx, ny, nz) == (240, 80, 80) else W.cantilever3d(nx, ny, nz)
        net = topo.Net.load(a.weights)
        evaluate(w, net, n_oc=tuple(int(v) for v in a.oc.split(",")), kinds=tuple(a.kinds.split(",")),
                 warm_max_rel=a.warm_max_rel)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
