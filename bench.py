"""Benchmark of the GB300 SIMP hot path.

Default workload: the 3D cantilever, 240 x 80 x 80 H8 elements (4,743,603
DOFs), x = 0 face clamped, unit line load along the bottom edge of the x = 240
face, volfrac 0.1, rmin 2.0, solved to true relative residual 1e-6 by
multigrid-preconditioned CG (FP32 operator and V-cycle, FP64 restarts), warm
started from the previous iteration's displacement.  One step = one SIMP
iteration (solve, sensitivities, filter, OC update) on device-resident data.
Metric: SIMP iterations per second (higher is better).  The 60 x 20 MBB beam,
the 600 x 200 three-case cantilever and the 120 x 40 x 40 cantilever are
reported beside it (`simp_configs`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
(the single-problem path does not shard); value = iterations of all ranks / the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on the host
cores for the same workload and metric (rank 0 only), on a bounded sample of
each step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SIMP iter/s; K(rho)u GDOF/s vs HBM roofline; learned+mixed vs plain PCG @1e-6"
WORKLOAD = "cantilever3d_240x80x80_line_load"
L2_FLUSH_BYTES = 256 << 20
# DRAM read + write of one finest-level 3D sweep launch at 240 x 80 x 80, from
# an ncu capture of the same kernel at the same size: the mean of three
# consecutive launches of a SIMP step (68.1, 45.7 and 65.5 MB; below the
# 82.0 MB of algorithmic bytes because the outputs stay in L2 for the next
# kernel).  None once the kernel changes, until it is captured again.
TRAFFIC_FINE_SWEEP_3D = 59.8e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def start(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def stop(self):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "", 1).isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if "Active" in s[2 + i]
                          and not s[2 + i].startswith("Not")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    from paper_2012_08208_gb300 import dist as D
    return D.env()


def algorithmic_bytes_pcg(info, n_dof, n_el, nc):
    """Algorithmic bytes of one mixed-precision CG launch: per CG iteration and
    per DOF and case 58 B (FP32 operator 10 B: read u, write y, moduli; CG vectors
    48 B), per FP64 true-residual update 60 B (FP64 operator 20 B, f, x64, x_l,
    r, z)."""
    return info.iters * nc * n_dof * 58.0 + info.updates * nc * n_dof * 60.0


# ---------------------------------------------------------------------------
# our arm


SOLVER_NAMES = {0: "Jacobi-PCG (persistent, FP32 + FP64 reliable updates)",
                1: "multigrid-preconditioned CG (FP32 V-cycle, FP32 correction segments, FP64 restarts; "
                   "graph-replayed iterations)",
                2: "multigrid-preconditioned CG (FP32 V-cycle, one persistent cooperative kernel per segment)"}


def step_opts(topo, w, solver):
    """Solver options of one SIMP step of workload w: its own tolerance and
    precision, previous displacement as the start."""
    prec = topo.TP_PREC_F64 if w.precision == "f64" else topo.TP_PREC_MIXED
    return topo.solve_opts(tol=w.tol, max_it=100000, precision=prec, warm_start=topo.TP_WARM_PREVIOUS,
                           update_drop=1e-1, precond=solver)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_2012_08208_gb300 import topo

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    w = W.cantilever3d_large()
    opts = step_opts(topo, w, args.solver)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    with torch.cuda.stream(stream):
        p = topo.Problem.from_workload(w, stream=stream)
        for _ in range(args.warmup):
            p.simp_step(opts, check=False)
            flush.add_(1.0)
        barrier()
        # the state after the warm-up: the e2e loop below restarts from it, so
        # both loops time the same SIMP iterations
        rho_w = p.get(topo.TP_RHO)
        u_w = p.get(topo.TP_U)
        clocks = ClockSampler(local)
        clocks.start()
        launches0 = p.launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        infos = []
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            infos.append(p.simp_step(opts, check=False))
            ev[k][1].record(stream)
            flush.add_(1.0)  # L2 flush between timed steps (outside the events)
        barrier()
        t_wall = time.perf_counter() - t_wall0
        launches = p.launch_count() - launches0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        # roofline pass: the same SIMP iterations again, with CUDA event pairs
        # around every finest-level sweep launch on the problem's stream (event
        # nodes in the replayed graph); kept out of the timed steps above
        prof = None
        if args.solver in (1, 2):
            p.set_density(torch.from_numpy(rho_w).to(dev))
            p.set(topo.TP_U, u_w)
            p.set_profile(True)
            for _ in range(min(args.steps, 3)):
                p.simp_step(opts, check=False)
                flush.add_(1.0)
            barrier()
            prof = p.get_profile()
            p.set_profile(False)
        # end-to-end through the public API with host buffers: H2D of the step's
        # design from pinned memory, the step, D2H of the updated design.
        rho_h = torch.empty(w.n_el, dtype=torch.float64, pin_memory=True)
        rho_h.numpy()[:] = rho_w
        out_h = torch.empty(w.n_el, dtype=torch.float64, pin_memory=True)
        e2e_steps = args.steps
        p.set(topo.TP_U, u_w)  # the warm start of the first timed step
        flush.add_(1.0)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            p.set_density(rho_h)
            p.simp_step(opts, check=False)
            p.get(topo.TP_RHO, out=out_h)
            rho_h.copy_(out_h)
            flush.add_(1.0)  # as in the device-timed loop
        barrier()
        t_e2e = time.perf_counter() - t0
        clk = clocks.stop()
        from paper_2012_08208_gb300 import dist as D
        total_ms, t_e2e = D.max_over_ranks([float(sum(step_ms)), t_e2e])
        extras = {}
        if not args.no_extras:
            extras["batch"] = batch_extra(topo, torch, dev, stream, ws=ws, rank=rank)
        if not args.no_extras and rank == 0:
            extras["simp_configs"] = simp_configs_extra(topo, torch, dev, stream, args.solver)
            extras["p1"] = p1_extra(topo, torch, dev, stream)
            extras["matvec"] = matvec_roofline(topo, torch, dev, stream, W.cantilever3d_large(),
                                               "cantilever3d_240x80x80 H8 FP32 K(rho)u")
            extras["matvec_2d"] = matvec_roofline(topo, torch, dev, stream, W.cantilever2d(),
                                                  "cantilever2d_600x200 Q4 FP32 K(rho)u", copies=96, reps=5)
            extras["learned"] = learned_extra(topo)
            extras["helmholtz"] = helmholtz_extra(topo, torch, dev, stream)
        p.close()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    hbm, peak_kind = _peaks()
    solve_ms = [i.solve.ms for i in infos]
    traffic = None
    avg_ms = float(np.mean(solve_ms))
    if args.solver in (1, 2):
        # dominant kernel, timed live by CUDA event pairs on the problem's
        # stream: the finest-level sweep launches (event nodes in the replayed
        # graph), or the persistent segment kernel (--solver 2)
        n_l, ms_l, bytes_l, levels = prof
        achieved = bytes_l / (ms_l * 1e-3) / 1e9 if ms_l > 0 else 0.0
        if args.solver == 1:
            roof_kernel = ("mg_sweep_kernel<3> (finest multigrid level: Chebyshev step or residual on the "
                           "strain-form FP32 H8 operator, graph-replayed PCG iterations)")
        else:
            roof_kernel = ("mg_seg_kernel<3,1> (persistent multigrid-preconditioned CG segment: FP32 correction "
                           "CG, Chebyshev V-cycle with grid barriers between phases)")
        roof_extra = {"launches_timed": n_l, "us_per_launch": round(1e3 * ms_l / max(n_l, 1), 3),
                      "bytes_per_launch": round(bytes_l / max(n_l, 1)), "levels": levels,
                      "bytes_note": "per launch: 4 B per element (moduli), 4 B per DOF (l1 scale), 12 B per DOF "
                                    "and case (u, b read, y written)",
                      "timing_note": "event pairs around each finest-sweep launch inside the replayed graph, in a "
                                     "separate pass over the first timed SIMP iterations (the events add the "
                                     "graph's node gaps to each launch)"}
        if args.solver == 1:
            traffic = TRAFFIC_FINE_SWEEP_3D
    else:
        byts = [algorithmic_bytes_pcg(i.solve, w.n_dof, w.n_el, w.n_cases) for i in infos]
        avg_bytes = float(np.mean(byts))
        achieved = avg_bytes / (avg_ms * 1e-3) / 1e9
        roof_kernel = "pcg_kernel<3,float,1> (persistent Jacobi-PCG)"
        roof_extra = {}
    value = ws * args.steps / (total_ms * 1e-3)
    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline(w, seconds=args.cpu_seconds)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "SIMP iter/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "240x80x80 H8", "n_dof": w.n_dof, "n_cases": w.n_cases,
                   "volfrac": w.volfrac, "rmin": w.rmin, "tol": w.tol,
                   "precision": "FP32 operator + FP64 reductions/restarts",
                   "warm_start": "previous iteration's displacement", "l2": "flushed between timed steps",
                   "solver": SOLVER_NAMES[args.solver], "parallelism": f"replicas x{ws}"},
        "e2e": {"value": round(ws * e2e_steps / t_e2e, 4), "unit": "SIMP iter/s",
                "h2d_bytes_per_step": w.n_el * 8, "d2h_bytes_per_step": w.n_el * 8},
        "gpu_launches": int(launches),
        "roofline": dict({"kernel": roof_kernel, "bound": "hbm",
                          "achieved": round(achieved, 2), "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                          "frac": round(achieved / hbm, 4), "traffic": traffic,
                          "solver_iters_per_step": float(np.mean([i.solve.iters for i in infos])),
                          "restarts_per_step": float(np.mean([i.solve.updates for i in infos])),
                          "solve_ms_per_step": round(avg_ms, 3),
                          "converged_steps": int(sum(i.solve.converged for i in infos)),
                          "max_true_rel_res": float(max(max(i.solve.rel_res[c] for c in range(w.n_cases))
                                                        for i in infos))}, **roof_extra),
        "clocks": clk,
        "cpu_baseline": cpu,
        "wall_s_timed": round(t_wall, 3),
    }
    line.update(extras)
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def simp_rate(topo, torch, dev, stream, w, solver, steps, warmup, profile=False):
    """SIMP iterations/s of workload w on device-resident data (L2 flushed
    between timed steps, outside the events), with the finest-sweep profile
    when asked."""
    opts = step_opts(topo, w, solver)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p = topo.Problem.from_workload(w, stream=stream)
    for _ in range(warmup):
        p.simp_step(opts, check=False)
        flush.add_(1.0)
    torch.cuda.synchronize(dev)
    rho_w, u_w = p.get(topo.TP_RHO), p.get(topo.TP_U)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = []
    for k in range(steps):
        ev[k][0].record(stream)
        infos.append(p.simp_step(opts, check=False))
        ev[k][1].record(stream)
        flush.add_(1.0)
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in ev]
    if profile:  # event pairs around the finest sweeps, in a pass of their own over the same iterations
        p.set_density(rho_w)
        p.set(topo.TP_U, u_w)
        p.set_profile(True)
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            ev2[k][0].record(stream)
            p.simp_step(opts, check=False)
            ev2[k][1].record(stream)
            flush.add_(1.0)
        torch.cuda.synchronize(dev)
        ms_prof = float(np.sum([a.elapsed_time(b) for a, b in ev2]))
    out = {"workload": w.name, "n_dof": w.n_dof, "n_cases": w.n_cases, "tol": w.tol,
           "precision": w.precision, "ms_per_step": round(float(np.mean(ms)), 3),
           "simp_iter_s": round(1e3 * steps / float(np.sum(ms)), 3),
           "solver_iters_per_step": float(np.mean([i.solve.iters for i in infos])),
           "converged_steps": int(sum(i.solve.converged for i in infos)), "steps": steps,
           "max_true_rel_res": float(max(max(i.solve.rel_res[c] for c in range(w.n_cases)) for i in infos))}
    if profile:
        n_l, ms_l, bytes_l, levels = p.get_profile()
        p.set_profile(False)
        out["fine_sweep"] = {"launches": n_l, "us_per_launch": round(1e3 * ms_l / max(n_l, 1), 3),
                             "bytes_per_launch": round(bytes_l / max(n_l, 1)),
                             "share_of_step": round(ms_l / ms_prof, 4), "levels": levels,
                             "note": "from a second pass over the same iterations with event pairs around each "
                                     "finest sweep"}
    p.close()
    return out


def simp_configs_extra(topo, torch, dev, stream, solver, steps=10, warmup=3):
    """SIMP iterations/s of the other single-problem configurations: the
    60 x 20 MBB beam (FP64, 1e-10), the 600 x 200 three-case cantilever with
    the passive disk (mixed, 1e-8) and the 120 x 40 x 40 cantilever (mixed,
    1e-6)."""
    import workloads as W
    out = {}
    for key, w in (("mbb2d_60x20", W.mbb2d()), ("cantilever2d_600x200", W.cantilever2d()),
                   ("cantilever3d_120x40x40", W.cantilever3d())):
        out[key] = simp_rate(topo, torch, dev, stream, w, solver, steps, warmup, profile=solver in (1, 2))
    out["solver"] = SOLVER_NAMES[solver]
    return out


def matvec_roofline(topo, torch, dev, stream, w, label, copies=8, reps=10):
    """K(rho)u in FP32 on workload w: GDOF/s and fraction of the HBM roofline.
    One library call applies the operator to `copies` vectors (one launch, the
    copies on the grid's y axis), so the per-call host synchronisation is
    amortised; u and y of all copies together exceed L2."""
    p = topo.Problem(topo.make_params(w.dim, w.nelx, w.nely, w.nelz, volfrac=w.volfrac, rmin=w.rmin),
                     stream=stream.cuda_stream)
    p.set_fixed(w.fixed)
    import workloads as W
    p.set_density(W.random_density(w.n_el, seed=1))
    u = torch.randn((copies, w.n_dof), dtype=torch.float32, device=dev)
    y = torch.empty_like(u)
    for _ in range(3):
        p.matvec(u, topo.TP_PREC_MIXED, ncopies=copies, out=y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        p.matvec(u, topo.TP_PREC_MIXED, ncopies=copies, out=y)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / (reps * copies)
    byts = w.n_nodes * w.dim * 4 * 2 + w.n_el * 4  # read u, write y (FP32), read E
    hbm, kind = _peaks()
    ach = byts / (ms * 1e-3) / 1e9
    p.close()
    return {"workload": label, "n_dof": w.n_dof, "us_per_apply": round(ms * 1e3, 2),
            "gdof_s": round(w.n_dof / (ms * 1e-3) / 1e9, 3), "achieved_gbs": round(ach, 1), "peak": hbm,
            "peak_kind": kind, "frac": round(ach / hbm, 4), "bytes_per_apply": byts,
            "note": f"{copies} vectors per launch, {reps} launches back to back"}


def learned_extra(topo, n_oc=(0, 5)):
    """Time to a true relative residual of 1e-6 on the 240 x 80 x 80 H8 cantilever
    (4.74M DOFs) at the densities after n_oc OC iterations: plain FP64
    Jacobi-PCG from u = 0, mixed-precision PCG from u = 0, and mixed PCG from the
    learned start (network time included; the start is dropped for u = 0 when
    its true residual exceeds that of u = 0), plus the learned start forced."""
    import workloads as W
    from paper_2012_08208_gb300 import warmstart as WS
    w = W.cantilever3d_large()
    net = topo.Net.load(WS.WEIGHTS)
    rows = []
    for k in n_oc:
        p = WS.density_after(w, k)
        r = {"oc_iter": k}
        for kind, kw in (("f64", {}), ("mixed", {}), ("learned", {}), ("learned_forced", {"warm_max_rel": 1e30}),
                         ("mg", {}), ("mg_learned", {})):
            t = WS.time_to_tol(p, "learned" if kind.startswith("learned") else kind, 1e-6, net, **kw)
            r[kind] = {"ms": round(t["ms"], 2), "iters": t["iters"], "rel_res": t["rel_res"],
                       "rel_res_init": round(t["rel_res_init"], 4), "fallback": t["fallback"],
                       "warm_ms": round(t["warm_ms"], 3)}
        r["speedup_vs_f64"] = round(r["f64"]["ms"] / r["learned"]["ms"], 3)
        r["mg_speedup_vs_f64"] = round(r["f64"]["ms"] / r["mg"]["ms"], 3)
        r["learned_gain_vs_mg"] = round(r["mg"]["ms"] / r["mg_learned"]["ms"], 4)
        r["learned_gain_vs_mixed"] = round(r["mixed"]["ms"] / r["learned"]["ms"], 4)
        rows.append(r)
        p.close()
    net.close()
    return {"workload": "cantilever3d_240x80x80 H8, time to true rel-res 1e-6", "rows": rows,
            "note": "ms = device time of the solve (+ the warm start for 'learned'); weights trained on "
                    "48x16x16 / 96x32x32 trajectories by paper_2012_08208_gb300.warmstart"}


def helmholtz_extra(topo, torch, dev, stream, reps=5, steps=5, warmup=3):
    """Helmholtz (PDE) filter mode: device time of one application rho~ = H rho
    (right-hand side, FP64 Jacobi-PCG as one persistent kernel, element means;
    the moduli and diagonal kernels that follow are included) at 600 x 200 and
    240 x 80 x 80 on a random density, and SIMP iterations/s of the 600 x 200
    cantilever in this filter mode with the multigrid solver."""
    import workloads as W
    out = {}
    for w, label in ((W.cantilever2d(), "cantilever2d_600x200"), (W.cantilever3d_large(), "cantilever3d_240x80x80")):
        p = topo.Problem.from_workload(w, stream=stream.cuda_stream)
        p.set_filter_mode(topo.TP_FILTER_HELMHOLTZ)
        rho = torch.tensor(W.random_density(w.n_el, seed=63, lo=0.001), dtype=torch.float64, device=dev)
        phys = torch.empty_like(rho)
        ms = []
        for k in range(reps + 1):
            p.set_density(rho)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.get(topo.TP_RHO_PHYS, out=phys)
            e1.record(stream)
            stream.synchronize()
            if k:
                ms.append(e0.elapsed_time(e1))
        out[label] = {"n_el": w.n_el, "ms_per_filter": round(float(np.median(ms)), 4)}
        p.close()
    w = W.cantilever2d()
    p = topo.Problem.from_workload(w, stream=stream.cuda_stream)
    p.set_filter_mode(topo.TP_FILTER_HELMHOLTZ)
    opts = topo.solve_opts(tol=w.tol, max_it=100000, warm_start=topo.TP_WARM_PREVIOUS, precond=topo.TP_PRECOND_MG)
    for _ in range(warmup):
        p.simp_step(opts, check=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    for _ in range(steps):
        p.simp_step(opts, check=False)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out["simp_cantilever2d_600x200"] = {"ms_per_step": round(ms, 3), "simp_iter_s": round(1e3 / ms, 3),
                                        "filter": "Helmholtz (two applications per step)", "solver": "multigrid-PCG"}
    p.close()
    return out


def p1_extra(topo, torch, dev, stream, steps=10, warmup=3):
    """The paper's own elements (P1 triangles with the "right/left" cut, Kuhn
    tetrahedra; FP64 Jacobi-PCG to 1e-8): SIMP iterations/s of the 2D cantilever
    with its traction strip at 60 x 20 and 300 x 100 squares, and of the
    tetrahedral cantilever at 48 x 16 x 8 cubes; and the FP64 P1 operator at
    300 x 100 (algorithmic bytes: u read and y written, 16 B per DOF, the cell
    moduli 8 B per cell, the fixed flags 1 B per DOF)."""
    import workloads as W
    out = {}
    opts = topo.solve_opts(tol=1e-8, max_it=200000, precision=topo.TP_PREC_F64, warm_start=topo.TP_WARM_PREVIOUS,
                           precond=topo.TP_PRECOND_JACOBI)
    for key, w in (("p1_cantilever2d_60x20_rightleft", W.p1_cantilever2d(60, 20)),
                   ("p1_cantilever2d_300x100_rightleft", W.p1_cantilever2d(300, 100, rmin=2.5)),
                   ("p1_cantilever3d_48x16x8_kuhn", W.p1_cantilever3d(48, 16, 8))):
        p = topo.P1Problem.from_workload(w, stream=stream)
        for _ in range(warmup):
            p.simp_step(opts)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        its = [p.simp_step(opts).solve.iters for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out[key] = {"cells": w.n_el, "n_dof": w.n_dof, "ms_per_step": round(ms, 3), "simp_iter_s": round(1e3 / ms, 3),
                    "cg_iters_per_step": float(np.mean(its))}
        p.close()
    w = W.p1_cantilever2d(300, 100)
    p = topo.P1Problem.from_workload(w, stream=stream)
    u = torch.randn(w.n_dof, dtype=torch.float64, device=dev)
    y = torch.empty_like(u)
    for _ in range(3):
        p.apply(u, out=y)
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        p.apply(u, out=y)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    us = 1e3 * e0.elapsed_time(e1) / reps
    byts = 16 * w.n_dof + 8 * w.n_el + w.n_dof
    hbm, kind = _peaks()
    out["p1_operator_300x100"] = {"us_per_apply": round(us, 2), "bytes": byts,
                                  "achieved_gbs": round(byts / (us * 1e-6) / 1e9, 1), "peak": hbm, "peak_kind": kind,
                                  "frac": round(byts / (us * 1e-6) / 1e9 / hbm, 4),
                                  "note": "FP64 node-gather parity operator; L2-resident (1.5 MB)"}
    p.close()
    return out


def batch_extra(topo, torch, dev, stream, steps=5, warmup=3, ws=1, rank=0):
    """64 uneven 2D cantilevers (batch2d, seed 0) in one persistent graph-captured
    launch per step with the autotuned tile shape: instance SIMP iterations/s.
    Over several ranks the instances are sharded by node count (no data crosses
    ranks); the value is all ranks' instance iterations over the slowest rank's
    time."""
    import workloads as W
    from paper_2012_08208_gb300 import dist as D
    allw = W.batch2d()
    mine = D.shard([w.n_nodes for w in allw], ws, rank)
    wl = [allw[i] for i in mine]
    b = topo.Batch(wl, stream=stream.cuda_stream)
    for i, w in enumerate(wl):
        b.set_density(i, w.initial_density())
    cache = os.path.join(ROOT, "_build", "batch_autotune.json")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    ty, cps = b.autotune(cache)
    opts = topo.solve_opts(tol=1e-6, max_it=100000, precision=topo.TP_PREC_MIXED,
                           warm_start=topo.TP_WARM_PREVIOUS, update_drop=0.1)
    for _ in range(warmup):
        b.step(opts, check=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    D.max_over_ranks([0.0])  # barrier
    e0.record(stream)
    infos = [b.step(opts, check=False)[0] for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = D.max_over_ranks([e0.elapsed_time(e1)])[0]
    b.close()
    return {"workload": "batch2d_64 (widths 40-320, seed 0)", "instances": len(allw), "ranks": ws,
            "value": round(len(allw) * steps / (ms * 1e-3), 2), "unit": "instance SIMP iter/s",
            "ms_per_step": round(ms / steps, 3), "tile_rows": ty, "ctas_per_sm": cps,
            "graph": int(all(i.graph for i in infos)), "max_cg_iters": max(i.max_iters for i in infos),
            "max_rel_res": max(i.max_rel_res for i in infos)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)


CG_COUNT_FILE = os.path.join(ROOT, "tests", "golden", "cg_iterations_cantilever3d_240x80x80.json")


def _oracle_cg_iterations():
    """The oracle's own Jacobi-CG iteration count to 1e-6 on the 240 x 80 x 80
    cantilever at the uniform start (written by
    tests/golden/make_trajectories.py cg_count, which runs oracle/ only)."""
    with open(CG_COUNT_FILE) as f:
        return int(json.load(f)["iterations"])


def oracle_step_sample(nz_slab=4, cg_iters=40):
    """One bounded sample of the oracle's SIMP iteration on the 240 x 80 x 80
    cantilever.  Its phases run on the 240 x 80 x nz_slab slab of the same
    cantilever (same supports, load and element arithmetic), and their times
    scale by the element ratio: assembly, sensitivities, the sensitivity filter
    and the OC bisection once each; SciPy's Jacobi-CG for `cg_iters` iterations,
    scaled per iteration to the oracle's own iteration count to 1e-6 (the
    solve of the first SIMP iteration).  Returns (seconds per full-size
    iteration, description, host threads used: process CPU time over wall
    time, which counts the threads of NumPy's and SciPy's libraries)."""
    import workloads as W
    from oracle import fem, filt, oc, sens
    c_start, w_start = time.process_time(), time.perf_counter()  # the threads used: CPU time / wall time
    full = W.cantilever3d_large()
    slab = W.cantilever3d(full.nelx, full.nely, nz_slab, volfrac=full.volfrac, rmin=full.rmin, tol=full.tol)
    scale = full.n_el / slab.n_el
    rho = slab.initial_density()
    Wm = filt.sparse_weights(slab)  # built once per oracle run, outside its loop
    t = {}
    t0 = time.perf_counter()
    K = fem.assemble(slab, rho)
    t["assembly"] = time.perf_counter() - t0
    def cg_run(iters):
        n = [0]
        t0 = time.perf_counter()
        try:
            fem.solve(slab, rho, method="cg", rtol=1e-30, K=K, maxiter=iters,
                      callback=lambda xk: n.__setitem__(0, n[0] + 1))
        except RuntimeError:
            pass  # stopped at maxiter by design
        return time.perf_counter() - t0, n[0]

    # two lengths separate the solve's set-up (free-DOF slicing, diagonal) from
    # the cost of one iteration
    ta, na = cg_run(cg_iters // 4)
    tb, nb = cg_run(cg_iters)
    t["cg_per_iteration"] = max(tb - ta, 0.0) / max(nb - na, 1)
    t["cg_setup"] = max(ta - na * t["cg_per_iteration"], 0.0)
    U = np.random.default_rng(3).normal(size=(1, slab.n_dof))
    U[:, slab.fixed.astype(bool)] = 0.0
    t0 = time.perf_counter()
    c, ce, dc = sens.sensitivities(slab, rho, U)
    t["sensitivities"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    dcf = filt.sensitivity_filter(Wm, rho, -np.abs(dc))
    t["filter"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    oc.bisect(rho, dcf, slab.volfrac, slab.move, slab.dmin)
    t["oc"] = time.perf_counter() - t0
    n_cg = _oracle_cg_iterations()
    per_iter = scale * (t["assembly"] + t["cg_setup"] + t["sensitivities"] + t["filter"] + t["oc"]
                        + n_cg * t["cg_per_iteration"])
    desc = (f"oracle phases on the 240x80x{nz_slab} slab ({slab.n_el} elements, 1/{scale:.0f} of the workload), "
            f"scaled by the element ratio: assembly {t['assembly']:.2f} s, sensitivities {t['sensitivities']:.2f} s, "
            f"filter {t['filter']:.3f} s, OC {t['oc']:.2f} s, CG set-up {t['cg_setup']:.2f} s, "
            f"SciPy Jacobi-CG {1e3 * t['cg_per_iteration']:.1f} ms "
            f"per iteration x {n_cg} iterations (the oracle's count to 1e-6 at the uniform start); "
            f"extrapolated, not a full-size run")
    threads = (time.process_time() - c_start) / max(time.perf_counter() - w_start, 1e-9)
    return per_iter, desc, threads


def cpu_baseline(w, seconds=20.0):
    """The oracle as it stands (SciPy assembly + Jacobi-CG + NumPy filter/OC),
    timed on the host on a bounded sample of the workload's SIMP iteration."""
    per_iter, desc, threads = oracle_step_sample()
    return {"value": round(1.0 / per_iter, 6), "unit": "SIMP iter/s", "cores": max(1, round(threads)),
            "kind": "oracle", "sample": desc, "host_cpus": os.cpu_count(),
            "cores_note": "threads used, measured as process CPU time / wall time over the sample"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    import workloads as W
    w = W.cantilever3d_large()
    budget = 240.0  # seconds of oracle samples (warm-up and timed), so the run ends within minutes
    t_warm0 = time.perf_counter()
    nwarm = 0
    for _ in range(args.warmup):
        oracle_step_sample()
        nwarm += 1
        if time.perf_counter() - t_warm0 > budget / 4:
            break
    per, t_wall, desc, thr = [], 0.0, "", []
    for k in range(args.steps):
        t0 = time.perf_counter()
        s, desc, th = oracle_step_sample()
        t_wall += time.perf_counter() - t0
        per.append(s)
        thr.append(th)
        if t_wall > budget:
            break
    tot = float(sum(per))
    value = len(per) / tot
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "SIMP iter/s",
            "n_gpus": ws, "steps": len(per), "warmup": nwarm,
            "ms_per_step": round(1e3 * tot / len(per), 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "240x80x80 H8", "n_dof": w.n_dof, "n_cases": w.n_cases,
                       "volfrac": w.volfrac, "rmin": w.rmin, "tol": w.tol,
                       "precision": "FP64 (SciPy Jacobi-CG, NumPy filter and OC)", "parallelism": "1 host core"},
            "cpu_baseline": {"value": round(value, 6), "unit": "SIMP iter/s", "cores": max(1, round(max(thr))),
                             "kind": "oracle", "sample": f"{len(per)} samples, each: {desc}",
                             "cores_note": "threads used, measured as process CPU time / wall time per sample"},
            "e2e": {"value": round(value, 6), "unit": "SIMP iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_only(args):
    """One extra measurement on its own (profiling entry point)."""
    import torch

    import workloads as W
    from paper_2012_08208_gb300 import topo
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        if args.only == "matvec3d":
            out = matvec_roofline(topo, torch, dev, stream, W.cantilever3d_large(),
                                  "cantilever3d_240x80x80 H8 FP32 K(rho)u", copies=args.copies, reps=args.reps)
        elif args.only == "matvec2d":
            out = matvec_roofline(topo, torch, dev, stream, W.cantilever2d(),
                                  "cantilever2d_600x200 Q4 FP32 K(rho)u", copies=args.copies, reps=args.reps)
        elif args.only == "batch":
            out = batch_extra(topo, torch, dev, stream)
        elif args.only in ("cg2d", "cg3d"):
            # one mixed-precision solve capped at --reps CG iterations (profiling entry)
            w = W.cantilever2d() if args.only == "cg2d" else W.cantilever3d_large()
            p = topo.Problem.from_workload(w, stream=stream.cuda_stream)
            info = p.solve(topo.solve_opts(tol=1e-8, max_it=args.reps, precision=topo.TP_PREC_MIXED,
                                           update_drop=0.1, precond=args.precond), check=False)
            out = {"workload": w.name, "n_dof": w.n_dof, "n_cases": w.n_cases, "iters": info.iters,
                   "updates": info.updates, "ms": round(info.ms, 3)}
            p.close()
        elif args.only == "helmholtz":
            out = helmholtz_extra(topo, torch, dev, stream)
        elif args.only == "p1":
            out = p1_extra(topo, torch, dev, stream)
        elif args.only == "simp":
            wl = {"mbb2d": W.mbb2d, "cantilever2d": W.cantilever2d, "cantilever3d": W.cantilever3d,
                  "cantilever3d_large": W.cantilever3d_large}[args.workload]()
            out = simp_rate(topo, torch, dev, stream, wl, args.solver, args.steps, args.warmup,
                            profile=args.solver in (1, 2))
        else:
            out = learned_extra(topo)
    print(json.dumps({args.only: out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--only", choices=["matvec3d", "matvec2d", "batch", "learned", "cg2d", "cg3d", "helmholtz",
                                       "simp", "p1"],
                    default=None,
                    help="run one extra measurement alone (for profiling)")
    ap.add_argument("--copies", type=int, default=8)
    ap.add_argument("--workload", default="cantilever3d_large",
                    choices=["mbb2d", "cantilever2d", "cantilever3d", "cantilever3d_large"],
                    help="workload of --only simp")
    ap.add_argument("--precond", type=int, default=0,
                    help="0 Jacobi-PCG, 1 multigrid-PCG, 2 multigrid-PCG persistent kernel (--only cg2d / cg3d)")
    ap.add_argument("--solver", type=int, default=1,
                    help="solver of the timed SIMP step: 0 Jacobi-PCG, 1 multigrid-PCG, 2 the same with persistent "
                         "segment kernels")
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
