"""Parity at the workloads' full sizes, in the launch configuration the bench
times, on outputs the oracle can compute (or check) at that size:

  * 600 x 200 Q4 cantilever (3 cases, passive disk): one SIMP iteration from the
    uniform start with the bench's solver options (mixed precision, true
    relative residual 1e-8, update drop 0.1) against the oracle's LU iteration.
    A true residual r = f - K u with ||r|| <= 1e-8 ||f|| moves the compliance by
    |r^T u*| <= 1e-8 ||f|| ||u*||; for these point loads ||f|| ||u*|| / f^T u* is
    about 50, so the bound is 5e-7 relative.  The element energies, the filtered
    sensitivities and the new densities inherit errors of that order (OC moves
    densities by at most the move limit, with sqrt damping): 5e-6 max-abs.
  * 120 x 40 x 40 and 240 x 80 x 80 H8 grids: sampled rows of K(rho)u in FP64
    and FP32 against the oracle's element-by-element rows, with the tolerances
    of the small-grid tests (1e-12 and 2e-5 of (|K||u|)_i).
  * 240 x 80 x 80 solve: the identity c = f^T u = u^T K u at the converged
    solution, the true residual reported by the solver recomputed with the FP64
    operator, and the solution's rows against the oracle's rows of K u = f.
  * 64-instance batch (widths 40-320): first-step compliance of sampled
    instances against the oracle's LU iteration on the same density.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, filt, simp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def topo():
    from paper_2012_08208_gb300 import topo as t
    return t


@pytest.mark.parametrize("precond", [0, 1, 2], ids=["jacobi", "multigrid", "multigrid_fused"])
def test_cantilever2d_full_step(topo, precond):
    w = W.cantilever2d()
    rho0 = w.initial_density()
    p = topo.Problem.from_workload(w)
    opts = topo.solve_opts(tol=w.tol, max_it=100000, precision=topo.TP_PREC_MIXED,
                           warm_start=topo.TP_WARM_PREVIOUS, update_drop=0.1, precond=precond)
    info = p.simp_step(opts)
    assert info.solve.converged == 1 and max(info.solve.rel_res[c] for c in range(3)) <= 1e-8
    rho1 = p.get(topo.TP_RHO)
    ref = simp.iteration(w, rho0, W=filt.weights_for(w))
    assert info.compliance == pytest.approx(ref["c"], rel=5e-7)
    assert np.max(np.abs(rho1 - ref["rho_new"])) <= 5e-6
    assert info.lambda_ == pytest.approx(ref["lam"], rel=5e-6)
    assert info.volume == pytest.approx(w.volfrac * w.n_el, rel=1e-9)
    p.close()


def _rows(n_dof, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, n_dof, size=n), [0, 1, 2, n_dof - 3, n_dof - 2, n_dof - 1]]))


@pytest.mark.parametrize("make", [W.cantilever3d, W.cantilever3d_large], ids=["120x40x40", "240x80x80"])
def test_h8_operator_sampled_rows(topo, make):
    w = make()
    rho = W.random_density(w.n_el, seed=1)
    u = W.random_vector(w.n_dof, seed=2)
    p = topo.Problem.from_workload(w)
    p.set_density(rho)
    rows = _rows(w.n_dof, 400, seed=3)
    y64 = p.matvec(u, topo.TP_PREC_F64)[rows]
    ref = fem.matvec_rows(w, rho, u, rows)
    scale = fem.matvec_rows(w, rho, u, rows, absolute=True)
    assert np.all(np.abs(y64 - ref) <= 1e-12 * scale + 1e-300)
    u32 = u.astype(np.float32)
    y32 = p.matvec(u32, topo.TP_PREC_MIXED).astype(np.float64)[rows]
    ref32 = fem.matvec_rows(w, rho, u32.astype(np.float64), rows)
    assert np.all(np.abs(y32 - ref32) <= 2e-5 * scale + 1e-30)
    p.close()


def test_h8_large_solve_properties(topo):
    w = W.cantilever3d_large()
    p = topo.Problem.from_workload(w)
    info = p.solve(topo.solve_opts(tol=1e-6, max_it=400000, precision=topo.TP_PREC_MIXED, update_drop=0.1))
    assert info.converged == 1 and info.rel_res[0] <= 1e-6
    u = p.get(topo.TP_U)
    c = p.sensitivities()
    f = w.loads[0]
    assert c == pytest.approx(float(f @ u), rel=1e-12)
    Ku = p.matvec(u, topo.TP_PREC_F64)
    free = ~w.fixed.astype(bool)
    r = np.where(free, f - Ku, 0.0)
    rel = np.linalg.norm(r) / np.linalg.norm(f[free])
    assert rel == pytest.approx(info.rel_res[0], rel=1e-6, abs=1e-12)
    # c = u^T K u up to the residual: |f^T u - u^T K u| = |r^T u| <= ||r|| ||u||
    assert abs(float(u @ np.where(free, Ku, 0.0)) - c) <= np.linalg.norm(r) * np.linalg.norm(u) * 1.01
    rows = _rows(w.n_dof, 300, seed=5)
    ref = fem.matvec_rows(w, w.initial_density(), u, rows)
    scale = fem.matvec_rows(w, w.initial_density(), u, rows, absolute=True)
    assert np.all(np.abs(Ku[rows] - ref) <= 1e-12 * scale + 1e-300)
    p.close()


def test_batch_full_size_sampled_instances(topo, tmp_path):
    ws = W.batch2d()
    B = topo.Batch(ws)
    B.autotune(str(tmp_path / "tiles.json"))
    opts = topo.solve_opts(tol=1e-8, max_it=100000, precision=topo.TP_PREC_MIXED, update_drop=0.1)
    info, comp = B.step(opts)
    assert info.converged == 1 and info.max_rel_res <= 1e-8
    order = np.argsort([w.n_nodes for w in ws])
    for i in [int(order[0]), int(order[len(ws) // 2]), int(order[-1])]:
        w = ws[i]
        ref = simp.iteration(w, w.initial_density(), W=filt.weights_for(w))
        assert comp[i] == pytest.approx(ref["c"], rel=5e-7), i
        rho1, sc = B.get(i, topo.TP_RHO)
        assert np.max(np.abs(rho1 - ref["rho_new"])) <= 5e-6, i
    B.close()
