"""GPU parity of the SIMP loop on the paper's own P1 cells (tp_p1_*, through the
C-ABI) against the FP64 oracle (oracle/p1.py) on the same seeded inputs.

Tolerances (as for Q4 / H8):
  * operator (FP64):     |y - y_ref| <= 1e-12 (|K| |u|)_i
  * solve:               true relative residual <= tol, compliance rel <= 1e-8
  * sensitivities, filter: rel <= 1e-12 (FP64 both sides, same formula)
  * SIMP iteration on identical densities: compliance rel <= 1e-8, densities
    max-abs <= 1e-6, lambda rel <= 1e-9 of the exact root of the volume
    constraint; final compliance within 1e-3 after the full iteration count
The meshes are the paper's (Section 4 "Discretization the problem": the
"right/left" cut; Section 5 "Working with 3D problems": tetrahedra), with its
traction-strip load in 2D and the line load in 3D.
"""
import numpy as np
import pytest

import workloads as W
from oracle import filt, oc, p1

pytestmark = pytest.mark.gpu

F64 = dict(precision=0, precond=0)


@pytest.fixture(scope="module")
def topo():
    from paper_2012_08208_gb300 import topo as t
    return t


def _random_loads(w, nc, seed):
    """nc load cases: the workload's own load, then seeded random forces on the
    free DOFs of the x = nelx face."""
    rng = np.random.default_rng(seed)
    f = np.zeros((nc, w.n_dof))
    f[0] = w.loads[0]
    X = p1.node_coords(w.dim, w.nelx, w.nely, w.nelz)
    face = np.flatnonzero(X[:, 0] == w.nelx)
    for c in range(1, nc):
        for n in face:
            f[c, w.dim * n: w.dim * n + w.dim] = rng.normal(size=w.dim)
    f[:, w.fixed.astype(bool)] = 0.0
    return f


PROBS = [W.p1_cantilever2d(7, 3, diagonal="right"), W.p1_cantilever2d(9, 4, diagonal="left"),
         W.p1_cantilever2d(30, 11, diagonal="right/left"), W.p1_cantilever2d(1, 1, diagonal="right/left"),
         W.p1_cantilever3d(5, 3, 4), W.p1_cantilever3d(9, 4, 3), W.p1_cantilever3d(1, 1, 1)]


@pytest.mark.parametrize("w", PROBS, ids=lambda w: w.name)
def test_p1_apply_against_assembled_operator(topo, w):
    rho = W.random_density(w.n_el, seed=81)
    p = topo.P1Problem.from_workload(w)
    p.set_density(rho)
    u = W.random_vector(w.n_dof, seed=82)
    y = p.apply(u)
    K = p1.assemble(w, rho)
    fixed = w.fixed.astype(bool)
    um = np.where(fixed, 0.0, u)
    ref = np.where(fixed, u, K @ um)
    bound = np.where(fixed, np.abs(u), abs(K) @ np.abs(um))
    assert np.all(np.abs(y - ref) <= 1e-12 * bound + 1e-300)
    p.close()


@pytest.mark.parametrize("w", [W.p1_cantilever2d(30, 11), W.p1_cantilever3d(9, 4, 3)], ids=lambda w: w.name)
@pytest.mark.parametrize("nc", [1, 2])
def test_p1_solve_matches_direct_solve(topo, w, nc):
    w.loads = _random_loads(w, nc, seed=83)
    rho = W.random_density(w.n_el, seed=84, lo=0.01)
    p = topo.P1Problem.from_workload(w)
    p.set_density(rho)
    info = p.solve(topo.solve_opts(tol=1e-11, max_it=100000, **F64))
    assert info.converged == 1 and info.iters > 0
    U = p.get(topo.TP_U).reshape(nc, -1)
    K = p1.assemble(w, rho)
    free = ~w.fixed.astype(bool)
    for c in range(nc):
        rel = np.linalg.norm((w.loads[c] - K @ U[c])[free]) / np.linalg.norm(w.loads[c][free])
        assert rel <= 1.2e-11
        assert info.rel_res[c] == pytest.approx(rel, rel=0.05, abs=1e-13)
    U_ref = p1.solve(w, rho, K)
    c_ref = float(sum(w.loads[c] @ U_ref[c] for c in range(nc)))
    assert p.sensitivities() == pytest.approx(c_ref, rel=1e-8)
    assert np.all(U[:, ~free] == 0.0)
    p.close()


@pytest.mark.parametrize("w", [W.p1_cantilever2d(13, 6, diagonal="right/left"), W.p1_cantilever3d(6, 3, 4)],
                         ids=lambda w: w.name)
def test_p1_sensitivities_on_identical_displacements(topo, w):
    w.loads = _random_loads(w, 2, seed=85)
    rho = W.random_density(w.n_el, seed=86)
    U = np.stack([W.random_vector(w.n_dof, seed=87 + c) for c in range(2)])
    U[:, w.fixed.astype(bool)] = 0.0
    p = topo.P1Problem.from_workload(w)
    p.set_density(rho)
    p.set(topo.TP_U, U.ravel())
    c = p.sensitivities()
    c_ref, ce_ref, dc_ref = p1.sensitivities(w, rho, U)
    assert c == pytest.approx(c_ref, rel=1e-12)
    assert np.allclose(p.get(topo.TP_CE), ce_ref, rtol=1e-12, atol=1e-12 * np.abs(ce_ref).max())
    assert np.allclose(p.get(topo.TP_DC), dc_ref, rtol=1e-12, atol=1e-12 * np.abs(dc_ref).max())
    p.close()


@pytest.mark.parametrize("w", [W.p1_cantilever2d(17, 9, diagonal="right", rmin=1.5),
                               W.p1_cantilever2d(14, 8, diagonal="left", rmin=2.5),
                               W.p1_cantilever2d(21, 10, diagonal="right/left", rmin=3.0),
                               W.p1_cantilever2d(1, 1, diagonal="right/left", rmin=1.5),
                               W.p1_cantilever3d(7, 4, 3, rmin=1.5), W.p1_cantilever3d(6, 5, 4, rmin=2.0)],
                         ids=lambda w: f"{w.name}_r{w.rmin}")
def test_p1_filter(topo, w):
    rho = W.random_density(w.n_el, seed=88)
    dc = W.random_sensitivity(w.n_el, seed=89)
    p = topo.P1Problem.from_workload(w)
    p.set_density(rho)
    p.set(topo.TP_DC, dc)
    p.filter()
    ref = filt.sensitivity_filter(p1.sparse_weights(w), rho, dc)
    assert np.allclose(p.get(topo.TP_DCF), ref, rtol=1e-12, atol=0)
    # the dense paper-literal weights give the same rows
    if w.n_el <= 2000:
        assert np.allclose(filt.sensitivity_filter(p1.dense_weights(w), rho, dc), ref, rtol=1e-12, atol=0)
    p.close()


def test_p1_oc_update_with_passive_cells(topo):
    w = W.p1_cantilever2d(40, 12)
    rng = np.random.default_rng(90)
    rho = rng.uniform(0.001, 1.0, w.n_el)
    dcf = W.random_sensitivity(w.n_el, seed=91)
    pas = (rng.uniform(size=w.n_el) < 0.1).astype(np.int8)
    rho[pas == 1] = w.dmin
    w.passive = pas
    p = topo.P1Problem.from_workload(w)
    p.set_density(rho)
    p.set(topo.TP_DCF, dcf)
    lam, vol, ch = p.oc_update()
    lam_exact = oc.exact_lambda(rho, dcf, w.volfrac, passive=pas)
    assert lam == pytest.approx(lam_exact, rel=1e-9)
    rho_new = p.get(topo.TP_RHO)
    assert np.max(np.abs(rho_new - oc.update(rho, dcf, lam_exact, passive=pas))) <= 1e-6
    assert np.all(rho_new[pas == 1] == w.dmin)
    assert vol == pytest.approx(w.volfrac * w.n_el, rel=1e-8)
    p.close()


@pytest.mark.parametrize("w,n_it", [(W.p1_cantilever2d(60, 20, diagonal="right/left"), 8),
                                    (W.p1_cantilever3d(24, 8, 4), 4)], ids=lambda x: getattr(x, "name", str(x)))
def test_p1_simp_iterations_on_identical_density(topo, w, n_it):
    """Each GPU iteration against the oracle's iteration on the GPU's own
    density (compliance <= 1e-8, rho <= 1e-6, lambda <= 1e-9)."""
    C = p1.cells(w)
    Ke = p1.unit_stiffness(w, C)
    Wm = p1.weights_for(w, C)
    p = topo.P1Problem.from_workload(w)
    opts = topo.solve_opts(tol=1e-11, max_it=100000, warm_start=topo.TP_WARM_PREVIOUS, **F64)
    rho = w.initial_density()
    for it in range(n_it):
        info = p.simp_step(opts)
        ref = p1.iteration(w, rho, W=Wm, Ke=Ke, C=C)
        assert abs(info.compliance - ref["c"]) <= 1e-8 * ref["c"], it
        lam_exact = oc.exact_lambda(rho, ref["dcf"], w.volfrac)
        assert info.lambda_ == pytest.approx(lam_exact, rel=1e-9), it
        rho_gpu = p.get(topo.TP_RHO)
        assert np.max(np.abs(rho_gpu - ref["rho_new"])) <= 1e-6, it
        assert info.volume == pytest.approx(w.volfrac * w.n_el, rel=1e-9)
        rho = rho_gpu
    p.close()


def test_p1_cantilever2d_50_iterations_final_compliance(topo):
    """The paper's 2D cantilever on its "right/left" mesh: 50 GPU iterations
    from the uniform start against 50 oracle iterations (final compliance
    within 1e-3; the first iteration within 1e-8)."""
    w = W.p1_cantilever2d(60, 20, diagonal="right/left")
    C = p1.cells(w)
    Ke = p1.unit_stiffness(w, C)
    Wm = p1.weights_for(w, C)
    rho = w.initial_density()
    cs_ref = []
    for it in range(50):
        ref = p1.iteration(w, rho, W=Wm, Ke=Ke, C=C)
        cs_ref.append(ref["c"])
        rho = ref["rho_new"]
    p = topo.P1Problem.from_workload(w)
    opts = topo.solve_opts(tol=1e-11, max_it=100000, warm_start=topo.TP_WARM_PREVIOUS, **F64)
    cs = [p.simp_step(opts).compliance for _ in range(50)]
    assert abs(cs[0] - cs_ref[0]) <= 1e-8 * cs_ref[0]
    assert abs(cs[-1] - cs_ref[-1]) <= 1e-3 * cs_ref[-1]
    p.close()


def test_p1_errors_keep_handle_usable(topo):
    w = W.p1_cantilever2d(6, 3)
    prm = topo.tp_p1_params(2, 6, 3, 0, 2, w.lam, w.mu, w.Emin, w.penal, w.volfrac, w.rmin, w.move, w.dmin, 1)
    p = topo.P1Problem(prm)
    with pytest.raises(topo.TopoError) as e:
        p.solve(topo.solve_opts(**F64))
    assert e.value.status == topo.TP_ERR_STATE
    with pytest.raises(topo.TopoError) as e:
        p.set_fixed(np.zeros(w.n_dof, np.uint8))
    assert e.value.status == topo.TP_ERR_ARG
    p.set_fixed(w.fixed)
    p.set_loads(w.loads)
    with pytest.raises(topo.TopoError):
        p.set_density(np.full(w.n_el, 1.5))
    p.set_density(w.initial_density())
    with pytest.raises(topo.TopoError) as e:
        p.solve(topo.solve_opts(precision=topo.TP_PREC_MIXED))
    assert e.value.status == topo.TP_ERR_ARG
    info = p.solve(topo.solve_opts(tol=1e-14, max_it=2, **F64), check=False)
    assert info.status == topo.TP_ERR_NOT_CONVERGED
    info = p.solve(topo.solve_opts(tol=1e-10, max_it=10000, **F64))
    assert info.converged == 1
    with pytest.raises(topo.TopoError) as e:
        p.oc_update()
    assert e.value.status == topo.TP_ERR_STATE
    p.close()
