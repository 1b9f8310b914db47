"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances (written per test):
  * FP64 operator:   |y - y_ref| <= 1e-12 * (|K| |u|)_i          (rounding order only)
  * FP32 operator:   |y - y_ref| <= 2e-5 * (|K| |u|)_i           (FP32 K0, E and sums)
  * double-word op.: |y - y_ref| <= 1e-12 * (|K| |u|)_i          (48-bit FP32 pairs, 3u^2 per addition)
  * solve / loop:    compliance rel <= 1e-8, densities max-abs <= 1e-6, lambda rel <= 1e-9
  * filter / sens:   rel <= 1e-12 (FP64 both sides, same formula; 3D element energies in double-word FP32)
"""
import numpy as np
import pytest

import workloads as W
from oracle import helm, fem, filt, oc, sens, simp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def topo():
    from paper_2012_08208_gb300 import topo as t
    return t


def _abs_product(prob, rho, u):
    K = fem.assemble(prob, rho)
    Ka = abs(K)
    fixed = prob.fixed.astype(bool)
    y = Ka @ np.abs(np.where(fixed, 0, u))
    return np.where(fixed, np.abs(u), y)


GRIDS = [
    W.small2d(1, 1), W.small2d(2, 1), W.small2d(70, 20), W.small2d(33, 9, n_cases=2),
    W.small3d(1, 1, 1), W.small3d(3, 2, 2), W.small3d(40, 9, 6), W.small3d(33, 5, 5, n_cases=2),
]


@pytest.mark.parametrize("prob", GRIDS, ids=lambda p: p.name + f"_nc{p.n_cases}")
def test_matvec_f64_and_f32(topo, prob):
    rho = W.random_density(prob.n_el, seed=31)
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    for k in range(2):
        u = W.random_vector(prob.n_dof, seed=32 + k)
        y_ref = fem.matvec_bc(prob, rho, u)
        bound = _abs_product(prob, rho, u)
        y64 = p.matvec(u, topo.TP_PREC_F64)
        assert np.all(np.abs(y64 - y_ref) <= 1e-12 * bound + 1e-300)
        u32 = u.astype(np.float32)
        y32 = p.matvec(u32, topo.TP_PREC_MIXED).astype(np.float64)
        y_ref32 = fem.matvec_bc(prob, rho, u32.astype(np.float64))
        assert np.all(np.abs(y32 - y_ref32) <= 2e-5 * bound + 1e-30)
    # several vectors in one call
    U = np.stack([W.random_vector(prob.n_dof, seed=40 + k) for k in range(3)])
    Y = p.matvec(U.ravel(), topo.TP_PREC_F64, ncopies=3).reshape(3, -1)
    for k in range(3):
        assert np.allclose(Y[k], fem.matvec_bc(prob, rho, U[k]), rtol=1e-12, atol=1e-12 * np.abs(Y[k]).max())
    p.close()


@pytest.mark.parametrize("prob", GRIDS, ids=lambda p: p.name + f"_nc{p.n_cases}")
def test_matvec_double_word(topo, prob):
    """The double-word FP32 operator (the multigrid solver's true residual at
    tolerances >= 1e-8 in 3D) against the FP64 oracle, on a density field with
    the void modulus (Emin = 1e-9) in a third of the elements and on smooth
    displacements (the case where the element strains cancel most)."""
    rng = np.random.default_rng(57)
    rho = np.where(rng.random(prob.n_el) < 0.33, 1e-3, W.random_density(prob.n_el, seed=58))
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    xs = np.linspace(0.0, 1.0, prob.n_dof)
    for u in (W.random_vector(prob.n_dof, seed=59), 1.0 + 1e-3 * np.sin(7.0 * xs)):
        u = np.where(prob.fixed.astype(bool), 0.0, u)
        y_ref = fem.matvec_bc(prob, rho, u)
        bound = _abs_product(prob, rho, u)
        ydw = p.matvec(u, topo.TP_PREC_DW)
        assert np.all(np.abs(ydw - y_ref) <= 1e-12 * bound + 1e-300), np.max(np.abs(ydw - y_ref) / (bound + 1e-300))
    p.close()


@pytest.mark.parametrize("prob", [W.small2d(37, 11, n_cases=3, passive_disk=(10, 5, 3)),
                                  W.small3d(17, 6, 5)], ids=lambda p: p.name)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_solve_matches_direct_solve(topo, prob, prec):
    rho = W.random_density(prob.n_el, seed=33, lo=0.01)
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    pr = topo.TP_PREC_F64 if prec == "f64" else topo.TP_PREC_MIXED
    info = p.solve(topo.solve_opts(tol=1e-11, max_it=100000, precision=pr))
    assert info.converged == 1
    U = p.get(topo.TP_U).reshape(prob.n_cases, -1)
    U_ref = fem.solve(prob, rho)
    res = fem.rel_residual(prob, rho, U)
    assert np.all(res <= 1.2e-11)
    # the reported residual is the FP64 true residual (differs from the oracle's
    # evaluation of it only by rounding order, ~1e-13 at this level)
    for c in range(prob.n_cases):
        assert info.rel_res[c] == pytest.approx(res[c], rel=0.05, abs=1e-13)
    c_gpu = p.sensitivities()
    c_ref = sens.compliance(prob, U_ref)
    assert abs(c_gpu - c_ref) <= 1e-8 * abs(c_ref)
    p.close()


@pytest.mark.parametrize("prob", [W.small2d(45, 13, n_cases=2), W.small3d(19, 7, 6)], ids=lambda p: p.name)
def test_sensitivities_on_identical_displacements(topo, prob):
    rho = W.random_density(prob.n_el, seed=34)
    U = np.stack([W.random_vector(prob.n_dof, seed=35 + c) for c in range(prob.n_cases)])
    U[:, prob.fixed.astype(bool)] = 0.0
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    p.set(topo.TP_U, U.ravel())
    c_gpu = p.sensitivities()
    c_ref, ce_ref, dc_ref = sens.sensitivities(prob, rho, U)
    assert c_gpu == pytest.approx(c_ref, rel=1e-12)
    assert np.allclose(p.get(topo.TP_CE), ce_ref, rtol=1e-12, atol=1e-12 * np.abs(ce_ref).max())
    assert np.allclose(p.get(topo.TP_DC), dc_ref, rtol=1e-12, atol=1e-12 * np.abs(dc_ref).max())
    p.close()


@pytest.mark.parametrize("prob", [W.small2d(70, 21, rmin=1.5), W.small2d(40, 17, rmin=3.0),
                                  W.small3d(35, 9, 7, rmin=1.5), W.small3d(33, 10, 6, rmin=2.0),
                                  W.small2d(1, 1, rmin=3.0), W.small3d(1, 2, 1, rmin=2.0)],
                         ids=lambda p: f"{p.name}_r{p.rmin}")
def test_filter(topo, prob):
    rho = W.random_density(prob.n_el, seed=36)
    dc = W.random_sensitivity(prob.n_el, seed=37)
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    p.set(topo.TP_DC, dc)
    p.filter()
    got = p.get(topo.TP_DCF)
    ref = filt.sensitivity_filter(filt.sparse_weights(prob), rho, dc)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    p.close()


@pytest.mark.parametrize("n,vf,passive", [(1200, 0.5, False), (4000, 0.3, True), (7, 0.6, False)])
def test_oc_update(topo, n, vf, passive):
    prob = W.small2d(n, 1, volfrac=vf)
    rng = np.random.default_rng(n)
    rho = rng.uniform(0.001, 1.0, n)
    dcf = W.random_sensitivity(n, seed=38)
    pas = None
    if passive:
        pas = (rng.uniform(size=n) < 0.1).astype(np.int8)
        rho[pas == 1] = 0.001
        prob.passive = pas
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    p.set(topo.TP_DCF, dcf)
    lam, vol, ch = p.oc_update()
    rho_new = p.get(topo.TP_RHO)
    lam_exact = oc.exact_lambda(rho, dcf, vf, passive=pas)
    assert lam == pytest.approx(lam_exact, rel=1e-9)
    ref = oc.update(rho, dcf, lam_exact, passive=pas)
    assert np.max(np.abs(rho_new - ref)) <= 1e-6
    assert vol == pytest.approx(vf * n, rel=1e-8)
    assert ch == pytest.approx(np.max(np.abs(rho_new - rho)), rel=1e-12)
    if passive:
        assert np.all(rho_new[pas == 1] == 0.001)
    p.close()


P1_CASES = [("right", (7, 5, 0), 1), ("left", (1, 1, 0), 1), ("right/left", (9, 6, 0), 2),
            ("kuhn", (1, 1, 1), 1), ("kuhn", (3, 2, 2), 1), ("kuhn", (5, 3, 4), 2)]


@pytest.mark.parametrize("diagonal,size,nc", P1_CASES, ids=lambda v: str(v).replace("/", ""))
def test_p1_matvec_against_oracle(topo, diagonal, size, nc):
    """The paper's P1 operator (tp_p1_matvec, FP64) against the oracle's
    assembled K(rho) on random densities and vectors, fixed rows y = u:
    |y - y_ref| <= 1e-12 (|K| |u|)_i (rounding order only)."""
    import torch
    nx, ny, nz = size
    prob = (W.p1_cantilever2d(nx, ny, diagonal=diagonal) if nz == 0 else W.p1_cantilever3d(nx, ny, nz))
    rho = W.random_density(prob.n_el, seed=21)
    U = np.stack([W.random_vector(prob.n_dof, seed=22 + c) for c in range(nc)])
    from oracle import p1
    K = p1.assemble(prob, rho)
    fixed = prob.fixed.astype(bool)
    dev = torch.device("cuda")
    y = torch.zeros((nc, prob.n_dof), dtype=torch.float64, device=dev)
    topo.p1_matvec(prob.dim, nx, ny, nz, diagonal, prob.lam, prob.mu, prob.Emin, prob.penal,
                   torch.tensor(rho, device=dev), torch.tensor(prob.fixed, device=dev),
                   torch.tensor(U, device=dev), y)
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    Ka = abs(K)
    for c in range(nc):
        um = np.where(fixed, 0.0, U[c])
        ref = np.where(fixed, U[c], K @ um)
        scale = np.where(fixed, np.abs(U[c]), Ka @ np.abs(um))
        assert np.all(np.abs(y[c] - ref) <= 1e-12 * scale + 1e-300), np.abs(y[c] - ref).max()


def test_p1_matvec_errors(topo):
    """Bad dimension, diagonal or material give TP_ERR_ARG before any launch."""
    import ctypes
    buf = np.zeros(64)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    f = topo.lib.tp_p1_matvec
    assert f(2, 2, 2, 0, 3, 0.6, 0.4, 1e-9, 3.0, ptr, ptr, ptr, ptr, 1, None) == topo.TP_ERR_ARG
    assert f(3, 2, 2, 2, 1, 0.6, 0.4, 1e-9, 3.0, ptr, ptr, ptr, ptr, 1, None) == topo.TP_ERR_ARG
    assert f(2, 2, 2, 0, 0, 0.6, -0.4, 1e-9, 3.0, ptr, ptr, ptr, ptr, 1, None) == topo.TP_ERR_ARG
    assert f(4, 2, 2, 0, 0, 0.6, 0.4, 1e-9, 3.0, ptr, ptr, ptr, ptr, 1, None) == topo.TP_ERR_ARG
    assert f(2, 2, 2, 0, 0, 0.6, 0.4, 1e-9, 3.0, ptr, ptr, ptr, ptr, 9, None) == topo.TP_ERR_ARG


@pytest.mark.parametrize("n", [1, 5, 64, 130, 300, 1000, 3952])
def test_spd_inverse_against_fp64(topo, n):
    """Dense FP32 inverse (the multigrid coarsest solve) against the FP64
    inverse of the same float32 matrix.  Sizes span one pivot block, ragged
    pivot blocks and trailing tiles, the scalar path (n = 130, 5: not a
    multiple of 4) and the coarsest size of the 600 x 200 cantilever (3952).
    Condition number 100: the FP32 sweep keeps |X - A^-1| / max|A^-1| within
    kappa * u * O(10) ~ 1e-4; the bound written is 1e-3.  The result is
    mirrored from one triangle, so it is exactly symmetric."""
    a = W.random_spd(n, cond=100.0, seed=n)
    x = topo.spd_inverse(a)
    ref = np.linalg.inv(a.astype(np.float64))
    err = np.abs(x - ref).max() / np.abs(ref).max()
    assert err <= 1e-3, err
    assert np.array_equal(x, x.T)


def test_spd_inverse_diagonal_exact(topo):
    """A diagonal matrix: every off-diagonal product is an exact zero, so the
    sweep returns the correctly rounded reciprocals bit for bit."""
    d = np.random.default_rng(3).uniform(0.5, 2.0, size=300).astype(np.float32)
    x = topo.spd_inverse(np.diag(d))
    assert np.array_equal(x, np.diag(np.float32(1.0) / d))


def test_spd_inverse_errors(topo):
    """A negative pivot (indefinite matrix) gives TP_ERR_BREAKDOWN; n out of
    range gives TP_ERR_ARG before any device work."""
    d = np.ones(200, dtype=np.float32)
    d[70] = -1.0
    with pytest.raises(topo.TopoError) as ei:
        topo.spd_inverse(np.diag(d))
    assert ei.value.status == topo.TP_ERR_BREAKDOWN
    import ctypes
    buf = np.zeros(4, dtype=np.float32)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    assert topo.lib.tp_spd_inverse_f32(ptr, ptr, 0, None) == topo.TP_ERR_ARG
    assert topo.lib.tp_spd_inverse_f32(ptr, ptr, topo.SPD_INVERSE_MAX_N + 1, None) == topo.TP_ERR_ARG
    assert topo.lib.tp_spd_inverse_f32(None, ptr, 2, None) == topo.TP_ERR_ARG


@pytest.mark.parametrize("n_special", [1, 100])
def test_oc_update_breakpoint_at_root(topo, n_special):
    """Clamp breakpoints exactly at the root (lambda* = 1): the FP64
    classification finds elements changing state inside the FP32 bracket.  One
    such element: the piecewise exact root decides; 100: more than the list
    holds, so FP64 bisection passes decide.  Lambda within 1e-9 of the exact
    root either way."""
    n = 4000
    rng = np.random.default_rng(77)
    rho = rng.uniform(0.3, 0.6, n)
    dcf = -np.ones(n)
    ks = rng.choice(n, size=n_special, replace=False)
    rho[ks] = 0.5
    dcf[ks] = -1.96  # B = 0.5 * 1.4 = rho + move: clamped high from lambda = 1 down
    vf = (rho.sum() + 0.2 * n_special) / n  # V(1) = sum rho + 0.2 per special element
    prob = W.small2d(n, 1, volfrac=vf)
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    p.set(topo.TP_DCF, dcf)
    lam, vol, ch = p.oc_update()
    lam_exact = oc.exact_lambda(rho, dcf, vf)
    assert lam_exact == pytest.approx(1.0, rel=1e-12)
    assert lam == pytest.approx(lam_exact, rel=1e-9)
    assert np.max(np.abs(p.get(topo.TP_RHO) - oc.update(rho, dcf, lam_exact))) <= 1e-6
    assert vol == pytest.approx(vf * n, rel=1e-8)
    p.close()


def test_simp_iterations_on_identical_density_mbb(topo):
    """Config 1 (MBB 60 x 20, FP64): every iteration compared with the oracle on the
    GPU's own density (compliance <= 1e-8, rho <= 1e-6, lambda <= 1e-9)."""
    prob = W.mbb2d()
    Wm = filt.weights_for(prob)
    p = topo.Problem.from_workload(prob)
    rho = prob.initial_density()
    opts = topo.solve_opts(tol=1e-10, max_it=50000, precision=topo.TP_PREC_F64, warm_start=topo.TP_WARM_PREVIOUS)
    for it in range(8):
        info = p.simp_step(opts)
        ref = simp.iteration(prob, rho, W=Wm)
        assert abs(info.compliance - ref["c"]) <= 1e-8 * ref["c"]
        rho_gpu = p.get(topo.TP_RHO)
        lam_exact = oc.exact_lambda(rho, ref["dcf"], prob.volfrac)
        assert info.lambda_ == pytest.approx(lam_exact, rel=1e-9)
        assert np.max(np.abs(rho_gpu - ref["rho_new"])) <= 1e-6
        rho = rho_gpu
    p.close()


def test_mbb_50_iterations_final_compliance(topo):
    prob = W.mbb2d()
    rho_ref, hist = simp.run(prob, n_iter=50)
    p = topo.Problem.from_workload(prob)
    opts = topo.solve_opts(tol=1e-10, max_it=50000, precision=topo.TP_PREC_F64, warm_start=topo.TP_WARM_PREVIOUS)
    cs = []
    for it in range(50):
        cs.append(p.simp_step(opts).compliance)
    assert abs(cs[-1] - hist[-1]["c"]) <= 1e-3 * hist[-1]["c"]
    assert abs(cs[0] - hist[0]["c"]) <= 1e-8 * hist[0]["c"]
    p.close()


def test_error_paths_keep_handle_usable(topo):
    prob = W.small2d(10, 5)
    p = topo.Problem(topo.make_params(2, 10, 5, volfrac=0.5))
    with pytest.raises(topo.TopoError) as e:
        p.solve(topo.solve_opts())
    assert e.value.status == topo.TP_ERR_STATE
    with pytest.raises(topo.TopoError) as e:
        p.set_fixed(np.zeros(prob.n_dof, np.uint8))
    assert e.value.status == topo.TP_ERR_ARG
    p.set_fixed(prob.fixed)
    bad = prob.loads.copy()
    bad[0, 5] = np.nan
    with pytest.raises(topo.TopoError) as e:
        p.set_loads(bad)
    assert e.value.status == topo.TP_ERR_ARG
    p.set_loads(prob.loads)
    with pytest.raises(topo.TopoError):
        p.set_density(np.full(prob.n_el, 1.5))
    p.set_density(np.full(prob.n_el, 0.5))
    info = p.solve(topo.solve_opts(tol=1e-14, max_it=3, precision=topo.TP_PREC_F64), check=False)
    assert info.status == topo.TP_ERR_NOT_CONVERGED and info.iters == 3
    info = p.solve(topo.solve_opts(tol=1e-10, max_it=10000, precision=topo.TP_PREC_F64))
    assert info.converged == 1
    p.close()


@pytest.mark.parametrize("prob", [W.mbb2d(), W.small3d(12, 6, 5, rmin=1.8, volfrac=0.3)], ids=lambda p: p.name)
def test_density_filter_mode_iterations(topo, prob):
    """Density-filter variant (the physical densities are W rho / rowsum, the
    sensitivities go back through the chain rule): every iteration against the
    oracle's filter_mode=1 iteration on the GPU's own design densities."""
    Wm = filt.weights_for(prob)
    p = topo.Problem.from_workload(prob)
    p.set_filter_mode(topo.TP_FILTER_DENSITY)
    rho = prob.initial_density()
    opts = topo.solve_opts(tol=1e-11, max_it=50000, precision=topo.TP_PREC_F64, warm_start=topo.TP_WARM_PREVIOUS)
    for it in range(4):
        phys = p.get(topo.TP_RHO_PHYS)
        assert np.allclose(phys, filt.density_filter(Wm, rho), rtol=1e-13, atol=0)
        info = p.simp_step(opts)
        ref = simp.iteration(prob, rho, W=Wm, filter_mode=1)
        assert abs(info.compliance - ref["c"]) <= 1e-8 * ref["c"]
        rho_gpu = p.get(topo.TP_RHO)
        lam_exact = oc.exact_lambda(rho, ref["dcf"], prob.volfrac)
        assert info.lambda_ == pytest.approx(lam_exact, rel=1e-8)
        assert np.max(np.abs(rho_gpu - ref["rho_new"])) <= 1e-6
        rho = rho_gpu
    # the mode is checked: a sensitivity-filter call on a density-filter problem is refused
    p.solve(opts)
    p.sensitivities()
    with pytest.raises(topo.TopoError):
        p.filter(topo.TP_FILTER_SENSITIVITY)
    p.close()


HELM_GRIDS = [W.small2d(37, 11, n_cases=2, rmin=2.5), W.small3d(13, 7, 5, rmin=1.8), W.small2d(1, 1, rmin=1.5)]


@pytest.mark.parametrize("prob", HELM_GRIDS, ids=lambda p: p.name)
def test_helmholtz_filter_matches_oracle(topo, prob):
    """Helmholtz (PDE) filter mode: the filtered densities and the chain rule
    dc~ = H dc against the oracle's sparse LU on the same inputs (FP64 PCG to
    relative residual 1e-14 on the GPU)."""
    rho = W.random_density(prob.n_el, seed=61, lo=0.01)
    p = topo.Problem.from_workload(prob)
    p.set_filter_mode(topo.TP_FILTER_HELMHOLTZ)
    p.set_density(rho)
    phys = p.get(topo.TP_RHO_PHYS)
    AT = helm.operator(prob)
    assert np.allclose(phys, helm.apply(prob, rho, AT=AT), rtol=1e-11, atol=1e-13)
    p.solve(topo.solve_opts(tol=1e-10, max_it=50000, precision=topo.TP_PREC_F64))
    p.sensitivities()
    p.filter(topo.TP_FILTER_HELMHOLTZ)
    dc = p.get(topo.TP_DC)
    ref = helm.apply(prob, dc, AT=AT)
    assert np.allclose(p.get(topo.TP_DCF), ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))
    p.close()


@pytest.mark.parametrize("prob", [W.mbb2d(), W.small3d(12, 6, 5, rmin=1.8, volfrac=0.3)], ids=lambda p: p.name)
def test_helmholtz_filter_mode_iterations(topo, prob):
    """SIMP iterations with the Helmholtz filter, each against the oracle's
    filter_mode=2 iteration on the GPU's own design densities."""
    p = topo.Problem.from_workload(prob)
    p.set_filter_mode(topo.TP_FILTER_HELMHOLTZ)
    rho = prob.initial_density()
    opts = topo.solve_opts(tol=1e-11, max_it=50000, precision=topo.TP_PREC_F64, warm_start=topo.TP_WARM_PREVIOUS)
    for it in range(4):
        info = p.simp_step(opts)
        ref = simp.iteration(prob, rho, filter_mode=2)
        assert abs(info.compliance - ref["c"]) <= 1e-8 * ref["c"]
        rho_gpu = p.get(topo.TP_RHO)
        lam_exact = oc.exact_lambda(rho, ref["dcf"], prob.volfrac)
        assert info.lambda_ == pytest.approx(lam_exact, rel=1e-8)
        assert np.max(np.abs(rho_gpu - ref["rho_new"])) <= 1e-6
        rho = rho_gpu
    p.close()


def test_helmholtz_filter_identities_full_size(topo):
    """At the 600 x 200 size of the SIMP bench: a constant density is a fixed
    point of the filter, and the filter conserves the total volume (both exact
    for the discrete operator).  With rmin = 3 (R^2 = 3/4 > 1/3) every
    off-diagonal entry of the 2D operator is negative, so it is an M-matrix and
    the filtered values stay within the range of the input."""
    prob = W.cantilever2d()
    p = topo.Problem.from_workload(prob)
    p.set_filter_mode(topo.TP_FILTER_HELMHOLTZ)
    p.set_density(np.full(prob.n_el, 0.4))
    assert np.allclose(p.get(topo.TP_RHO_PHYS), 0.4, rtol=0, atol=1e-13)
    rho = W.random_density(prob.n_el, seed=62, lo=0.001)
    p.set_density(rho)
    phys = p.get(topo.TP_RHO_PHYS)
    assert phys.sum() == pytest.approx(rho.sum(), rel=1e-12)
    assert phys.min() >= rho.min() - 1e-12 and phys.max() <= rho.max() + 1e-12
    p.close()


MG_GRIDS = [W.small2d(40, 12, n_cases=3, passive_disk=(12, 6, 3)), W.small2d(60, 20), W.small3d(16, 8, 6),
            W.small3d(20, 10, 10, n_cases=2)]


MG_KINDS = ["graph", "fused"]


def _mg(topo, kind):
    return topo.TP_PRECOND_MG if kind == "graph" else topo.TP_PRECOND_MG_FUSED


@pytest.mark.parametrize("kind", MG_KINDS)
@pytest.mark.parametrize("prob", MG_GRIDS, ids=lambda p: p.name + f"_nc{p.n_cases}")
def test_multigrid_solve_matches_direct_solve(topo, prob, kind):
    """Multigrid-preconditioned CG (FP32 correction segments with FP64
    restarts, FP32 V-cycle), graph-replayed and as a persistent kernel, against
    the oracle's LU solve on a random density: true residual <= tol,
    compliance rel <= 1e-8, displacements rel <= 1e-6."""
    rho = W.random_density(prob.n_el, seed=51, lo=0.05)
    p = topo.Problem.from_workload(prob)
    p.set_density(rho)
    info = p.solve(topo.solve_opts(tol=1e-11, max_it=5000, precond=_mg(topo, kind)))
    assert info.converged == 1 and max(info.rel_res[c] for c in range(prob.n_cases)) <= 1e-11
    assert info.iters < 200
    U = fem.solve(prob, rho)
    u = p.get(topo.TP_U).reshape(prob.n_cases, -1)
    for c in range(prob.n_cases):
        assert float(prob.loads[c] @ u[c]) == pytest.approx(float(prob.loads[c] @ U[c]), rel=1e-8)
        assert np.linalg.norm(u[c] - U[c]) <= 1e-6 * np.linalg.norm(U[c])
    p.close()


@pytest.mark.parametrize("kind", MG_KINDS)
def test_multigrid_simp_iterations_mbb(topo, kind):
    """Config 1 SIMP iterations with the multigrid solver, each against the
    oracle on the GPU's own density (compliance <= 1e-8, rho <= 1e-6, lambda
    <= 1e-9 of the exact root)."""
    prob = W.mbb2d()
    Wm = filt.weights_for(prob)
    p = topo.Problem.from_workload(prob)
    rho = prob.initial_density()
    opts = topo.solve_opts(tol=1e-10, max_it=5000, warm_start=topo.TP_WARM_PREVIOUS, precond=_mg(topo, kind))
    for it in range(8):
        info = p.simp_step(opts)
        assert info.solve.iters < 100
        ref = simp.iteration(prob, rho, W=Wm)
        assert abs(info.compliance - ref["c"]) <= 1e-8 * ref["c"]
        rho_gpu = p.get(topo.TP_RHO)
        assert info.lambda_ == pytest.approx(oc.exact_lambda(rho, ref["dcf"], prob.volfrac), rel=1e-9)
        assert np.max(np.abs(rho_gpu - ref["rho_new"])) <= 1e-6
        rho = rho_gpu
    p.close()


def test_multigrid_needs_a_hierarchy(topo):
    prob = W.small2d(37, 11)  # prime element counts: no coarse grid
    p = topo.Problem.from_workload(prob)
    for kind in MG_KINDS:
        with pytest.raises(topo.TopoError) as e:
            p.solve(topo.solve_opts(tol=1e-8, precond=_mg(topo, kind)))
        assert e.value.status == topo.TP_ERR_ARG
    info = p.solve(topo.solve_opts(tol=1e-8, max_it=20000))  # the handle stays usable
    assert info.converged == 1
    with pytest.raises(topo.TopoError) as e:
        p.solve(topo.solve_opts(tol=1e-8, precond=7))
    assert e.value.status == topo.TP_ERR_ARG
    p.close()


@pytest.mark.parametrize("prob", [W.small2d(40, 12, n_cases=3, passive_disk=(12, 6, 3)), W.small3d(16, 8, 6)],
                         ids=lambda p: p.name)
def test_multigrid_variants_agree(topo, prob):
    """The graph-replayed and the persistent-kernel solvers run the same
    method; their reductions differ in rounding order only: iteration counts
    within 10 %, solutions within 1e-6."""
    rho = W.random_density(prob.n_el, seed=52, lo=0.05)
    out = {}
    for kind in MG_KINDS:
        p = topo.Problem.from_workload(prob)
        p.set_density(rho)
        info = p.solve(topo.solve_opts(tol=1e-10, max_it=5000, precond=_mg(topo, kind)))
        out[kind] = (info.iters, info.updates, p.get(topo.TP_U))
        p.close()
    assert abs(out["graph"][0] - out["fused"][0]) <= max(2, 0.1 * out["graph"][0])
    ug, uf = out["graph"][2], out["fused"][2]
    assert np.linalg.norm(ug - uf) <= 1e-6 * np.linalg.norm(ug)
