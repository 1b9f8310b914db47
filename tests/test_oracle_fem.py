"""Pins for the oracle's operator and solve (discrete system of Section 3.1,
Eq. "fe_form"; modified SIMP stiffness; direct solve as in Section 4.3)."""
import numpy as np
import pytest

import workloads as W
from oracle import element, fem, mesh, sens


def _rigid(prob):
    X = mesh.node_coords(prob.dim, prob.nelx, prob.nely, prob.nelz)
    dim = prob.dim
    modes = []
    for d in range(dim):
        v = np.zeros_like(X)
        v[:, d] = 1
        modes.append(v.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        v = np.zeros_like(X)
        v[:, a] = -X[:, b]
        v[:, b] = X[:, a]
        modes.append(v.ravel())
    return modes


CASES = [W.small2d(5, 3), W.small2d(7, 4, n_cases=2), W.small3d(3, 2, 2), W.small3d(4, 3, 2)]


@pytest.mark.parametrize("prob", CASES, ids=lambda p: p.name)
def test_three_statements_of_the_product_agree(prob):
    rho = W.random_density(prob.n_el, seed=11)
    u = W.random_vector(prob.n_dof, seed=12)
    K = fem.assemble(prob, rho)
    y1 = fem.matvec_bc(prob, rho, u, K)
    fixed = prob.fixed.astype(bool)
    y2 = fem.matvec_elementwise(prob, rho, np.where(fixed, 0, u))
    y2 = np.where(fixed, u, y2)
    dofs = np.arange(prob.n_dof)
    y3 = fem.matvec_rows(prob, rho, u, dofs)
    assert np.allclose(y1, y2, rtol=1e-13, atol=1e-13)
    assert np.allclose(y1, y3, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prob", CASES, ids=lambda p: p.name)
def test_unconstrained_rigid_modes_and_symmetry(prob):
    rho = W.random_density(prob.n_el, seed=13)
    K = fem.assemble(prob, rho)
    for m in _rigid(prob):
        assert np.abs(K @ m).max() < 1e-12 * max(1.0, np.abs(m).max())
    v = W.random_vector(prob.n_dof, 14)
    w = W.random_vector(prob.n_dof, 15)
    assert v @ (K @ w) == pytest.approx(w @ (K @ v), rel=1e-12)


def test_uniform_density_scaling_is_exact():
    prob = W.small2d(6, 3)
    u1 = fem.solve(prob, np.ones(prob.n_el))
    c = 0.37
    uc = fem.solve(prob, np.full(prob.n_el, c))
    Ec = prob.Emin + c ** 3 * (prob.E0 - prob.Emin)
    assert np.allclose(uc, u1 / Ec, rtol=1e-10, atol=0)


def _bar(dim, nx, ny, nz, sigma):
    fixed, f = W._empty(dim, nx, ny, nz, 1)
    nn = (nx + 1) * (ny + 1) * ((nz + 1) if dim == 3 else 1)
    X = mesh.node_coords(dim, nx, ny, nz)
    for n in range(nn):
        x = X[n]
        if x[0] == 0:
            fixed[dim * n] = 1
            if x[1] == 0:
                fixed[dim * n + 1] = 1
            if dim == 3 and x[2] == 0:
                fixed[dim * n + 2] = 1
        if x[0] == nx:
            share = 1.0
            if x[1] in (0, ny):
                share *= 0.5
            if dim == 3 and x[2] in (0, nz):
                share *= 0.5
            f[0, dim * n] = sigma * share
    return W.Problem("bar", dim, nx, ny, nz, 0.5, 1.5, fixed, f), X


@pytest.mark.parametrize("dim,shape", [(2, (6, 3, 0)), (3, (4, 2, 3))])
def test_uniaxial_bar_closed_form(dim, shape):
    """Rollers on x = 0 and a uniform traction sigma on x = nx: the exact field
    u_x = sigma x / E, u_y = -nu sigma y / E (and u_z = -nu sigma z / E in 3D) is
    reproduced by bilinear/trilinear elements (plane stress in 2D)."""
    sigma = 0.8
    prob, X = _bar(dim, *shape, sigma)
    rho = np.ones(prob.n_el)
    u = fem.solve(prob, rho)[0].reshape(-1, dim)
    E, nu = prob.E0, prob.nu
    assert np.allclose(u[:, 0], sigma * X[:, 0] / E, atol=1e-12)
    assert np.allclose(u[:, 1], -nu * sigma * X[:, 1] / E, atol=1e-12)
    if dim == 3:
        assert np.allclose(u[:, 2], -nu * sigma * X[:, 2] / E, atol=1e-12)


@pytest.mark.parametrize("prob", CASES, ids=lambda p: p.name)
def test_compliance_equals_energy_and_residual(prob):
    rho = W.random_density(prob.n_el, seed=16)
    K = fem.assemble(prob, rho)
    U = fem.solve(prob, rho, K=K)
    assert np.all(fem.rel_residual(prob, rho, U, K) < 1e-10)
    c, ce, dc = sens.sensitivities(prob, rho, U)
    E = fem.young(rho, prob.E0, prob.Emin, prob.penal)
    uKu = sum(U[k] @ (K @ U[k]) for k in range(prob.n_cases))
    assert c == pytest.approx(uKu, rel=1e-10)
    assert c == pytest.approx(float(E @ ce), rel=1e-10)


def test_lu_and_cg_agree():
    prob = W.small3d(4, 3, 2)
    rho = W.random_density(prob.n_el, seed=17, lo=0.2)
    U1 = fem.solve(prob, rho, method="lu")
    U2 = fem.solve(prob, rho, method="cg", rtol=1e-14)
    assert np.allclose(U1, U2, rtol=1e-8, atol=1e-10 * np.abs(U1).max())


def test_matvec_rows_at_config_scale_sample():
    """The row-by-row evaluator (used for sampled checks at full size) agrees
    with the assembled product on a mid-size 3D grid."""
    prob = W.cantilever3d(12, 4, 4)
    rho = W.random_density(prob.n_el, seed=18)
    u = W.random_vector(prob.n_dof, seed=19)
    y = fem.matvec_bc(prob, rho, u)
    dofs = np.random.default_rng(0).choice(prob.n_dof, 200, replace=False)
    assert np.allclose(fem.matvec_rows(prob, rho, u, dofs), y[dofs], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prob", [W.small2d(3, 2, n_cases=2), W.small3d(2, 2, 2)], ids=lambda p: p.name)
def test_sensitivity_finite_differences(prob):
    """Adjoint identity dc/drho_e = -u_e^T (dK_e/drho_e) u_e against central finite
    differences of c(rho) (Section 3.2 sensitivity)."""
    rho = W.random_density(prob.n_el, seed=20, lo=0.3)
    U = fem.solve(prob, rho)
    _, _, dc = sens.sensitivities(prob, rho, U)
    h = 1e-6
    for e in range(prob.n_el):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        cp = sens.compliance(prob, fem.solve(prob, rp))
        cm = sens.compliance(prob, fem.solve(prob, rm))
        assert (cp - cm) / (2 * h) == pytest.approx(dc[e], rel=1e-6)


def test_workload_sizes_match_configs():
    p = W.mbb2d()
    assert (p.n_el, p.n_nodes, p.n_dof, int(p.fixed.sum())) == (1200, 1281, 2562, 22)
    p = W.cantilever2d()
    assert (p.n_el, p.n_dof, int(p.fixed.sum()), p.n_cases) == (120000, 241602, 402, 3)
    p = W.cantilever3d()
    assert (p.n_el, p.n_dof, int(p.fixed.sum())) == (192000, 610203, 3 * 41 * 41)
    assert p.loads.sum() == pytest.approx(-40.0)
