"""Pins for the oracle of the learned warm start's problem-side steps:
hand-computed features on a 2 x 2 x 2 grid, closed forms of the target and
averaging maps on affine fields, and the optimality of the energy scale."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, nn, warm


def _cube2():
    """2 x 2 x 2 elements, x = 0 face clamped, f_y = -1 at node (2, 0, 1)."""
    fixed, f = W._empty(3, 2, 2, 2, 1)
    W._fix_face_x0(fixed, 3, 2, 2, 2)
    n = 2 + 3 * (0 + 3 * 1)
    f[0, 3 * n + 1] = -1.0
    return W.Problem("cube2", 3, 2, 2, 2, volfrac=0.3, rmin=1.5, fixed=fixed, loads=f)


def test_features_hand_computed():
    p = _cube2()
    rho = np.arange(1, 9) / 10.0
    F = warm.features(p, rho)
    assert F.shape == (8, 2, 2, 2)
    # element (i, j, k) sits at F[:, k, j, i]
    assert np.allclose(F[0].ravel(), rho)
    # elements with i = 0 have their 4 nodes of the x = 0 face clamped
    assert np.allclose(F[1][:, :, 0], 0.5) and np.allclose(F[1][:, :, 1], 0.0)
    # node (2, 0, 1) belongs to elements (1, 0, 0) and (1, 0, 1): share -1/8 in y
    fy = np.zeros((2, 2, 2))
    fy[0, 0, 1] = fy[1, 0, 1] = -1.0 / 8.0
    assert np.allclose(F[3], fy) and np.allclose(F[2], 0.0) and np.allclose(F[4], 0.0)
    # centres (i + 0.5) / 2 etc.
    assert np.allclose(F[5][0, 0], [0.25, 0.75]) and np.allclose(F[6][0, :, 0], [0.25, 0.75])
    assert np.allclose(F[7][:, 0, 0], [0.25, 0.75])


def test_targets_of_affine_field_are_centre_values():
    p = W.small3d(4, 3, 2)
    xyz = np.stack(np.meshgrid(np.arange(5), np.arange(4), np.arange(3), indexing="ij"), -1)
    xyz = xyz.transpose(2, 1, 0, 3).reshape(-1, 3)      # node order: x fastest
    A = np.array([[0.1, 0.2, -0.3], [0.0, 1.0, 0.5], [2.0, 0.0, 0.1]])
    u = (xyz @ A.T + np.array([1.0, -2.0, 0.5])).ravel()
    T = warm.targets(p, u)
    cen = np.stack(np.meshgrid(np.arange(4) + .5, np.arange(3) + .5, np.arange(2) + .5, indexing="ij"), -1)
    cen = cen.transpose(2, 1, 0, 3).reshape(-1, 3)
    m = cen @ A.T + np.array([1.0, -2.0, 0.5])
    assert np.allclose(T.reshape(3, -1).T, m / np.max(np.abs(m)))
    assert np.isclose(np.max(np.abs(T)), 1.0)


def test_node_average_reproduces_affine_fields_at_interior_nodes():
    p = W.small3d(4, 4, 4)
    cen = np.stack(np.meshgrid(np.arange(4) + .5, np.arange(4) + .5, np.arange(4) + .5, indexing="ij"), -1)
    cen = cen.transpose(2, 1, 0, 3).reshape(-1, 3)
    A = np.array([[1.0, 0.5, 0.0], [0.2, -1.0, 0.3], [0.0, 0.1, 2.0]])
    y = (cen @ A.T).T.reshape(3, 4, 4, 4)
    u = warm.node_average(p, y).reshape(-1, 3)
    for (i, j, k) in [(1, 1, 1), (2, 3, 1), (3, 2, 2)]:
        n = i + 5 * (j + 5 * k)
        assert np.allclose(u[n], A @ np.array([i, j, k], float))
    # a constant field stays constant on free nodes and is zero on the clamped face
    u = warm.node_average(p, np.ones((3, 4, 4, 4))).reshape(-1, 3)
    free = ~p.fixed.reshape(-1, 3).astype(bool)
    assert np.allclose(u[free], 1.0) and np.allclose(u[~free], 0.0)


def test_alpha_is_the_energy_optimal_scale():
    p = W.small3d(4, 3, 2)
    rho = W.random_density(p.n_el, seed=11, lo=0.2)
    ustar = fem.solve(p, rho)[0]
    # scaling the exact solution is undone exactly
    assert warm.alpha(p, rho, ustar / 3.0) == pytest.approx(3.0, rel=1e-9)
    # for any direction, alpha minimises the energy norm of the error
    K = fem.assemble(p, rho)
    uh = np.where(p.fixed.astype(bool), 0.0, W.random_vector(p.n_dof, seed=12))
    a = warm.alpha(p, rho, uh, K=K)
    def err(s):
        e = ustar - s * uh
        return float(e @ fem.matvec_bc(p, rho, e, K=K))
    assert err(a) < err(a * 1.01) and err(a) < err(a * 0.99)
    assert err(a) <= err(0.0)


def test_quantised_forward_stores_representable_activations():
    rng = np.random.default_rng(7)
    params = nn.init_params(seed=8, c_in=2, c_out=3, widths=(4, 4, 4, 4))
    x = nn.to_bf16(rng.normal(size=(2, 8, 8, 8)))
    y0 = nn.forward(params, x)
    y, cache = nn.forward(params, x, keep=True, quant=nn.to_bf16)
    for (_, i, a, act_out, act) in cache:
        if act:
            assert np.array_equal(nn.to_bf16(act_out), act_out)
    # the quantised network stays close to the exact one (bf16 has 8 significant bits)
    assert np.linalg.norm(y - y0) <= 0.05 * np.linalg.norm(y0)


def test_node_average_adjoint_identity():
    p = W.small3d(4, 3, 2)
    rng = np.random.default_rng(13)
    y = rng.normal(size=(3, 2, 3, 4))
    g = rng.normal(size=p.n_dof)
    assert float(warm.node_average(p, y) @ g) == pytest.approx(float(np.sum(y * warm.node_average_adjoint(p, g))),
                                                                rel=1e-12)


def test_energy_loss_value_and_gradient():
    p = W.small3d(4, 3, 2)
    rho = W.random_density(p.n_el, seed=14, lo=0.2)
    U = fem.solve(p, rho)[0]
    comp = float(p.loads[0] @ U)
    rng = np.random.default_rng(15)
    y = rng.normal(size=(3, 2, 3, 4))
    K = fem.assemble(p, rho)
    L, g = warm.energy_loss(p, rho, y, comp, K=K)
    # the value is the relative energy error of the optimally scaled start
    uh = warm.node_average(p, y)
    a = warm.alpha(p, rho, uh, K=K)
    e = U - a * uh
    assert L == pytest.approx(float(e @ fem.matvec_bc(p, rho, e, K=K)) / comp, rel=1e-9)
    assert 0.0 <= L <= 1.0
    # central differences of the loss
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 1, 2, 3), (2, 1, 1, 2)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += h
        ym[idx] -= h
        fd = (warm.energy_loss(p, rho, yp, comp, K=K)[0] - warm.energy_loss(p, rho, ym, comp, K=K)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-10)
