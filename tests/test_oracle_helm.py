"""Pins of the oracle's Helmholtz (PDE) filter (oracle/helm.py) against facts
that do not depend on its code: textbook element matrices, exact identities of
the discrete operator (constants kept, mass conserved, symmetry), the limit of
a large radius, and the reduction of an x-only field to a 1D problem solved
densely from the 1D element matrices."""
import numpy as np
import pytest

import workloads as W
from oracle import helm


def _hamming_class(dim):
    C = helm._corners(dim)
    return (C[:, None, :] != C[None, :, :]).sum(axis=2)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrices_closed_forms(dim):
    """Bilinear / trilinear unit element: Laplacian stiffness and consistent mass
    depend only on how many coordinates two corners differ in."""
    K, M, t = helm.element_matrices(dim)
    h = _hamming_class(dim)
    if dim == 2:
        Kx = np.choose(h, [4 / 6, -1 / 6, -2 / 6])
        Mx = np.choose(h, [4 / 36, 2 / 36, 1 / 36])
    else:
        Kx = np.choose(h, [4 / 12, 0.0, -1 / 12, -1 / 12])
        Mx = np.choose(h, [8 / 216, 4 / 216, 2 / 216, 1 / 216])
    assert np.allclose(K, Kx, rtol=0, atol=1e-15)
    assert np.allclose(M, Mx, rtol=0, atol=1e-15)
    assert np.allclose(t, 0.5 ** dim, rtol=0, atol=1e-15)


PROBS = [W.small2d(17, 9, rmin=2.0), W.small3d(7, 5, 4, rmin=1.5)]


@pytest.mark.parametrize("prob", PROBS, ids=lambda p: p.name)
def test_constants_kept_and_mass_conserved(prob):
    """K_F 1 = 0 and T 1 = M_F 1, so a constant density is a fixed point; and
    1^T H x = 1^T x for every x (the filter conserves the total volume)."""
    AT = helm.operator(prob)
    one = np.ones(prob.n_el)
    assert np.allclose(helm.apply(prob, one, AT=AT), one, rtol=0, atol=1e-12)
    x = np.random.default_rng(3).uniform(0.0, 1.0, prob.n_el)
    assert helm.apply(prob, x, AT=AT).sum() == pytest.approx(x.sum(), rel=1e-12)


@pytest.mark.parametrize("prob", PROBS, ids=lambda p: p.name)
def test_symmetric(prob):
    AT = helm.operator(prob)
    rng = np.random.default_rng(4)
    x, y = rng.normal(size=prob.n_el), rng.normal(size=prob.n_el)
    assert float(x @ helm.apply(prob, y, AT=AT)) == pytest.approx(float(y @ helm.apply(prob, x, AT=AT)), rel=1e-11)


@pytest.mark.parametrize("prob", PROBS, ids=lambda p: p.name)
def test_large_radius_gives_the_mean(prob):
    x = np.random.default_rng(5).uniform(0.0, 1.0, prob.n_el)
    out = helm.apply(prob, x, R=1e4)
    assert np.allclose(out, x.mean(), rtol=0, atol=1e-6)


@pytest.mark.parametrize("prob", [W.small2d(23, 4, rmin=3.0), W.small3d(9, 3, 2, rmin=2.0)], ids=lambda p: p.name)
def test_x_only_field_reduces_to_1d(prob):
    """A density that varies along x only: the tensor-product operator reduces
    to the 1D problem (R^2 K1 + M1) psi = T1 rho with K1 = [[1, -1], [-1, 1]],
    M1 = [[2, 1], [1, 2]] / 6, T1 = 1/2 per node, solved densely here."""
    n = prob.nelx
    rho1 = np.random.default_rng(6).uniform(0.0, 1.0, n)
    reps = prob.n_el // n
    rho = np.tile(rho1, reps)  # x fastest in the element numbering
    R = helm.radius(prob.rmin)
    A1 = np.zeros((n + 1, n + 1))
    T1 = np.zeros((n + 1, n))
    for e in range(n):
        idx = [e, e + 1]
        A1[np.ix_(idx, idx)] += R * R * np.array([[1.0, -1.0], [-1.0, 1.0]]) + np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
        T1[idx, e] += 0.5
    ref1 = T1.T @ np.linalg.solve(A1, T1 @ rho1)
    out = helm.apply(prob, rho)
    assert np.allclose(out, np.tile(ref1, reps), rtol=0, atol=1e-12)


def test_simp_compliance_gradient_through_the_helmholtz_filter():
    """The oracle's SIMP iteration with the Helmholtz filter: dc~ = H dc is the
    gradient of the compliance c(H rho) -- central finite differences through
    the full chain (filter, assembly, LU solve, compliance) on a small MBB."""
    from oracle import fem, simp
    prob = W.small2d(8, 5, rmin=2.0)
    rho = np.random.default_rng(8).uniform(0.3, 0.9, prob.n_el)
    out = simp.iteration(prob, rho, filter_mode=2)
    AT = helm.operator(prob)

    def comp(r):
        rt = helm.apply(prob, r, AT=AT)
        U = fem.solve(prob, rt)
        return float(sum(prob.loads[c] @ U[c] for c in range(prob.n_cases)))

    assert comp(rho) == pytest.approx(out["c"], rel=1e-12)
    h = 1e-6
    for e in (0, 11, prob.n_el - 1):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        assert (comp(rp) - comp(rm)) / (2 * h) == pytest.approx(out["dcf"][e], rel=1e-5)
