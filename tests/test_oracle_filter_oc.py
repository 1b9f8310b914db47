"""Pins for the oracle's filter (Section 3.2.2, Eq. "filter", "filter_cond";
Section 4.5, Eq. "filter_mat") and OC update with bisection (Section 3.2,
Eq. "update"; Section 3.2.1; code of Section 4.4)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import filt, oc


def test_closed_form_weights_rmin_1p5():
    offs, wts = filt.stencil_offsets(2, 1.5)
    got = sorted(set(np.round(wts, 14)))
    assert got == sorted(set(np.round([1.5, 0.5, 1.5 - math.sqrt(2)], 14)))
    assert len(offs) == 9
    assert sum(wts) == pytest.approx(1.5 + 4 * 0.5 + 4 * (1.5 - math.sqrt(2)), abs=1e-14)
    assert sum(wts) == pytest.approx(3.8431, abs=1e-4)


def test_stencil_sizes():
    # rmin 3.0 in 2D: offsets with |d| < 3 -> the 5 x 5 block (corner 2.83 in, 3 out)
    assert len(filt.stencil_offsets(2, 3.0)[0]) == 25
    # rmin 1.5 in 3D: 19-point (face 1, edge 1.41 in; corner 1.73 out)
    assert len(filt.stencil_offsets(3, 1.5)[0]) == 19
    # rmin 2.0 in 3D: |d| < 2 -> 27 + 6 ... only 27-point block (dist 2 gives weight 0)
    assert len(filt.stencil_offsets(3, 2.0)[0]) == 27


def _brute_filter(prob, rho, dc):
    """Pure-Python double loop over element pairs, straight from Eq. "filter"."""
    n = prob.n_el
    cx = [((e % prob.nelx) + 0.5, ((e // prob.nelx) % prob.nely) + 0.5,
           (e // (prob.nelx * prob.nely)) + 0.5 if prob.dim == 3 else 0.0) for e in range(n)]
    out = np.zeros(n)
    for a in range(n):
        num = 0.0
        den = 0.0
        for b in range(n):
            d = math.sqrt(sum((cx[a][i] - cx[b][i]) ** 2 for i in range(3)))
            w = max(0.0, prob.rmin - d)
            num += w * rho[b] * dc[b]
            den += w
        out[a] = num / (rho[a] * den)
    return out


@pytest.mark.parametrize("prob", [W.small2d(6, 4, rmin=1.5), W.small2d(7, 5, rmin=3.0),
                                  W.small3d(4, 3, 3, rmin=1.5), W.small3d(4, 4, 3, rmin=2.0)],
                         ids=lambda p: f"{p.name}_r{p.rmin}")
def test_dense_edm_sparse_and_brute_force_agree(prob):
    rho = W.random_density(prob.n_el, seed=21)
    dc = W.random_sensitivity(prob.n_el, seed=22)
    Wd = filt.dense_weights(prob)
    Ws = filt.sparse_weights(prob)
    assert np.allclose(Wd, Ws.toarray(), atol=1e-14)
    a = filt.sensitivity_filter(Wd, rho, dc)
    b = filt.sensitivity_filter(Ws, rho, dc)
    c = _brute_filter(prob, rho, dc)
    assert np.allclose(a, b, rtol=1e-13)
    assert np.allclose(a, c, rtol=1e-13)


@pytest.mark.parametrize("prob", [W.small2d(9, 5, rmin=3.0), W.small3d(5, 4, 3, rmin=2.0)],
                         ids=lambda p: p.name)
def test_normalisation_and_linearity(prob):
    Ws = filt.sparse_weights(prob)
    rho = np.full(prob.n_el, 0.42)
    dc = np.full(prob.n_el, -3.5)
    # uniform rho and constant dc are returned unchanged, boundary elements included
    assert np.allclose(filt.sensitivity_filter(Ws, rho, dc), dc, rtol=1e-14)
    rho = W.random_density(prob.n_el, seed=23)
    d1 = W.random_sensitivity(prob.n_el, 24)
    d2 = W.random_sensitivity(prob.n_el, 25)
    lhs = filt.sensitivity_filter(Ws, rho, 2.0 * d1 + 3.0 * d2)
    rhs = 2.0 * filt.sensitivity_filter(Ws, rho, d1) + 3.0 * filt.sensitivity_filter(Ws, rho, d2)
    assert np.allclose(lhs, rhs, rtol=1e-12)
    # density filter preserves constants too
    assert np.allclose(filt.density_filter(Ws, np.full(prob.n_el, 0.3)), 0.3)


def _oc_case(n, seed, passive_frac=0.0):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.001, 1.0, n)
    dcf = W.random_sensitivity(n, seed + 1)
    passive = (rng.uniform(size=n) < passive_frac).astype(np.int8) if passive_frac else None
    if passive is not None:
        rho[passive == 1] = 0.001
    return rho, dcf, passive


@pytest.mark.parametrize("n,seed,vf,pf", [(50, 1, 0.4, 0.0), (1000, 2, 0.5, 0.0),
                                          (3000, 3, 0.3, 0.1), (7, 4, 0.6, 0.0)])
def test_bisection_matches_exact_root_and_constraints(n, seed, vf, pf):
    rho, dcf, passive = _oc_case(n, seed, pf)
    new, lam, vol, change, it = oc.bisect(rho, dcf, vf, passive=passive)
    lam_exact = oc.exact_lambda(rho, dcf, vf, passive=passive)
    assert lam == pytest.approx(lam_exact, rel=2e-9)
    # exact root satisfies the constraint to rounding
    assert oc.volume_at(rho, dcf, lam_exact, passive=passive) == pytest.approx(vf * n, rel=1e-12)
    assert vol == pytest.approx(vf * n, rel=1e-7)
    # bounds and move limits
    assert np.all(new >= 0.001 - 1e-15) and np.all(new <= 1.0 + 1e-15)
    assert np.all(np.abs(new - rho) <= 0.2 + 1e-12)
    assert change == pytest.approx(np.max(np.abs(new - rho)))
    if passive is not None:
        assert np.all(new[passive == 1] == 0.001)
    # KKT for unclamped elements: rho_new = rho sqrt(-dc~/lambda)
    lo = np.maximum(0.001, rho - 0.2)
    hi = np.minimum(1.0, rho + 0.2)
    free = (new > lo + 1e-9) & (new < hi - 1e-9)
    if passive is not None:
        free &= passive == 0
    assert free.sum() > 0
    assert np.allclose(new[free], rho[free] * np.sqrt(-dcf[free] / lam), rtol=1e-12)
    assert 40 <= it <= 120


def test_bisection_paper_rule_ties_move_upper_bound():
    """All elements pinned at the same bound: V(lambda) is flat; the paper's rule
    (positive -> lower bound up, else upper bound down) still terminates."""
    rho = np.full(10, 0.5)
    dcf = np.full(10, -1.0)
    new, lam, vol, change, it = oc.bisect(rho, dcf, 0.5)
    assert vol == pytest.approx(5.0, rel=1e-8)
    assert lam == pytest.approx(1.0, rel=1e-8)


def test_density_filter_chain_rule_is_the_adjoint_and_the_gradient():
    """d/d rho of phi(W rho / rowsum) is W^T (g / rowsum): the adjoint identity
    <density_filter(x), y> = <x, chain(y)> and central finite differences of a
    smooth function of the filtered densities."""
    prob = W.small2d(9, 7, rmin=2.2)
    Wd = filt.weights_for(prob)
    rng = np.random.default_rng(17)
    x, y = rng.uniform(0.1, 1, prob.n_el), rng.normal(size=prob.n_el)
    assert float(filt.density_filter(Wd, x) @ y) == pytest.approx(float(x @ filt.density_filter_chain(Wd, y)), rel=1e-12)
    phi = lambda r: float(np.sum(np.sin(filt.density_filter(Wd, r)) ** 2))
    g = np.sin(2 * filt.density_filter(Wd, x))  # d phi / d rho~
    grad = filt.density_filter_chain(Wd, g)
    h = 1e-6
    for e in (0, 17, prob.n_el - 1):
        xp, xm = x.copy(), x.copy()
        xp[e] += h
        xm[e] -= h
        assert (phi(xp) - phi(xm)) / (2 * h) == pytest.approx(grad[e], rel=1e-6)
