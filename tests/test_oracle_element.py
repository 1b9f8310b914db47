"""Pins for the oracle's element stiffness (energy density of Section 2.1, Eq.
"str_energy"; bilinear/trilinear elements allowed by the Remark of Section 3.1)."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from oracle import element


def psi0(eps, lam, mu):
    """Closed-form strain energy density psi0 = lambda/2 tr(eps)^2 + mu tr(eps^2)
    (Eq. "str_energy"), written out independently of any element code."""
    return 0.5 * lam * np.trace(eps) ** 2 + mu * np.trace(eps @ eps)


def rigid_modes(nodes):
    dim = len(nodes[0])
    X = np.array(nodes, dtype=float)
    modes = []
    for d in range(dim):
        v = np.zeros((len(nodes), dim))
        v[:, d] = 1.0
        modes.append(v.ravel())
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (0, 2)]
    for a, b in pairs:
        v = np.zeros((len(nodes), dim))
        v[:, a] = -X[:, b]
        v[:, b] = X[:, a]
        modes.append(v.ravel())
    return np.array(modes)


@pytest.mark.parametrize("nu", [0.3, 0.0, 0.25, 0.45])
def test_q4_gauss_equals_exact_rational(nu):
    Kg = element.k0_q4(1.0, nu)
    Kq = element.to_float(element.k0_q4_exact(Fraction(1), Fraction(nu).limit_denominator(1000)))
    assert np.allclose(Kg, Kq, rtol=0, atol=1e-14)


@pytest.mark.parametrize("nu", [0.3, 0.2])
def test_h8_gauss_equals_exact_rational(nu):
    Kg = element.k0_h8(1.0, nu)
    Kq = element.to_float(element.k0_h8_exact(Fraction(1), Fraction(nu).limit_denominator(1000)))
    assert np.allclose(Kg, Kq, rtol=0, atol=1e-14)


def test_q4_closed_form_entries():
    """The eight distinct entries of the plane-stress unit-square K0, times
    (1 - nu^2)/E, are 1/2 - nu/6, 1/8 + nu/8, -1/4 - nu/12, -1/8 + 3nu/8,
    -1/4 + nu/12, -1/8 - nu/8, nu/6, 1/8 - 3nu/8 (textbook closed form)."""
    for nu in (0.3, 0.1, 0.4):
        K = element.k0_q4(1.0, nu) * (1 - nu * nu)
        expect = [1 / 2 - nu / 6, 1 / 8 + nu / 8, -1 / 4 - nu / 12, -1 / 8 + 3 * nu / 8,
                  -1 / 4 + nu / 12, -1 / 8 - nu / 8, nu / 6, 1 / 8 - 3 * nu / 8]
        got = np.unique(np.round(K, 12))
        assert np.allclose(sorted(got), sorted(np.round(expect, 12)), atol=1e-12)
        # the diagonal is the 1/2 - nu/6 entry
        assert np.allclose(np.diag(K), 1 / 2 - nu / 6)


@pytest.mark.parametrize("which", ["q4", "h8"])
def test_symmetric_psd_and_rigid_null_space(which):
    K = element.k0_q4(1.0, 0.3) if which == "q4" else element.k0_h8(1.0, 0.3)
    nodes = element.Q4_NODES if which == "q4" else element.H8_NODES
    assert np.allclose(K, K.T, atol=1e-15)
    ev = np.linalg.eigvalsh(K)
    n_rigid = 3 if which == "q4" else 6
    assert np.all(ev > -1e-14)
    assert np.sum(np.abs(ev) < 1e-12) == n_rigid
    R = rigid_modes(nodes)
    assert np.abs(K @ R.T).max() < 1e-14
    # row sums vanish (translations)
    dim = len(nodes[0])
    for d in range(dim):
        assert np.abs(K[:, d::dim].sum(axis=1)).max() < 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_q4_patch_test_plane_stress(seed):
    """u = A x + b on the unit square: u^T K0 u = 2 * psi0(sym A) * area with the
    plane-stress Lame parameter lambda* = E nu / (1 - nu^2), mu = E / (2 (1 + nu))."""
    rng = np.random.default_rng(seed)
    E, nu = 1.7, 0.3
    A = rng.normal(size=(2, 2))
    b = rng.normal(size=2)
    u = np.concatenate([A @ np.array(x, float) + b for x in element.Q4_NODES])
    eps = 0.5 * (A + A.T)
    lam_ps = E * nu / (1 - nu * nu)
    mu = E / (2 * (1 + nu))
    assert u @ element.k0_q4(E, nu) @ u == pytest.approx(2 * psi0(eps, lam_ps, mu), rel=1e-13)
    # plane strain would give a different value: the pin distinguishes them
    lam_pe = E * nu / ((1 + nu) * (1 - 2 * nu))
    if abs(np.trace(eps)) > 1e-3:
        assert abs(2 * psi0(eps, lam_pe, mu) - 2 * psi0(eps, lam_ps, mu)) > 1e-6


@pytest.mark.parametrize("seed", range(5))
def test_h8_patch_test(seed):
    rng = np.random.default_rng(seed)
    E, nu = 2.3, 0.3
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)
    u = np.concatenate([A @ np.array(x, float) + b for x in element.H8_NODES])
    eps = 0.5 * (A + A.T)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    assert u @ element.k0_h8(E, nu) @ u == pytest.approx(2 * psi0(eps, lam, mu), rel=1e-13)


def test_golden_k0_fixture_matches():
    """Stored exact K0 entries (written by tests/golden/make_golden.py from the exact
    rational derivation) still match the quadrature derivation."""
    import os
    d = os.path.join(os.path.dirname(__file__), "golden")
    for name, K in (("k0_q4_nu0.3.txt", element.k0_q4(1.0, 0.3)),
                    ("k0_h8_nu0.3.txt", element.k0_h8(1.0, 0.3))):
        rows = [l.split() for l in open(os.path.join(d, name)) if not l.startswith("#")]
        G = np.array([[float(Fraction(x)) for x in r] for r in rows])
        assert np.allclose(G, K, atol=1e-15)
