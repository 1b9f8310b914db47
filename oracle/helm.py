"""Helmholtz (PDE) filter: the filter the paper switches to for its parallel
runs (Section "Parallel implementation of topology optimization"), where the
mesh-independency filter of Section 3.2.2 needs element centres that a mesh
partition does not hold.  The paper cites Lazarov & Sigmund (2011) for it and
gives no formula; this module states the filter in its usual finite-element
form.  TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU legs use this package.

The filtered nodal field psi solves  -R^2 lap(psi) + psi = rho  on the design
domain with homogeneous Neumann conditions, discretised with the bilinear (Q4)
/ trilinear (H8) elements of the displacement:

    (R^2 K_F + M_F) psi = T rho,     T[n, e] = integral over element e of N_n,

K_F the Laplacian stiffness and M_F the consistent mass.  The filtered element
density is the element mean of psi, rho~_e = sum_n T[n, e] psi_n / |e|.  With
unit elements

    rho~ = T^T (R^2 K_F + M_F)^-1 T rho =: H rho,

and H is symmetric, so the chain rule of a function phi of rho~ is
d phi / d rho = H (d phi / d rho~).  R = rmin / (2 sqrt 3): the radius at which
the PDE filter matches the cone filter of radius rmin (Lazarov & Sigmund).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mesh


def radius(rmin):
    """PDE filter length scale R for a cone-filter radius rmin."""
    return rmin / (2.0 * np.sqrt(3.0))


def _corners(dim):
    """Corner coordinates of the unit element in oracle.mesh's local order."""
    en = mesh.element_nodes(dim, 1, 1, 1 if dim == 3 else 0)[0]
    n = 2
    return np.array([[(v % n), (v // n) % n] + ([v // (n * n)] if dim == 3 else []) for v in en], dtype=np.float64)


def element_matrices(dim):
    """K_F, M_F (nc x nc) and t (integral of each shape function) of the unit
    element, by 2-point Gauss quadrature per axis (exact for these
    polynomials).  N_a(x) = prod_i (x_i if corner_a,i = 1 else 1 - x_i)."""
    C = _corners(dim)
    nc = C.shape[0]
    g = [0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)]
    K = np.zeros((nc, nc))
    M = np.zeros((nc, nc))
    t = np.zeros(nc)
    for pt in itertools.product(g, repeat=dim):
        x = np.array(pt)
        w = 0.5 ** dim  # Gauss weights on [0, 1]
        N = np.array([np.prod([x[i] if C[a, i] == 1 else 1.0 - x[i] for i in range(dim)]) for a in range(nc)])
        dN = np.zeros((nc, dim))
        for a in range(nc):
            for i in range(dim):
                d = 1.0 if C[a, i] == 1 else -1.0
                others = [x[j] if C[a, j] == 1 else 1.0 - x[j] for j in range(dim) if j != i]
                dN[a, i] = d * np.prod(others)
        K += w * dN @ dN.T
        M += w * np.outer(N, N)
        t += w * N
    return K, M, t


def operator(prob, R=None):
    """Assembled A = R^2 K_F + M_F (nodes x nodes) and T (nodes x elements)."""
    R = radius(prob.rmin) if R is None else R
    Ke, Me, te = element_matrices(prob.dim)
    Ae = R * R * Ke + Me
    en = mesh.element_nodes(prob.dim, prob.nelx, prob.nely, prob.nelz)
    ne, nc = en.shape
    nn = mesh.n_nodes(prob.dim, prob.nelx, prob.nely, prob.nelz)
    rows = np.repeat(en, nc, axis=1).ravel()
    cols = np.tile(en, (1, nc)).ravel()
    A = sp.coo_matrix((np.tile(Ae.ravel(), ne), (rows, cols)), shape=(nn, nn)).tocsc()
    T = sp.coo_matrix((np.tile(te, ne), (en.ravel(), np.repeat(np.arange(ne), nc))), shape=(nn, ne)).tocsr()
    return A, T


def apply(prob, x, R=None, AT=None):
    """H x = T^T (R^2 K_F + M_F)^-1 T x (element values in, element values
    out).  Filters densities and, by symmetry, maps d phi / d rho~ back to
    d phi / d rho."""
    A, T = operator(prob, R) if AT is None else AT
    psi = spla.spsolve(A, T @ np.asarray(x, dtype=np.float64))
    return T.T @ psi
