"""Unit-element stiffness matrices K0 = integral of B^T D B over the unit element.

Energy density (Section 2.1, Eq. "str_energy"): psi0 = lambda/2 tr(eps)^2 + mu tr(eps^2),
so the element energy is u_e^T K0 u_e = 2 * integral(psi0).  The paper uses P1
triangles/tets and notes (Remark in Section 3.1) that quadrilaterals/hexahedra
may be used instead; we use bilinear Q4 (2D plane stress) and trilinear H8 (3D).

Local node order: Q4 (0,0),(1,0),(1,1),(0,1); H8 the same four at z = 0 then at
z = 1.  DOF order inside an element: node-major, component-minor.
Strain (Voigt): 2D [exx, eyy, gxy]; 3D [exx, eyy, ezz, gyz, gxz, gxy] with
engineering shears g = 2 eps.

Two independent derivations:
  k0_q4 / k0_h8            Gauss-Legendre quadrature (2 points per axis) in FP64
  k0_q4_exact / k0_h8_exact exact polynomial integration in rational arithmetic
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product

import numpy as np

Q4_NODES = [(0, 0), (1, 0), (1, 1), (0, 1)]
H8_NODES = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
            (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def d_plane_stress(E, nu):
    """2D plane-stress constitutive matrix in Voigt form [exx, eyy, gxy]."""
    c = E / (1.0 - nu * nu)
    return c * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]])


def d_iso3d(E, nu):
    """3D isotropic constitutive matrix from the Lame parameters
    lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu))."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] = lam + 2 * mu
        D[3 + i, 3 + i] = mu
    return D


def _shape_grad(nodes, xi):
    """Gradients of the multilinear shape functions N_a(xi) = prod_d (x_ad ? xi_d : 1 - xi_d)
    on the unit element, returned as array [n_nodes, dim]."""
    dim = len(xi)
    g = np.zeros((len(nodes), dim))
    for a, xa in enumerate(nodes):
        for d in range(dim):
            v = 1.0
            for e in range(dim):
                if e == d:
                    v *= 1.0 if xa[e] == 1 else -1.0
                else:
                    v *= xi[e] if xa[e] == 1 else (1.0 - xi[e])
            g[a, d] = v
    return g


def _b_matrix(grad, dim):
    n = grad.shape[0]
    if dim == 2:
        B = np.zeros((3, 2 * n))
        for a in range(n):
            dx, dy = grad[a]
            B[0, 2 * a] = dx
            B[1, 2 * a + 1] = dy
            B[2, 2 * a] = dy
            B[2, 2 * a + 1] = dx
        return B
    B = np.zeros((6, 3 * n))
    for a in range(n):
        dx, dy, dz = grad[a]
        B[0, 3 * a] = dx
        B[1, 3 * a + 1] = dy
        B[2, 3 * a + 2] = dz
        B[3, 3 * a + 1] = dz
        B[3, 3 * a + 2] = dy
        B[4, 3 * a] = dz
        B[4, 3 * a + 2] = dx
        B[5, 3 * a] = dy
        B[5, 3 * a + 1] = dx
    return B


def _gauss_k0(nodes, D, dim):
    g = 0.5 / np.sqrt(3.0)
    pts = [0.5 - g, 0.5 + g]
    w = 0.5 ** dim  # each 1D weight is 1/2 on [0, 1]
    K = np.zeros((dim * len(nodes), dim * len(nodes)))
    for xi in product(pts, repeat=dim):
        B = _b_matrix(_shape_grad(nodes, xi), dim)
        K += w * B.T @ D @ B
    return K


def k0_q4(E=1.0, nu=0.3):
    """Q4 plane-stress unit-square stiffness (8 x 8) by 2 x 2 Gauss quadrature."""
    return _gauss_k0(Q4_NODES, d_plane_stress(E, nu), 2)


def k0_h8(E=1.0, nu=0.3):
    """H8 isotropic unit-cube stiffness (24 x 24) by 2 x 2 x 2 Gauss quadrature."""
    return _gauss_k0(H8_NODES, d_iso3d(E, nu), 3)


# ---------------------------------------------------------------------------
# Exact rational derivation: shape-function derivatives are products of
# monomials in (x, y[, z]); the integral of x^a over [0,1] is 1/(a+1).


def _poly_mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(i + j for i, j in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return out


def _poly_int(p):
    s = Fraction(0)
    for e, c in p.items():
        t = Fraction(c)
        for a in e:
            t /= (a + 1)
        s += t
    return s


def _shape_grad_poly(node, d, dim):
    """d N_a / d x_d as a polynomial {exponent tuple: coefficient}."""
    poly = {tuple([0] * dim): Fraction(1)}
    for e in range(dim):
        if e == d:
            fac = {tuple([0] * dim): Fraction(1 if node[e] == 1 else -1)}
        else:
            unit = [0] * dim
            unit[e] = 1
            if node[e] == 1:
                fac = {tuple(unit): Fraction(1)}
            else:
                fac = {tuple([0] * dim): Fraction(1), tuple(unit): Fraction(-1)}
        poly = _poly_mul(poly, fac)
    return poly


def _exact_k0(nodes, Dq, dim):
    """K0 in exact arithmetic; Dq is the constitutive matrix as Fractions."""
    n = len(nodes)
    # G[a][d] = polynomial of dN_a/dx_d
    G = [[_shape_grad_poly(nd, d, dim) for d in range(dim)] for nd in nodes]
    # Integrals of products of gradients I[a][b][d][e] = int dNa/dxd dNb/dxe
    I = [[[[_poly_int(_poly_mul(G[a][d], G[b][e])) for e in range(dim)] for d in range(dim)]
          for b in range(n)] for a in range(n)]
    # B rows expressed as lists of (node, component, derivative-direction)
    if dim == 2:
        rows = [[(0, 0)], [(1, 1)], [(0, 1), (1, 0)]]  # (component, direction)
    else:
        rows = [[(0, 0)], [(1, 1)], [(2, 2)], [(1, 2), (2, 1)], [(0, 2), (2, 0)],
                [(0, 1), (1, 0)]]
    nv = len(rows)
    K = [[Fraction(0)] * (dim * n) for _ in range(dim * n)]
    for a in range(n):
        for b in range(n):
            for ci in range(dim):
                for cj in range(dim):
                    s = Fraction(0)
                    for p in range(nv):
                        for q in range(nv):
                            if Dq[p][q] == 0:
                                continue
                            for (comp_p, dir_p) in rows[p]:
                                if comp_p != ci:
                                    continue
                                for (comp_q, dir_q) in rows[q]:
                                    if comp_q != cj:
                                        continue
                                    s += Dq[p][q] * I[a][b][dir_p][dir_q]
                    K[dim * a + ci][dim * b + cj] = s
    return K


def k0_q4_exact(E=Fraction(1), nu=Fraction(3, 10)):
    """Q4 plane-stress K0 in exact rational arithmetic (list of lists of Fraction)."""
    E, nu = Fraction(E), Fraction(nu)
    c = E / (1 - nu * nu)
    Dq = [[c, c * nu, 0], [c * nu, c, 0], [0, 0, c * (1 - nu) / 2]]
    return _exact_k0(Q4_NODES, Dq, 2)


def k0_h8_exact(E=Fraction(1), nu=Fraction(3, 10)):
    """H8 isotropic K0 in exact rational arithmetic (list of lists of Fraction)."""
    E, nu = Fraction(E), Fraction(nu)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    Dq = [[0] * 6 for _ in range(6)]
    for i in range(3):
        for j in range(3):
            Dq[i][j] = lam
        Dq[i][i] = lam + 2 * mu
        Dq[3 + i][3 + i] = mu
    return _exact_k0(H8_NODES, Dq, 3)


def to_float(Kq):
    return np.array([[float(v) for v in row] for row in Kq])
