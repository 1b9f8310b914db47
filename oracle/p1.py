"""The paper's own discretisation: vector P1 displacements on a triangulated
(tetrahedralised) structured grid with one density per cell.  TEST
INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU legs use
this package.

The paper meshes the design domain with RectangleMesh(..., "right/left"), which
splits each unit square into two triangles, and BoxMesh in 3D (Section 4
"Discretization the problem", Section 5 "Working with 3D problems").  The
displacement is a continuous piecewise-linear vector field and the density is
constant per cell (DG0).  The bilinear form is the integral of
d^p sigma(u) : grad(v), with sigma(u) = 2 mu eps(u) + lambda tr(eps(u)) I, the
same formula in 2D and 3D (Section 4.3 listing).

Readings (the paper leaves them to the mesh generator):
  * "right" diagonal: each square [i, i+1] x [j, j+1] is cut along
    (i, j)-(i+1, j+1) into the cells (v00, v10, v11) and (v00, v11, v01);
    "left": along (i+1, j)-(i, j+1) into (v00, v10, v01) and (v10, v11, v01);
    "right/left": rows j = 0, 2, 4, ... cut "right", odd rows "left".
  * 3D: each cube is cut into the 6 tetrahedra of the Kuhn (Freudenthal)
    subdivision, which all share the diagonal from the cube's lowest corner to its
    highest; for each ordering (a, b, c) of the axes, the path v0, v0 + e_a,
    v0 + e_a + e_b, v0 + e_a + e_b + e_c.  Orderings are taken lexicographically,
    and each tetrahedron is stored with positive orientation.
  * Modified SIMP as for Q4 / H8: the cell's sigma is scaled by
    E_e = Emin + rho_e^p (1 - Emin).
  * Objective and sensitivity: the paper projects d^p psi(u) onto DG0. For P1,
    psi is constant per cell, so this is psi_e = u_e^T K_e u_e / (2 |T_e|).
    Every cell of the structured grid has the same measure, so the oracle uses
    the cell energy ce_e = u_e^T K_e u_e (unit modulus), as for Q4 / H8: a
    uniform factor, which leaves the OC update unchanged.
  * Filter distances are measured between cell midpoints (centroids), as in the
    paper's listing.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.spatial import cKDTree

from . import filt, oc


# ---------------------------------------------------------------- mesh ----

def node_coords(dim, nelx, nely, nelz=0):
    """Node coordinates, x fastest (node (i, j, k) at (i, j, k))."""
    if dim == 2:
        j, i = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel()], axis=1).astype(np.float64)
    k, j, i = np.meshgrid(np.arange(nelz + 1), np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)


def _cut(diagonal, j):
    if diagonal == "right/left":
        return "right" if j % 2 == 0 else "left"
    if diagonal in ("right", "left"):
        return diagonal
    raise ValueError(f"unknown diagonal pattern {diagonal!r}")


KUHN_ORDERS = list(itertools.permutations(range(3)))  # lexicographic


def cells(prob):
    """Vertex node indices of every cell, shape [n_el, dim + 1], each cell with
    positive orientation; cell index = (2 or 6) * square / cube index + local."""
    nx, ny = prob.nelx, prob.nely
    if prob.dim == 2:
        out = np.zeros((2 * nx * ny, 3), dtype=np.int64)
        for j in range(ny):
            cut = _cut(prob.diagonal, j)
            for i in range(nx):
                v00 = i + (nx + 1) * j
                v10, v01, v11 = v00 + 1, v00 + nx + 1, v00 + nx + 2
                e = i + nx * j
                if cut == "right":
                    out[2 * e] = (v00, v10, v11)
                    out[2 * e + 1] = (v00, v11, v01)
                else:
                    out[2 * e] = (v00, v10, v01)
                    out[2 * e + 1] = (v10, v11, v01)
        return out
    nz = prob.nelz
    X = node_coords(3, nx, ny, nz)
    out = np.zeros((6 * nx * ny * nz, 4), dtype=np.int64)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                for t, order in enumerate(KUHN_ORDERS):
                    p = [i, j, k]
                    verts = [i + (nx + 1) * (j + (ny + 1) * k)]
                    for a in order:
                        p[a] += 1
                        verts.append(p[0] + (nx + 1) * (p[1] + (ny + 1) * p[2]))
                    M = X[verts[1:]] - X[verts[0]]
                    if np.linalg.det(M) < 0:
                        verts[2], verts[3] = verts[3], verts[2]
                    out[6 * e + t] = verts
    return out


def cell_midpoints(prob, C=None):
    """Centroid of every cell, shape [n_el, dim]."""
    C = cells(prob) if C is None else C
    X = node_coords(prob.dim, prob.nelx, prob.nely, prob.nelz)
    return X[C].mean(axis=1)


def cell_dofs(prob, C=None):
    C = cells(prob) if C is None else C
    d = prob.dim * C[:, :, None] + np.arange(prob.dim)[None, None, :]
    return d.reshape(C.shape[0], -1)


# ---------------------------------------------------- element matrices ----

def bary_gradients(V):
    """Gradients of the barycentric coordinates of the simplex with vertex
    coordinates V [d + 1, d] (rows = vertices), and its measure.  lambda_i is the
    affine function equal to 1 at vertex i and 0 at the others, so its
    coefficients are the columns of [1 | V]^-1."""
    d = V.shape[1]
    M = np.hstack([np.ones((d + 1, 1)), V])
    Cm = np.linalg.inv(M)
    G = Cm[1:, :].T  # G[i] = grad lambda_i
    meas = abs(np.linalg.det(M)) / float(np.prod(np.arange(1, d + 1)))
    return G, meas


def elasticity_voigt(dim, lam, mu):
    """sigma = 2 mu eps + lambda tr(eps) I in Voigt form (engineering shears)."""
    if dim == 2:
        return np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[[0, 1, 2], [0, 1, 2]] = lam + 2 * mu
    C[[3, 4, 5], [3, 4, 5]] = mu
    return C


def strain_matrix(G):
    """B with eps_voigt = B u_e for the P1 cell with gradients G [d + 1, d];
    2D rows (xx, yy, 2xy), 3D rows (xx, yy, zz, 2yz, 2xz, 2xy)."""
    nv, d = G.shape
    if d == 2:
        B = np.zeros((3, 2 * nv))
        for i, (gx, gy) in enumerate(G):
            B[:, 2 * i:2 * i + 2] = [[gx, 0.0], [0.0, gy], [gy, gx]]
        return B
    B = np.zeros((6, 3 * nv))
    for i, (gx, gy, gz) in enumerate(G):
        B[:, 3 * i:3 * i + 3] = [[gx, 0, 0], [0, gy, 0], [0, 0, gz], [0, gz, gy], [gz, 0, gx], [gy, gx, 0]]
    return B


def cell_stiffness(V, lam, mu):
    """K_e = |T| B^T C B for unit modulus (the strain is constant on the cell,
    so one evaluation integrates the form exactly)."""
    G, meas = bary_gradients(V)
    B = strain_matrix(G)
    return meas * B.T @ elasticity_voigt(V.shape[1], lam, mu) @ B


def cell_stiffness_tensor(V, lam, mu):
    """The same matrix from the bilinear form in tensor notation:
    a(N_i e_a, N_j e_b) = |T| (mu (delta_ab g_i.g_j + g_i[b] g_j[a]) + lambda g_i[a] g_j[b])."""
    G, meas = bary_gradients(V)
    nv, d = G.shape
    K = np.zeros((d * nv, d * nv))
    for i in range(nv):
        for j in range(nv):
            for a in range(d):
                for b in range(d):
                    v = mu * ((G[i] @ G[j]) * (a == b) + G[i][b] * G[j][a]) + lam * G[i][a] * G[j][b]
                    K[d * i + a, d * j + b] = meas * v
    return K


def psi(eps, lam, mu):
    """Strain energy density lambda / 2 tr(eps)^2 + mu eps : eps (the paper's psi)."""
    return 0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps)


# ------------------------------------------------------------- analysis ----

def young(rho, Emin=1e-9, penal=3.0):
    return Emin + np.power(rho, penal) * (1.0 - Emin)


def unit_stiffness(prob, C=None):
    """K_e of every cell for unit modulus, shape [n_el, nd, nd]."""
    C = cells(prob) if C is None else C
    X = node_coords(prob.dim, prob.nelx, prob.nely, prob.nelz)
    return np.stack([cell_stiffness(X[c], prob.lam, prob.mu) for c in C])


def assemble(prob, rho, Ke=None, C=None):
    """K(rho) = sum_e E_e P_e^T K_e P_e as CSR (no boundary conditions)."""
    C = cells(prob) if C is None else C
    Ke = unit_stiffness(prob, C) if Ke is None else Ke
    dofs = cell_dofs(prob, C)
    E = young(rho, prob.Emin, prob.penal)
    nd = dofs.shape[1]
    rows = np.repeat(dofs, nd, axis=1).ravel()
    cols = np.tile(dofs, (1, nd)).ravel()
    vals = (E[:, None, None] * Ke).reshape(len(E), -1).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(prob.n_dof, prob.n_dof)).tocsr()
    K.sum_duplicates()
    return K


def solve(prob, rho, K=None):
    """u[n_cases, n_dof] from K_ff u_f = f_f by SuperLU, u = 0 on fixed DOFs
    (the paper's default sparse LU)."""
    K = assemble(prob, rho) if K is None else K
    free = np.flatnonzero(prob.fixed == 0)
    lu = spla.splu(K[free][:, free].tocsc(), permc_spec="COLAMD")
    U = np.zeros((prob.n_cases, prob.n_dof))
    for c in range(prob.n_cases):
        U[c, free] = lu.solve(prob.loads[c, free])
    return U


def sensitivities(prob, rho, U, Ke=None, C=None):
    """(c, ce, dc): compliance sum_k f_k^T u_k, cell energies
    ce_e = sum_k u_e^T K_e u_e (unit modulus), dc_e = -p rho^(p-1) (1 - Emin) ce_e."""
    C = cells(prob) if C is None else C
    Ke = unit_stiffness(prob, C) if Ke is None else Ke
    dofs = cell_dofs(prob, C)
    ce = np.zeros(len(dofs))
    for k in range(U.shape[0]):
        ue = U[k][dofs]
        ce += np.einsum("ei,eij,ej->e", ue, Ke, ue)
    c = float(sum(prob.loads[k] @ U[k] for k in range(U.shape[0])))
    dc = -prob.penal * np.power(rho, prob.penal - 1.0) * (1.0 - prob.Emin) * ce
    return c, ce, dc


def dense_weights(prob, C=None):
    """Paper-literal dense W = max(0, rmin - |m_a - m_b|) over cell midpoints."""
    M = cell_midpoints(prob, C)
    D = np.sqrt(np.maximum(((M[:, None, :] - M[None, :, :]) ** 2).sum(-1), 0.0))
    W = prob.rmin - D
    W[W < 0] = 0.0
    return W


def sparse_weights(prob, C=None):
    """The same W as a sparse matrix from the midpoint pairs closer than rmin
    (a k-d tree query), the cell itself included."""
    M = cell_midpoints(prob, C)
    pairs = cKDTree(M).query_pairs(prob.rmin, output_type="ndarray")
    n = len(M)
    d = np.linalg.norm(M[pairs[:, 0]] - M[pairs[:, 1]], axis=1)
    w = prob.rmin - d
    keep = w > 0
    r = np.concatenate([pairs[keep, 0], pairs[keep, 1], np.arange(n)])
    q = np.concatenate([pairs[keep, 1], pairs[keep, 0], np.arange(n)])
    v = np.concatenate([w[keep], w[keep], np.full(n, prob.rmin)])
    return sp.csr_matrix((v, (r, q)), shape=(n, n))


def weights_for(prob, C=None, dense_max=4000):
    return dense_weights(prob, C) if prob.n_el <= dense_max else sparse_weights(prob, C)


def iteration(prob, rho, W=None, Ke=None, C=None):
    """One SIMP iteration of the paper's loop on its own mesh: solve,
    sensitivities, sensitivity filter, OC bisection."""
    C = cells(prob) if C is None else C
    Ke = unit_stiffness(prob, C) if Ke is None else Ke
    W = weights_for(prob, C) if W is None else W
    K = assemble(prob, rho, Ke, C)
    U = solve(prob, rho, K)
    c, ce, dc = sensitivities(prob, rho, U, Ke, C)
    dcf = filt.sensitivity_filter(W, rho, dc)
    rho_new, lam, vol, change, nb = oc.bisect(rho, dcf, prob.volfrac, prob.move, prob.dmin, prob.passive)
    return dict(u=U, c=c, ce=ce, dc=dc, dcf=dcf, rho_new=rho_new, lam=lam, vol=vol, change=change, n_bisect=nb)
