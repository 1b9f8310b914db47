"""Oracle of the learned warm start's problem-side steps (test infrastructure:
only tests, the smoke check and the benchmark's CPU baseline use it).

The paper has no warm start: it factorises every state equation afresh
(Section 4.3).  These functions define, in plain NumPy/SciPy, what the GPU
path computes around the network (3D H8 problems):

  features   per element: density; fraction of its 8 nodes with a fixed DOF;
             its load share sum_nodes f / (8 max|f|) (3 components); its
             centre's coordinates divided by (nelx, nely, nelz).
  targets    per element: the mean of u over its 8 nodes, divided by the
             largest magnitude of those means (all elements and components).
  node_average   the network's per-element output averaged onto each node over
             its adjacent elements (1 to 8), zero on fixed DOFs.
  alpha      the scale minimising the energy norm of the error of alpha*u^,
             alpha = f^T u^ / (u^T K u^)  (K symmetric positive definite).

Pinned in tests/test_oracle_warm.py by hand-computed features on a 2x2x2
grid, invariants of the averaging, and the optimality of alpha.
"""
from __future__ import annotations

import numpy as np

from . import fem, mesh


def _grid_shape(prob):
    return prob.nelz, prob.nely, prob.nelx


def features(prob, rho, case=0):
    """[8][nelz][nely][nelx] float64 network input of one load case."""
    en = mesh.element_nodes(3, prob.nelx, prob.nely, prob.nelz)       # [n_el, 8]
    fixed_node = prob.fixed.reshape(-1, 3).any(axis=1)
    f = prob.loads[case].reshape(-1, 3)
    free = ~prob.fixed.reshape(-1, 3).astype(bool)
    fmax = np.max(np.abs(f[free])) if np.any(free) else 0.0
    fmask = np.where(free, f, 0.0)                                      # loads on fixed DOFs are ignored
    share = fmask[en].sum(axis=1) / (8.0 * fmax)                       # [n_el, 3]
    cen = mesh.element_centres(3, prob.nelx, prob.nely, prob.nelz)     # [n_el, 3] (x, y, z)
    out = np.empty((8, prob.n_el))
    out[0] = rho
    out[1] = fixed_node[en].sum(axis=1) / 8.0
    out[2:5] = share.T
    out[5] = cen[:, 0] / prob.nelx
    out[6] = cen[:, 1] / prob.nely
    out[7] = cen[:, 2] / prob.nelz
    return out.reshape((8,) + _grid_shape(prob))


def targets(prob, u):
    """[3][nelz][nely][nelx]: element means of u (ABI layout [n_dof]) / max |mean|."""
    en = mesh.element_nodes(3, prob.nelx, prob.nely, prob.nelz)
    m = u.reshape(-1, 3)[en].mean(axis=1)                               # [n_el, 3]
    mx = np.max(np.abs(m))
    return (m / mx if mx > 0 else m).T.reshape((3,) + _grid_shape(prob))


def node_average(prob, y):
    """y: [3][nelz][nely][nelx] per-element output -> u^ [n_dof] (ABI layout)."""
    en = mesh.element_nodes(3, prob.nelx, prob.nely, prob.nelz)
    ye = y.reshape(3, -1).T                                             # [n_el, 3]
    nn = prob.n_nodes
    s = np.zeros((nn, 3))
    cnt = np.zeros(nn)
    for c in range(8):
        np.add.at(s, en[:, c], ye)
        np.add.at(cnt, en[:, c], 1.0)
    u = (s / cnt[:, None]).ravel()
    return np.where(prob.fixed.astype(bool), 0.0, u)


def alpha(prob, rho, uhat, case=0, K=None):
    """alpha = f^T u^ / (u^T K_bc u^) with the Dirichlet-restricted operator."""
    Ku = fem.matvec_bc(prob, rho, uhat, K=K)
    a = float(prob.loads[case] @ np.where(prob.fixed.astype(bool), 0.0, uhat))
    b = float(uhat @ Ku)
    return a / b if b > 0 else 0.0


def node_average_adjoint(prob, g):
    """Adjoint of node_average: g [n_dof] (ABI) -> [3][nelz][nely][nelx];
    element e receives sum over its nodes n of g_n / (elements adjacent to n),
    with g read as zero on fixed DOFs."""
    en = mesh.element_nodes(3, prob.nelx, prob.nely, prob.nelz)
    cnt = np.zeros(prob.n_nodes)
    for c in range(8):
        np.add.at(cnt, en[:, c], 1.0)
    gn = np.where(prob.fixed.astype(bool), 0.0, g).reshape(-1, 3) / cnt[:, None]
    return gn[en].sum(axis=1).T.reshape((3,) + _grid_shape(prob))


def energy_loss(prob, rho, y, comp, case=0, K=None):
    """Energy-norm error left by the best multiple of the averaged prediction,
    relative to the solution's energy c = f^T u* (the compliance):
        L(y) = ||u* - alpha u^||_K^2 / c = 1 - (f^T u^)^2 / ((u^T K u^) c),
    u^ = node_average(y).  Returns (L, dL/dy).  With alpha = f^T u^ / u^T K u^,
    dL/du^ = -(2 alpha / c) (f - alpha K u^) on free DOFs."""
    K = fem.assemble(prob, rho) if K is None else K
    uh = node_average(prob, y)
    Ku = fem.matvec_bc(prob, rho, uh, K=K)
    fixed = prob.fixed.astype(bool)
    f = np.where(fixed, 0.0, prob.loads[case])
    a, b = float(f @ uh), float(uh @ Ku)
    al = a / b
    g = -(2.0 * al / comp) * (f - al * np.where(fixed, 0.0, Ku))
    return 1.0 - a * al / comp, node_average_adjoint(prob, g)
