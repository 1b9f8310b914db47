"""Mesh-independency filter (Section 3.2.2, Eq. "filter", Eq. "filter_cond";
matrix form Eq. "filter_mat"; vectorised construction in Section 4.5).

Weights W_ab = max(0, rmin - dist(a, b)), dist = Euclidean distance between
element midpoints, the element itself included (dist 0, weight rmin), and only
elements that exist in the mesh (rows are truncated at the domain boundary).
Sensitivity filter:   dc~_a = sum_b W_ab rho_b dc_b / (rho_a sum_b W_ab).
Density filter (variant, mode 1): rho~_a = sum_b W_ab rho_b / sum_b W_ab.

The paper writes the distance matrix through the expansion
||x_i||^2 - 2 x_i^T x_j + ||x_j||^2 (which is the *squared* distance) and then
uses it as a distance; we read the weight as rmin minus the (non-squared)
Euclidean distance, clipped at 0.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

from . import mesh


def dense_weights(prob):
    """Paper-literal dense W (n_el x n_el) from the Euclidean distance matrix of
    element midpoints.  Only for small meshes (memory is n_el^2)."""
    X = mesh.element_centres(prob.dim, prob.nelx, prob.nely, prob.nelz)
    sq = np.sum(X * X, axis=1)
    D2 = sq[:, None] - 2.0 * (X @ X.T) + sq[None, :]
    D = np.sqrt(np.maximum(D2, 0.0))
    W = prob.rmin - D
    W[W < 0] = 0.0
    return W


def stencil_offsets(dim, rmin):
    """Integer offsets d with weight rmin - |d| > 0, and those weights."""
    r = int(math.ceil(rmin))
    offs, wts = [], []
    rng = range(-r, r + 1)
    for d in itertools.product(rng, repeat=dim):
        dist = math.sqrt(sum(x * x for x in d))
        w = rmin - dist
        if w > 0:
            offs.append(d)
            wts.append(w)
    return offs, wts


def sparse_weights(prob):
    """The same W as a sparse matrix built from explicit neighbour offsets."""
    dim, nx, ny, nz = prob.dim, prob.nelx, prob.nely, prob.nelz
    offs, wts = stencil_offsets(dim, prob.rmin)
    n = prob.n_el
    idx = np.arange(n)
    ei = idx % nx
    ej = (idx // nx) % ny
    ek = idx // (nx * ny) if dim == 3 else np.zeros_like(idx)
    rows, cols, vals = [], [], []
    for d, w in zip(offs, wts):
        ni, nj = ei + d[0], ej + d[1]
        nk = ek + d[2] if dim == 3 else ek
        ok = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny)
        if dim == 3:
            ok &= (nk >= 0) & (nk < nz)
        rows.append(idx[ok])
        cols.append((ni + nx * (nj + ny * nk))[ok])
        vals.append(np.full(int(ok.sum()), w))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def sensitivity_filter(W, rho, dc):
    """dc~ = (W (rho . dc)) / (rho . rowsum(W))  (Eq. "filter_mat")."""
    rowsum = np.asarray(W.sum(axis=1)).ravel()
    return (W @ (rho * dc)) / (rho * rowsum)


def density_filter(W, rho):
    """rho~ = (W rho) / rowsum(W)."""
    rowsum = np.asarray(W.sum(axis=1)).ravel()
    return (W @ rho) / rowsum


def density_filter_chain(W, g):
    """Chain rule through the density filter: d/d rho of phi(rho~) given
    g = d phi / d rho~ is W^T (g / rowsum)."""
    rowsum = np.asarray(W.sum(axis=1)).ravel()
    return W.T @ (g / rowsum)


def weights_for(prob, dense_max=6000):
    return dense_weights(prob) if prob.n_el <= dense_max else sparse_weights(prob)
