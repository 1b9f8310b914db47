"""Structured-grid bookkeeping for the oracle (unit elements, x-fastest numbering).

The paper builds its mesh with RectangleMesh / BoxMesh (Section 4 "Mesh", Section
5.1) and reads element midpoints for the filter (Section 4.5).  Here the mesh is
the structured grid of unit squares / cubes: node (i, j, k) sits at (i, j, k) and
element (i, j, k) spans [i, i+1] x [j, j+1] x [k, k+1].
"""
from __future__ import annotations

import numpy as np

from .element import H8_NODES, Q4_NODES


def n_nodes(dim, nelx, nely, nelz=0):
    return (nelx + 1) * (nely + 1) * ((nelz + 1) if dim == 3 else 1)


def element_nodes(dim, nelx, nely, nelz=0):
    """Global node indices of every element, shape [n_el, 4 or 8], in the local
    node order of oracle.element."""
    if dim == 2:
        ej, ei = np.meshgrid(np.arange(nely), np.arange(nelx), indexing="ij")
        ei, ej = ei.ravel(), ej.ravel()
        cols = [(ei + dx) + (nelx + 1) * (ej + dy) for (dx, dy) in Q4_NODES]
        return np.stack(cols, axis=1)
    ek, ej, ei = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    cols = [(ei + dx) + (nelx + 1) * ((ej + dy) + (nely + 1) * (ek + dz))
            for (dx, dy, dz) in H8_NODES]
    return np.stack(cols, axis=1)


def element_dofs(dim, nelx, nely, nelz=0):
    """Global DOF indices of every element, shape [n_el, dim * nodes_per_el]."""
    en = element_nodes(dim, nelx, nely, nelz)
    d = dim * en[:, :, None] + np.arange(dim)[None, None, :]
    return d.reshape(en.shape[0], -1)


def element_centres(dim, nelx, nely, nelz=0):
    """Midpoint coordinates of every element, shape [n_el, dim] (Section 4.5:
    the filter distance is measured between element midpoints)."""
    if dim == 2:
        ej, ei = np.meshgrid(np.arange(nely), np.arange(nelx), indexing="ij")
        return np.stack([ei.ravel() + 0.5, ej.ravel() + 0.5], axis=1).astype(np.float64)
    ek, ej, ei = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx), indexing="ij")
    return np.stack([ei.ravel() + 0.5, ej.ravel() + 0.5, ek.ravel() + 0.5], axis=1).astype(np.float64)


def node_coords(dim, nelx, nely, nelz=0):
    if dim == 2:
        j, i = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel()], axis=1).astype(np.float64)
    k, j, i = np.meshgrid(np.arange(nelz + 1), np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
