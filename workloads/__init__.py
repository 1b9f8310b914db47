"""Seeded synthetic problem data shared by the oracle, the tests and the benchmark.

This module holds problem *data* only: grid sizes, material constants, boundary
masks, load vectors, passive-element masks and seeded random fields.  It contains
none of the method's arithmetic (no stiffness, no solve, no filter, no OC update),
so both the CPU oracle and the CUDA path may draw their inputs from it.

Numbering used for every array produced here:
  node (i, j[, k])   -> i + (nelx+1) * (j + (nely+1) * k)      (x fastest)
  element (i, j[, k]) -> i + nelx * (j + nely * k)
  DOF                -> dim * node + component   (component 0=x, 1=y, 2=z)

The problems follow the paper's examples (Section 4 "FEniCS implementation" and
Section 5 "Model extensions": cantilever, MBB-type roller supports, several load
cases, a passive hole, the 3D cantilever) on structured grids of unit Q4/H8
elements with point or line loads.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Problem:
    """One topology-optimisation problem instance (inputs only)."""

    name: str
    dim: int
    nelx: int
    nely: int
    nelz: int  # 0 in 2D
    volfrac: float
    rmin: float
    fixed: np.ndarray  # uint8[n_dof], 1 = Dirichlet DOF (u = 0)
    loads: np.ndarray  # float64[n_cases, n_dof]
    passive: Optional[np.ndarray] = None  # int8[n_el], 1 = void held at dmin
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    penal: float = 3.0
    move: float = 0.2
    dmin: float = 1e-3
    n_iter: int = 50
    tol: float = 1e-10
    precision: str = "f64"  # "f64" or "mixed"
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        n = (self.nelx + 1) * (self.nely + 1)
        return n * (self.nelz + 1) if self.dim == 3 else n

    @property
    def n_el(self) -> int:
        n = self.nelx * self.nely
        return n * self.nelz if self.dim == 3 else n

    @property
    def n_dof(self) -> int:
        return self.dim * self.n_nodes

    @property
    def n_cases(self) -> int:
        return int(self.loads.shape[0])

    def passive_mask(self) -> np.ndarray:
        if self.passive is None:
            return np.zeros(self.n_el, dtype=np.int8)
        return self.passive

    def initial_density(self) -> np.ndarray:
        """Uniform volfrac start (the paper initialises density to volfrac);
        passive elements start at dmin."""
        rho = np.full(self.n_el, self.volfrac, dtype=np.float64)
        rho[self.passive_mask() == 1] = self.dmin
        return rho


def node_id(p: Problem, i, j, k=0):
    return i + (p.nelx + 1) * (j + (p.nely + 1) * k)


def _empty(dim, nelx, nely, nelz, n_cases):
    nn = (nelx + 1) * (nely + 1) * ((nelz + 1) if dim == 3 else 1)
    return np.zeros(dim * nn, dtype=np.uint8), np.zeros((n_cases, dim * nn), dtype=np.float64)


def _fix_face_x0(fixed, dim, nelx, nely, nelz):
    """Clamp every DOF of the nodes on the plane x = 0."""
    ks = range(nelz + 1) if dim == 3 else [0]
    for k in ks:
        for j in range(nely + 1):
            n = (nelx + 1) * (j + (nely + 1) * k)
            fixed[dim * n: dim * n + dim] = 1


def mbb2d(nelx: int = 60, nely: int = 20) -> Problem:
    """MBB half-beam: symmetry rollers (u_x = 0) on the left edge, a roller
    (u_y = 0) at the bottom-right node, unit downward load at the top-left node."""
    fixed, f = _empty(2, nelx, nely, 0, 1)
    for j in range(nely + 1):
        fixed[2 * ((nelx + 1) * j) + 0] = 1
    fixed[2 * nelx + 1] = 1  # node (nelx, 0), y component
    f[0, 2 * ((nelx + 1) * nely) + 1] = -1.0  # node (0, nely), y component
    return Problem("mbb2d", 2, nelx, nely, 0, volfrac=0.5, rmin=1.5, fixed=fixed,
                   loads=f, n_iter=50, tol=1e-10, precision="f64")


def cantilever2d(nelx: int = 600, nely: int = 200, disk_r: float = 40.0,
                 disk_c=(150.0, 100.0)) -> Problem:
    """2D cantilever, left edge clamped, three load cases: unit downward point
    loads at the mid-right, top-right and bottom-right nodes, with a passive void
    disk (element centre inside the closed disk)."""
    fixed, f = _empty(2, nelx, nely, 0, 3)
    _fix_face_x0(fixed, 2, nelx, nely, 0)
    for c, j in enumerate((nely // 2, nely, 0)):
        f[c, 2 * (nelx + (nelx + 1) * j) + 1] = -1.0
    ex = np.arange(nelx) + 0.5
    ey = np.arange(nely) + 0.5
    X, Y = np.meshgrid(ex, ey)  # shape (nely, nelx): x fastest after ravel
    passive = (((X - disk_c[0]) ** 2 + (Y - disk_c[1]) ** 2) <= disk_r ** 2).astype(np.int8).ravel()
    if disk_r <= 0:
        passive[:] = 0
    return Problem("cantilever2d", 2, nelx, nely, 0, volfrac=0.4, rmin=3.0, fixed=fixed,
                   loads=f, passive=passive, n_iter=50, tol=1e-8, precision="mixed")


def cantilever3d(nelx: int = 120, nely: int = 40, nelz: int = 40, volfrac: float = 0.12,
                 rmin: float = 1.5, n_iter: int = 30, tol: float = 1e-6) -> Problem:
    """3D cantilever: x = 0 face clamped, unit line load (downward, -y) along the
    bottom edge (y = 0) of the x = nelx face.  The line load of intensity 1 is
    lumped consistently: -1 at interior edge nodes and -0.5 at the two end nodes."""
    fixed, f = _empty(3, nelx, nely, nelz, 1)
    _fix_face_x0(fixed, 3, nelx, nely, nelz)
    for k in range(nelz + 1):
        n = nelx + (nelx + 1) * (0 + (nely + 1) * k)
        f[0, 3 * n + 1] = -0.5 if k in (0, nelz) else -1.0
    return Problem("cantilever3d", 3, nelx, nely, nelz, volfrac=volfrac, rmin=rmin,
                   fixed=fixed, loads=f, n_iter=n_iter, tol=tol, precision="mixed")


def cantilever3d_large() -> Problem:
    """240 x 80 x 80 H8 cantilever (about 4.7M DOFs)."""
    return cantilever3d(240, 80, 80, volfrac=0.1, rmin=2.0, n_iter=30, tol=1e-6)


def batch2d(n: int = 64, seed: int = 0, w_range=(40, 320)) -> list:
    """Uneven batch of 2D cantilevers.  Per instance, in this draw order:
    width w ~ uniform even integer in [w_lo, w_hi], height h = w / 2, load node
    row j ~ uniform integer in [0, h] on the right edge (unit downward load),
    volfrac ~ U(0.3, 0.6).  Left edge clamped, rmin = 1.5."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = w_range[0] // 2, w_range[1] // 2
    for b in range(n):
        w = 2 * int(rng.integers(lo, hi + 1))
        h = w // 2
        j = int(rng.integers(0, h + 1))
        vf = float(rng.uniform(0.3, 0.6))
        fixed, f = _empty(2, w, h, 0, 1)
        _fix_face_x0(fixed, 2, w, h, 0)
        f[0, 2 * (w + (w + 1) * j) + 1] = -1.0
        out.append(Problem(f"batch{b}", 2, w, h, 0, volfrac=vf, rmin=1.5, fixed=fixed,
                           loads=f, n_iter=50, tol=1e-6, precision="mixed",
                           extra={"load_row": j}))
    return out


def small2d(nelx: int, nely: int, n_cases: int = 1, rmin: float = 1.5, volfrac: float = 0.5,
            passive_disk=None, seed: int = 3) -> Problem:
    """Small clamped-left 2D cantilever for parity tests on ragged grids; loads are
    seeded random nodal forces on the right edge (one vector per case)."""
    rng = np.random.default_rng(seed)
    fixed, f = _empty(2, nelx, nely, 0, n_cases)
    _fix_face_x0(fixed, 2, nelx, nely, 0)
    for c in range(n_cases):
        for j in range(nely + 1):
            n = nelx + (nelx + 1) * j
            f[c, 2 * n: 2 * n + 2] = rng.normal(size=2)
    passive = None
    if passive_disk is not None:
        (cx, cy, r) = passive_disk
        ex = np.arange(nelx) + 0.5
        ey = np.arange(nely) + 0.5
        X, Y = np.meshgrid(ex, ey)
        passive = (((X - cx) ** 2 + (Y - cy) ** 2) <= r * r).astype(np.int8).ravel()
    return Problem(f"small2d_{nelx}x{nely}", 2, nelx, nely, 0, volfrac=volfrac, rmin=rmin,
                   fixed=fixed, loads=f, passive=passive, n_iter=10, tol=1e-12, precision="f64")


def small3d(nelx: int, nely: int, nelz: int, n_cases: int = 1, rmin: float = 1.5,
            volfrac: float = 0.3, seed: int = 4) -> Problem:
    """Small clamped-x0 3D cantilever with seeded random nodal forces on the
    x = nelx face."""
    rng = np.random.default_rng(seed)
    fixed, f = _empty(3, nelx, nely, nelz, n_cases)
    _fix_face_x0(fixed, 3, nelx, nely, nelz)
    for c in range(n_cases):
        for k in range(nelz + 1):
            for j in range(nely + 1):
                n = nelx + (nelx + 1) * (j + (nely + 1) * k)
                f[c, 3 * n: 3 * n + 3] = rng.normal(size=3)
    return Problem(f"small3d_{nelx}x{nely}x{nelz}", 3, nelx, nely, nelz, volfrac=volfrac,
                   rmin=rmin, fixed=fixed, loads=f, n_iter=10, tol=1e-12, precision="f64")


def warmstart3d(nelx: int, nely: int, nelz: int, seed: int) -> Problem:
    """Seeded 3D cantilever variant for the warm-start network's training
    trajectories (x = 0 face clamped).  Draw order: volfrac ~ U(0.08, 0.3),
    rmin ~ U(1.2, 2.5), load kind (0 full line load along z on the bottom edge
    of the x = nelx face, as in the 3D cantilever; 1 a line segment of that edge;
    2 a point load on it), the segment or point position, then 0 to 2 passive
    boxes (void), each with corner and extent uniform over the inner domain.
    Loads act in -y with unit intensity (line loads lumped as in cantilever3d)."""
    rng = np.random.default_rng(seed)
    vf = float(rng.uniform(0.08, 0.3))
    rmin = float(rng.uniform(1.2, 2.5))
    kind = int(rng.integers(0, 3))
    fixed, f = _empty(3, nelx, nely, nelz, 1)
    _fix_face_x0(fixed, 3, nelx, nely, nelz)
    if kind == 0:
        k0, k1 = 0, nelz
    elif kind == 1:
        a, b = sorted(int(v) for v in rng.integers(0, nelz + 1, size=2))
        k0, k1 = a, max(b, a + 1)
    else:
        k0 = k1 = int(rng.integers(0, nelz + 1))
    for k in range(k0, k1 + 1):
        n = nelx + (nelx + 1) * (0 + (nely + 1) * k)
        f[0, 3 * n + 1] = -1.0 if k0 == k1 else (-0.5 if k in (k0, k1) else -1.0)
    passive = np.zeros(nelx * nely * nelz, dtype=np.int8)
    ek, ej, ei = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx), indexing="ij")
    for _ in range(int(rng.integers(0, 3))):
        lo = rng.uniform([0.2, 0.1, 0.1], [0.7, 0.6, 0.6]) * np.array([nelx, nely, nelz])
        ext = rng.uniform(0.1, 0.3, size=3) * np.array([nelx, nely, nelz])
        box = ((ei + 0.5 >= lo[0]) & (ei + 0.5 <= lo[0] + ext[0]) & (ej + 0.5 >= lo[1]) &
               (ej + 0.5 <= lo[1] + ext[1]) & (ek + 0.5 >= lo[2]) & (ek + 0.5 <= lo[2] + ext[2]))
        passive[box.ravel()] = 1
    return Problem(f"warmstart3d_{nelx}x{nely}x{nelz}_s{seed}", 3, nelx, nely, nelz, volfrac=vf, rmin=rmin,
                   fixed=fixed, loads=f, passive=passive if passive.any() else None, n_iter=30, tol=1e-6,
                   precision="mixed", extra={"load_kind": kind, "k0": k0, "k1": k1})


def random_density(n_el: int, seed: int = 1, lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    """rho ~ U(lo, hi), seeded."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n_el)


def random_vector(n: int, seed: int = 2) -> np.ndarray:
    """u ~ N(0, 1), seeded."""
    return np.random.default_rng(seed).normal(size=n)


def random_sensitivity(n_el: int, seed: int = 5) -> np.ndarray:
    """Negative sensitivities dc ~ -U(1e-4, 1) * 10^U(-2, 2) (spread over decades)."""
    rng = np.random.default_rng(seed)
    return -rng.uniform(1e-4, 1.0, size=n_el) * 10.0 ** rng.uniform(-2, 2, size=n_el)


@dataclass
class SimplexProblem:
    """A problem on the paper's own elements (inputs only): the structured grid
    of unit squares (cubes) with each square split into 2 triangles along the
    diagonal pattern `diagonal` ("right", "left" or "right/left"), each cube into
    6 tetrahedra, vector P1 displacements and one density per cell.  Nodes and
    DOFs are numbered as for the Q4 / H8 problems; cells are numbered
    (2 or 6) * (element of the square / cube) + local cell.  The material is
    given by its Lame constants (the paper: mu = 0.4, lambda = 0.6), which set
    sigma = 2 mu eps + lambda tr(eps) I in 2D and 3D alike."""

    name: str
    dim: int
    nelx: int
    nely: int
    nelz: int
    diagonal: str
    volfrac: float
    rmin: float
    fixed: np.ndarray  # uint8[n_dof]
    loads: np.ndarray  # float64[n_cases, n_dof]
    passive: Optional[np.ndarray] = None  # int8[n_el] (cells)
    lam: float = 0.6
    mu: float = 0.4
    Emin: float = 1e-9
    penal: float = 3.0
    move: float = 0.2
    dmin: float = 1e-3
    n_iter: int = 50

    @property
    def n_nodes(self) -> int:
        n = (self.nelx + 1) * (self.nely + 1)
        return n * (self.nelz + 1) if self.dim == 3 else n

    @property
    def n_el(self) -> int:
        """Number of cells (triangles or tetrahedra)."""
        return 2 * self.nelx * self.nely if self.dim == 2 else 6 * self.nelx * self.nely * self.nelz

    @property
    def n_dof(self) -> int:
        return self.dim * self.n_nodes

    @property
    def n_cases(self) -> int:
        return int(self.loads.shape[0])

    def passive_mask(self) -> np.ndarray:
        return np.zeros(self.n_el, dtype=np.int8) if self.passive is None else self.passive

    def initial_density(self) -> np.ndarray:
        rho = np.full(self.n_el, self.volfrac, dtype=np.float64)
        rho[self.passive_mask() == 1] = self.dmin
        return rho


def p1_cantilever2d(nelx: int = 60, nely: int = 20, volfrac: float = 0.5, rmin: float = 1.5,
                    diagonal: str = "right/left", n_iter: int = 50) -> SimplexProblem:
    """The paper's 2D cantilever on its own mesh: x = 0 clamped; a downward
    traction of unit intensity on the right edge x = nelx over y in [0, 2] (the
    facets whose points all satisfy x = nelx, y <= 2).  Its consistent nodal
    loads on the linear edge segments are -0.5, -1, -0.5 at y = 0, 1, 2."""
    fixed, f = _empty(2, nelx, nely, 0, 1)
    _fix_face_x0(fixed, 2, nelx, nely, 0)
    top = min(2, nely)
    for j in range(top + 1):
        w = 0.5 if j in (0, top) else 1.0
        f[0, 2 * (nelx + (nelx + 1) * j) + 1] = -w
    return SimplexProblem(f"p1_cantilever2d_{nelx}x{nely}_{diagonal.replace('/', '')}", 2, nelx, nely, 0,
                          diagonal, volfrac, rmin, fixed, f, n_iter=n_iter)


def p1_cantilever3d(nelx: int = 60, nely: int = 20, nelz: int = 4, volfrac: float = 0.3, rmin: float = 1.5,
                    n_iter: int = 30) -> SimplexProblem:
    """The paper's 3D cantilever on tetrahedra (6 per cube): x = 0 face
    clamped, the unit downward line load along the bottom edge (y = 0) of the
    x = nelx face, lumped as -0.5 at the end nodes and -1 between."""
    fixed, f = _empty(3, nelx, nely, nelz, 1)
    _fix_face_x0(fixed, 3, nelx, nely, nelz)
    for k in range(nelz + 1):
        n = nelx + (nelx + 1) * (0 + (nely + 1) * k)
        f[0, 3 * n + 1] = -0.5 if k in (0, nelz) else -1.0
    return SimplexProblem(f"p1_cantilever3d_{nelx}x{nely}x{nelz}", 3, nelx, nely, nelz, "kuhn", volfrac, rmin,
                          fixed, f, n_iter=n_iter)


def random_spd(n: int, cond: float = 100.0, seed: int = 7) -> np.ndarray:
    """Symmetric positive definite float32 matrix Q diag(lam) Q^T: Q from the QR
    factorisation of a Gaussian matrix, lam log-uniform in [1, cond], seeded."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = cond ** rng.uniform(0.0, 1.0, size=n)
    a = (q * lam) @ q.T
    return (0.5 * (a + a.T)).astype(np.float32)


CONFIGS = {
    "mbb2d_60x20": mbb2d,
    "cantilever2d_600x200": cantilever2d,
    "cantilever3d_120x40x40": cantilever3d,
    "batch2d_64": batch2d,
    "cantilever3d_240x80x80": cantilever3d_large,
}
