"""Pins of the P1 simplex oracle (oracle/p1.py): the paper's own elements
(vector P1 on RectangleMesh / BoxMesh cells, DG0 density), checked against
geometry, closed forms, two independent statements of the element matrix,
exact reproduction of affine fields, energy identities and finite differences."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import p1

LAM, MU = 0.6, 0.4  # the paper's Lame constants


def _prob2d(nx, ny, diagonal="right/left"):
    return W.p1_cantilever2d(nx, ny, diagonal=diagonal)


def _prob3d(nx, ny, nz):
    return W.p1_cantilever3d(nx, ny, nz)


def _signed_measure(V):
    M = V[1:] - V[0]
    return np.linalg.det(M) / (2.0 if V.shape[1] == 2 else 6.0)


@pytest.mark.parametrize("diagonal", ["right", "left", "right/left"])
def test_triangles_measure_orientation_conformity(diagonal):
    """Every triangle has area 1/2 with counter-clockwise vertices; the cells
    tile the rectangle conformingly: each interior edge is shared by exactly
    two cells, the boundary has 2 (nx + ny) edges, and V - E + F = 1."""
    prob = _prob2d(5, 4, diagonal)
    C = p1.cells(prob)
    X = p1.node_coords(2, 5, 4)
    areas = np.array([_signed_measure(X[c]) for c in C])
    assert np.allclose(areas, 0.5, atol=0, rtol=0)
    edges = {}
    for c in C:
        for a, b in itertools.combinations(sorted(c), 2):
            edges[(a, b)] = edges.get((a, b), 0) + 1
    counts = np.array(list(edges.values()))
    assert counts.max() == 2
    assert (counts == 1).sum() == 2 * (5 + 4)
    assert prob.n_nodes - len(edges) + len(C) == 1


def test_diagonal_patterns():
    """"right" cuts square (0, 0) along (0, 0)-(1, 1), "left" along
    (1, 0)-(0, 1); "right/left" alternates by row."""
    for diagonal, row, want in (("right", 0, "right"), ("left", 0, "left"),
                                ("right/left", 0, "right"), ("right/left", 1, "left"),
                                ("right/left", 2, "right")):
        prob = _prob2d(3, 3, diagonal)
        C = p1.cells(prob)
        e = 0 + 3 * row
        shared = set(C[2 * e]) & set(C[2 * e + 1])
        v00 = 0 + 4 * row
        diag = {v00, v00 + 5} if want == "right" else {v00 + 1, v00 + 4}
        assert shared == diag


def test_tetrahedra_kuhn():
    """Six tetrahedra of volume 1/6 per cube, positively oriented, all holding
    the cube's main diagonal; the mesh is conforming: every interior face is
    shared by two cells, the boundary has 2 triangles per boundary square, and
    V - E + F - T = 1."""
    nx, ny, nz = 3, 2, 2
    prob = _prob3d(nx, ny, nz)
    C = p1.cells(prob)
    X = p1.node_coords(3, nx, ny, nz)
    vols = np.array([_signed_measure(X[c]) for c in C])
    assert np.allclose(vols, 1.0 / 6.0, atol=1e-15)
    for e in range(nx * ny * nz):
        i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
        lo = i + (nx + 1) * (j + (ny + 1) * k)
        hi = (i + 1) + (nx + 1) * ((j + 1) + (ny + 1) * (k + 1))
        for t in range(6):
            assert lo in C[6 * e + t] and hi in C[6 * e + t]
    faces, edges = {}, set()
    for c in C:
        for f in itertools.combinations(sorted(c), 3):
            faces[f] = faces.get(f, 0) + 1
        for a, b in itertools.combinations(sorted(c), 2):
            edges.add((a, b))
    counts = np.array(list(faces.values()))
    assert counts.max() == 2
    assert (counts == 1).sum() == 2 * 2 * (nx * ny + ny * nz + nx * nz)
    assert prob.n_nodes - len(edges) + len(faces) - len(C) == 1


def _random_simplex(dim, rng):
    while True:
        V = rng.normal(size=(dim + 1, dim))
        if abs(_signed_measure(V)) > 0.2:
            return V


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrix_two_statements(dim):
    """K_e from the Voigt form |T| B^T C B equals K_e from the bilinear form in
    tensor notation; in 2D the barycentric gradients equal the textbook
    constant-strain-triangle formulas b_i / 2A, c_i / 2A."""
    rng = np.random.default_rng(dim)
    for _ in range(5):
        V = _random_simplex(dim, rng)
        K1 = p1.cell_stiffness(V, LAM, MU)
        K2 = p1.cell_stiffness_tensor(V, LAM, MU)
        assert np.allclose(K1, K2, rtol=1e-12, atol=1e-12 * np.abs(K1).max())
        if dim == 2:
            (x1, y1), (x2, y2), (x3, y3) = V
            two_a = x1 * (y2 - y3) + x2 * (y3 - y1) + x3 * (y1 - y2)
            b = np.array([y2 - y3, y3 - y1, y1 - y2]) / two_a
            c = np.array([x3 - x2, x1 - x3, x2 - x1]) / two_a
            G, meas = p1.bary_gradients(V)
            assert np.allclose(G[:, 0], b, rtol=1e-12) and np.allclose(G[:, 1], c, rtol=1e-12)
            assert meas == pytest.approx(abs(two_a) / 2, rel=1e-13)


def _rigid_modes(V):
    d = V.shape[1]
    modes = []
    for a in range(d):
        t = np.zeros_like(V)
        t[:, a] = 1.0
        modes.append(t.ravel())
    for a, b in itertools.combinations(range(d), 2):
        r = np.zeros_like(V)
        r[:, a] = -V[:, b]
        r[:, b] = V[:, a]
        modes.append(r.ravel())
    return np.array(modes)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrix_null_space_and_patch(dim):
    """Symmetric positive semidefinite with the rigid motions as exact null space
    (3 in 2D, 6 in 3D); for an affine field u = A x + t the cell energy
    u^T K_e u equals 2 |T| psi(sym A) (patch test)."""
    rng = np.random.default_rng(10 + dim)
    V = _random_simplex(dim, rng)
    K = p1.cell_stiffness(V, LAM, MU)
    assert np.allclose(K, K.T, atol=1e-13 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    nrig = 3 if dim == 2 else 6
    assert np.all(ev[:nrig] < 1e-12 * ev[-1]) and ev[nrig] > 1e-6 * ev[-1]
    for m in _rigid_modes(V):
        assert np.abs(K @ m).max() < 1e-12 * np.abs(K).max() * np.abs(m).max()
    _, meas = p1.bary_gradients(V)
    for _ in range(3):
        A = rng.normal(size=(dim, dim))
        t = rng.normal(size=dim)
        u = (V @ A.T + t).ravel()
        eps = 0.5 * (A + A.T)
        assert u @ K @ u == pytest.approx(2 * meas * p1.psi(eps, LAM, MU), rel=1e-11)


@pytest.mark.parametrize("case", ["2d_right", "2d_rightleft", "3d"])
def test_uniaxial_bar_exact(case):
    """A bar stretched by prescribed end displacements u_x = 0 on x = 0 and
    u_x = e_xx nx on x = nx, free lateral faces, with rigid motions pinned.  P1
    represents the affine solution, so the discrete solution is exactly
    u = (e_xx x, e_yy y[, e_yy z]) with e_yy / e_xx = -lambda / (lambda + 2 mu)
    (2D) or -nu (3D), and the end reaction equals sigma * area with
    sigma = 4 mu (lambda + mu) / (lambda + 2 mu) e_xx (2D) or E e_xx (3D)."""
    if case.startswith("2d"):
        prob = _prob2d(6, 3, "right" if case == "2d_right" else "right/left")
        nx, ny, nz = 6, 3, 0
        ratio = -LAM / (LAM + 2 * MU)
        stiff = 4 * MU * (LAM + MU) / (LAM + 2 * MU)
        area = ny
    else:
        prob = _prob3d(4, 2, 3)
        nx, ny, nz = 4, 2, 3
        E = MU * (3 * LAM + 2 * MU) / (LAM + MU)
        ratio = -LAM / (2 * (LAM + MU))
        stiff = E
        area = ny * nz
    dim = prob.dim
    X = p1.node_coords(dim, nx, ny, nz)
    exx = 1e-3
    exact = np.zeros((prob.n_nodes, dim))
    exact[:, 0] = exx * X[:, 0]
    for a in range(1, dim):
        exact[:, a] = ratio * exx * X[:, a]
    exact = exact.ravel()
    fixed = np.zeros(prob.n_dof, dtype=bool)
    ends = np.flatnonzero((X[:, 0] == 0) | (X[:, 0] == nx))
    fixed[dim * ends] = True
    origin = 0
    fixed[dim * origin + 1:dim * origin + dim] = True  # u_y (u_z) at the origin
    if dim == 3:
        fixed[dim * (ny * (nx + 1)) + 2] = True  # u_z at (0, ny, 0): rotation about x
    K = p1.assemble(prob, np.ones(prob.n_el))
    free = np.flatnonzero(~fixed)
    fx = np.flatnonzero(fixed)
    import scipy.sparse.linalg as spla
    u = exact.copy()
    u[free] = 0.0
    u[free] = spla.spsolve(K[free][:, free].tocsc(), -(K[free][:, fx] @ exact[fx]))
    assert np.abs(u - exact).max() < 1e-12
    reaction = K @ u
    right = np.flatnonzero(X[:, 0] == nx)
    assert reaction[dim * right].sum() == pytest.approx(stiff * exx * area, rel=1e-11)


def test_loads_and_energy_identities():
    """The paper's traction strip sums to -2 (unit traction on a strip of length 2);
    c = f^T u = u^T K u = sum_e E_e ce_e on random densities, 2D and 3D."""
    prob = _prob2d(8, 4)
    assert prob.loads[0].sum() == pytest.approx(-2.0)
    assert prob.loads[0][1::2].sum() == pytest.approx(-2.0)
    for prob in (_prob2d(8, 4), _prob2d(7, 5, "left"), _prob3d(4, 2, 2)):
        rho = W.random_density(prob.n_el, seed=4)
        K = p1.assemble(prob, rho)
        U = p1.solve(prob, rho, K)
        c, ce, dc = p1.sensitivities(prob, rho, U)
        assert c == pytest.approx(float(U[0] @ (K @ U[0])), rel=1e-10)
        assert c == pytest.approx(float(np.sum(p1.young(rho) * ce)), rel=1e-10)
        free = prob.fixed == 0
        r = (prob.loads[0] - K @ U[0])[free]
        assert np.linalg.norm(r) < 1e-10 * np.linalg.norm(prob.loads[0])


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_sensitivities_finite_differences(which):
    """dc_e = d c / d rho_e against central differences of the compliance
    (step 1e-6) on every cell of a small mesh."""
    prob = _prob2d(3, 2) if which == "2d" else _prob3d(2, 1, 1)
    rho = W.random_density(prob.n_el, seed=9, lo=0.3)

    def comp(r):
        return p1.sensitivities(prob, r, p1.solve(prob, r))[0]

    _, _, dc = p1.sensitivities(prob, rho, p1.solve(prob, rho))
    h = 1e-6
    for e in range(prob.n_el):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (comp(rp) - comp(rm)) / (2 * h)
        assert fd == pytest.approx(dc[e], rel=1e-6, abs=1e-9 * np.abs(dc).max())


def test_filter_on_cell_midpoints():
    """Midpoints of the two cells of a "right" square are (i + 2/3, j + 1/3)
    and (i + 1/3, j + 2/3); the dense (paper-literal) and k-d tree weights agree;
    a uniform density and a constant sensitivity pass the filter unchanged."""
    prob = _prob2d(9, 5, "right")
    M = p1.cell_midpoints(prob)
    assert np.allclose(M[0], [2 / 3, 1 / 3]) and np.allclose(M[1], [1 / 3, 2 / 3])
    for pr in (prob, _prob2d(9, 5), _prob3d(3, 2, 2)):
        Wd = p1.dense_weights(pr)
        Ws = p1.sparse_weights(pr).toarray()
        assert np.allclose(Wd, Ws, atol=1e-14)
        from oracle import filt
        rho = np.full(pr.n_el, 0.4)
        dc = np.full(pr.n_el, -2.5)
        assert np.allclose(filt.sensitivity_filter(p1.sparse_weights(pr), rho, dc), dc, rtol=1e-14)


def test_iteration_volume_and_bounds():
    """One SIMP iteration of the paper's cantilever on its own mesh: the new
    density meets the volume target to the bisection tolerance, stays in
    [dmin, 1] and within the move limit."""
    prob = W.p1_cantilever2d(16, 6, volfrac=0.5, rmin=1.5)
    rho = prob.initial_density()
    out = p1.iteration(prob, rho)
    rn = out["rho_new"]
    assert rn.sum() == pytest.approx(prob.volfrac * prob.n_el, rel=1e-7)
    assert rn.min() >= prob.dmin and rn.max() <= 1.0
    assert np.abs(rn - rho).max() <= prob.move + 1e-15
    assert out["c"] > 0 and np.all(out["dc"] <= 0)
