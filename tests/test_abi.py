"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU and
exports every entry point that include/topo.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tp[a-z]*_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2012_08208_gb300 import topo
    return topo


def test_library_exports_every_declared_symbol(lib):
    names = _declared("topo.h") + _declared("topo_nn.h")
    assert len(names) >= 15
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(names) <= set(lib.EXPORTED)


def test_create_rejects_bad_params_without_touching_the_gpu(lib):
    import ctypes as C
    h = C.c_void_p()
    for bad in [lib.make_params(4, 10, 5), lib.make_params(2, 0, 5), lib.make_params(2, 10, 5, volfrac=0.0),
                lib.make_params(2, 10, 5, rmin=-1.0), lib.make_params(2, 10, 5, n_cases=9),
                lib.make_params(2, 10, 5, nu=0.5)]:
        assert lib.lib.tp_create_problem(C.byref(bad), None, C.byref(h)) == lib.TP_ERR_ARG


@pytest.mark.parametrize("dim", [2, 3])
def test_p1_shape_matrices_match_the_oracle(lib, dim):
    """Host arithmetic of the P1 operator (tp_p1_shape_matrices, no device
    work): each cell shape's unit matrix equals the oracle's element matrix of
    the same simplex, and the shapes are the oracle's cells of one square
    ("right" then "left" cut) or one cube (Kuhn order)."""
    import numpy as np
    import workloads as W
    from oracle import p1
    lam, mu = 0.6, 0.4
    K, off = lib.p1_shape_matrices(dim, lam, mu)
    for t in range(K.shape[0]):
        ref = p1.cell_stiffness(off[t].astype(float), lam, mu)
        assert np.allclose(K[t], ref, rtol=1e-13, atol=1e-14)
    if dim == 2:
        probs = [(W.p1_cantilever2d(1, 1, diagonal=d), 2 * i) for i, d in enumerate(["right", "left"])]
    else:
        probs = [(W.p1_cantilever3d(1, 1, 1), 0)]
    for prob, t0 in probs:
        X = p1.node_coords(dim, 1, 1, 1 if dim == 3 else 0).astype(int)
        for c, cell in enumerate(p1.cells(prob)):
            got = {tuple(v) for v in off[t0 + c]}
            assert got == {tuple(X[n]) for n in cell}
    with pytest.raises(lib.TopoError):
        lib.p1_shape_matrices(dim, lam, -1.0)


def test_dense_and_p1_entry_points_reject_bad_arguments_without_the_gpu(lib):
    """Argument checks of tp_spd_inverse_f32 and tp_p1_matvec return
    TP_ERR_ARG before any CUDA call (so they run without a GPU)."""
    import ctypes as C
    import numpy as np
    buf = np.zeros(64)
    p = buf.ctypes.data_as(C.c_void_p)
    f = lib.lib.tp_spd_inverse_f32
    assert f(p, p, 0, None) == lib.TP_ERR_ARG
    assert f(p, p, lib.SPD_INVERSE_MAX_N + 1, None) == lib.TP_ERR_ARG
    assert f(None, p, 4, None) == lib.TP_ERR_ARG and f(p, None, 4, None) == lib.TP_ERR_ARG
    g = lib.lib.tp_p1_matvec
    ok = (0.6, 0.4, 1e-9, 3.0)
    assert g(1, 2, 2, 0, 0, *ok, p, p, p, p, 1, None) == lib.TP_ERR_ARG        # dim
    assert g(2, 0, 2, 0, 0, *ok, p, p, p, p, 1, None) == lib.TP_ERR_ARG        # nelx
    assert g(2, 2, 2, 1, 0, *ok, p, p, p, p, 1, None) == lib.TP_ERR_ARG        # nelz in 2D
    assert g(3, 2, 2, 0, 0, *ok, p, p, p, p, 1, None) == lib.TP_ERR_ARG        # nelz in 3D
    assert g(2, 2, 2, 0, 3, *ok, p, p, p, p, 1, None) == lib.TP_ERR_ARG        # diagonal
    assert g(2, 2, 2, 0, 0, 0.6, 0.0, 1e-9, 3.0, p, p, p, p, 1, None) == lib.TP_ERR_ARG  # mu
    assert g(2, 2, 2, 0, 0, -1.0, 0.4, 1e-9, 3.0, p, p, p, p, 1, None) == lib.TP_ERR_ARG  # lambda + mu
    assert g(2, 2, 2, 0, 0, 0.6, 0.4, 1.0, 3.0, p, p, p, p, 1, None) == lib.TP_ERR_ARG   # Emin
    assert g(2, 2, 2, 0, 0, 0.6, 0.4, 1e-9, 0.5, p, p, p, p, 1, None) == lib.TP_ERR_ARG  # penal
    assert g(2, 2, 2, 0, 0, *ok, p, p, p, p, 0, None) == lib.TP_ERR_ARG        # ncases
    assert g(2, 2, 2, 0, 0, *ok, None, p, p, p, 1, None) == lib.TP_ERR_ARG     # NULL rho


@pytest.mark.parametrize("dim,diagonal,rmin", [(2, "right", 1.5), (2, "left", 2.5), (2, "right/left", 1.5),
                                               (2, "right/left", 3.0), (3, "kuhn", 1.5), (3, "kuhn", 2.0)])
def test_p1_filter_stencil_rebuilds_the_oracle_weights(lib, dim, diagonal, rmin):
    """The host stencil of the P1 midpoint filter (tp_p1_filter_stencil), laid
    over a small grid with neighbours outside it skipped, gives exactly the
    oracle's paper-literal dense weight matrix."""
    import numpy as np
    import workloads as W
    from oracle import p1
    if dim == 2:
        prob = W.p1_cantilever2d(7, 6, diagonal=diagonal, rmin=rmin)
    else:
        prob = W.p1_cantilever3d(4, 3, 3, rmin=rmin)
    count, ent, w = lib.p1_filter_stencil(dim, diagonal, rmin)
    nx, ny, nz = prob.nelx, prob.nely, max(prob.nelz, 1)
    nc = 2 if dim == 2 else 6
    starts = np.concatenate([[0], np.cumsum(count)])
    Wg = np.zeros((prob.n_el, prob.n_el))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                for l0 in range(nc):
                    if dim == 2:
                        cut = {"right": 0, "left": 1}.get(diagonal, j % 2)
                        t = 2 * cut + l0
                    else:
                        t = l0
                    for q in range(starts[t], starts[t + 1]):
                        dx, dy, dz, l = ent[q]
                        i2, j2, k2 = i + dx, j + dy, k + dz
                        if not (0 <= i2 < nx and 0 <= j2 < ny and 0 <= k2 < nz):
                            continue
                        e2 = i2 + nx * (j2 + ny * k2)
                        Wg[nc * e + l0, nc * e2 + l] = w[q]
    assert np.allclose(Wg, p1.dense_weights(prob), rtol=0, atol=1e-13)


def test_binding_rejects_bad_tensors_before_the_library(lib):
    """The device-pointer wrappers (oc_update_noalloc, p1_matvec) check each
    tensor's dtype, contiguity, element count and device before any call, so a
    wrong tensor raises instead of letting a kernel read or write out of
    bounds.  CPU tensors reach only the checks (no device work)."""
    import torch
    n = 100
    good = torch.zeros(n, dtype=torch.float64)
    with pytest.raises(ValueError, match="dtype"):
        lib.oc_update_noalloc(good, torch.zeros(n, dtype=torch.float32), good.clone(), 0.5)
    with pytest.raises(ValueError, match="elements"):
        lib.oc_update_noalloc(good, torch.zeros(n - 1, dtype=torch.float64), good.clone(), 0.5)
    with pytest.raises(ValueError, match="contiguous"):
        lib.oc_update_noalloc(good, torch.zeros(2 * n, dtype=torch.float64)[::2], good.clone(), 0.5)
    with pytest.raises(ValueError, match="dtype"):
        lib.oc_update_noalloc(good, good.clone(), good.clone(), 0.5, passive=torch.zeros(n, dtype=torch.uint8))
    with pytest.raises(ValueError, match="CUDA"):
        lib.oc_update_noalloc(good, good.clone(), good.clone(), 0.5)
    with pytest.raises(TypeError):
        lib.oc_update_noalloc(good.numpy(), good, good, 0.5)
    # P1 operator on a 3 x 2 grid "right": 6 cells, 12 nodes, 24 DOFs
    rho = torch.full((12,), 0.5, dtype=torch.float64)
    fixed = torch.zeros(24, dtype=torch.uint8)
    u = torch.zeros((2, 24), dtype=torch.float64)
    y = torch.zeros((2, 24), dtype=torch.float64)
    args = (2, 3, 2, 0, "right", 0.6, 0.4, 1e-9, 3.0)
    with pytest.raises(ValueError, match="elements"):
        lib.p1_matvec(*args, rho[:6], fixed, u, y)                       # one density per cell
    with pytest.raises(ValueError, match="elements"):
        lib.p1_matvec(*args, rho, fixed, u, y[:1])                       # y shorter than u
    with pytest.raises(ValueError, match="dtype"):
        lib.p1_matvec(*args, rho, fixed.to(torch.int32), u, y)
    with pytest.raises(ValueError, match="dtype"):
        lib.p1_matvec(*args, rho, fixed, u.float(), y)
    with pytest.raises(ValueError, match="CUDA"):
        lib.p1_matvec(*args, rho, fixed, u, y)


def test_stream_argument_forms(lib):
    """A stream may be given as None, a raw handle or an object with a
    cuda_stream attribute (torch.cuda.Stream)."""
    class FakeStream:
        cuda_stream = 12345
    assert lib._stream_handle(FakeStream()) == 12345
    assert lib._stream_handle(678) == 678
    assert isinstance(lib._stream_handle(None), int)


def test_p1_create_rejects_bad_params_without_the_gpu(lib):
    """tp_p1_create validates its parameters before any CUDA call."""
    import ctypes as C
    h = C.c_void_p()
    good = dict(dim=2, nelx=6, nely=3, nelz=0, diagonal=2, lam=0.6, mu=0.4, Emin=1e-9, penal=3.0, volfrac=0.5,
                rmin=1.5, move=0.2, dmin=1e-3, n_cases=1)
    for k, v in [("dim", 4), ("nelx", 0), ("nelz", 2), ("diagonal", 3), ("mu", 0.0), ("Emin", 0.0), ("penal", 0.5),
                 ("volfrac", 0.0), ("rmin", 5.0), ("move", 0.0), ("dmin", 1.0), ("n_cases", 9)]:
        prm = dict(good, **{k: v})
        args = lib.tp_p1_params(*[prm[f] for f, _ in lib.tp_p1_params._fields_])
        assert lib.lib.tp_p1_create(C.byref(args), None, C.byref(h)) == lib.TP_ERR_ARG, k
    three = dict(good, dim=3, nelz=0, diagonal=0)
    args = lib.tp_p1_params(*[three[f] for f, _ in lib.tp_p1_params._fields_])
    assert lib.lib.tp_p1_create(C.byref(args), None, C.byref(h)) == lib.TP_ERR_ARG
