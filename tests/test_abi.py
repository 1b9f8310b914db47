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
