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
