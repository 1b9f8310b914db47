"""Thin ctypes binding of libtopo.so (C-ABI declared in include/topo.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA
kernels.  Arrays may be NumPy arrays (host) or CUDA torch tensors (device); the
binding passes their pointers through.  If the library has not been built the
import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libtopo.so")

TP_OK, TP_ERR_ARG, TP_ERR_CUDA, TP_ERR_OOM, TP_ERR_NOT_CONVERGED, TP_ERR_BREAKDOWN, TP_ERR_TIMEOUT, \
    TP_ERR_STATE = range(8)
STATUS_NAMES = ["TP_OK", "TP_ERR_ARG", "TP_ERR_CUDA", "TP_ERR_OOM", "TP_ERR_NOT_CONVERGED",
                "TP_ERR_BREAKDOWN", "TP_ERR_TIMEOUT", "TP_ERR_STATE"]
TP_PREC_F64, TP_PREC_MIXED, TP_PREC_DW = 0, 1, 2
TP_WARM_ZERO, TP_WARM_PREVIOUS, TP_WARM_USER = 0, 1, 2
TP_FILTER_SENSITIVITY = 0
TP_FILTER_DENSITY = 1
TP_FILTER_HELMHOLTZ = 2
TP_PRECOND_JACOBI = 0
TP_PRECOND_MG = 1
TP_PRECOND_MG_FUSED = 2
TP_RHO, TP_U, TP_DC, TP_DCF, TP_CE, TP_RHO_PHYS = range(6)


class tp_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelx", C.c_int), ("nely", C.c_int), ("nelz", C.c_int),
                ("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double), ("penal", C.c_double),
                ("volfrac", C.c_double), ("rmin", C.c_double), ("move", C.c_double),
                ("dmin", C.c_double), ("n_cases", C.c_int)]


class tp_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_it", C.c_int), ("precision", C.c_int),
                ("warm_start", C.c_int), ("update_drop", C.c_double), ("warm_max_rel", C.c_double),
                ("precond", C.c_int)]


class tp_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("updates", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("rel_res", C.c_double * 8), ("ms", C.c_double), ("rel_res_init", C.c_double * 8),
                ("warm_fallback", C.c_int)]


class tp_batch_info(C.Structure):
    _fields_ = [("max_iters", C.c_int), ("updates", C.c_int), ("converged", C.c_int), ("graph", C.c_int),
                ("tile_rows", C.c_int), ("ctas", C.c_int), ("max_rel_res", C.c_double), ("ms", C.c_double)]


class tp_step_info(C.Structure):
    _fields_ = [("solve", tp_solve_info), ("compliance", C.c_double), ("lambda_", C.c_double),
                ("volume", C.c_double), ("change", C.c_double), ("oc_passes", C.c_int), ("oc_root", C.c_int)]


class tp_p1_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nelx", C.c_int), ("nely", C.c_int), ("nelz", C.c_int), ("diagonal", C.c_int),
                ("lam", C.c_double), ("mu", C.c_double), ("Emin", C.c_double), ("penal", C.c_double),
                ("volfrac", C.c_double), ("rmin", C.c_double), ("move", C.c_double), ("dmin", C.c_double),
                ("n_cases", C.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sigs = {
        "tp_create_problem": (C.c_int, [C.POINTER(tp_params), P, C.POINTER(P)]),
        "tp_destroy_problem": (None, [P]),
        "tp_last_error": (C.c_char_p, [P]),
        "tp_launch_count": (C.c_longlong, [P]),
        "tp_set_fixed": (C.c_int, [P, P]),
        "tp_set_loads": (C.c_int, [P, P]),
        "tp_set_passive": (C.c_int, [P, P]),
        "tp_set_density": (C.c_int, [P, P, C.c_int]),
        "tp_solve": (C.c_int, [P, C.POINTER(tp_solve_opts), C.POINTER(tp_solve_info)]),
        "tp_sensitivities": (C.c_int, [P, C.POINTER(C.c_double)]),
        "tp_filter": (C.c_int, [P, C.c_int]),
        "tp_set_filter_mode": (C.c_int, [P, C.c_int]),
        "tp_oc_update": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "tp_simp_step": (C.c_int, [P, C.POINTER(tp_solve_opts), C.POINTER(tp_step_info)]),
        "tp_get": (C.c_int, [P, C.c_int, P, C.c_int]),
        "tp_set": (C.c_int, [P, C.c_int, P, C.c_int]),
        "tp_matvec": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int]),
        "tp_set_trace": (C.c_int, [P, C.c_int]),
        "tp_set_wait_budget": (C.c_int, [P, C.c_longlong]),
        "tp_batch_create": (C.c_int, [C.c_int, C.POINTER(tp_params), P, C.POINTER(P)]),
        "tp_batch_destroy": (None, [P]),
        "tp_batch_last_error": (C.c_char_p, [P]),
        "tp_batch_set_fixed": (C.c_int, [P, C.c_int, P]),
        "tp_batch_set_loads": (C.c_int, [P, C.c_int, P]),
        "tp_batch_set_density": (C.c_int, [P, C.c_int, P]),
        "tp_batch_set_tiles": (C.c_int, [P, C.c_int, C.c_int]),
        "tp_batch_autotune": (C.c_int, [P, C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "tp_batch_step": (C.c_int, [P, C.POINTER(tp_solve_opts), C.POINTER(tp_batch_info), P]),
        "tp_batch_get": (C.c_int, [P, C.c_int, C.c_int, P, P]),
        "tp_batch_launch_count": (C.c_longlong, [P]),
        "tp_oc_update_noalloc": (C.c_int, [P, P, P, C.c_longlong, C.c_double, C.c_double, C.c_double, P, P,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "tp_spd_inverse_f32": (C.c_int, [P, P, C.c_int, P]),
        "tp_p1_shape_matrices": (C.c_int, [C.c_int, C.c_double, C.c_double, P, P]),
        "tp_p1_filter_stencil": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_int, P, P, P,
                                           C.POINTER(C.c_int)]),
        "tp_p1_matvec": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, P, P, P, P, C.c_int, P]),
        "tp_p1_create": (C.c_int, [C.POINTER(tp_p1_params), P, C.POINTER(P)]),
        "tp_p1_destroy": (None, [P]),
        "tp_p1_last_error": (C.c_char_p, [P]),
        "tp_p1_launch_count": (C.c_longlong, [P]),
        "tp_p1_set_fixed": (C.c_int, [P, P]),
        "tp_p1_set_loads": (C.c_int, [P, P]),
        "tp_p1_set_passive": (C.c_int, [P, P]),
        "tp_p1_set_density": (C.c_int, [P, P, C.c_int]),
        "tp_p1_solve": (C.c_int, [P, C.POINTER(tp_solve_opts), C.POINTER(tp_solve_info)]),
        "tp_p1_sensitivities": (C.c_int, [P, C.POINTER(C.c_double)]),
        "tp_p1_filter": (C.c_int, [P]),
        "tp_p1_oc_update": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "tp_p1_simp_step": (C.c_int, [P, C.POINTER(tp_solve_opts), C.POINTER(tp_step_info)]),
        "tp_p1_apply": (C.c_int, [P, P, P, C.c_int]),
        "tp_p1_get": (C.c_int, [P, C.c_int, P, C.c_int]),
        "tp_p1_set": (C.c_int, [P, C.c_int, P, C.c_int]),
        "tp_get_trace": (C.c_int, [P, P]),
        "tp_set_profile": (C.c_int, [P, C.c_int]),
        "tp_get_profile": (C.c_int, [P, P]),
        "tpnn_create": (C.c_int, [C.c_int, C.c_int, P, P, C.POINTER(P)]),
        "tpnn_destroy": (None, [P]),
        "tpnn_last_error": (C.c_char_p, [P]),
        "tpnn_param_count": (C.c_longlong, [P]),
        "tpnn_info": (C.c_int, [P, P, P, P]),
        "tpnn_set_params": (C.c_int, [P, P]),
        "tpnn_get_params": (C.c_int, [P, P]),
        "tpnn_get_grads": (C.c_int, [P, P]),
        "tpnn_forward": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P]),
        "tpnn_backward": (C.c_int, [P, P]),
        "tpnn_zero_grad": (C.c_int, [P]),
        "tpnn_adam": (C.c_int, [P, C.c_float, C.c_float, C.c_float, C.c_float]),
        "tpnn_mse": (C.c_int, [P, P, P, C.c_longlong, P, C.POINTER(C.c_double)]),
        "tpnn_train_step": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                      C.POINTER(C.c_double)]),
        "tpnn_features": (C.c_int, [P, P]),
        "tpnn_targets": (C.c_int, [P, P]),
        "tpnn_energy_grad": (C.c_int, [P, P, P, P, P]),
        "tp_warm_start_nn": (C.c_int, [P, P, P, P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# Every name the header declares (checked by the CPU test suite).
EXPORTED = ["tp_create_problem", "tp_destroy_problem", "tp_last_error", "tp_launch_count", "tp_set_fixed",
            "tp_set_loads", "tp_set_passive", "tp_set_density", "tp_solve", "tp_sensitivities", "tp_filter",
            "tp_oc_update", "tp_simp_step", "tp_get", "tp_set", "tp_matvec", "tp_set_trace", "tp_get_trace", "tp_set_wait_budget",
            "tp_oc_update_noalloc", "tp_spd_inverse_f32", "tp_p1_matvec", "tp_p1_shape_matrices", "tp_p1_filter_stencil",
            "tp_p1_create", "tp_p1_destroy", "tp_p1_last_error", "tp_p1_launch_count", "tp_p1_set_fixed",
            "tp_p1_set_loads", "tp_p1_set_passive", "tp_p1_set_density", "tp_p1_solve", "tp_p1_sensitivities",
            "tp_p1_filter", "tp_p1_oc_update", "tp_p1_simp_step", "tp_p1_apply", "tp_p1_get", "tp_p1_set", "tp_set_filter_mode", "tp_set_profile", "tp_get_profile", "tp_batch_create", "tp_batch_destroy", "tp_batch_last_error",
            "tp_batch_set_fixed", "tp_batch_set_loads", "tp_batch_set_density", "tp_batch_set_tiles",
            "tp_batch_autotune", "tp_batch_step", "tp_batch_get", "tp_batch_launch_count",
            "tpnn_create", "tpnn_destroy", "tpnn_last_error", "tpnn_param_count", "tpnn_info",
            "tpnn_set_params", "tpnn_get_params", "tpnn_get_grads", "tpnn_forward", "tpnn_backward",
            "tpnn_zero_grad", "tpnn_adam", "tpnn_mse", "tpnn_train_step", "tpnn_features", "tpnn_targets", "tpnn_energy_grad",
            "tp_warm_start_nn"]
TPNN_FEATURES = 8
NOALLOC_MAX_ELEMENTS = 1048576
SPD_INVERSE_MAX_N = 16384


def _stream_handle(stream):
    """cudaStream_t of `stream` as an int: a torch.cuda.Stream (its
    cuda_stream), a raw handle, or None for torch's current stream on the
    current device (the legacy default stream, 0, when CUDA is unavailable)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return 0
    cs = getattr(stream, "cuda_stream", None)
    return int(cs if cs is not None else stream)


def _device_tensors(*specs):
    """Pointers of tensors the C-ABI reads or writes as device memory of the
    current device.  specs: (tensor, name, dtype, numel).  Every tensor's type,
    dtype, contiguity and element count is checked first, then that each is a
    CUDA tensor on the current device.  A mismatch raises (the library would
    otherwise read or write out of bounds)."""
    import torch
    for t, name, dtype, numel in specs:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: a torch tensor is required, got {type(t).__name__}")
        if t.dtype != dtype:
            raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: the tensor must be contiguous")
        if t.numel() != numel:
            raise ValueError(f"{name}: {t.numel()} elements, expected {numel}")
    for t, name, _, _ in specs:
        if not t.is_cuda:
            raise ValueError(f"{name}: a CUDA tensor is required")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name}: on {t.device}, but the current device is cuda:{torch.cuda.current_device()}")
    return [C.c_void_p(t.data_ptr()) for t, _, _, _ in specs]


def oc_update_noalloc(rho, dcf, rho_new, volfrac, move=0.2, dmin=1e-3, passive=None, stream=None):
    """Allocation-free OC update on device tensors (see tp_oc_update_noalloc in
    include/topo.h).  rho, dcf, rho_new: contiguous CUDA float64 tensors of n_el
    elements on the current device; passive: CUDA int8 tensor of n_el elements
    or None.  stream: torch.cuda.Stream, raw handle, or None for torch's current
    stream.  Returns (lambda, volume, change)."""
    import torch
    n = rho.numel() if isinstance(rho, torch.Tensor) else -1
    specs = [(rho, "rho", torch.float64, n), (dcf, "dcf", torch.float64, n), (rho_new, "rho_new", torch.float64, n)]
    if passive is not None:
        specs.append((passive, "passive", torch.int8, n))
    ptrs = _device_tensors(*specs)
    pr, pd, po = ptrs[:3]
    pp = ptrs[3] if passive is not None else None
    lam, vol, ch = C.c_double(), C.c_double(), C.c_double()
    st = lib.tp_oc_update_noalloc(pr, pd, pp, n, volfrac, move, dmin, po, C.c_void_p(_stream_handle(stream)),
                                  C.byref(lam), C.byref(vol), C.byref(ch))
    if st != TP_OK:
        raise TopoError(st, "tp_oc_update_noalloc failed")
    return lam.value, vol.value, ch.value


def spd_inverse(a, stream=None):
    """Inverse of a symmetric positive definite matrix in FP32 by the library's
    dense blocked sweep (tp_spd_inverse_f32 in include/topo.h; the multigrid
    coarsest-level solve).  a: (n, n) NumPy array, read as float32 (upper
    triangle).  Returns the (n, n) float32 inverse."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("a must be square")
    out = np.empty_like(a)
    st = lib.tp_spd_inverse_f32(a.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p), a.shape[0],
                                C.c_void_p(_stream_handle(stream)))
    if st != TP_OK:
        raise TopoError(st, "tp_spd_inverse_f32 failed")
    return out


P1_DIAGONALS = {"right": 0, "left": 1, "right/left": 2, "kuhn": 0}


def p1_matvec(dim, nelx, nely, nelz, diagonal, lam, mu, Emin, penal, rho, fixed, u, y, stream=None):
    """y = K(rho) u for the paper's P1 cells (tp_p1_matvec in include/topo.h).
    rho (float64, one per cell), fixed (uint8, n_dof), u and y (float64,
    [ncases, n_dof] or [n_dof]): contiguous CUDA tensors on the current device;
    diagonal: "right", "left", "right/left" (2D) or "kuhn" (3D)."""
    import torch
    nn = (nelx + 1) * (nely + 1) * ((nelz + 1) if dim == 3 else 1)
    n_dof = dim * nn
    n_cells = (2 * nelx * nely) if dim == 2 else 6 * nelx * nely * nelz
    if not isinstance(u, torch.Tensor) or u.dim() not in (1, 2):
        raise ValueError("u: a 1D or 2D torch tensor is required")
    nc = u.shape[0] if u.dim() == 2 else 1
    pu, py, pr, pf = _device_tensors((u, "u", torch.float64, nc * n_dof), (y, "y", torch.float64, nc * n_dof),
                                     (rho, "rho", torch.float64, n_cells), (fixed, "fixed", torch.uint8, n_dof))
    st = lib.tp_p1_matvec(dim, nelx, nely, nelz, P1_DIAGONALS[diagonal], lam, mu, Emin, penal,
                          pr, pf, pu, py, nc, C.c_void_p(_stream_handle(stream)))
    if st != TP_OK:
        raise TopoError(st, "tp_p1_matvec failed")
    return y


def p1_shape_matrices(dim, lam, mu):
    """(K[ntypes, nd, nd], offsets[ntypes, dim + 1, dim]) of the P1 cell
    shapes (tp_p1_shape_matrices in include/topo.h); host only."""
    nt, nd = (4, 6) if dim == 2 else (6, 12)
    K = np.zeros((nt, nd, nd))
    off = np.zeros((nt, dim + 1, dim), dtype=np.int32)
    st = lib.tp_p1_shape_matrices(dim, lam, mu, K.ctypes.data_as(C.c_void_p), off.ctypes.data_as(C.c_void_p))
    if st != TP_OK:
        raise TopoError(st, "tp_p1_shape_matrices failed")
    return K, off


def p1_filter_stencil(dim, diagonal, rmin, cap=65536):
    """(count[ntypes], entries[n, 4], weights[n]) of the P1 midpoint filter
    (tp_p1_filter_stencil in include/topo.h); host only."""
    nt = 4 if dim == 2 else 6
    count = np.zeros(nt, dtype=np.int32)
    ent = np.zeros((cap, 4), dtype=np.int32)
    w = np.zeros(cap)
    n = C.c_int()
    st = lib.tp_p1_filter_stencil(dim, P1_DIAGONALS[diagonal], rmin, cap, count.ctypes.data_as(C.c_void_p),
                                  ent.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p), C.byref(n))
    if st != TP_OK:
        raise TopoError(st, "tp_p1_filter_stencil failed")
    return count, ent[:n.value].copy(), w[:n.value].copy()


class TopoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _ptr(a):
    """(pointer, on_device) of a NumPy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p), 0
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def make_params(dim, nelx, nely, nelz=0, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0, volfrac=0.5, rmin=1.5,
                move=0.2, dmin=1e-3, n_cases=1):
    return tp_params(dim, nelx, nely, nelz, E0, Emin, nu, penal, volfrac, rmin, move, dmin, n_cases)


def solve_opts(tol=1e-8, max_it=20000, precision=TP_PREC_MIXED, warm_start=TP_WARM_ZERO, update_drop=1e-2,
               warm_max_rel=0.0, precond=0):
    return tp_solve_opts(tol, max_it, precision, warm_start, update_drop, warm_max_rel, precond)


class Problem:
    """Owns a tp_problem handle.  Method names follow the C-ABI."""

    def __init__(self, params: tp_params, stream=None):
        h = C.c_void_p()
        s = C.c_void_p(_stream_handle(stream))
        st = lib.tp_create_problem(C.byref(params), s, C.byref(h))
        if st != TP_OK:
            raise TopoError(st, "tp_create_problem rejected the parameters")
        self.h = h
        self.params = params
        self.dim = params.dim
        nz = (params.nelz + 1) if params.dim == 3 else 1
        self.n_nodes = (params.nelx + 1) * (params.nely + 1) * nz
        self.n_dof = self.dim * self.n_nodes
        self.n_el = params.nelx * params.nely * (params.nelz if params.dim == 3 else 1)
        self.n_cases = params.n_cases

    @classmethod
    def from_workload(cls, w, stream=None):
        """Create and configure from a `workloads.Problem` (fixed DOFs, loads,
        passive mask, initial density)."""
        prm = make_params(w.dim, w.nelx, w.nely, w.nelz, w.E0, w.Emin, w.nu, w.penal, w.volfrac, w.rmin,
                          w.move, w.dmin, w.n_cases)
        p = cls(prm, stream)
        p.set_fixed(w.fixed)
        p.set_loads(w.loads)
        if w.passive is not None:
            p.set_passive(w.passive)
        p.set_density(w.initial_density())
        return p

    def close(self):
        if getattr(self, "h", None):
            lib.tp_destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != TP_OK:
            raise TopoError(st, lib.tp_last_error(self.h).decode())

    def last_error(self):
        return lib.tp_last_error(self.h).decode()

    def launch_count(self):
        return int(lib.tp_launch_count(self.h))

    def set_trace(self, enable=True):
        self._check(lib.tp_set_trace(self.h, 1 if enable else 0))

    def set_wait_budget(self, cycles=0):
        """Grid-barrier wait limit in SM cycles (0 = the default, about 1 s)."""
        self._check(lib.tp_set_wait_budget(self.h, int(cycles)))

    def get_trace(self):
        out = np.zeros((32, 8), dtype=np.int64)
        self._check(lib.tp_get_trace(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_profile(self, enable=True):
        self._check(lib.tp_set_profile(self.h, 1 if enable else 0))

    def get_profile(self):
        """(timed multigrid launches -- finest-level sweeps, or persistent
        segments with TP_PRECOND_MG_FUSED -- their total ms, their total
        algorithmic bytes, levels)."""
        out = np.zeros(4)
        self._check(lib.tp_get_profile(self.h, out.ctypes.data_as(C.c_void_p)))
        return int(out[0]), float(out[1]), float(out[2]), int(out[3])

    def set_fixed(self, fixed):
        a = np.ascontiguousarray(fixed, dtype=np.uint8)
        assert a.size == self.n_dof
        self._check(lib.tp_set_fixed(self.h, a.ctypes.data_as(C.c_void_p)))

    def set_loads(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64)
        assert a.size == self.n_cases * self.n_dof
        self._check(lib.tp_set_loads(self.h, a.ctypes.data_as(C.c_void_p)))

    def set_passive(self, passive):
        a = np.ascontiguousarray(passive, dtype=np.int8)
        assert a.size == self.n_el
        self._check(lib.tp_set_passive(self.h, a.ctypes.data_as(C.c_void_p)))

    def set_density(self, rho):
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64)
        ptr, dev = _ptr(rho)
        self._check(lib.tp_set_density(self.h, ptr, dev))

    def solve(self, opts: tp_solve_opts, check=True):
        info = tp_solve_info()
        st = lib.tp_solve(self.h, C.byref(opts), C.byref(info))
        if check:
            self._check(st)
        return info

    def sensitivities(self):
        c = C.c_double()
        self._check(lib.tp_sensitivities(self.h, C.byref(c)))
        return c.value

    def filter(self, mode=None):
        self._check(lib.tp_filter(self.h, getattr(self, "filter_mode", TP_FILTER_SENSITIVITY) if mode is None else mode))

    def set_filter_mode(self, mode):
        self._check(lib.tp_set_filter_mode(self.h, mode))
        self.filter_mode = mode

    def oc_update(self):
        lam, vol, ch = C.c_double(), C.c_double(), C.c_double()
        self._check(lib.tp_oc_update(self.h, C.byref(lam), C.byref(vol), C.byref(ch)))
        return lam.value, vol.value, ch.value

    def simp_step(self, opts: tp_solve_opts, check=True):
        info = tp_step_info()
        st = lib.tp_simp_step(self.h, C.byref(opts), C.byref(info))
        if check:
            self._check(st)
        return info

    def _size(self, what):
        return self.n_cases * self.n_dof if what == TP_U else self.n_el

    def get(self, what, out=None):
        if out is None:
            out = np.empty(self._size(what), dtype=np.float64)
        ptr, dev = _ptr(out)
        self._check(lib.tp_get(self.h, what, ptr, dev))
        return out

    def set(self, what, src):
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.float64)
        ptr, dev = _ptr(src)
        self._check(lib.tp_set(self.h, what, ptr, dev))

    def features(self, out):
        """Network input of every load case into `out` (CUDA bfloat16 tensor
        [n_cases, 8, nelz, nely, nelx])."""
        self._check(lib.tpnn_features(self.h, _dev_ptr(out, 2, self.n_cases * TPNN_FEATURES * self.n_el)))
        return out

    def targets(self, out):
        """Normalised element means of the current displacement into `out` (CUDA
        bfloat16 tensor [n_cases, 3, nelz, nely, nelx])."""
        self._check(lib.tpnn_targets(self.h, _dev_ptr(out, 2, self.n_cases * 3 * self.n_el)))
        return out

    def energy_grad(self, y, comp, gy):
        """Relative energy error of the scaled, node-averaged prediction y (CUDA
        float32 [n_cases, 3, nelz, nely, nelx]) and its gradient into gy.
        comp: the solution's compliance per case.  Returns the losses."""
        cm = np.ascontiguousarray(np.atleast_1d(comp), np.float64)
        loss = np.zeros(self.n_cases)
        n = self.n_cases * 3 * self.n_el
        self._check(lib.tpnn_energy_grad(self.h, _dev_ptr(y, 4, n), cm.ctypes.data_as(C.c_void_p),
                                         _dev_ptr(gy, 4, n), loss.ctypes.data_as(C.c_void_p)))
        return loss

    def warm_start_nn(self, net):
        """Store alpha * u^ from the network as the start of the next solve with
        warm_start=TP_WARM_USER.  Returns (alpha per case, device ms)."""
        alpha = np.zeros(self.n_cases)
        ms = C.c_double()
        self._check(lib.tp_warm_start_nn(self.h, net.h, alpha.ctypes.data_as(C.c_void_p), C.byref(ms)))
        return alpha, ms.value

    def matvec(self, u, precision=TP_PREC_F64, ncopies=1, out=None):
        if isinstance(u, np.ndarray):
            dt = np.float32 if precision == TP_PREC_MIXED else np.float64
            u = np.ascontiguousarray(u, dtype=dt)
            if out is None:
                out = np.empty_like(u)
        ptr_u, dev = _ptr(u)
        ptr_y, dev2 = _ptr(out)
        assert dev == dev2
        self._check(lib.tp_matvec(self.h, ptr_u, ptr_y, precision, ncopies, dev))
        return out


class P1Problem:
    """Owns a tp_p1_problem handle: the SIMP loop on the paper's own P1 cells
    (triangles / Kuhn tetrahedra).  Method names follow the C-ABI."""

    def __init__(self, params: tp_p1_params, stream=None):
        h = C.c_void_p()
        st = lib.tp_p1_create(C.byref(params), C.c_void_p(_stream_handle(stream)), C.byref(h))
        if st != TP_OK:
            raise TopoError(st, "tp_p1_create rejected the parameters")
        self.h = h
        self.params = params
        self.dim = params.dim
        nz = (params.nelz + 1) if params.dim == 3 else 1
        self.n_nodes = (params.nelx + 1) * (params.nely + 1) * nz
        self.n_dof = self.dim * self.n_nodes
        self.n_el = (2 * params.nelx * params.nely if params.dim == 2
                     else 6 * params.nelx * params.nely * params.nelz)
        self.n_cases = params.n_cases

    @classmethod
    def from_workload(cls, w, stream=None):
        """Create and configure from a `workloads.SimplexProblem`."""
        prm = tp_p1_params(w.dim, w.nelx, w.nely, w.nelz if w.dim == 3 else 0, P1_DIAGONALS[w.diagonal],
                           w.lam, w.mu, w.Emin, w.penal, w.volfrac, w.rmin, w.move, w.dmin, w.n_cases)
        p = cls(prm, stream)
        p.set_fixed(w.fixed)
        p.set_loads(w.loads)
        if w.passive is not None:
            p.set_passive(w.passive)
        p.set_density(w.initial_density())
        return p

    def close(self):
        if getattr(self, "h", None):
            lib.tp_p1_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != TP_OK:
            raise TopoError(st, lib.tp_p1_last_error(self.h).decode())

    def launch_count(self):
        return int(lib.tp_p1_launch_count(self.h))

    def set_fixed(self, fixed):
        a = np.ascontiguousarray(fixed, dtype=np.uint8)
        if a.size != self.n_dof:
            raise ValueError(f"fixed: {a.size} entries, expected {self.n_dof}")
        self._check(lib.tp_p1_set_fixed(self.h, a.ctypes.data_as(C.c_void_p)))

    def set_loads(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64)
        if a.size != self.n_cases * self.n_dof:
            raise ValueError(f"loads: {a.size} entries, expected {self.n_cases * self.n_dof}")
        self._check(lib.tp_p1_set_loads(self.h, a.ctypes.data_as(C.c_void_p)))

    def set_passive(self, passive):
        a = np.ascontiguousarray(passive, dtype=np.int8)
        if a.size != self.n_el:
            raise ValueError(f"passive: {a.size} entries, expected {self.n_el}")
        self._check(lib.tp_p1_set_passive(self.h, a.ctypes.data_as(C.c_void_p)))

    def _sized(self, a, n, name):
        """a as a contiguous float64 array (NumPy) or the float64 tensor itself,
        after checking its element count."""
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float64)
            size = a.size
        else:
            import torch
            if not isinstance(a, torch.Tensor) or a.dtype != torch.float64:
                raise ValueError(f"{name}: a float64 NumPy array or torch tensor is required")
            size = a.numel()
        if size != n:
            raise ValueError(f"{name}: {size} entries, expected {n}")
        return a

    def set_density(self, rho):
        rho = self._sized(rho, self.n_el, "rho")
        ptr, dev = _ptr(rho)
        self._check(lib.tp_p1_set_density(self.h, ptr, dev))

    def solve(self, opts: tp_solve_opts, check=True):
        info = tp_solve_info()
        st = lib.tp_p1_solve(self.h, C.byref(opts), C.byref(info))
        if check:
            self._check(st)
        return info

    def sensitivities(self):
        c = C.c_double()
        self._check(lib.tp_p1_sensitivities(self.h, C.byref(c)))
        return c.value

    def filter(self):
        self._check(lib.tp_p1_filter(self.h))

    def oc_update(self):
        lam, vol, ch = C.c_double(), C.c_double(), C.c_double()
        self._check(lib.tp_p1_oc_update(self.h, C.byref(lam), C.byref(vol), C.byref(ch)))
        return lam.value, vol.value, ch.value

    def simp_step(self, opts: tp_solve_opts, check=True):
        info = tp_step_info()
        st = lib.tp_p1_simp_step(self.h, C.byref(opts), C.byref(info))
        if check:
            self._check(st)
        return info

    def _size(self, what):
        return self.n_cases * self.n_dof if what == TP_U else self.n_el

    def get(self, what, out=None):
        if out is None:
            out = np.empty(self._size(what), dtype=np.float64)
        out = self._sized(out, self._size(what), "out") if isinstance(out, np.ndarray) else out
        ptr, dev = _ptr(out)
        self._check(lib.tp_p1_get(self.h, what, ptr, dev))
        return out

    def set(self, what, src):
        src = self._sized(src, self._size(what), "src")
        ptr, dev = _ptr(src)
        self._check(lib.tp_p1_set(self.h, what, ptr, dev))

    def apply(self, u, out=None):
        """y = K(rho) u for all cases (u [n_cases * n_dof], float64)."""
        u = self._sized(u, self.n_cases * self.n_dof, "u")
        if out is None:
            out = np.empty_like(u) if isinstance(u, np.ndarray) else u.new_empty(u.shape)
        out = self._sized(out, self.n_cases * self.n_dof, "out")
        pu, dev = _ptr(u)
        py, dev2 = _ptr(out)
        if dev != dev2:
            raise ValueError("u and out must both be host or both be device memory")
        self._check(lib.tp_p1_apply(self.h, pu, py, dev))
        return out


class Batch:
    """Owns a tp_batch handle (independent 2D problems solved together)."""

    def __init__(self, workloads_list, stream=None):
        n = len(workloads_list)
        arr = (tp_params * n)(*[make_params(w.dim, w.nelx, w.nely, w.nelz, w.E0, w.Emin, w.nu, w.penal,
                                             w.volfrac, w.rmin, w.move, w.dmin, w.n_cases)
                                 for w in workloads_list])
        h = C.c_void_p()
        st = lib.tp_batch_create(n, arr, C.c_void_p(_stream_handle(stream)), C.byref(h))
        if st != TP_OK:
            raise TopoError(st, "tp_batch_create rejected the parameters")
        self.h = h
        self.n = n
        self.w = list(workloads_list)
        for i, w in enumerate(self.w):
            self._check(lib.tp_batch_set_fixed(h, i, np.ascontiguousarray(w.fixed, np.uint8).ctypes.data_as(C.c_void_p)))
            self._check(lib.tp_batch_set_loads(h, i, np.ascontiguousarray(w.loads[0], np.float64).ctypes.data_as(C.c_void_p)))

    def _check(self, st):
        if st != TP_OK:
            raise TopoError(st, lib.tp_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib.tp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_density(self, i, rho):
        a = np.ascontiguousarray(rho, np.float64)
        self._check(lib.tp_batch_set_density(self.h, i, a.ctypes.data_as(C.c_void_p)))

    def set_tiles(self, tile_rows, ctas_per_sm):
        self._check(lib.tp_batch_set_tiles(self.h, tile_rows, ctas_per_sm))

    def autotune(self, cache_path=None):
        ty, cps = C.c_int(), C.c_int()
        self._check(lib.tp_batch_autotune(self.h, None if cache_path is None else cache_path.encode(),
                                          C.byref(ty), C.byref(cps)))
        return ty.value, cps.value

    def step(self, opts, check=True):
        info = tp_batch_info()
        comp = np.zeros(self.n)
        st = lib.tp_batch_step(self.h, C.byref(opts), C.byref(info), comp.ctypes.data_as(C.c_void_p))
        if check:
            self._check(st)
        return info, comp

    def get(self, i, what):
        w = self.w[i]
        size = 2 * w.n_nodes if what == TP_U else w.n_el
        out = np.empty(size)
        sc = np.empty(6)
        self._check(lib.tp_batch_get(self.h, i, what, out.ctypes.data_as(C.c_void_p), sc.ctypes.data_as(C.c_void_p)))
        return out, sc

    def launch_count(self):
        return int(lib.tp_batch_launch_count(self.h))


def _dev_ptr(t, itemsize, numel):
    """Device pointer of a contiguous CUDA tensor with the expected size."""
    ptr, dev = _ptr(t)
    if not dev:
        raise ValueError("a CUDA tensor is required")
    if t.numel() != numel or t.element_size() != itemsize:
        raise ValueError(f"expected {numel} elements of {itemsize} bytes, got {t.numel()} of {t.element_size()}")
    return ptr


def layer_shapes(c_in=TPNN_FEATURES, c_out=3, widths=(16, 32, 64, 64)):
    """(c_out, c_in) of the 11 convolutions in network order."""
    c0, c1, c2, c3 = widths
    return [(c0, c_in), (c0, c0), (c1, c0), (c1, c1), (c2, c1), (c2, c2), (c3, c2), (c1, c3), (c0, c1),
            (c0, c0), (c_out, c0)]


def pack_params(params):
    """[(w[co][ci][27], b[co])] -> the packed FP32 vector of the C-ABI."""
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for w, b in params]).astype(np.float32)


def unpack_params(flat, shapes):
    out, o = [], 0
    for co, ci in shapes:
        nw = co * ci * 27
        out.append((np.asarray(flat[o:o + nw], np.float64).reshape(co, ci, 27),
                    np.asarray(flat[o + nw:o + nw + co], np.float64)))
        o += nw + co
    assert o == len(flat)
    return out


class Net:
    """Owns a tpnn handle: the warm-start U-Net with hand-written BF16/FP32
    kernels.  Tensor arguments are CUDA tensors (bfloat16 inputs/targets,
    float32 outputs/gradients) on the network's stream."""

    def __init__(self, c_in=TPNN_FEATURES, widths=(16, 32, 64, 64), stream=None):
        h = C.c_void_p()
        wd = (C.c_int * 4)(*widths)
        st = lib.tpnn_create(c_in, 3, wd, C.c_void_p(_stream_handle(stream)), C.byref(h))
        if st != TP_OK:
            raise TopoError(st, "tpnn_create rejected the configuration")
        self.h = h
        self.c_in = c_in
        self.widths = tuple(widths)
        self.shapes = layer_shapes(c_in, 3, widths)
        self.n_params = int(lib.tpnn_param_count(h))

    def _check(self, st):
        if st != TP_OK:
            raise TopoError(st, lib.tpnn_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib.tpnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        flat = params if isinstance(params, np.ndarray) else pack_params(params)
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.n_params
        self._check(lib.tpnn_set_params(self.h, flat.ctypes.data_as(C.c_void_p)))

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        self._check(lib.tpnn_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def get_grads(self):
        out = np.empty(self.n_params, np.float32)
        self._check(lib.tpnn_get_grads(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, x, y):
        n, c, D, H, W = x.shape
        assert c == self.c_in
        self._check(lib.tpnn_forward(self.h, _dev_ptr(x, 2, x.numel()), n, D, H, W,
                                     _dev_ptr(y, 4, n * 3 * D * H * W)))
        return y

    def backward(self, gy):
        self._check(lib.tpnn_backward(self.h, _dev_ptr(gy, 4, gy.numel())))

    def zero_grad(self):
        self._check(lib.tpnn_zero_grad(self.h))

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(lib.tpnn_adam(self.h, lr, beta1, beta2, eps))

    def mse(self, y, t, gy):
        loss = C.c_double()
        self._check(lib.tpnn_mse(self.h, _dev_ptr(y, 4, y.numel()), _dev_ptr(t, 2, y.numel()), y.numel(),
                                 _dev_ptr(gy, 4, y.numel()), C.byref(loss)))
        return loss.value

    def train_step(self, x, t, lr):
        n, c, D, H, W = x.shape
        loss = C.c_double()
        self._check(lib.tpnn_train_step(self.h, _dev_ptr(x, 2, x.numel()), _dev_ptr(t, 2, n * 3 * D * H * W),
                                        n, D, H, W, lr, C.byref(loss)))
        return loss.value

    def save(self, path):
        np.savez(path, params=self.get_params(), widths=np.array(self.widths), c_in=self.c_in)

    @classmethod
    def load(cls, path, stream=None):
        d = np.load(path)
        net = cls(int(d["c_in"]), tuple(int(v) for v in d["widths"]), stream)
        net.set_params(d["params"])
        return net
