"""ctypes front end of the oracle's C quadrature (test infrastructure only).

Builds ``nl_quad.c`` with gcc on first use (or through ``build_oracle()``) into
``oracle/_build``.  Every function returns FP64 numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_quad.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    src = os.path.join(_HERE, "nl_quad.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int64), ("xy", C.c_void_p), ("n_elems", C.c_int64),
                ("elems", C.c_void_p), ("node_dir", C.c_void_p), ("elem_dir", C.c_void_p)]


class _Kernel(C.Structure):
    _fields_ = [("type", C.c_int), ("delta", C.c_double), ("s", C.c_double), ("c", C.c_double), ("ball", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle())
            lib.oracle_pair_matrix.restype = C.c_int
            lib.oracle_pair_matrix.argtypes = [C.POINTER(_Mesh), C.POINTER(_Kernel), C.c_int64, C.c_int64,
                                               C.c_void_p, C.c_void_p]
            lib.oracle_point_integral.restype = C.c_int
            lib.oracle_point_integral.argtypes = [C.POINTER(_Mesh), C.POINTER(_Kernel), C.c_int64, C.c_int64,
                                                  C.c_double, C.c_double, C.c_void_p, C.c_void_p]
            lib.oracle_assemble.restype = C.c_int
            lib.oracle_assemble.argtypes = [C.POINTER(_Mesh), C.POINTER(_Kernel), C.c_void_p, C.c_int, C.c_int,
                                            C.c_void_p,
                                            C.c_int64, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_int]
            lib.oracle_assemble_rows.restype = C.c_int
            lib.oracle_assemble_rows.argtypes = [C.POINTER(_Mesh), C.POINTER(_Kernel), C.c_void_p, C.c_int64,
                                                 C.c_void_p, C.c_int]
            _lib = lib
    return _lib


def _threads(n):
    if n is not None:
        return int(n)
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


class _Ctx:
    """Keeps the numpy buffers alive for the duration of a C call."""

    def __init__(self, mesh, kernel, scale):
        self.xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self.el = np.ascontiguousarray(mesh.elems, dtype=np.int32)
        self.nd = np.ascontiguousarray(mesh.node_is_dirichlet, dtype=np.int8)
        self.ed = np.ascontiguousarray(mesh.elem_is_dirichlet, dtype=np.int8)
        self.m = _Mesh(mesh.dim, mesh.n_nodes, self.xy.ctypes.data, mesh.n_elems, self.el.ctypes.data,
                       self.nd.ctypes.data, self.ed.ctypes.data)
        self.k = _Kernel(kernel.type, kernel.delta, kernel.s, scale, int(getattr(kernel, "ball", 0)))


def pair_matrix(mesh, kernel, scale, e, ep):
    """Local matrix of the ordered element pair (E=e outer, E'=ep inner) and its node list."""
    if not (0 <= e < mesh.n_elems and 0 <= ep < mesh.n_elems):
        raise IndexError("element index out of range")
    lib = _load()
    ctx = _Ctx(mesh, kernel, scale)
    nc = kernel.ncomp
    out = np.zeros((12 * 12,), dtype=np.float64)
    nodes = np.zeros(6, dtype=np.int32)
    nl = lib.oracle_pair_matrix(C.byref(ctx.m), C.byref(ctx.k), int(e), int(ep), out.ctypes.data,
                                nodes.ctypes.data)
    ld = nl * nc
    return out[: ld * ld].reshape(ld, ld).copy(), nodes[:nl].copy()


def point_integral(mesh, kernel, scale, e, ep, x):
    """Inner integral of the ordered pair (E=e, E'=ep) at an arbitrary outer point x (2-D)."""
    if not (0 <= e < mesh.n_elems and 0 <= ep < mesh.n_elems):
        raise IndexError("element index out of range")
    lib = _load()
    ctx = _Ctx(mesh, kernel, scale)
    nc = kernel.ncomp
    out = np.zeros((12 * 12,), dtype=np.float64)
    nodes = np.zeros(6, dtype=np.int32)
    nl = lib.oracle_point_integral(C.byref(ctx.m), C.byref(ctx.k), int(e), int(ep), float(x[0]), float(x[1]),
                                   out.ctypes.data, nodes.ctypes.data)
    ld = nl * nc
    return out[: ld * ld].reshape(ld, ld).copy(), nodes[:nl].copy()


def assemble(mesh, kernel, scale, dof_of, n_dofs, elem_mask=None, k=-1, band=None, g=None, nthreads=None,
             matrix=True):
    """Assemble the (sub)domain matrix over the dofs given by ``dof_of`` ((n_nodes*nc,) int32, -1 = none).

    Returns (A, Bg): A dense (n_dofs, n_dofs) or, with ``band=kd``, the lower band (kd+1, n_dofs);
    Bg = sum over Dirichlet columns of A_ij g_j when ``g`` is given (else None)."""
    lib = _load()
    ctx = _Ctx(mesh, kernel, scale)
    dof_of = np.ascontiguousarray(dof_of, dtype=np.int32)
    if not matrix:
        A = None
        mode, kd = 0, 0
    elif band is None:
        A = np.zeros((n_dofs, n_dofs), dtype=np.float64)
        mode, kd = 0, 0
    else:
        A = np.zeros((band + 1, n_dofs), dtype=np.float64)
        mode, kd = 1, band
    mask = None
    mask_words = 1
    if elem_mask is not None:
        mask = np.ascontiguousarray(elem_mask, dtype=np.uint64)
        if mask.ndim == 1:
            mask = mask.reshape(-1, 1)
        mask_words = mask.shape[1]
    gbuf = None
    Bg = None
    if g is not None:
        gbuf = np.ascontiguousarray(g, dtype=np.float64)
        Bg = np.zeros(n_dofs, dtype=np.float64)
    st = lib.oracle_assemble(C.byref(ctx.m), C.byref(ctx.k), None if mask is None else mask.ctypes.data,
                             int(mask_words), int(k),
                             dof_of.ctypes.data, int(n_dofs), mode, int(kd), None if A is None else A.ctypes.data,
                             None if gbuf is None else gbuf.ctypes.data, None if Bg is None else Bg.ctypes.data,
                             _threads(nthreads))
    if st != 0:
        raise RuntimeError("band overflow in oracle assembly")
    return A, Bg


def assemble_rows(mesh, kernel, scale, rows, nthreads=None):
    """Full rows (all n_nodes*nc columns, Dirichlet columns included) of the single-domain matrix."""
    lib = _load()
    ctx = _Ctx(mesh, kernel, scale)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= mesh.n_nodes * kernel.ncomp):
        raise IndexError("row index out of range")
    ncols = mesh.n_nodes * kernel.ncomp
    out = np.zeros((rows.size, ncols), dtype=np.float64)
    lib.oracle_assemble_rows(C.byref(ctx.m), C.byref(ctx.k), rows.ctypes.data, rows.size, out.ctypes.data,
                             _threads(nthreads))
    return out
