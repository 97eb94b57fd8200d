"""ctypes binding of ``libnlfeti.so`` (argument marshalling only; all computation is in the library).

The names follow the C ABI in ``include/nlfeti.h``.  PyTorch, when importable with a
CUDA device, provides the stream and the device memory (its caching allocator is
passed to ``nlfeti_create`` as the allocator callback); otherwise the library uses
``cudaMalloc`` on the legacy stream.  There is no CPU fallback: without a GPU every
constructor raises ``NlfetiError``.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

from . import build as _build

OK, E_INVALID, E_NOMEM, E_NOT_SPD, E_NOT_CONVERGED, E_TIMEOUT, E_CUDA, E_BUSY = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "OK", -1: "INVALID", -2: "NOMEM", -3: "NOT_SPD", -4: "NOT_CONVERGED", -5: "TIMEOUT",
                -6: "CUDA", -7: "BUSY"}

EXPORTED = ["nlfeti_default_options", "nlfeti_create", "nlfeti_destroy", "nlfeti_last_error", "nlfeti_problem_create",
            "nlfeti_problem_destroy", "nlfeti_problem_info", "nlfeti_problem_set_options", "nlfeti_factor",
            "nlfeti_solve", "nlfeti_solve_device", "nlfeti_get_decomposition", "nlfeti_get_operator",
            "nlfeti_apply", "nlfeti_set_profiling", "nlfeti_get_profile", "nlfeti_server_create", "nlfeti_submit",
            "nlfeti_wait", "nlfeti_server_destroy", "nlfeti_apply_schur_noalloc", "nlfeti_cg_prepare",
            "nlfeti_solve_cg", "nlfeti_solve_cg_device", "nlfeti_problem_set_matrix",
            "nlfeti_debug_apply_waits", "nlfeti_submit_mesh", "nlfeti_server_get_info",
            "nlfeti_autotune", "nlfeti_set_apply_choice"]


class NlfetiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"nlfeti {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_it", C.c_int), ("max_refine", C.c_int),
                ("inner_tol", C.c_double), ("refine_tol", C.c_double), ("batched", C.c_int),
                ("hbm_budget", C.c_size_t), ("graph_loop", C.c_int),
                ("precond_fp16", C.c_int), ("factor_tc", C.c_int), ("residual_format", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refine_sweeps", C.c_int), ("final_rel_residual", C.c_double),
                ("rel_correction", C.c_double), ("ms_setup", C.c_double), ("ms_factor", C.c_double),
                ("ms_solve", C.c_double), ("ms_queue", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("K", C.c_int32), ("ncomp", C.c_int32), ("n_floating", C.c_int32), ("n_coarse", C.c_int32),
                ("n_lambda", C.c_int64), ("n_u", C.c_int64), ("sum_nk", C.c_int64), ("sum_nk2", C.c_int64),
                ("sum_ngamma2", C.c_int64), ("max_nk", C.c_int32), ("max_ngamma", C.c_int32),
                ("residual_nnz", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("apply_launches", C.c_int64), ("apply_ms", C.c_double),
                ("apply_bytes", C.c_double), ("half_apply_launches", C.c_int64), ("half_apply_ms", C.c_double),
                ("half_apply_bytes", C.c_double)]


class ServerInfo(C.Structure):
    _fields_ = [("requests_done", C.c_int64), ("batches", C.c_int64), ("merged_requests", C.c_int64),
                ("problem_hits", C.c_int64), ("problem_misses", C.c_int64), ("problems_evicted", C.c_int64),
                ("problems_cached", C.c_int32), ("peak_active", C.c_int32), ("queued", C.c_int32),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t)]


class TuneEntry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nrhs", C.c_int32), ("rc", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("us", C.c_double), ("from_cache", C.c_int32), ("rows_per_warp", C.c_int32)]


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int64), ("xy", C.c_void_p), ("n_elems", C.c_int64),
                ("elems", C.c_void_p), ("node_is_dirichlet", C.c_void_p), ("elem_is_dirichlet", C.c_void_p)]


class Kernel(C.Structure):
    _fields_ = [("type", C.c_int), ("delta", C.c_double), ("s", C.c_double), ("scale", C.c_double), ("ball", C.c_int)]


class Decomp(C.Structure):
    _fields_ = [("K", C.c_int32), ("elem_subdomain", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building in-tree if needed) the CUDA library and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise NlfetiError(E_CUDA, f"CUDA library not built: {path}")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "nlfeti_default_options": (None, [C.POINTER(Options)]),
        "nlfeti_create": (i32, [C.POINTER(vp), C.POINTER(Options), vp, ALLOC_FN, FREE_FN, vp]),
        "nlfeti_destroy": (None, [vp]),
        "nlfeti_last_error": (C.c_char_p, [vp]),
        "nlfeti_problem_create": (i32, [vp, C.POINTER(Mesh), C.POINTER(Kernel), C.POINTER(Decomp), C.POINTER(vp)]),
        "nlfeti_problem_destroy": (None, [vp]),
        "nlfeti_problem_info": (i32, [vp, C.POINTER(Info)]),
        "nlfeti_problem_set_options": (i32, [vp, C.POINTER(Options)]),
        "nlfeti_factor": (i32, [vp, i32]),
        "nlfeti_solve": (i32, [vp, i32, i32, vp, vp, vp, C.POINTER(Stats)]),
        "nlfeti_solve_device": (i32, [vp, i32, i32, vp, vp, vp, C.POINTER(Stats)]),
        "nlfeti_cg_prepare": (i32, [vp]),
        "nlfeti_solve_cg": (i32, [vp, i32, i32, vp, vp, vp, C.POINTER(Stats)]),
        "nlfeti_solve_cg_device": (i32, [vp, i32, i32, vp, vp, vp, C.POINTER(Stats)]),
        "nlfeti_get_decomposition": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "nlfeti_get_operator": (i32, [vp, i32, i32, i32, vp]),
        "nlfeti_problem_set_matrix": (i32, [vp, i32, vp]),
        "nlfeti_debug_apply_waits": (i32, [vp, C.c_longlong, i32]),
        "nlfeti_autotune": (i32, [vp, i32, C.c_char_p, C.POINTER(TuneEntry), C.POINTER(C.c_int)]),
        "nlfeti_set_apply_choice": (i32, [vp, i32, i32, i32, i32, i32]),
        "nlfeti_apply": (i32, [vp, i32, i32, i32, vp, vp]),
        "nlfeti_set_profiling": (i32, [vp, i32]),
        "nlfeti_get_profile": (i32, [vp, C.POINTER(Profile)]),
        "nlfeti_server_create": (i32, [vp, C.c_size_t, i32, C.POINTER(vp)]),
        "nlfeti_submit": (i32, [vp, vp, i32, i32, vp, vp, C.POINTER(C.c_uint64)]),
        "nlfeti_wait": (i32, [vp, C.c_uint64, i32, vp, C.POINTER(Stats)]),
        "nlfeti_server_destroy": (None, [vp]),
        "nlfeti_submit_mesh": (i32, [vp, C.POINTER(Mesh), C.POINTER(Kernel), C.POINTER(Decomp), C.POINTER(Options),
                                     i32, i32, vp, vp, C.POINTER(C.c_uint64)]),
        "nlfeti_server_get_info": (i32, [vp, C.POINTER(ServerInfo)]),
        "nlfeti_apply_schur_noalloc": (i32, [vp, i32, i32, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_options(**kw) -> Options:
    lib = load()
    o = Options()
    lib.nlfeti_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    return None if a is None else a.ctypes.data


class Context:
    """A library context bound to torch's current CUDA stream and caching allocator."""

    def __init__(self, options: Options | None = None, use_torch: bool = True, alloc_filter=None):
        """alloc_filter(nbytes) -> bool, optional: when it returns False the allocator callback
        returns NULL for that request (the library then reports NLFETI_E_NOMEM)."""
        self.lib = load()
        self._keep = []
        stream = None
        alloc, free = ALLOC_FN(), FREE_FN()
        if use_torch:
            try:
                import torch
                if torch.cuda.is_available():
                    dev = torch.cuda.current_device()
                    s = torch.cuda.current_stream()
                    stream = s.cuda_stream

                    def _alloc(n, user):
                        if alloc_filter is not None and not alloc_filter(int(n)):
                            return None
                        return torch.cuda.caching_allocator_alloc(int(n), dev, s)

                    def _free(p, user):
                        torch.cuda.caching_allocator_delete(int(p))

                    alloc, free = ALLOC_FN(_alloc), FREE_FN(_free)
            except ImportError:
                pass
        self._keep += [alloc, free]
        h = C.c_void_p()
        st = self.lib.nlfeti_create(C.byref(h), C.byref(options) if options else None, stream, alloc, free, None)
        if st != OK:
            raise NlfetiError(st, "cannot create a context (no CUDA device or driver?)")
        self.h = h

    def check(self, st):
        if st != OK:
            raise NlfetiError(st, self.lib.nlfeti_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None):
            self.lib.nlfeti_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter shutdown torch (whose allocator frees our device memory) may already be
        # torn down; the process exit releases everything, so nothing is done then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """A nonlocal FETI problem: setup and GPU assembly on construction."""

    def __init__(self, ctx: Context, dim, xy, elems, node_is_dirichlet, elem_is_dirichlet, kernel_type, delta, s,
                 scale, labels, K, ball=0):
        self.ctx = ctx
        lib = ctx.lib
        self._xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._el = np.ascontiguousarray(elems, dtype=np.int32)
        self._nd = np.ascontiguousarray(node_is_dirichlet, dtype=np.int8)
        self._ed = np.ascontiguousarray(elem_is_dirichlet, dtype=np.int8)
        self._lab = np.ascontiguousarray(labels, dtype=np.int32)
        mesh = Mesh(dim, self._nd.size, self._xy.ctypes.data, self._ed.size, self._el.ctypes.data,
                    self._nd.ctypes.data, self._ed.ctypes.data)
        kern = Kernel(int(kernel_type), float(delta), float(s), float(scale), int(ball))
        dec = Decomp(int(K), self._lab.ctypes.data)
        h = C.c_void_p()
        ctx.check(lib.nlfeti_problem_create(ctx.h, C.byref(mesh), C.byref(kern), C.byref(dec), C.byref(h)))
        self.h = h
        self.n_nodes = self._nd.size
        inf = self.info()
        self.ncomp = inf["ncomp"]
        self.n_dofs = self.n_nodes * self.ncomp

    @classmethod
    def from_workload(cls, ctx, w):
        m, k = w.mesh, w.kernel
        return cls(ctx, m.dim, m.xy, m.elems, m.node_is_dirichlet, m.elem_is_dirichlet, k.type, k.delta, k.s,
                   k.scale, w.labels, w.K, getattr(k, "ball", 0))

    def info(self):
        i = Info()
        self.ctx.check(self.ctx.lib.nlfeti_problem_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def set_options(self, opt: Options):
        self.ctx.check(self.ctx.lib.nlfeti_problem_set_options(self.h, C.byref(opt)))

    def factor(self, mask: int = 1):
        self.ctx.check(self.ctx.lib.nlfeti_factor(self.h, int(mask)))

    def solve(self, rhs, rhs_kind, g=None, raise_on_error=True):
        rhs = np.asfortranarray(rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs.reshape(-1, 1, order="F")
        nrhs = rhs.shape[1]
        gg = None if g is None else np.asfortranarray(np.broadcast_to(np.asarray(g, np.float64).reshape(rhs.shape[0], -1), rhs.shape))
        out = np.zeros(rhs.shape, dtype=np.float64, order="F")
        st = Stats()
        code = self.ctx.lib.nlfeti_solve(self.h, nrhs, int(rhs_kind), rhs.ctypes.data, _ptr(gg), out.ctypes.data,
                                         C.byref(st))
        if raise_on_error:
            self.ctx.check(code)
        return out, st.as_dict()

    def cg_prepare(self):
        """Assemble the single-domain matrix for the CG baseline (once per problem)."""
        self.ctx.check(self.ctx.lib.nlfeti_cg_prepare(self.h))

    def solve_cg(self, rhs, rhs_kind, g=None, raise_on_error=True):
        """The paper's baseline: diagonally preconditioned CG on the single-domain system."""
        rhs = np.asfortranarray(rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs.reshape(-1, 1, order="F")
        nrhs = rhs.shape[1]
        gg = None if g is None else np.asfortranarray(np.broadcast_to(np.asarray(g, np.float64).reshape(rhs.shape[0], -1), rhs.shape))
        out = np.zeros(rhs.shape, dtype=np.float64, order="F")
        st = Stats()
        code = self.ctx.lib.nlfeti_solve_cg(self.h, nrhs, int(rhs_kind), rhs.ctypes.data, _ptr(gg), out.ctypes.data,
                                            C.byref(st))
        if raise_on_error:
            self.ctx.check(code)
        return out, st.as_dict()

    def solve_cg_device(self, d_rhs, rhs_kind, d_out, d_g=None, nrhs=None):
        """CG baseline on device arrays (as solve_device)."""
        ptr = lambda t: None if t is None else (t if isinstance(t, int) else t.data_ptr())
        if nrhs is None:
            nrhs = d_rhs.shape[0]
        st = Stats()
        self.ctx.check(self.ctx.lib.nlfeti_solve_cg_device(self.h, int(nrhs), int(rhs_kind), ptr(d_rhs), ptr(d_g),
                                                           ptr(d_out), C.byref(st)))
        return st.as_dict()

    def solve_host_ptr(self, rhs_ptr, rhs_kind, out_ptr, nrhs, g_ptr=None):
        """Host arrays given by address (e.g. pinned torch tensors), column-major n_dofs x nrhs."""
        st = Stats()
        self.ctx.check(self.ctx.lib.nlfeti_solve(self.h, int(nrhs), int(rhs_kind), rhs_ptr, g_ptr, out_ptr,
                                                 C.byref(st)))
        return st.as_dict()

    def set_profiling(self, on: bool):
        self.ctx.check(self.ctx.lib.nlfeti_set_profiling(self.h, 1 if on else 0))

    def profile(self):
        pr = Profile()
        self.ctx.check(self.ctx.lib.nlfeti_get_profile(self.h, C.byref(pr)))
        return {k: getattr(pr, k) for k, _ in Profile._fields_}

    def solve_device(self, d_rhs, rhs_kind, d_out, d_g=None, nrhs=None):
        """Device pointers (ints) or torch tensors (column-major, n_dofs x nrhs as contiguous (nrhs, n_dofs))."""
        ptr = lambda t: None if t is None else (t if isinstance(t, int) else t.data_ptr())
        if nrhs is None:
            nrhs = d_rhs.shape[0]
        st = Stats()
        self.ctx.check(self.ctx.lib.nlfeti_solve_device(self.h, int(nrhs), int(rhs_kind), ptr(d_rhs), ptr(d_g),
                                                        ptr(d_out), C.byref(st)))
        return st.as_dict()

    def decomposition(self):
        inf = self.info()
        K = inf["K"]
        nk = np.zeros(K, np.int32)
        ng = np.zeros(K, np.int32)
        fl = np.zeros(K, np.int8)
        nodes = np.zeros(inf["sum_nk"] // inf["ncomp"], np.int32)
        bp = np.zeros(max(inf["n_lambda"], 1), np.int64)
        bm = np.zeros(max(inf["n_lambda"], 1), np.int64)
        self.ctx.check(self.ctx.lib.nlfeti_get_decomposition(self.h, nk.ctypes.data, ng.ctypes.data, nodes.ctypes.data,
                                                             bp.ctypes.data, bm.ctypes.data, fl.ctypes.data))
        n = inf["n_lambda"]
        return dict(n_k=nk, n_gamma=ng, nodes=nodes, B_plus=bp[:n], B_minus=bm[:n], floating=fl)

    def autotune(self, nrhs, cache_path=None):
        """Time the apply shapes for nrhs right-hand sides and keep the fastest (see nlfeti_autotune);
        returns one dict per operator kind."""
        arr = (TuneEntry * 3)()
        n = C.c_int(0)
        self.ctx.check(self.ctx.lib.nlfeti_autotune(self.h, int(nrhs), cache_path.encode() if cache_path else None,
                                                    arr, C.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in TuneEntry._fields_} for i in range(n.value)]

    def set_apply_choice(self, kind, nrhs, rc, ctas_per_sm=2, rows_per_warp=4, raise_on_error=True):
        code = self.ctx.lib.nlfeti_set_apply_choice(self.h, int(kind), int(nrhs), int(rc), int(ctas_per_sm),
                                                    int(rows_per_warp))
        if raise_on_error:
            self.ctx.check(code)
        return code

    def debug_apply_waits(self, wait_tries=0, withhold_copies=0):
        """Fault injection for tests of the apply's bounded waits (see nlfeti_debug_apply_waits)."""
        self.ctx.check(self.ctx.lib.nlfeti_debug_apply_waits(self.h, int(wait_tries), int(withhold_copies)))

    def set_matrix(self, k, A, raise_on_error=True):
        """Replace the assembled subdomain matrix A^k (n_k x n_k); the factorizations are dropped."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        code = self.ctx.lib.nlfeti_problem_set_matrix(self.h, int(k), A.ctypes.data)
        if raise_on_error:
            self.ctx.check(code)
        return code

    def operator(self, k, which, precision=0):
        d = self.decomposition()
        n = int(d["n_k"][k]) if which == 0 else int(d["n_gamma"][k])
        out = np.zeros((n, n), np.float64)
        self.ctx.check(self.ctx.lib.nlfeti_get_operator(self.h, int(k), int(which), int(precision), out.ctypes.data))
        return out

    def apply_schur_noalloc(self, which, precision, d_in, d_out, nrhs, raise_on_error=True):
        """S^+ (which 0) or S (which 1) on device arrays (ints or torch tensors; column-major
        n_u x nrhs = contiguous (nrhs, n_u)) without device allocation; returns the status."""
        ptr = lambda t: t if isinstance(t, int) else t.data_ptr()
        code = self.ctx.lib.nlfeti_apply_schur_noalloc(self.h, int(which), int(precision), int(nrhs), ptr(d_in),
                                                       ptr(d_out))
        if raise_on_error:
            self.ctx.check(code)
        return code

    def apply(self, op, precision, X):
        X = np.asfortranarray(X, dtype=np.float64)
        if X.ndim == 1:
            X = X.reshape(-1, 1, order="F")
        out = np.zeros(X.shape, np.float64, order="F")
        self.ctx.check(self.ctx.lib.nlfeti_apply(self.h, int(op), int(precision), X.shape[1], X.ctypes.data,
                                                 out.ctypes.data))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.nlfeti_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter shutdown torch (whose allocator frees our device memory) may already be
        # torn down; the process exit releases everything, so nothing is done then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over a context (one worker thread and stream per slot;
    requests on the same problem share batched solves)."""

    def __init__(self, ctx: Context, hbm_budget: int = 0, max_slots: int = 4):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(ctx.lib.nlfeti_server_create(ctx.h, int(hbm_budget), int(max_slots), C.byref(h)))
        self.h = h
        self._pending = {}

    def submit(self, prob: Problem, rhs, rhs_kind, g=None):
        rhs = np.asfortranarray(rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs.reshape(-1, 1, order="F")
        gg = None if g is None else np.asfortranarray(np.broadcast_to(np.asarray(g, np.float64).reshape(rhs.shape[0], -1), rhs.shape))
        t = C.c_uint64()
        self.ctx.check(self.ctx.lib.nlfeti_submit(self.h, prob.h, rhs.shape[1], int(rhs_kind), rhs.ctypes.data,
                                                  _ptr(gg), C.byref(t)))
        self._pending[t.value] = (rhs.shape, prob)
        return t.value

    def submit_workload(self, w, rhs=None, opt: Options | None = None, g=None):
        """A request on the problem given by a workload's inputs (the server's factorization
        cache creates and factors it on first use)."""
        m, k = w.mesh, w.kernel
        xy = np.ascontiguousarray(m.xy, dtype=np.float64)
        el = np.ascontiguousarray(m.elems, dtype=np.int32)
        nd = np.ascontiguousarray(m.node_is_dirichlet, dtype=np.int8)
        ed = np.ascontiguousarray(m.elem_is_dirichlet, dtype=np.int8)
        lab = np.ascontiguousarray(w.labels, dtype=np.int32)
        mesh = Mesh(m.dim, nd.size, xy.ctypes.data, ed.size, el.ctypes.data, nd.ctypes.data, ed.ctypes.data)
        kern = Kernel(int(k.type), float(k.delta), float(k.s), float(k.scale), int(getattr(k, "ball", 0)))
        dec = Decomp(int(w.K), lab.ctypes.data)
        rhs = np.asfortranarray(w.rhs if rhs is None else rhs, dtype=np.float64)
        if rhs.ndim == 1:
            rhs = rhs.reshape(-1, 1, order="F")
        gg = None if g is None else np.asfortranarray(np.broadcast_to(np.asarray(g, np.float64).reshape(rhs.shape[0], -1), rhs.shape))
        t = C.c_uint64()
        self.ctx.check(self.ctx.lib.nlfeti_submit_mesh(self.h, C.byref(mesh), C.byref(kern), C.byref(dec),
                                                       C.byref(opt) if opt is not None else None, rhs.shape[1],
                                                       int(w.rhs_kind), rhs.ctypes.data, _ptr(gg), C.byref(t)))
        self._pending[t.value] = (rhs.shape, None)
        return t.value

    def info(self):
        i = ServerInfo()
        self.ctx.check(self.ctx.lib.nlfeti_server_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in ServerInfo._fields_}

    def wait(self, ticket, timeout_ms=-1):
        shape, _ = self._pending[ticket]
        out = np.zeros(shape, np.float64, order="F")
        st = Stats()
        code = self.ctx.lib.nlfeti_wait(self.h, C.c_uint64(ticket), int(timeout_ms), out.ctypes.data, C.byref(st))
        if code == E_TIMEOUT:
            raise NlfetiError(code, "wait timed out")
        del self._pending[ticket]
        self.ctx.check(code)
        return out, st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.nlfeti_server_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter shutdown torch (whose allocator frees our device memory) may already be
        # torn down; the process exit releases everything, so nothing is done then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass
