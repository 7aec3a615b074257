"""Python binding of liblrs, the GB300 hierarchical sparse solver.

The functions mirror the C ABI of include/lrs.h one to one (lrs_analyze,
lrs_plan_export, lrs_factor, lrs_apply, lrs_solve, lrs_factor_export,
lrs_factor_sigma, lrs_factor_stats) and only marshal arguments: every step of
the method runs in the CUDA library.  Device memory comes from PyTorch's
caching allocator through the library's allocator hooks; vectors may be host
NumPy arrays (copied by the library) or CUDA torch tensors (used in place).

Importing this module never builds or loads CUDA code; the first call that
needs the library loads liblrs.so and raises LrsLibraryMissing when it was
not built (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrs.so")

LRS_OK = 0
LRS_ERR_INVALID_ARG = 1
LRS_ERR_OOM = 2
LRS_ERR_SINGULAR_PIVOT = 3
LRS_ERR_NOT_CONVERGED = 4
LRS_ERR_TIMEOUT = 5
LRS_ERR_CUDA = 6
LRS_ERR_NUMERIC = 7
LRS_ERR_STATE = 8

EXPORT_PERM, EXPORT_LEAF_OFF, EXPORT_BATCHES, EXPORT_COMPRESS, EXPORT_ELIM, EXPORT_INSTANCES = range(6)
SYM_DETECT, SYM_GENERAL, SYM_SYMMETRIC = 0, 1, 2
PREC_FP64, PREC_TF32 = 0, 1
PREC_FP32 = PREC_TF32      # the precision form under its storage type's name
GMRES_RIGHT, GMRES_LEFT = 0, 1
TRUNC_CUTOFF1, TRUNC_CUROFF6 = 0, 1
GEMM_AUTO, GEMM_FP64, GEMM_EMU, GEMM_TF32 = 0, 1, 2, 3
EXPORT_RANKS, EXPORT_PIVOT_SIZES, EXPORT_ITERS = 5, 6, 7

# Every symbol declared in include/lrs.h.
ABI_SYMBOLS = ("lrs_analyze", "lrs_analyze_batch", "lrs_plan_export", "lrs_plan_destroy", "lrs_factor", "lrs_apply", "lrs_apply_static",
               "lrs_solve",
               "lrs_factor_export", "lrs_factor_sigma", "lrs_factor_stats", "lrs_factor_profile",
               "lrs_factor_destroy", "lrs_status_string", "lrs_selftest_bounded_wait", "lrs_block_gemm",
               "lrs_server_create", "lrs_server_factor", "lrs_server_solve", "lrs_server_wait",
               "lrs_server_evict", "lrs_server_stats", "lrs_server_destroy")

PROF_CLASSES = ("factor_gemm", "invert", "spectrum", "copy", "assemble", "apply_gemm", "spmv", "vector",
                "factor_gemm_f32", "factor_gemm_emu")


class LrsLibraryMissing(RuntimeError):
    pass


class LrsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("dim", ctypes.c_int), ("coords", ctypes.c_void_p)]


class _AnalyzeOpts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("depth", ctypes.c_int), ("separation", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class _FactorOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("profile", ctypes.c_int),
                ("symmetry", ctypes.c_int), ("precision", ctypes.c_int), ("trunc_rule", ctypes.c_int),
                ("gemm", ctypes.c_int)]


class _ProfEntry(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("tol", ctypes.c_double),
                ("side", ctypes.c_int), ("precond_residual", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("rel_res_precond", ctypes.c_double)]


EXEC_FACTOR_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t))
EXEC_SOLVE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int, ctypes.POINTER(_SolveOpts), ctypes.POINTER(SolveInfo))
EXEC_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class _ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("workers", ctypes.c_int), ("max_batch_rhs", ctypes.c_int),
                ("factor_fn", EXEC_FACTOR_FN), ("solve_fn", EXEC_SOLVE_FN), ("release_fn", EXEC_RELEASE_FN),
                ("exec_ctx", ctypes.c_void_p)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("batch_rhs", ctypes.c_int), ("bytes", ctypes.c_size_t), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("n", ctypes.c_int64), ("ext_n", ctypes.c_int64),
                ("n_compress", ctypes.c_int64), ("n_batches", ctypes.c_int64), ("factor_ms", ctypes.c_double),
                ("flops_factor", ctypes.c_double), ("eig_flops", ctypes.c_double),
                ("eig_cycles", ctypes.c_double * 5), ("factor_bytes", ctypes.c_int64),
                ("apply_bytes", ctypes.c_int64), ("max_rank", ctypes.c_int), ("max_pivot", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("precision", ctypes.c_int), ("flops_factor_f32", ctypes.c_double),
                ("host_ms", ctypes.c_double), ("host_wait_ms", ctypes.c_double), ("host_elim_ms", ctypes.c_double),
                ("host_merge_ms", ctypes.c_double), ("host_compress_ms", ctypes.c_double),
                ("eig_lead_ms", ctypes.c_double * 5)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k in ("eig_cycles", "eig_lead_ms") else v
        return out


_lib = None


def load(path: str = LIB_PATH):
    """Load liblrs.so (built by build.build()); raise LrsLibraryMissing if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LrsLibraryMissing(f"{path} is missing: run paper_1510_07363_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.lrs_analyze.argtypes = [ctypes.POINTER(_Csr), ctypes.POINTER(_AnalyzeOpts), ctypes.POINTER(P)]
    lib.lrs_analyze_batch.argtypes = [I32, ctypes.POINTER(_Csr), ctypes.POINTER(_AnalyzeOpts), ctypes.POINTER(P)]
    lib.lrs_plan_export.argtypes = [P, I32, P, ctypes.POINTER(I64)]
    lib.lrs_plan_destroy.argtypes = [P]
    lib.lrs_plan_destroy.restype = None
    lib.lrs_factor.argtypes = [P, P, I32, ctypes.POINTER(_FactorOpts), ctypes.POINTER(P)]
    lib.lrs_apply.argtypes = [P, P, P, I32, I32]
    lib.lrs_selftest_bounded_wait.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.lrs_block_gemm.argtypes = [I32, I32, I32, I32, P, I32, I32, P, I32, I32, P, I32, I32, I32,
                                   ctypes.POINTER(ctypes.c_double)]
    lib.lrs_apply_static.argtypes = [P, P, P, I32]
    lib.lrs_solve.argtypes = [P, P, P, I32, I32, ctypes.POINTER(_SolveOpts), ctypes.POINTER(SolveInfo)]
    lib.lrs_factor_export.argtypes = [P, I32, P, ctypes.POINTER(I64)]
    lib.lrs_factor_sigma.argtypes = [P, I64, P, ctypes.POINTER(I64)]
    lib.lrs_factor_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.lrs_factor_profile.argtypes = [P, ctypes.POINTER(_ProfEntry), I32]
    lib.lrs_factor_destroy.argtypes = [P]
    lib.lrs_factor_destroy.restype = None
    lib.lrs_server_create.argtypes = [ctypes.POINTER(_ServerOpts), ctypes.POINTER(P)]
    lib.lrs_server_factor.argtypes = [P, P, P, ctypes.c_double, I32, ctypes.c_size_t, ctypes.POINTER(I64)]
    lib.lrs_server_solve.argtypes = [P, I64, P, P, I32, ctypes.POINTER(_SolveOpts), ctypes.POINTER(I64)]
    lib.lrs_server_wait.argtypes = [P, I64, ctypes.POINTER(RequestInfo)]
    lib.lrs_server_evict.argtypes = [P, I64]
    lib.lrs_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(I32), ctypes.POINTER(I32)]
    lib.lrs_server_destroy.argtypes = [P]
    lib.lrs_server_destroy.restype = None
    lib.lrs_status_string.argtypes = [I32]
    lib.lrs_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().lrs_status_string(code).decode()
    except LrsLibraryMissing:
        return str(code)


def _check(code, where):
    if code != LRS_OK:
        raise LrsError(code, where)


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Plan:
    """Result of lrs_analyze: the H-tree and the elimination program."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lrs_plan_destroy(self._h)
            self._h = None

    def export(self, what: int) -> np.ndarray:
        return lrs_plan_export(self, what)


def lrs_analyze(csr, leaf_size: int = 64, depth: int = 0, separation: int = 0) -> Plan:
    lib = load()
    rowptr = np.ascontiguousarray(csr.rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(csr.colind, dtype=np.int32)
    coords = np.ascontiguousarray(csr.coords, dtype=np.float64)
    A = _Csr(int(csr.n), _np_ptr(rowptr), _np_ptr(colind), None, int(coords.shape[1]), _np_ptr(coords))
    opts = _AnalyzeOpts(int(leaf_size), int(depth), int(separation))
    h = ctypes.c_void_p()
    _check(lib.lrs_analyze(ctypes.byref(A), ctypes.byref(opts), ctypes.byref(h)), "lrs_analyze")
    plan = Plan(h, (rowptr, colind, coords))
    plan.n = int(csr.n)
    plan.nnz = int(rowptr[-1])
    return plan


def lrs_analyze_batch(csrs, leaf_size: int = 64, depth: int = 0, separation: int = 0) -> Plan:
    """The batched form: one plan over independent matrices (lrs_analyze_batch).

    Values for lrs_factor are the instances' values concatenated in order;
    right-hand sides are the instances' rows stacked in the same order.
    """
    lib = load()
    keep, structs = [], (_Csr * len(csrs))()
    for k, csr in enumerate(csrs):
        rowptr = np.ascontiguousarray(csr.rowptr, dtype=np.int64)
        colind = np.ascontiguousarray(csr.colind, dtype=np.int32)
        coords = np.ascontiguousarray(csr.coords, dtype=np.float64)
        keep.append((rowptr, colind, coords))
        structs[k] = _Csr(int(csr.n), _np_ptr(rowptr), _np_ptr(colind), None, int(coords.shape[1]),
                          _np_ptr(coords))
    opts = _AnalyzeOpts(int(leaf_size), int(depth), int(separation))
    h = ctypes.c_void_p()
    _check(lib.lrs_analyze_batch(len(csrs), structs, ctypes.byref(opts), ctypes.byref(h)), "lrs_analyze_batch")
    plan = Plan(h, keep)
    plan.n = int(sum(int(c.n) for c in csrs))
    plan.nnz = int(sum(int(r[0][-1]) for r in keep))
    return plan


def lrs_plan_export(plan: Plan, what: int) -> np.ndarray:
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.lrs_plan_export(plan._h, what, None, ctypes.byref(cnt)), "lrs_plan_export")
    out = np.zeros(cnt.value, dtype=np.int32)
    _check(lib.lrs_plan_export(plan._h, what, _np_ptr(out), ctypes.byref(cnt)), "lrs_plan_export")
    return out


class _TorchAllocator:
    """Allocator hooks backed by torch.cuda's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device()
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
        except Exception:
            return None

    def _free(self, ptr, nbytes, stream, ctx):
        self.torch.cuda.caching_allocator_delete(int(ptr))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Factor:
    """Result of lrs_factor: the hierarchical factorization resident on the GPU."""

    def __init__(self, handle, plan, allocator, stream):
        self._h = handle
        self.plan = plan
        self._allocator = allocator
        self.stream = stream

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lrs_factor_destroy(self._h)
            self._h = None

    def apply(self, b):
        return lrs_apply(self, b)

    def solve(self, b, **kw):
        return lrs_solve(self, b, **kw)

    def export(self, what):
        return lrs_factor_export(self, what)

    def ranks(self):
        return lrs_factor_export(self, EXPORT_RANKS)

    def sigma(self, k):
        return lrs_factor_sigma(self, k)

    def stats(self) -> dict:
        return lrs_factor_stats(self)


def lrs_factor(plan: Plan, val, eps: float, stream=None, allocator: str = "torch",
               profile: bool = False, symmetry: int = SYM_DETECT, precision: int = PREC_FP64,
               trunc_rule: int = TRUNC_CUTOFF1, gemm: int = 0) -> Factor:
    """Factor A (values `val` in CSR order: NumPy host array or CUDA tensor).

    symmetry: SYM_DETECT (take the symmetric path when the values are exactly
    symmetric), SYM_GENERAL or SYM_SYMMETRIC (the caller asserts A = A^T).
    precision: PREC_FP64, or PREC_FP32 for the precision form (block products
    on the tensor cores, see include/lrs.h).  trunc_rule: TRUNC_CUTOFF1
    (sigma_k / sigma_0 >= eps, Sec. 6.1) or TRUNC_CUROFF6 (Frobenius tail
    against all levels below, Sec. 6.3).  gemm: GEMM_AUTO, GEMM_FP64 or GEMM_EMU,
    the engine of the FP64 block products (see include/lrs.h)."""
    lib = load()
    alloc = _TorchAllocator() if allocator == "torch" else None
    sh = 0
    if stream is not None:
        sh = int(getattr(stream, "cuda_stream", stream))
    opts = _FactorOpts(float(eps), ctypes.c_void_p(sh) if sh else None,
                       alloc.alloc if alloc else ALLOC_FN(), alloc.free if alloc else FREE_FN(), None,
                       int(bool(profile)), int(symmetry), int(precision), int(trunc_rule), int(gemm))
    h = ctypes.c_void_p()
    if _is_torch(val):
        assert val.is_cuda and val.dtype.is_floating_point and val.is_contiguous()
        code = lib.lrs_factor(plan._h, ctypes.c_void_p(val.data_ptr()), 1, ctypes.byref(opts), ctypes.byref(h))
    else:
        v = np.ascontiguousarray(val, dtype=np.float64)
        code = lib.lrs_factor(plan._h, _np_ptr(v), 0, ctypes.byref(opts), ctypes.byref(h))
    _check(code, "lrs_factor")
    return Factor(h, plan, alloc, sh)


def lrs_block_gemm(engine: int, A, B, C, transa: bool = False, transb: bool = False,
                   accumulate: bool = False, subtract: bool = False) -> float:
    """C = init + sign op(A) op(B) on the GPU with the given engine
    (GEMM_FP64, GEMM_EMU or GEMM_TF32); A, B, C: CUDA float64 tensors in
    column-major order (the transpose of a contiguous row-major tensor, e.g.
    X.t().contiguous().t()).  Returns the kernel's duration in ms."""
    lib = load()

    def cm(X):
        assert X.is_cuda and X.dtype.is_floating_point and X.element_size() == 8 and X.dim() == 2
        assert X.stride(0) == 1, "column-major (stride(0) == 1) expected"
        return X.shape[0], X.shape[1], max(1, X.stride(1))
    ra, ca, lda = cm(A)
    rb, cb, ldb = cm(B)
    rc, cc, ldc = cm(C)
    rows, k = (ca, ra) if transa else (ra, ca)
    kb, cols = (cb, rb) if transb else (rb, cb)
    assert kb == k and rc == rows and cc == cols
    ms = ctypes.c_double()
    _check(lib.lrs_block_gemm(int(engine), rows, cols, k, ctypes.c_void_p(A.data_ptr()), lda, int(transa),
                              ctypes.c_void_p(B.data_ptr()), ldb, int(transb), ctypes.c_void_p(C.data_ptr()), ldc,
                              int(accumulate), int(subtract), ctypes.byref(ms)), "lrs_block_gemm")
    return ms.value


def _vec_args(f: Factor, b):
    """(pointer to b, pointer to a new x, nrhs, on_device, x, reshape)."""
    n = f.plan.n
    if _is_torch(b):
        import torch
        vec = b.dim() == 1
        # column-major n x nrhs == row-major nrhs x n
        B = b.reshape(1, n) if vec else b.t().contiguous()
        X = torch.empty_like(B)
        back = (lambda X: X.reshape(n)) if vec else (lambda X: X.t())
        return ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()), B.shape[0], 1, X, back, B
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    B = np.asfortranarray(b.reshape(n, -1))
    X = np.zeros_like(B, order="F")
    back = (lambda X: X[:, 0]) if vec else (lambda X: X)
    return _np_ptr(B), _np_ptr(X), B.shape[1], 0, X, back, B


def lrs_apply(f: Factor, b):
    """x = M b (Algorithms 2-4) for a vector or an n x nrhs block."""
    pb, px, k, dev, X, back, _keep = _vec_args(f, b)
    _check(load().lrs_apply(f._h, pb, px, k, dev), "lrs_apply")
    return back(X)


def lrs_apply_static(f: Factor, b, out=None):
    """x = M b through lrs_apply_static (no device allocation inside the call).

    b: CUDA tensor (n,) or (n, nrhs).  The caller provides the output buffer
    `out` (same shape) or lets this binding create it before the call."""
    import torch
    n = f.plan.n
    vec = b.dim() == 1
    B = b.reshape(1, n) if vec else b.t().contiguous()
    X = torch.empty_like(B) if out is None else (out.reshape(1, n) if vec else out.t())
    if not X.is_contiguous():
        raise ValueError("out must be contiguous in column-major order")
    _check(load().lrs_apply_static(f._h, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()), B.shape[0]),
           "lrs_apply_static")
    return X.reshape(n) if vec else X.t()


def lrs_solve(f: Factor, b, restart: int = 30, maxit: int = 500, tol: float = 1e-10, check: bool = False,
              side: int = GMRES_RIGHT, precond_residual: bool = False):
    """GMRES preconditioned by the factor; returns (x, SolveInfo, per-column iterations).

    side: GMRES_RIGHT (stop on the true residual) or GMRES_LEFT (the paper's
    form, stop on ||M(b - Ax)|| / ||Mb||); info.rel_res_precond is that
    preconditioned residual (left side, or right side with precond_residual)."""
    pb, px, k, dev, X, back, _keep = _vec_args(f, b)
    opts = _SolveOpts(int(restart), int(maxit), float(tol), int(side), int(bool(precond_residual)))
    info = SolveInfo()
    code = load().lrs_solve(f._h, pb, px, k, dev, ctypes.byref(opts), ctypes.byref(info))
    if code not in (LRS_OK, LRS_ERR_NOT_CONVERGED) or (check and code != LRS_OK):
        raise LrsError(code, "lrs_solve")
    return back(X), info, lrs_factor_export(f, EXPORT_ITERS)


def lrs_factor_export(f: Factor, what: int) -> np.ndarray:
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.lrs_factor_export(f._h, what, None, ctypes.byref(cnt)), "lrs_factor_export")
    out = np.zeros(cnt.value, dtype=np.int32)
    _check(lib.lrs_factor_export(f._h, what, _np_ptr(out), ctypes.byref(cnt)), "lrs_factor_export")
    return out


def lrs_factor_sigma(f: Factor, k: int) -> np.ndarray:
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.lrs_factor_sigma(f._h, k, None, ctypes.byref(cnt)), "lrs_factor_sigma")
    out = np.zeros(cnt.value, dtype=np.float64)
    _check(lib.lrs_factor_sigma(f._h, k, _np_ptr(out), ctypes.byref(cnt)), "lrs_factor_sigma")
    return out


def lrs_factor_profile(f: Factor, reset: bool = False) -> dict:
    """{class: {launches, ms, flops, bytes}} of the launches timed so far."""
    arr = (_ProfEntry * len(PROF_CLASSES))()
    _check(load().lrs_factor_profile(f._h, arr, int(reset)), "lrs_factor_profile")
    return {name: {"launches": e.launches, "ms": e.ms, "flops": e.flops, "bytes": e.bytes}
            for name, e in zip(PROF_CLASSES, arr)}


def lrs_factor_stats(f: Factor) -> dict:
    st = Stats()
    _check(load().lrs_factor_stats(f._h, ctypes.byref(st)), "lrs_factor_stats")
    return st.as_dict()


def lrs_selftest_bounded_wait():
    """(status code, milliseconds the wait took): LRS_ERR_TIMEOUT is the pass."""
    ms = ctypes.c_double(0.0)
    code = load().lrs_selftest_bounded_wait(ctypes.byref(ms))
    return code, ms.value


class Server:
    """The serving form (lrs_server_*): factorizations kept resident, admitted
    by an HBM budget, and a request loop whose solves against one factor are
    merged into one multi-column GMRES.  Host arrays in and out; the arrays of
    a request are kept alive here until its wait.

    executor: None for the library's GPU executor, or an object with
    factor(plan_ptr, val_ptr, eps, precision) -> (status, handle, bytes),
    solve(handle, b_ptr, x_ptr, nrhs, restart, maxit, tol) -> (status, iters, rel_res)
    and release(handle), called from the server's worker threads."""

    def __init__(self, hbm_budget: int, workers: int = 2, max_batch_rhs: int = 16, executor=None):
        lib = load()
        self._keep = {}
        self._cb = None
        o = _ServerOpts(int(hbm_budget), int(workers), int(max_batch_rhs))
        if executor is not None:
            # an exception in a hook fails its request (a ctypes callback that
            # raised would otherwise return 0, i.e. success)
            def f_fn(ctx, plan, val, eps, prec, out, nbytes):
                try:
                    st, handle, b = executor.factor(plan, val, eps, prec)
                    out[0] = handle
                    nbytes[0] = b
                    return st
                except Exception:
                    out[0] = None
                    nbytes[0] = 0
                    return LRS_ERR_STATE

            def s_fn(ctx, handle, b, x, nrhs, opts, info):
                try:
                    st, iters, rel = executor.solve(handle, b, x, nrhs, opts[0].restart, opts[0].maxit, opts[0].tol)
                    info[0].iters, info[0].status, info[0].rel_res = iters, st, rel
                    return st
                except Exception:
                    return LRS_ERR_STATE

            def r_fn(ctx, handle):
                try:
                    executor.release(handle)
                except Exception:
                    pass

            self._cb = (EXEC_FACTOR_FN(f_fn), EXEC_SOLVE_FN(s_fn), EXEC_RELEASE_FN(r_fn))
            o.factor_fn, o.solve_fn, o.release_fn = self._cb
        h = ctypes.c_void_p()
        _check(lib.lrs_server_create(ctypes.byref(o), ctypes.byref(h)), "lrs_server_create")
        self._h = h

    def factor(self, plan: Plan, val, eps: float, precision: int = PREC_FP64, reserve_bytes: int = 0) -> int:
        v = np.ascontiguousarray(val, dtype=np.float64)
        t = ctypes.c_int64()
        _check(load().lrs_server_factor(self._h, plan._h, _np_ptr(v), float(eps), int(precision),
                                        int(reserve_bytes), ctypes.byref(t)), "lrs_server_factor")
        self._keep[t.value] = (v, plan)
        return t.value

    def solve(self, factor: int, b, tol: float = 1e-10, restart: int = 30, maxit: int = 300,
              side: int = GMRES_RIGHT) -> int:
        b = np.asarray(b, dtype=np.float64)
        vec = b.ndim == 1
        B = np.asfortranarray(b.reshape(b.shape[0], -1))
        X = np.zeros_like(B, order="F")
        opts = _SolveOpts(int(restart), int(maxit), float(tol), int(side), 0)
        t = ctypes.c_int64()
        _check(load().lrs_server_solve(self._h, int(factor), _np_ptr(B), _np_ptr(X), B.shape[1], ctypes.byref(opts),
                                       ctypes.byref(t)), "lrs_server_solve")
        self._keep[t.value] = (B, X, vec)
        return t.value

    def wait(self, ticket: int):
        """(x or None for a factorization, RequestInfo) once the request is done."""
        info = RequestInfo()
        _check(load().lrs_server_wait(self._h, int(ticket), ctypes.byref(info)), "lrs_server_wait")
        kept = self._keep.pop(int(ticket), None)
        if kept is not None and len(kept) == 3:
            X = kept[1]
            return (X[:, 0] if kept[2] else X), info
        return None, info

    def evict(self, factor: int) -> None:
        _check(load().lrs_server_evict(self._h, int(factor)), "lrs_server_evict")

    def stats(self) -> dict:
        held, res, q = ctypes.c_size_t(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().lrs_server_stats(self._h, ctypes.byref(held), ctypes.byref(res), ctypes.byref(q)),
               "lrs_server_stats")
        return {"held_bytes": held.value, "resident": res.value, "queued": q.value}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().lrs_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        if _lib is not None:
            self.close()
