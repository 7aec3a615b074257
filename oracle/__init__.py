"""Python handle on the FP64 CPU oracle (lrs_oracle.cpp).

TEST INFRASTRUCTURE: only the tests, the package smoke check and the CPU
baseline of bench.py use this module.  The CUDA library never imports it.

The oracle follows the paper's Algorithm 1 (factorization), Algorithms 2-4
(solve) and restarted GMRES, sequentially in FP64; see lrs_oracle.cpp for the
passages each routine follows and for the readings where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lrs_oracle.cpp")
_LIB = os.path.join(_HERE, "liblrs_oracle.so")
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 3: "singular pivot", 4: "not converged"}

EXPORT_PERM, EXPORT_LEAF_OFF, EXPORT_BATCHES, EXPORT_COMPRESS, EXPORT_ELIM, \
    EXPORT_RANKS, EXPORT_PIVOT_SIZES = range(7)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no machine-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.lrso_create.argtypes = [I64, P, P, P, I32, P, I32, I32, ctypes.POINTER(P)]
        lib.lrso_destroy.argtypes = [P]
        lib.lrso_depth.argtypes = [P]
        lib.lrso_set_separation.argtypes = [P, I32]
        lib.lrso_set_order.argtypes = [P, I32]
        lib.lrso_gmres_left.argtypes = [P, P, P, I32, I32, I32, D, P, P, P]
        lib.lrso_set_values.argtypes = [P, P]
        lib.lrso_factor.argtypes = [P, D, I32]
        lib.lrso_factor_partial.argtypes = [P, D, I32]
        lib.lrso_ext_size.argtypes = [P]
        lib.lrso_ext_size.restype = I64
        lib.lrso_apply.argtypes = [P, P, P, I32]
        lib.lrso_spmv.argtypes = [P, P, P, I32]
        lib.lrso_gmres.argtypes = [P, P, P, I32, I32, I32, D, I32, P, P]
        lib.lrso_export_size.argtypes = [P, I32]
        lib.lrso_export_size.restype = I64
        lib.lrso_export.argtypes = [P, I32, P]
        lib.lrso_compress_count.argtypes = [P]
        lib.lrso_compress_info.argtypes = [P, I32, P]
        lib.lrso_compress_sigma.argtypes = [P, I32, P]
        lib.lrso_compress_matrix.argtypes = [P, I32, P]
        lib.lrso_compress_v.argtypes = [P, I32, P]
        lib.lrso_compress_below.argtypes = [P, I32]
        lib.lrso_compress_below.restype = ctypes.c_double
        lib.lrso_set_trunc_rule.argtypes = [P, I32]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class Oracle:
    """One matrix pattern + values, its H-tree, and (after factor) its factorization."""

    def __init__(self, csr, leaf_size: int = 64, depth: int = 0, separation: int = 2, order: str = "greedy",
                 trunc_rule: str = "cutoff1"):
        lib = _load()
        self._keep = (csr.rowptr, csr.colind, csr.val, csr.coords)
        self.n = csr.n
        h = ctypes.c_void_p()
        st = lib.lrso_create(csr.n, _ptr(csr.rowptr), _ptr(csr.colind), _ptr(csr.val), csr.dim,
                             _ptr(csr.coords), leaf_size, depth, ctypes.byref(h))
        if st:
            raise OracleError(st, "lrso_create")
        self._h = h
        self.depth = lib.lrso_depth(h)
        st = lib.lrso_set_separation(h, int(separation))
        if st:
            raise OracleError(st, "lrso_set_separation")
        if order not in ("greedy", "natural"):
            raise ValueError("order: 'greedy' (batches) or 'natural' (one super-node at a time)")
        lib.lrso_set_order(h, int(order == "natural"))
        if trunc_rule not in ("cutoff1", "curoff6"):
            raise ValueError("trunc_rule: 'cutoff1' (sigma_k / sigma_0 >= eps, Sec. 6.1) or 'curoff6' "
                             "(Frobenius tail against all levels below, Sec. 6.3)")
        lib.lrso_set_trunc_rule(h, int(trunc_rule == "curoff6"))

    def __del__(self):
        if getattr(self, "_h", None):
            _load().lrso_destroy(self._h)
            self._h = None

    def set_values(self, val):
        val = np.ascontiguousarray(val, dtype=np.float64)
        self._keep = self._keep[:2] + (val,) + self._keep[3:]
        _load().lrso_set_values(self._h, _ptr(val))

    def factor(self, eps: float, capture: bool = False):
        st = _load().lrso_factor(self._h, float(eps), int(capture))
        if st:
            raise OracleError(st, "lrso_factor")

    def factor_partial(self, eps: float, max_batches: int):
        """Run only the first max_batches batches (records of a sample)."""
        st = _load().lrso_factor_partial(self._h, float(eps), int(max_batches))
        if st:
            raise OracleError(st, "lrso_factor_partial")

    @property
    def ext_size(self) -> int:
        return int(_load().lrso_ext_size(self._h))

    def _cols(self, b):
        b = np.asarray(b, dtype=np.float64)
        vec = b.ndim == 1
        B = np.asfortranarray(b.reshape(self.n, -1))
        return vec, B

    def apply(self, b):
        """x = M b: one forward + backward traversal (Algorithms 2-4)."""
        vec, B = self._cols(b)
        X = np.zeros_like(B, order="F")
        st = _load().lrso_apply(self._h, _ptr(B), _ptr(X), B.shape[1])
        if st:
            raise OracleError(st, "lrso_apply")
        return X[:, 0] if vec else X

    def spmv(self, x):
        vec, X = self._cols(x)
        Y = np.zeros_like(X, order="F")
        _load().lrso_spmv(self._h, _ptr(X), _ptr(Y), X.shape[1])
        return Y[:, 0] if vec else Y

    def gmres(self, b, restart=30, maxit=500, tol=1e-10, precond=True, check=False):
        """Right-preconditioned restarted GMRES; returns (x, iters, relres, status)."""
        vec, B = self._cols(b)
        X = np.zeros_like(B, order="F")
        k = B.shape[1]
        iters = np.zeros(k, dtype=np.int32)
        rel = np.zeros(k, dtype=np.float64)
        st = _load().lrso_gmres(self._h, _ptr(B), _ptr(X), k, restart, maxit, tol, int(precond),
                                _ptr(iters), _ptr(rel))
        if check and st:
            raise OracleError(st, "lrso_gmres")
        return (X[:, 0] if vec else X), iters, rel, st

    def gmres_left(self, b, restart=30, maxit=500, tol=1e-10):
        """The paper's left-preconditioned GMRES (stops on ||M(b - Ax)|| / ||Mb||);
        returns (x, iters, true relres, preconditioned relres, status)."""
        vec, B = self._cols(b)
        X = np.zeros_like(B, order="F")
        k = B.shape[1]
        iters = np.zeros(k, dtype=np.int32)
        rel = np.zeros(k, dtype=np.float64)
        prec = np.zeros(k, dtype=np.float64)
        st = _load().lrso_gmres_left(self._h, _ptr(B), _ptr(X), k, restart, maxit, tol, _ptr(iters), _ptr(rel),
                                     _ptr(prec))
        return (X[:, 0] if vec else X), iters, rel, prec, st

    def export(self, what: int) -> np.ndarray:
        lib = _load()
        n = lib.lrso_export_size(self._h, what)
        out = np.zeros(n, dtype=np.int32)
        lib.lrso_export(self._h, what, _ptr(out))
        return out

    def compressions(self, with_matrices: bool = False):
        """List of dicts (snode, rho, m, r, sigma, below[, M, V]) in compression
        order; below is eq. curOff6's ||all levels below||_F at that compression."""
        lib = _load()
        out = []
        info = np.zeros(4, dtype=np.int32)
        for k in range(lib.lrso_compress_count(self._h)):
            lib.lrso_compress_info(self._h, k, _ptr(info))
            snode, rho, m, r = (int(v) for v in info)
            sig = np.zeros(min(rho, m), dtype=np.float64)
            if sig.size:
                lib.lrso_compress_sigma(self._h, k, _ptr(sig))
            rec = dict(snode=snode, rho=rho, m=m, r=r, sigma=sig, below=lib.lrso_compress_below(self._h, k))
            if with_matrices:
                M = np.zeros((rho, m), dtype=np.float64, order="F")
                V = np.zeros((m, r), dtype=np.float64, order="F")
                if lib.lrso_compress_matrix(self._h, k, _ptr(M)) == 0 and \
                        lib.lrso_compress_v(self._h, k, _ptr(V)) == 0:
                    rec["M"], rec["V"] = M, V
            out.append(rec)
        return out
