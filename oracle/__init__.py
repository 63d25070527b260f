"""CPU oracle for the PPE hot path.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2604_01800_gb300``) and never imports it.

* ``ppe_oracle.c`` (FP64, plain loops): CSR assembly of the volume-scaled
  variable-spacing 5-point operator, Jacobi PCG with range projection, the
  full solve with compatibility check and zero-mean normalisation.
* ``net_oracle.py`` (FP64 numpy): distance-vector maps, Mesh-Conv weights,
  the U-Net-branch DeepONet forward and backward, the loss of Eq. 18 and one
  SAM + Adam step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppe_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libppe_oracle.so")
_LIB_OMP = os.path.join(_LIBDIR, "libppe_oracle_omp.so")
_lib = None
_lib_omp = None

OR_OK, OR_ERR_ARG, OR_ERR_INCOMPATIBLE, OR_ERR_NOT_CONVERGED = 0, 1, 4, 5


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no vector extensions).  The
    tests use the single-thread build; ``openmp=True`` builds the all-core
    variant that only the benchmark's CPU timing uses."""
    os.makedirs(_LIBDIR, exist_ok=True)
    path = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".{os.getpid()}.tmp"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def lib(openmp: bool = False):
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = _declare(ctypes.CDLL(build(openmp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    """Argument and result types of the exported functions."""
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_long)
    ip = ctypes.POINTER(ctypes.c_int)
    L.or_nnz.restype = ctypes.c_long
    L.or_nnz.argtypes = [ctypes.c_int, ctypes.c_int]
    L.or_assemble.restype = ctypes.c_int
    L.or_assemble.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, lp, ip, dp]
    L.or_spmv.restype = None
    L.or_spmv.argtypes = [ctypes.c_long, lp, ip, dp, dp, dp]
    L.or_jpcg.restype = ctypes.c_long
    L.or_jpcg.argtypes = [ctypes.c_long, lp, ip, dp, dp, dp, ctypes.c_double, ctypes.c_long]
    L.or_scaled_rhs.restype = None
    L.or_scaled_rhs.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
    L.or_solve.restype = ctypes.c_int
    L.or_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, ctypes.c_long, dp]
    return L


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class CSR:
    """The assembled operator A = -V M (scipy-free container)."""

    def __init__(self, dx, dy):
        dx, dy = _c64(dx), _c64(dy)
        self.nx, self.ny = dx.size, dy.size
        n = self.nx * self.ny
        nnz = lib().or_nnz(self.nx, self.ny)
        self.rowptr = np.zeros(n + 1, dtype=np.int64)
        self.col = np.zeros(nnz, dtype=np.int32)
        self.val = np.zeros(nnz, dtype=np.float64)
        st = lib().or_assemble(self.nx, self.ny, _d(dx), _d(dy),
                               self.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                               self.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(self.val))
        assert st == OR_OK

    @property
    def n(self):
        return self.nx * self.ny

    def matvec(self, x):
        x = _c64(x).reshape(-1)
        y = np.empty_like(x)
        lib().or_spmv(self.n, self.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                      self.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(self.val), _d(x), _d(y))
        return y

    def dense(self):
        A = np.zeros((self.n, self.n))
        for r in range(self.n):
            for k in range(self.rowptr[r], self.rowptr[r + 1]):
                A[r, self.col[k]] = self.val[k]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def apply(dx, dy, x):
    """y = A x for a field x [ny, nx] (A = -V M)."""
    A = CSR(dx, dy)
    return A.matvec(x).reshape(len(dy), len(dx))


def scaled_rhs(dx, dy, S):
    dx, dy, S = _c64(dx), _c64(dy), _c64(S)
    b = np.empty_like(S)
    lib().or_scaled_rhs(dx.size, dy.size, _d(dx), _d(dy), _d(S), _d(b))
    return b


def solve(dx, dy, S, tol_rel=1e-8, x0=None, maxit=10_000_000, openmp=False):
    """Solve M x = S; returns (x [ny, nx], info dict, status).  ``openmp``
    runs the all-core build (benchmark timing only)."""
    dx, dy, S = _c64(dx), _c64(dy), _c64(S)
    x = np.zeros_like(S) if x0 is None else _c64(x0).copy()
    out = np.zeros(3)
    st = lib(openmp).or_solve(dx.size, dy.size, _d(dx), _d(dy), _d(S), _d(x), tol_rel, maxit, _d(out))
    return x, {"rel_res_true": out[0], "iters": int(out[1]), "incompat": out[2]}, st


def true_relres(dx, dy, S, x):
    """||P(b - A x)|| / ||P b|| with b = -V S and P the zero-sum projection."""
    b = scaled_rhs(dx, dy, S).reshape(-1)
    b = b - b.mean()
    r = b - apply(dx, dy, x).reshape(-1)
    r = r - r.mean()
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def volume_mean_free(dx, dy, x):
    V = np.outer(dy, dx)
    return x - (V * x).sum() / V.sum()
