"""Python access to the CPU FP64 oracle (``tpfa_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark.  The CUDA library and its binding never
import, link or call anything here, and nothing here imports them.

Every function takes and returns numpy arrays in the flat X-innermost layout
``c = i + nx*(j + ny*k)`` and computes in double precision.  What each one
computes, and which passage of the paper it follows, is stated in the C
source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpfa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt oracle library may be named in TPFA_ORACLE_LIB; the oracle's
# own mutation test uses this to run the pins against deliberately broken
# copies of the source.
_LIB_OVERRIDE = os.environ.get("TPFA_ORACLE_LIB")


def compile_to(src: str, out: str) -> str:
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, -O2, OpenMP)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_to(_SRC, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("mu", C.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        G = C.POINTER(_Grid)
        _lib.orc_assemble.argtypes = [G, P, P, P, C.c_double, C.c_int, P, P, P]
        _lib.orc_assemble.restype = C.c_int64
        _lib.orc_rhs.argtypes = [G, P, P, P, P, C.c_int, P]
        _lib.orc_rhs_transient.argtypes = [G, P, P, P, P, P, C.c_double, P, P]
        _lib.orc_coefficients.argtypes = [G, P, P, P, C.c_double, P, P, P, P]
        _lib.orc_face_trans.argtypes = [G, P, P, P, P]
        _lib.orc_extra_diagonal.argtypes = [G, P, P, P, C.c_double, P]
        _lib.orc_apply_rows.argtypes = [G, P, P, P, C.c_double, P, C.c_int64, P, P]
        _lib.orc_abs_apply_rows.argtypes = [G, P, P, P, C.c_double, P, C.c_int64, P, P]
        _lib.orc_net_flux.argtypes = [G, P, P, P]
        _lib.orc_spmv.argtypes = [C.c_int64, P, P, P, P, P]
        _lib.orc_cg.argtypes = [C.c_int64, P, P, P, P, P, C.c_double, C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(C.c_double), P, C.c_int64]
        _lib.orc_cg.restype = C.c_int
        _lib.orc_pcg_jacobi.argtypes = _lib.orc_cg.argtypes
        _lib.orc_pcg_jacobi.restype = C.c_int
        _lib.orc_threads.argtypes = []
        _lib.orc_threads.restype = C.c_int
        _lib.orc_cholesky_solve.argtypes = [C.c_int64, P, P, P]
        _lib.orc_cholesky_solve.restype = C.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


class Grid:
    """Structured grid: nx, ny, nz cells of size dx, dy, dz; viscosity mu."""

    def __init__(self, nx, ny, nz, dx=1.0, dy=1.0, dz=1.0, mu=1.0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy, self.dz, self.mu = float(dx), float(dy), float(dz), float(mu)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def _c(self):
        return C.byref(_Grid(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.mu))


def _dargs(d):
    """d may be a per-cell array or a scalar applied to every cell."""
    if d is None:
        return None, 0.0
    if np.isscalar(d):
        return None, float(d)
    return _f64(d), 0.0


class CSR:
    def __init__(self, n, rowptr, cols, vals):
        self.n, self.rowptr, self.cols, self.vals = n, rowptr, cols, vals

    def dense(self):
        A = np.zeros((self.n, self.n))
        for r in range(self.n):
            s, e = self.rowptr[r], self.rowptr[r + 1]
            A[r, self.cols[s:e]] += self.vals[s:e]
        return A

    def matvec(self, x):
        y = np.empty(self.n)
        x = _f64(x)
        _L().orc_spmv(self.n, _p(self.rowptr), _p(self.cols), _p(self.vals), _p(x), _p(y))
        return y


def assemble(g: Grid, K, mask=None, d=None, literal=False) -> CSR:
    """Explicit CSR of the operator (symmetric eliminated form, or Eq. 6 as printed)."""
    K, mask = _f64(K), _u8(mask)
    da, d0 = _dargs(d)
    n = g.n
    rowptr = np.empty(n + 1, np.int64)
    cols = np.empty(7 * n, np.int64)
    vals = np.empty(7 * n, np.float64)
    nnz = _L().orc_assemble(g._c(), _p(K), _p(mask), _p(da), d0, int(bool(literal)),
                            _p(rowptr), _p(cols), _p(vals))
    # views of the first nnz entries (no copy: the paper-scale matrix is tens of GB)
    return CSR(n, rowptr, cols[:nnz], vals[:nnz])


def rhs(g: Grid, K, mask=None, q=None, pD=None, literal=False):
    b = np.empty(g.n)
    _L().orc_rhs(g._c(), _p(_f64(K)), _p(_u8(mask)), _p(_f64(q)), _p(_f64(pD)),
                 int(bool(literal)), _p(b))
    return b


def rhs_transient(g: Grid, K, mask, q, pD, d, p_prev):
    """Right-hand side of one backward-Euler step: rhs + d * p_prev on interior cells."""
    da, d0 = _dargs(d)
    b = np.empty(g.n)
    _L().orc_rhs_transient(g._c(), _p(_f64(K)), _p(_u8(mask)), _p(_f64(q)), _p(_f64(pD)),
                           _p(da), d0, _p(_f64(p_prev)), _p(b))
    return b


def transient(g: Grid, K, mask, d, q, pD, p0, steps, tol=1e-12):
    """Backward-Euler steps: A p^{n+1} = q + d p^n (+ Dirichlet lifts), each
    solved by CG from p^n.  Returns the list [p^1, ..., p^steps]."""
    A = assemble(g, K, mask, d)
    out, p = [], _f64(p0).copy()
    for _ in range(steps):
        b = rhs_transient(g, K, mask, q, pD, d, p)
        p, st, _, _ = cg(A, b, x0=p, tol=tol)
        if st < 0:
            raise RuntimeError(f"oracle CG failed with status {st}")
        out.append(p.copy())
    return out


def coefficients(g: Grid, K, mask=None, d=None):
    """(Tx, Ty, Tz, D) of the eliminated operator, float64 each."""
    K, mask = _f64(K), _u8(mask)
    da, d0 = _dargs(d)
    out = [np.empty(g.n) for _ in range(4)]
    _L().orc_coefficients(g._c(), _p(K), _p(mask), _p(da), d0, *[_p(o) for o in out])
    return tuple(out)


def extra_diagonal(g: Grid, K, mask=None, d=None):
    """E with (A x)_K = sum_f T'_f (x_K - x_L) + E_K x_K (see the C source)."""
    K, mask = _f64(K), _u8(mask)
    da, d0 = _dargs(d)
    E = np.empty(g.n)
    _L().orc_extra_diagonal(g._c(), _p(K), _p(mask), _p(da), d0, _p(E))
    return E


def face_trans(g: Grid, K):
    out = [np.empty(g.n) for _ in range(3)]
    _L().orc_face_trans(g._c(), _p(_f64(K)), *[_p(o) for o in out])
    return tuple(out)


def apply_rows(g: Grid, K, mask, d, rows, x):
    """(A x) at the listed rows only, evaluated row by row from K."""
    K, mask, x = _f64(K), _u8(mask), _f64(x)
    da, d0 = _dargs(d)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(len(rows))
    _L().orc_apply_rows(g._c(), _p(K), _p(mask), _p(da), d0, _p(rows), len(rows), _p(x), _p(y))
    return y


def abs_apply_rows(g: Grid, K, mask, d, rows, x):
    """(|A| |x|) at the listed rows: the rounding scale of (A x) there."""
    K, mask, x = _f64(K), _u8(mask), _f64(x)
    da, d0 = _dargs(d)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(len(rows))
    _L().orc_abs_apply_rows(g._c(), _p(K), _p(mask), _p(da), d0, _p(rows), len(rows), _p(x),
                            _p(y))
    return y


def net_flux(g: Grid, K, x):
    y = np.empty(g.n)
    _L().orc_net_flux(g._c(), _p(_f64(K)), _p(_f64(x)), _p(y))
    return y


def cg(A: CSR, b, x0=None, tol=1e-12, maxit=None, history=0):
    """Textbook CG.  Returns (x, status, iterations, recursive relative residual[, history])."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    maxit = 10 * A.n + 10 if maxit is None else int(maxit)
    it, rr = C.c_int64(0), C.c_double(0.0)
    hist = np.zeros((history, A.n)) if history else None
    st = _L().orc_cg(A.n, _p(A.rowptr), _p(A.cols), _p(A.vals), _p(b), _p(x), float(tol), maxit,
                     C.byref(it), C.byref(rr), _p(hist), int(history))
    if history:
        return x, st, it.value, rr.value, hist
    return x, st, it.value, rr.value


def pcg_jacobi(A: CSR, b, x0=None, tol=1e-12, maxit=None, history=0):
    """CG preconditioned with diag(A).  Returns (x, status, iterations,
    recursive relative residual[, history]) like cg()."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    maxit = 10 * A.n + 10 if maxit is None else int(maxit)
    it, rr = C.c_int64(0), C.c_double(0.0)
    hist = np.zeros((history, A.n)) if history else None
    st = _L().orc_pcg_jacobi(A.n, _p(A.rowptr), _p(A.cols), _p(A.vals), _p(b), _p(x),
                             float(tol), maxit, C.byref(it), C.byref(rr), _p(hist), int(history))
    if history:
        return x, st, it.value, rr.value, hist
    return x, st, it.value, rr.value


def threads():
    """Host threads the oracle's parallel loops use (OpenMP)."""
    return int(_L().orc_threads())


def cholesky_solve(Adense, b):
    A = np.array(Adense, dtype=np.float64, order="C")
    x = np.empty(A.shape[0])
    st = _L().orc_cholesky_solve(A.shape[0], _p(A), _p(_f64(b)), _p(x))
    if st != 0:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    return x


def solve(g: Grid, K, mask=None, d=None, q=None, pD=None, tol=1e-12, maxit=None, x0=None,
          jacobi=False):
    """Assemble and solve A p = b (plain CG, or Jacobi PCG with jacobi=True);
    returns (p, iterations)."""
    A = assemble(g, K, mask, d)
    b = rhs(g, K, mask, q, pD)
    x, st, it, _ = (pcg_jacobi if jacobi else cg)(A, b, x0=x0, tol=tol, maxit=maxit)
    if st < 0:
        raise RuntimeError(f"oracle CG failed with status {st}")
    return x, it


def rel_residual(g: Grid, K, mask, d, q, pD, x):
    """||b - A x||_2 / ||b||_2 evaluated with the assembled FP64 operator."""
    A = assemble(g, K, mask, d)
    b = rhs(g, K, mask, q, pD)
    r = b - A.matvec(x)
    nb = np.linalg.norm(b)
    return np.linalg.norm(r) / (nb if nb > 0 else 1.0)
