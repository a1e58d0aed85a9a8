"""FP64 CPU oracle for iterative sketching (Epperly, arXiv:2311.04362).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never imports, links or calls it, and it shares no code with the
CUDA path (see ``ls_oracle.c`` for the per-function citations).

This module is a ctypes binding of ``ls_oracle.c``; arrays are numpy float64 /
int32 / uint32 / int64.  ``A`` is row-major (C order) ``m x n``; sketch and R
matrices are returned as Fortran-ordered numpy arrays, matching the
column-major layout the C code uses.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ls_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ls_oracle.c into oracle/liboracle.so with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    I64 = C.c_int64
    lib.or_philox4x32_10.argtypes = [P, P, P]
    lib.or_bounded_draw_test.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, P]
    lib.or_sparse_sign_column.argtypes = [C.c_uint64, I64, I64, C.c_int, P, P]
    lib.or_sketch_indices.argtypes = [I64, I64, C.c_int, C.c_uint64, P, P]
    lib.or_sketch_csr.argtypes = [I64, I64, C.c_int, P, P, P, P]
    lib.or_sketch_apply.argtypes = [P, I64, I64, I64, P, I64, P, P, C.c_double, P, I64]
    lib.or_householder_qr.argtypes = [P, I64, I64, I64, I64, P]
    lib.or_factor.argtypes = [P, I64, I64, I64, P, I64, P, C.c_uint64, P, P]
    lib.or_normest.argtypes = [P, I64, I64, C.c_uint64]
    lib.or_normest.restype = C.c_double
    lib.or_condest.argtypes = [P, I64, I64, C.c_uint64, C.c_double]
    lib.or_condest.restype = C.c_double
    lib.or_power_steps.argtypes = [I64]
    lib.or_power_steps.restype = I64
    lib.or_residual_gradient.argtypes = [P, I64, I64, I64, P, P, P, P]
    lib.or_iterate.argtypes = [P, I64, I64, I64, P, P, I64, P, C.c_int, C.c_int, C.c_int,
                               C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_int, C.c_double, C.c_double, P]
    lib.or_qr_solve.argtypes = [P, I64, I64, I64, P, P]
    lib.or_solve.argtypes = [P, P, I64, I64, I64, I64, C.c_int, C.c_int, C.c_uint64,
                             C.c_int, C.c_int, P, P]
    lib.or_inv_norm1_est.argtypes = [P, I64, I64]
    lib.or_inv_norm1_est.restype = C.c_double
    lib.or_norm1_upper.argtypes = [P, I64, I64]
    lib.or_norm1_upper.restype = C.c_double
    lib.or_trsv_upper.argtypes = [P, I64, I64, P, P]
    lib.or_trsv_upper_T.argtypes = [P, I64, I64, P, P]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _rowmajor(A):
    A = np.asarray(A, dtype=np.float64)
    if A.ndim != 2 or A.strides[1] != 8 or A.strides[0] % 8:
        A = np.ascontiguousarray(A)
    return A, A.strides[0] // 8


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def bounded_draws(seed: int, j: int, rng: int, ndraws: int):
    """Draws uniform in [0, rng) from column j's word stream (no sign word)."""
    lib = _load()
    out = np.zeros(ndraws, dtype=np.uint32)
    lib.or_bounded_draw_test(seed, j, rng, ndraws, _p(out))
    return out


def sparse_sign_column(seed: int, j: int, d: int, zeta: int):
    lib = _load()
    rows = np.zeros(zeta, dtype=np.int32)
    mask = np.zeros(1, dtype=np.uint32)
    rc = lib.or_sparse_sign_column(seed, j, d, zeta, _p(rows), _p(mask))
    if rc != 0:
        raise ValueError("invalid (d, zeta)")
    return rows, int(mask[0])


def sketch_indices(m: int, d: int, zeta: int, seed: int):
    lib = _load()
    rows = np.zeros((m, zeta), dtype=np.int32)
    signs = np.zeros(m, dtype=np.uint32)
    if lib.or_sketch_indices(m, d, zeta, seed, _p(rows), _p(signs)) != 0:
        raise ValueError("invalid (d, zeta)")
    return rows, signs


def sketch_csr(m: int, d: int, zeta: int, rows, signs):
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    signs = np.ascontiguousarray(signs, dtype=np.uint32)
    row_ptr = np.zeros(d + 1, dtype=np.int64)
    ent = np.zeros(m * zeta, dtype=np.uint32)
    if lib.or_sketch_csr(m, d, zeta, _p(rows), _p(signs), _p(row_ptr), _p(ent)) != 0:
        raise MemoryError
    return row_ptr, ent


def sketch_scale(zeta: int) -> float:
    return 1.0 / np.sqrt(np.float64(zeta))


def sketch_apply(A, b, d: int, row_ptr, ent, s: float):
    """B_aug = s * S [A b], returned as a Fortran-ordered (d, n+1) array."""
    lib = _load()
    A, lda = _rowmajor(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    B = np.zeros((d, n + 1), dtype=np.float64, order="F")
    lib.or_sketch_apply(_p(A), m, n, lda, _p(b), d, _p(np.ascontiguousarray(row_ptr, dtype=np.int64)),
                        _p(np.ascontiguousarray(ent, dtype=np.uint32)), float(s), _p(B), d)
    return B


def sketch(A, b, d: int, zeta: int, seed: int):
    A, _ = _rowmajor(A)
    m = A.shape[0]
    rows, signs = sketch_indices(m, d, zeta, seed)
    row_ptr, ent = sketch_csr(m, d, zeta, rows, signs)
    return sketch_apply(A, b, d, row_ptr, ent, sketch_scale(zeta))


def householder_qr(B, nref: int | None = None):
    """In-place-style Householder QR of a copy of B (column-major); returns (F, tau, rc)."""
    lib = _load()
    F = np.array(B, dtype=np.float64, order="F", copy=True)
    rows, ncols = F.shape
    nref = ncols if nref is None else nref
    tau = np.zeros(max(nref, 1), dtype=np.float64)
    rc = lib.or_householder_qr(_p(F), rows, ncols, nref, rows, _p(tau))
    return F, tau[:nref], rc


def factor(B_aug, seed: int = 0):
    """QR of B_aug (d x (n+1)) -> (R, x0, normest, condest, rc)."""
    lib = _load()
    F = np.array(B_aug, dtype=np.float64, order="F", copy=True)
    d, n1 = F.shape
    n = n1 - 1
    R = np.zeros((n, n), dtype=np.float64, order="F")
    x0 = np.zeros(n, dtype=np.float64)
    ne = np.zeros(1)
    ce = np.zeros(1)
    rc = lib.or_factor(_p(F), d, n, d, _p(R), n, _p(x0), seed, _p(ne), _p(ce))
    return R, x0, float(ne[0]), float(ce[0]), rc


def power_steps(n: int) -> int:
    return int(_load().or_power_steps(n))


def normest(R, seed: int = 0) -> float:
    R = np.asfortranarray(R, dtype=np.float64)
    return float(_load().or_normest(_p(R), R.shape[0], R.shape[0], seed))


def condest(R, seed: int = 0, normest_value: float | None = None) -> float:
    R = np.asfortranarray(R, dtype=np.float64)
    ne = normest(R, seed) if normest_value is None else normest_value
    return float(_load().or_condest(_p(R), R.shape[0], R.shape[0], seed, ne))


def inv_norm1_est(R) -> float:
    R = np.asfortranarray(R, dtype=np.float64)
    return float(_load().or_inv_norm1_est(_p(R), R.shape[0], R.shape[0]))


def norm1_upper(R) -> float:
    R = np.asfortranarray(R, dtype=np.float64)
    return float(_load().or_norm1_upper(_p(R), R.shape[0], R.shape[0]))


def trsv_upper(R, z):
    R = np.asfortranarray(R, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    x = np.zeros_like(z)
    _load().or_trsv_upper(_p(R), R.shape[0], R.shape[0], _p(z), _p(x))
    return x


def trsv_upper_T(R, c):
    R = np.asfortranarray(R, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    y = np.zeros_like(c)
    _load().or_trsv_upper_T(_p(R), R.shape[0], R.shape[0], _p(c), _p(y))
    return y


def residual_gradient(A, b, x):
    """r = b - A x, c = A^T r (plain ascending loops)."""
    A, lda = _rowmajor(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.zeros(m)
    c = np.zeros(n)
    _load().or_residual_gradient(_p(A), m, n, lda, _p(b), _p(x), _p(r), _p(c))
    return r, c


def _veltkamp(a):
    """a = hi + lo exactly, hi with at most 26 significant bits (Veltkamp's
    splitting with the constant 2^27 + 1; no overflow for |a| < 2^996)."""
    c = 134217729.0 * a
    hi = c - (c - a)
    return hi, a - hi


def two_product(a, b):
    """p + e = a b exactly (Dekker's product from the splitting above), for
    FP64 arrays whose products neither overflow nor underflow."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p = a * b
    ah, al = _veltkamp(a)
    bh, bl = _veltkamp(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def residual_exact(A, b, x, rows=None):
    """r_j = b_j - sum_k A_jk x_k rounded once to FP64 (the residual of the
    Algorithm 2 loop in exact arithmetic): every product split exactly into
    two doubles, then math.fsum (exact sum, one rounding).  rows: indices to
    compute (default all).  For the error analysis of Sec. 4.3 this is r(x)
    with f = 0 up to a final rounding."""
    import math

    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    rows = range(A.shape[0]) if rows is None else rows
    out = []
    for j in rows:
        p, e = two_product(A[j], x)
        out.append(math.fsum([float(b[j]), *(-p).tolist(), *(-e).tolist()]))
    return np.array(out)


def gradient_exact(A, r, cols=None):
    """c_k = sum_j A_jk r_j rounded once to FP64 (A^T r in exact arithmetic,
    same construction as residual_exact)."""
    import math

    A = np.asarray(A, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    cols = range(A.shape[1]) if cols is None else cols
    out = []
    for k in cols:
        p, e = two_product(A[:, k], r)
        out.append(math.fsum([*p.tolist(), *e.tolist()]))
    return np.array(out)


def iterate(A, b, R, x0, q: int, normest_value: float, condest_value: float, *,
            use_stop: bool = True, extra: int = 0, gamma: float = 1.0, rho: float = 0.04,
            variant: int = 0, alpha: float = 1.0, beta: float = 0.0):
    """Algorithm 2 loop from x0.  Returns (x, info dict)."""
    A, lda = _rowmajor(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    R = np.asfortranarray(R, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    out = np.zeros(4)
    rc = _load().or_iterate(_p(A), m, n, lda, _p(b), _p(R), R.shape[0], _p(x), q, int(use_stop), extra,
                            gamma, rho, normest_value, condest_value, variant, alpha, beta, _p(out))
    if rc != 0:
        raise MemoryError
    return x, {"iters": int(out[0]), "converged": bool(out[1]), "res_norm": out[2], "step_norm": out[3]}


def qr_solve(A, b):
    """Direct Householder-QR least-squares solution (the forward-error yardstick)."""
    A, lda = _rowmajor(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    rc = _load().or_qr_solve(_p(A), m, n, lda, _p(b), _p(x))
    if rc != 0:
        raise ArithmeticError(f"rank deficiency at column {rc - 1}")
    return x


def solve(A, b, d: int, zeta: int, q: int, seed: int, *, use_stop: bool = True, extra: int = 0):
    """Whole method: sketch, factor, sketch-and-solve start, iterate."""
    A, lda = _rowmajor(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    info = np.zeros(6)
    rc = _load().or_solve(_p(A), _p(b), m, n, lda, d, zeta, q, seed, int(use_stop), extra, _p(x), _p(info))
    if rc != 0:
        raise ArithmeticError(f"oracle solve failed: {rc}")
    return x, {"iters": int(info[0]), "converged": bool(info[1]), "res_norm": info[2],
               "step_norm": info[3], "normest": info[4], "condest": info[5]}


def forward_error(x_hat, x) -> float:
    return float(np.linalg.norm(x - x_hat) / np.linalg.norm(x))


def qr_solve_lapack(A, b):
    """Householder QR least-squares solve through LAPACK (numpy.linalg.qr is
    dgeqrf/dorgqr, blocked Householder) -- the same method as ``qr_solve``
    for matrices too large for the plain loops.  x = R^{-1} (Q^T b)."""
    import scipy.linalg as sl

    A = np.asarray(A, dtype=np.float64)
    Q, R = np.linalg.qr(A, mode="reduced")
    z = Q.T @ np.asarray(b, dtype=np.float64)
    del Q
    return sl.solve_triangular(R, z, lower=False)
