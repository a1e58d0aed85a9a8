"""Python binding of libls (include/ls.h): iterative sketching for
overdetermined least squares on GB300 (Epperly, arXiv:2311.04362).

Argument marshalling only: every step runs in the CUDA kernels of
``libls.so``.  Array arguments are torch CUDA tensors (float64 / int32 /
uint32 / int64, contiguous as documented in ``include/ls.h``) or raw
integer pointers.  PyTorch provides device memory and the stream.

The library must have been built (``python -m paper_2311_04362_gb300.build``
or ``__graft_entry__.build()``); importing the binding without it raises.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB as _LIB_PATH

LS_OK, LS_EINVAL, LS_ENOMEM, LS_ECUDA, LS_ERANK, LS_ENONFINITE, LS_ETIMEOUT, LS_ENOTCONV = range(8)
LS_FAULT_NONE, LS_FAULT_SKIP_TILE, LS_FAULT_ALLOC = range(3)
STATUS_NAMES = ["LS_OK", "LS_EINVAL", "LS_ENOMEM", "LS_ECUDA", "LS_ERANK", "LS_ENONFINITE", "LS_ETIMEOUT",
                "LS_ENOTCONV"]


class LsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class ls_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("stop_reason", C.c_int), ("res_norm", C.c_double),
                ("step_norm", C.c_double), ("normest", C.c_double), ("condest", C.c_double),
                ("ms_sketch", C.c_float), ("ms_factor", C.c_float), ("ms_iterate", C.c_float),
                ("ms_pass", C.c_float), ("n_pass", C.c_int), ("launches", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ls_opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("rho", C.c_double), ("extra_iters", C.c_int), ("use_stop", C.c_int),
                ("alpha", C.c_double), ("beta", C.c_double)]


class ls_problem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p), ("m", C.c_int64), ("n", C.c_int64),
                ("lda", C.c_int64), ("d", C.c_int64), ("seed", C.c_uint64), ("B_out", C.c_void_p),
                ("R_out", C.c_void_p)]


class ls_server_stats(C.Structure):
    _fields_ = [("inflight", C.c_int64), ("queued", C.c_int64), ("completed", C.c_int64), ("steps", C.c_int64),
                ("admitted_bytes", C.c_size_t), ("workspace_bytes_used", C.c_size_t)]


_lib = None


def lib():
    """The loaded libls.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libls.so not built at {_LIB_PATH}; run paper_2311_04362_gb300.build.build()")
    L = C.CDLL(_LIB_PATH)
    P, I64, I = C.c_void_p, C.c_int64, C.c_int
    S = C.c_int
    L.ls_default_opts.argtypes = [C.POINTER(ls_opts)]
    L.ls_create.argtypes = [C.POINTER(P), I, P]
    L.ls_create.restype = S
    L.ls_destroy.argtypes = [P]
    L.ls_destroy.restype = S
    L.ls_last_error.argtypes = [P]
    L.ls_last_error.restype = C.c_char_p
    L.ls_workspace_bytes.argtypes = [I64, I64, I64, I]
    L.ls_workspace_bytes.restype = C.c_size_t
    L.ls_sketch_indices.argtypes = [P, I64, I64, I, C.c_uint64, P, P]
    L.ls_sketch_indices.restype = S
    L.ls_sketch_csr.argtypes = [P, I64, I64, I, P, P, P, P]
    L.ls_sketch_csr.restype = S
    L.ls_sketch.argtypes = [P, P, I64, I64, I64, P, I64, I, C.c_uint64, P, I64]
    L.ls_sketch.restype = S
    L.ls_factor.argtypes = [P, P, I64, I64, I64, P, I64, P, C.c_uint64, C.POINTER(ls_info)]
    L.ls_factor.restype = S
    L.ls_residual_gradient.argtypes = [P, P, I64, I64, I64, P, P, P, P, P, P]
    L.ls_residual_gradient.restype = S
    L.ls_correct.argtypes = [P, P, I64, I64, P, P, P, P]
    L.ls_correct.restype = S
    L.ls_iterate.argtypes = [P, P, I64, I64, I64, P, P, I64, P, I, C.POINTER(ls_opts), C.POINTER(ls_info)]
    L.ls_iterate.restype = S
    L.ls_solve.argtypes = [P, P, P, I64, I64, I64, I64, I, I, C.c_uint64, P, C.POINTER(ls_info)]
    L.ls_solve.restype = S
    L.ls_solve_ex.argtypes = [P, P, P, I64, I64, I64, I64, I, I, C.c_uint64, C.POINTER(ls_opts), P,
                              C.POINTER(ls_info)]
    L.ls_solve_ex.restype = S
    L.ls_opts_damping.argtypes = [C.POINTER(ls_opts), I64, I64]
    L.ls_opts_momentum.argtypes = [C.POINTER(ls_opts), I64, I64]
    L.ls_solve_batched.argtypes = [P, C.POINTER(ls_problem), I, I, I, C.POINTER(ls_opts), C.POINTER(ls_info)]
    L.ls_solve_batched.restype = S
    L.ls_solve_batched_mixed.argtypes = [P, C.POINTER(ls_problem), I, I, I, C.POINTER(ls_opts), C.POINTER(ls_info)]
    L.ls_solve_batched_mixed.restype = S
    L.ls_tune_batched.argtypes = [P, C.POINTER(ls_problem), I, I, C.c_char_p, C.c_size_t]
    L.ls_tune_batched.restype = S
    L.ls_reset_tuning.argtypes = [P]
    L.ls_reset_tuning.restype = S
    L.ls_sketch_sparse.argtypes = [P, P, P, P, I64, I64, P, I64, I, C.c_uint64, P, I64]
    L.ls_sketch_sparse.restype = S
    L.ls_solve_sparse.argtypes = [P, P, P, P, I64, I64, I64, P, I64, I, I, C.c_uint64, C.POINTER(ls_opts), P,
                                  C.POINTER(ls_info)]
    L.ls_solve_sparse.restype = S
    L.ls_server_request_bytes.argtypes = [I64, I64, I64, I64]
    L.ls_server_request_bytes.restype = C.c_size_t
    L.ls_server_create.argtypes = [P, I, I64, C.c_size_t, C.c_size_t, I, I, C.POINTER(ls_opts), C.POINTER(P)]
    L.ls_server_create.restype = S
    L.ls_server_destroy.argtypes = [P]
    L.ls_server_destroy.restype = S
    L.ls_server_submit.argtypes = [P, C.POINTER(ls_problem), C.POINTER(C.c_int64)]
    L.ls_server_submit.restype = S
    L.ls_server_step.argtypes = [P, C.POINTER(I)]
    L.ls_server_step.restype = S
    L.ls_server_poll.argtypes = [P, P, C.POINTER(ls_info), I, C.POINTER(I)]
    L.ls_server_poll.restype = S
    L.ls_server_get_stats.argtypes = [P, C.POINTER(ls_server_stats)]
    L.ls_server_get_stats.restype = S
    L.ls_residual_gradient_noalloc.argtypes = [P, P, I64, I64, I64, P, P, P, P, P, P]
    L.ls_residual_gradient_noalloc.restype = S
    L.ls_fixed_point.argtypes = [P, P, I64, I64, I64, P, I64, P]
    L.ls_fixed_point.restype = S
    L.ls_residual_gradient_fx.argtypes = [P, P, P, I64, I64, I64, P, P, P, P, P, P]
    L.ls_residual_gradient_fx.restype = S
    L.ls_set_wait_limit.argtypes = [P, C.c_uint64]
    L.ls_set_wait_limit.restype = S
    L.ls_iterate_rows.argtypes = [P, I, C.POINTER(P), C.POINTER(I64), I64, I64, C.POINTER(P), P, I64, P, I,
                                  C.POINTER(ls_opts), C.POINTER(ls_info)]
    L.ls_iterate_rows.restype = S
    L.ls_inject_fault.argtypes = [P, I, I64]
    L.ls_inject_fault.restype = S
    _lib = L
    return L


def _ptr(t):
    """Pointer of a tensor / numpy array / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(t)}")


def default_opts() -> ls_opts:
    o = ls_opts()
    lib().ls_default_opts(C.byref(o))
    return o


def damping_opts(n: int, d: int) -> ls_opts:
    """Defaults with the damping weights of App. B, Eq. (B.2), e = sqrt(n/d)."""
    o = default_opts()
    lib().ls_opts_damping(C.byref(o), n, d)
    return o


def momentum_opts(n: int, d: int) -> ls_opts:
    """Defaults with the momentum weights of App. B, Eq. (B.3), e = sqrt(n/d)."""
    o = default_opts()
    lib().ls_opts_momentum(C.byref(o), n, d)
    return o


def workspace_bytes(m, n, d, zeta) -> int:
    return int(lib().ls_workspace_bytes(m, n, d, zeta))


class Context:
    """Owns an ls_ctx (device scratch arena) bound to a device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self._h = C.c_void_p()
        sp = None
        if stream is not None:
            sp = stream if isinstance(stream, int) else stream.cuda_stream
        st = lib().ls_create(C.byref(self._h), device, sp)
        if st != LS_OK:
            raise LsError(st, "ls_create failed (needs an sm_103 GPU)")

    def close(self):
        if self._h:
            lib().ls_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def _check(self, st, allow=(LS_OK,)):
        if st not in allow:
            raise LsError(st, lib().ls_last_error(self._h).decode())
        return st

    # ---- entry points (same names as the C ABI) -----------------------------
    def ls_sketch_indices(self, m, d, zeta, seed, rows, signs):
        return self._check(lib().ls_sketch_indices(self._h, m, d, zeta, seed, _ptr(rows), _ptr(signs)))

    def ls_sketch_csr(self, m, d, zeta, rows, signs, row_ptr, ent):
        return self._check(lib().ls_sketch_csr(self._h, m, d, zeta, _ptr(rows), _ptr(signs), _ptr(row_ptr),
                                               _ptr(ent)))

    def ls_sketch(self, A, m, n, lda, b, d, zeta, seed, B, ldb):
        return self._check(lib().ls_sketch(self._h, _ptr(A), m, n, lda, _ptr(b), d, zeta, seed, _ptr(B), ldb))

    def ls_factor(self, B, d, n, ldb, R, ldr, x0, seed, info=None):
        info = info if info is not None else ls_info()
        self._check(lib().ls_factor(self._h, _ptr(B), d, n, ldb, _ptr(R), ldr, _ptr(x0), seed, C.byref(info)))
        return info

    def ls_residual_gradient(self, A, m, n, lda, b, x, r_prev, r_out, c, norms):
        return self._check(lib().ls_residual_gradient(self._h, _ptr(A), m, n, lda, _ptr(b), _ptr(x),
                                                      _ptr(r_prev), _ptr(r_out), _ptr(c), _ptr(norms)))

    def ls_fixed_point(self, A, m, n, lda, A_fx, ldf, row_exp):
        return self._check(lib().ls_fixed_point(self._h, _ptr(A), m, n, lda, _ptr(A_fx), ldf, _ptr(row_exp)))

    def ls_residual_gradient_fx(self, A_fx, row_exp, m, n, ldf, b, x, r_prev, r_out, c, norms):
        return self._check(lib().ls_residual_gradient_fx(self._h, _ptr(A_fx), _ptr(row_exp), m, n, ldf, _ptr(b),
                                                         _ptr(x), _ptr(r_prev), _ptr(r_out), _ptr(c), _ptr(norms)))

    def ls_iterate_rows(self, A_parts, m_parts, n, lda, b_parts, R, ldr, x, q, opts=None, info=None):
        info = info if info is not None else ls_info()
        k = len(A_parts)
        Ap = (C.c_void_p * k)(*[_ptr(a) for a in A_parts])
        bp = (C.c_void_p * k)(*[_ptr(b) for b in b_parts])
        mp = (C.c_int64 * k)(*m_parts)
        st = lib().ls_iterate_rows(self._h, k, Ap, mp, n, lda, bp, _ptr(R), ldr, _ptr(x), q,
                                   C.byref(opts) if opts is not None else None, C.byref(info))
        self._check(st, allow=(LS_OK, LS_ENOTCONV))
        return st, info

    def ls_set_wait_limit(self, ns):
        return self._check(lib().ls_set_wait_limit(self._h, ns))

    def ls_inject_fault(self, kind, arg=0):
        return self._check(lib().ls_inject_fault(self._h, kind, arg))

    def ls_correct(self, R, ldr, n, c, x, y_out=None, d_out=None):
        return self._check(lib().ls_correct(self._h, _ptr(R), ldr, n, _ptr(c), _ptr(x), _ptr(y_out), _ptr(d_out)))

    def ls_iterate(self, A, m, n, lda, b, R, ldr, x, q, opts=None, info=None):
        info = info if info is not None else ls_info()
        st = lib().ls_iterate(self._h, _ptr(A), m, n, lda, _ptr(b), _ptr(R), ldr, _ptr(x), q,
                              C.byref(opts) if opts is not None else None, C.byref(info))
        self._check(st, allow=(LS_OK, LS_ENOTCONV))
        return st, info

    def ls_solve_ex(self, A, b, m, n, lda, d, zeta, q, seed, opts, x, info=None):
        info = info if info is not None else ls_info()
        st = lib().ls_solve_ex(self._h, _ptr(A), _ptr(b), m, n, lda, d, zeta, q, seed,
                               C.byref(opts) if opts is not None else None, _ptr(x), C.byref(info))
        self._check(st, allow=(LS_OK, LS_ENOTCONV))
        return st, info

    def ls_sketch_sparse(self, row_ptr, col, val, m, n, b, d, zeta, seed, B, ldb):
        return self._check(lib().ls_sketch_sparse(self._h, _ptr(row_ptr), _ptr(col), _ptr(val), m, n, _ptr(b), d,
                                                  zeta, seed, _ptr(B), ldb))

    def ls_solve_sparse(self, row_ptr, col, val, m, n, nnz, b, d, zeta, q, seed, x, opts=None, info=None):
        info = info if info is not None else ls_info()
        st = lib().ls_solve_sparse(self._h, _ptr(row_ptr), _ptr(col), _ptr(val), m, n, nnz, _ptr(b), d, zeta, q,
                                   seed, C.byref(opts) if opts is not None else None, _ptr(x), C.byref(info))
        self._check(st, allow=(LS_OK, LS_ENOTCONV))
        return st, info

    def ls_solve(self, A, b, m, n, lda, d, zeta, q, seed, x, info=None):
        info = info if info is not None else ls_info()
        st = lib().ls_solve(self._h, _ptr(A), _ptr(b), m, n, lda, d, zeta, q, seed, _ptr(x), C.byref(info))
        self._check(st, allow=(LS_OK, LS_ENOTCONV))
        return st, info

    def ls_solve_batched(self, probs, zeta, q, opts=None, infos=None, mixed=False):
        """probs: sequence of ls_problem (or dicts with its fields; tensors are
        taken by pointer).  Returns the ls_info array (one per problem).
        mixed=True calls ls_solve_batched_mixed (FP32 sketch and QR)."""
        arr = (ls_problem * len(probs))()
        for i, p in enumerate(probs):
            if isinstance(p, ls_problem):
                arr[i] = p
                continue
            arr[i] = ls_problem(_ptr(p["A"]), _ptr(p["b"]), _ptr(p["x"]), p["m"], p["n"], p["lda"], p["d"],
                                p.get("seed", i), _ptr(p.get("B_out")), _ptr(p.get("R_out")))
        infos = infos if infos is not None else (ls_info * len(probs))()
        fn = lib().ls_solve_batched_mixed if mixed else lib().ls_solve_batched
        self._check(fn(self._h, arr, len(probs), zeta, q, C.byref(opts) if opts is not None else None, infos))
        return infos

    def ls_tune_batched(self, probs, reps=3) -> str:
        arr = (ls_problem * len(probs))()
        for i, p in enumerate(probs):
            arr[i] = p if isinstance(p, ls_problem) else ls_problem(
                _ptr(p["A"]), _ptr(p["b"]), _ptr(p.get("x")), p["m"], p["n"], p["lda"], p["d"], p.get("seed", i),
                None, None)
        buf = C.create_string_buffer(4096)
        self._check(lib().ls_tune_batched(self._h, arr, len(probs), reps, buf, 4096))
        return buf.value.decode()

    def ls_reset_tuning(self):
        return self._check(lib().ls_reset_tuning(self._h))

    def ls_solve_batched_mixed(self, probs, zeta, q, opts=None, infos=None):
        return self.ls_solve_batched(probs, zeta, q, opts, infos, mixed=True)


def server_request_bytes(m, n, lda, d) -> int:
    return int(lib().ls_server_request_bytes(m, n, lda, d))


class Server:
    """Continuous-batching server (ls_server_*): submit requests, step, poll.
    Runs on its own CUDA stream; A and b must be ready before submit and x is
    final once the request comes back from poll."""

    def __init__(self, ctx: Context, max_inflight: int, max_n: int, workspace_bytes: int, admit_bytes: int = 0,
                 zeta: int = 8, q: int = 100, opts: ls_opts | None = None):
        self._ctx = ctx
        self._h = C.c_void_p()
        st = lib().ls_server_create(ctx.handle, max_inflight, max_n, workspace_bytes, admit_bytes, zeta, q,
                                    C.byref(opts) if opts is not None else None, C.byref(self._h))
        ctx._check(st)

    def close(self):
        if self._h:
            lib().ls_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def ls_server_submit(self, prob: dict) -> int:
        p = ls_problem(_ptr(prob["A"]), _ptr(prob["b"]), _ptr(prob["x"]), prob["m"], prob["n"], prob["lda"],
                       prob["d"], prob.get("seed", 0), None, None)
        t = C.c_int64()
        self._ctx._check(lib().ls_server_submit(self._h, C.byref(p), C.byref(t)))
        return t.value

    def ls_server_step(self) -> int:
        nd = C.c_int()
        self._ctx._check(lib().ls_server_step(self._h, C.byref(nd)))
        return nd.value

    def ls_server_poll(self, cap: int = 4096):
        tickets = (C.c_int64 * cap)()
        infos = (ls_info * cap)()
        n = C.c_int()
        self._ctx._check(lib().ls_server_poll(self._h, tickets, infos, cap, C.byref(n)))
        return [(tickets[i], ls_info.from_buffer_copy(infos[i])) for i in range(n.value)]

    def ls_server_get_stats(self) -> dict:
        st = ls_server_stats()
        self._ctx._check(lib().ls_server_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}


def solve(A, b, d=None, zeta=8, q=100, seed=0, ctx: Context | None = None):
    """Convenience: x = argmin ||b - A x|| for torch float64 tensors A (m x n,
    row-major; CUDA or host) and b.  Returns (x, info dict)."""
    import torch

    m, n = A.shape
    d = 20 * n if d is None else d
    if A.stride(1) != 1 or A.stride(0) % 2 or A.data_ptr() % 16:
        A = A.contiguous()
        if n % 2:
            Ap = torch.zeros(m, n + 1, dtype=A.dtype, device=A.device)
            Ap[:, :n] = A
            A = Ap
    lda = A.stride(0)
    x = torch.empty(n, dtype=torch.float64, device=b.device)
    own = ctx is None
    ctx = ctx or Context(A.device.index if A.is_cuda else 0,
                         torch.cuda.current_stream() if A.is_cuda else None)
    try:
        st, info = ctx.ls_solve(A, b.contiguous(), m, n, lda, d, zeta, q, seed, x)
    finally:
        if own:
            ctx.close()
    out = info.as_dict()
    out["status"] = STATUS_NAMES[st]
    return x, out
