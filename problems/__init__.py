"""Seeded synthetic least-squares problems shaped like the paper's experiments.

Shared by the tests, ``bench.py`` and ``__graft_entry__.smoke()``.  This module
holds none of the solver's arithmetic (no sketching, no solver QR, no
iteration): it only draws inputs.

Construction (Sec. 1.1.1 of the paper): ``A = U diag(sigma) V^T`` with ``U``
an ``m x n`` orthonormalised Gaussian (Haar after the sign fix), ``V`` an
``n x n`` orthonormalised Gaussian, ``sigma_k = kappa^{-k/(n-1)}`` (log-spaced
from 1 to 1/kappa, so ``||A|| = 1``), ``x = w/||w||`` for Gaussian ``w``,
``r = beta (I - U U^T) g / ||(I - U U^T) g||`` for Gaussian ``g`` (projected
twice), and ``b = A x + r``.
"""
from __future__ import annotations

import numpy as np


def _haar_columns(G):
    Q, Rg = np.linalg.qr(G)
    s = np.sign(np.diag(Rg))
    s[s == 0] = 1.0
    return Q * s


def sigmas(n: int, kappa: float) -> np.ndarray:
    if n == 1:
        return np.ones(1)
    return kappa ** (-np.arange(n, dtype=np.float64) / (n - 1))


def make_problem(m: int, n: int, kappa: float, resnorm: float, seed: int):
    """numpy problem: returns dict with A (C-contiguous m x n), b, x, r, U, sigma."""
    rng = np.random.default_rng(seed)
    U = _haar_columns(rng.standard_normal((m, n)))
    V = _haar_columns(rng.standard_normal((n, n)))
    sig = sigmas(n, kappa)
    A = np.ascontiguousarray((U * sig) @ V.T)
    w = rng.standard_normal(n)
    x = w / np.linalg.norm(w)
    g = rng.standard_normal(m)
    r = g - U @ (U.T @ g)
    r = r - U @ (U.T @ r)
    nr = np.linalg.norm(r)
    r = r * (resnorm / nr) if nr > 0 else r
    b = A @ x + r
    return {"A": A, "b": b, "x": x, "r": r, "U": U, "V": V, "sigma": sig,
            "kappa": kappa, "resnorm": resnorm, "m": m, "n": n, "seed": seed}


def torch_key(seed: int) -> int:
    """Key of torch's generator for data seed ``seed``.  torch's CUDA
    generator is Philox4x32-10 as well; keyed with the same integer as a
    problem's sparse sign embedding, the Gaussian draws behind A and the
    embedding's words come from overlapping Philox streams, and the embedding
    is then measurably worse for that A (distortion of A R^{-1} up to 1.38
    instead of about 1.25 at d = 20 n, and iterations that stall).  Hashing the
    seed through SeedSequence keeps the data stream independent."""
    st = np.random.SeedSequence([int(seed), 0x70C4]).generate_state(1, np.uint64)[0]
    return int(st) & ((1 << 63) - 1)


def make_problem_torch(m: int, n: int, kappa: float, resnorm: float, seed: int, device="cuda"):
    """Same construction drawn with torch on ``device`` (for problems too large
    for host numpy); returns torch float64 tensors A (m x n row-major), b, x."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(torch_key(seed))
    G = torch.randn(m, n, dtype=torch.float64, device=device, generator=gen)
    Q, Rg = torch.linalg.qr(G, mode="reduced")
    del G
    s = torch.sign(torch.diagonal(Rg))
    s[s == 0] = 1.0
    Q.mul_(s)
    H = torch.randn(n, n, dtype=torch.float64, device=device, generator=gen)
    V, Rv = torch.linalg.qr(H)
    sv = torch.sign(torch.diagonal(Rv))
    sv[sv == 0] = 1.0
    V = V * sv
    sig = torch.as_tensor(sigmas(n, kappa), dtype=torch.float64, device=device)
    w = torch.randn(n, dtype=torch.float64, device=device, generator=gen)
    x = w / torch.linalg.norm(w)
    g = torch.randn(m, dtype=torch.float64, device=device, generator=gen)
    r = g - Q @ (Q.T @ g)
    r = r - Q @ (Q.T @ r)
    r = r * (resnorm / torch.linalg.norm(r))
    A = (Q * sig) @ V.T
    del Q
    A = A.contiguous()
    b = A @ x + r
    return {"A": A, "b": b, "x": x, "r": r, "sigma": sig, "kappa": kappa,
            "resnorm": resnorm, "m": m, "n": n, "seed": seed}


# The paper-shaped configurations (Sec. 1.1.1; Sec. 3.3: d = 20 n, zeta = 8).
SMALL = dict(m=4000, n=50, kappa=1e10, resnorm=1e-6, d=1000, zeta=8, seed=0, q=100)
LARGE = dict(m=2_000_000, n=1000, kappa=1e8, resnorm=1e-4, d=20_000, zeta=8, seed=0, q=100)
# Mixed-precision comparison problem.
MIXED = dict(m=1_000_000, n=200, kappa=1e4, resnorm=1e-3, d=4000, zeta=8, seed=0, q=100)


# Batched uneven problems (4096 independent problems, Sec. 1.1.1 construction
# per problem): n log-uniform in [10, 200], then m log-uniform in
# [max(500, 20 n), 20000] so that m >= 20 n holds, kappa log-uniform in
# [1e2, 1e12], ||r|| log-uniform in [1e-10, 1e-2], d = 20 n, zeta = 8,
# sparse-sign seed = problem index.
BATCH = dict(count=4096, m_lo=500, m_hi=20_000, n_lo=10, n_hi=200, kappa_lo=1e2, kappa_hi=1e12,
             res_lo=1e-10, res_hi=1e-2, d_over_n=20, zeta=8, q=100, seed=0)


def batch_shapes(count, m_lo, m_hi, n_lo, n_hi, kappa_lo, kappa_hi, res_lo, res_hi, d_over_n, seed, **_):
    """Per-problem (m, n, d, kappa, resnorm, data seed) of a batch, drawn from
    one generator keyed by ``seed``."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7C4]))

    def logu(lo, hi, size=None):
        return np.exp(rng.uniform(np.log(lo), np.log(hi), size))

    out = []
    for i in range(count):
        n = int(np.clip(np.rint(logu(n_lo, n_hi)), n_lo, n_hi))
        mlo = max(m_lo, d_over_n * n)
        m = int(np.clip(np.rint(logu(mlo, max(mlo, m_hi))), mlo, max(mlo, m_hi)))
        out.append(dict(m=m, n=n, d=d_over_n * n, kappa=float(logu(kappa_lo, kappa_hi)),
                        resnorm=float(logu(res_lo, res_hi)), data_seed=seed * 1_000_003 + i, index=i))
    return out


def make_batch_torch(shapes, device="cuda", lda_even=True):
    """Draw every problem of ``shapes`` on ``device`` (make_problem_torch);
    A is stored row-major with an even leading dimension (16-byte rows)."""
    import torch

    probs = []
    for s in shapes:
        P = make_problem_torch(s["m"], s["n"], s["kappa"], s["resnorm"], s["data_seed"], device=device)
        A = P["A"]
        n = s["n"]
        if lda_even and n % 2:
            Ap = torch.zeros(s["m"], n + 1, dtype=torch.float64, device=device)
            Ap[:, :n] = A
            A = Ap
        probs.append(dict(A=A, b=P["b"], x=torch.empty(n, dtype=torch.float64, device=device), x_true=P["x"],
                          m=s["m"], n=n, lda=A.stride(0), d=s["d"],
                          kappa=s["kappa"], resnorm=s["resnorm"], seed=s["index"]))
    return probs


# Serving stream (requests drawn from a pool of such problems): n log-uniform
# in [20, 500], then m log-uniform in [max(1000, 20 n), 5e5], kappa
# log-uniform in [1e2, 1e10], ||r|| log-uniform in [1e-8, 1e-2], d = 20 n,
# zeta = 8; Poisson arrivals at each rate of the sweep.
SERVE = dict(count=96, m_lo=1000, m_hi=500_000, n_lo=20, n_hi=500, kappa_lo=1e2, kappa_hi=1e10,
             res_lo=1e-8, res_hi=1e-2, d_over_n=20, zeta=8, q=100, seed=5,
             rates=(50, 200, 500, 1000, 2000, 5000), requests_per_rate=400, budget_bytes=150 * 10**9)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream of the given rate."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, int(rate), 0xA77]))
    return np.cumsum(rng.exponential(1.0 / rate, count))


# The sparse workload of Sec. 3.5: m = 3e6 rows with three nonzeros each in
# uniformly random distinct columns, values +-1 uniformly, b standard
# Gaussian, d = 30 n.
SPARSE = dict(m=3_000_000, n=500, nnz_per_row=3, d_over_n=30, zeta=8, seed=0, q=100)


def make_sparse(m: int, n: int, seed: int, nnz_per_row: int = 3):
    """CSR (row_ptr int64, col int32 ascending within rows, val float64) and
    b, numpy.  Distinct columns per row by the successive-shift method: the
    k-th draw is uniform over n - k values and is shifted past the k smaller
    columns already taken."""
    assert nnz_per_row <= n
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5BA5E]))
    cols = np.empty((m, nnz_per_row), dtype=np.int64)
    for k in range(nnz_per_row):
        c = rng.integers(0, n - k, m)
        taken = np.sort(cols[:, :k], axis=1)
        for t in range(k):
            c = c + (c >= taken[:, t])
        cols[:, k] = c
    cols.sort(axis=1)
    val = (rng.integers(0, 2, (m, nnz_per_row)) * 2 - 1).astype(np.float64)
    b = rng.standard_normal(m)
    row_ptr = np.arange(0, m * nnz_per_row + 1, nnz_per_row, dtype=np.int64)
    return {"row_ptr": row_ptr, "col": cols.reshape(-1).astype(np.int32), "val": val.reshape(-1), "b": b,
            "m": m, "n": n, "nnz": m * nnz_per_row}


def sparse_to_dense(S):
    A = np.zeros((S["m"], S["n"]))
    rows = np.repeat(np.arange(S["m"]), np.diff(S["row_ptr"]))
    A[rows, S["col"]] = S["val"]
    return A
