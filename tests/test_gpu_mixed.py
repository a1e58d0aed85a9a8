"""GPU checks of the mixed-precision solver (ls_solve_batched_mixed): FP32
sketch and FP32 Householder QR, FP64 residual, gradient, solves and update.

Per stage, against the FP64 oracle on the same seeded inputs:
 * sketch: every entry is an FP32 sum of k_t terms (each A entry rounded to
   FP32) scaled once, so |B32 - B| <= (k_t + 3) u32 s sum_bucket |[A b]_jc|
   (k_t = bucket size, s = 1/sqrt(zeta), u32 = 2^-24);
 * QR: backward stable in FP32 on its own input:
   |R^T R - B32^T B32| <= 10 d n u32 ||B32||^2;
 * the whole method: forward error <= 10x that of the oracle's FP64
   Householder-QR solution (iterative refinement in FP64 removes the FP32
   error of R; only the contraction rate depends on it), for kappa up to 1e5.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import problems
from gpu_common import U, dev, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


CASES = [(4000, 50, 1e4, 1e-3), (3000, 20, 1e2, 1e-6), (6000, 120, 1e5, 1e-4), (2500, 33, 1e3, 1e-2),
         (8000, 200, 1e4, 1e-3), (1000, 10, 1.0, 1e-3)]


def _run(env, cases, mixed=True):
    torch, ls, ctx = env
    probs, hps = [], []
    for i, (m, n, kappa, res) in enumerate(cases):
        P = problems.make_problem(m, n, kappa, res, 40 + i)
        lda = n + (n % 2)
        d = 20 * n
        probs.append(dict(A=dev(torch, padded_rowmajor(P["A"], lda)), b=dev(torch, P["b"]),
                          x=torch.empty(n, dtype=torch.float64, device="cuda"), m=m, n=n, lda=lda, d=d, seed=i,
                          B_out=torch.empty(d * (n + 1), dtype=torch.float64, device="cuda"),
                          R_out=torch.empty(n * n, dtype=torch.float64, device="cuda")))
        hps.append(P)
    infos = ctx.ls_solve_batched(probs, 8, 100, mixed=mixed)
    torch.cuda.synchronize()
    return probs, hps, infos


@pytest.fixture(scope="module")
def mixed_run(env):
    return _run(env, CASES)


def test_mixed_sketch_within_fp32_bound(env, mixed_run):
    probs, hps, _ = mixed_run
    for i, (p, P) in enumerate(zip(probs, hps)):
        m, n, d = p["m"], p["n"], p["d"]
        Bg = host(p["B_out"]).reshape(n + 1, d).T
        Bo = oracle.sketch(P["A"], P["b"], d, 8, i)
        rows, signs = oracle.sketch_indices(m, d, 8, i)
        # bucket sizes and sum_bucket |[A b]_j| through the pattern of S
        S = sp.csr_matrix((np.ones(m * 8), (np.asarray(rows).reshape(m, 8).ravel(), np.repeat(np.arange(m), 8))),
                          shape=(d, m))
        k = np.asarray(S.sum(axis=1)).ravel()
        Ab = np.abs(np.column_stack([P["A"], P["b"]]))
        bound = (k[:, None] + 3) * U32 * (1.0 / np.sqrt(8.0)) * (S @ Ab) * 1.0001
        assert np.all(np.abs(Bg - Bo) <= bound), i
        assert not np.array_equal(Bg, Bo)                # it really is FP32


def test_mixed_qr_backward_stable_in_fp32(env, mixed_run):
    probs, hps, _ = mixed_run
    L = np.longdouble
    for p in probs:
        n, d = p["n"], p["d"]
        B32 = host(p["B_out"]).reshape(n + 1, d).T[:, :n]
        R = host(p["R_out"]).reshape(n, n).T
        assert np.all(np.tril(R, -1) == 0.0)
        err = np.max(np.abs(R.astype(L).T @ R.astype(L) - B32.astype(L).T @ B32.astype(L)))
        assert err <= 10 * d * n * U32 * np.linalg.norm(B32, 2) ** 2
        assert np.all(R.astype(np.float32).astype(np.float64) == R)   # an FP32 factor, widened


def test_mixed_solution_meets_fp64_acceptance(env, mixed_run):
    probs, hps, infos = mixed_run
    for p, P, inf in zip(probs, hps, infos):
        fe = oracle.forward_error(host(p["x"]), P["x"])
        fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
        # the rule may not fire when ||r_i - r_{i-1}|| settles just above its
        # threshold (small kappa and residual); x is then converged all the same
        assert inf.stop_reason in (0, 1), inf.as_dict()
        assert fe <= 10 * fe_qr, (p["m"], p["n"], fe, fe_qr)


def test_mixed_iterations_near_fp64(env, mixed_run):
    """The FP32 R perturbs the preconditioned matrix by ~kappa u32; the
    iteration count grows but stays of the FP64 path's order at kappa <= 1e5."""
    probs, hps, infos = mixed_run
    ref = _run(env, CASES, mixed=False)[2]
    for a, b in zip(infos, ref):
        assert a.iters <= 2 * b.iters + 10, (a.iters, b.iters)


def test_mixed_deterministic(env, mixed_run):
    torch, ls, ctx = env
    probs, hps, infos = mixed_run
    again = [dict(p, x=torch.empty_like(p["x"]), B_out=None, R_out=None) for p in probs]
    infos2 = ctx.ls_solve_batched(again, 8, 100, mixed=True)
    for p, q, a, b in zip(probs, again, infos, infos2):
        assert np.array_equal(host(p["x"]), host(q["x"])) and a.iters == b.iters
