"""GPU parity of the factor step (a4 Householder QR + start, a5 estimates).

Tolerances (derived, not fitted):
 * backward error of the GPU R: |R^T R - B^T B| <= 10 d n u ||B||^2 (Householder
   QR is backward stable: B + dB = Q R, ||dB|| <= c d n u ||B||);
 * R against the oracle's R up to row signs: both are R-factors of B plus a
   backward error of size c d n u ||B||, so they differ by at most
   c d n u kappa(B) ||B|| (QR perturbation bound) -- checked on a
   well-conditioned case where that bound is tight;
 * x0 against the oracle's x0: both solve the sketched problem backward
   stably, so each is within Wedin's bound (Fact 2.1) with eps = 10 d n u of
   the exact sketched solution;
 * normest: same start vector and steps, products in a different order:
   relative 1e-10;  condest: relative 1e-6 (substitutions on R amplify
   rounding by kappa(R) u at most 1e-6 here; only its scale enters the rule).
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import U, dev, host, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


def run_factor(env, Bo, seed=0):
    torch, ls, ctx = env
    d, n1 = Bo.shape
    n = n1 - 1
    B = dev(torch, np.asfortranarray(Bo).ravel(order="F"))
    R = torch.empty(n * n, dtype=torch.float64, device="cuda")
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    info = ctx.ls_factor(B, d, n, d, R, n, x0, seed)
    return host(R).reshape(n, n).T, host(x0), info


# d = 70,000 and 100,000 give row slices of 461 and 658 per CTA on 152 SMs:
# above the lookahead kernel's 436 (two panel buffers) and the single-buffer
# kernel's 600, so they take the single-buffer and the unblocked kernel.
@pytest.mark.parametrize("m,n,kappa,res,d", [(4000, 50, 1e10, 1e-6, 1000), (4000, 50, 10.0, 1e-3, 1000),
                                             (2000, 1, 1.0, 1e-2, 20), (3000, 33, 1e6, 1e-8, 660),
                                             (20000, 257, 1e4, 1e-4, 5140), (500, 5, 1e2, 1e-1, 10),
                                             (100000, 40, 1e6, 1e-6, 70000), (120000, 12, 1e3, 1e-4, 100000),
                                             # n = 720: 23 column groups of 32, so the lookahead factors its
                                             # panels with 2 warps (>= 20 groups left), then 4 (>= 10), then 8
                                             (30000, 720, 1e3, 1e-4, 14000)])
def test_factor_parity(env, m, n, kappa, res, d):
    P = problems.make_problem(m, n, kappa, res, n)
    Bo = oracle.sketch(P["A"], P["b"], d, 8, 0)
    Rg, x0g, info = run_factor(env, Bo)
    Ro, x0o, ne, ce, rc = oracle.factor(Bo, 0)
    assert rc == 0
    Bm, Sb = Bo[:, :n], Bo[:, n]
    nB = np.linalg.norm(Bm, 2)
    kB = np.linalg.cond(Bm)
    # upper triangular, backward stable
    assert np.all(np.tril(Rg, -1) == 0.0)
    # (extended precision where affordable; in FP64 the check's own rounding,
    # at most d u ||B||^2, is 1/(10 n) of the bound)
    L = np.longdouble if d * n * n < 2e9 else np.float64
    err = np.max(np.abs(Rg.astype(L).T @ Rg.astype(L) - Bm.astype(L).T @ Bm.astype(L)))
    assert err <= 10 * d * n * U * nB ** 2
    # R vs oracle R up to row signs
    D = np.sign(np.diag(Rg)) * np.sign(np.diag(Ro))
    dev_R = np.linalg.norm(D[:, None] * Rg - Ro) / np.linalg.norm(Ro)
    assert dev_R <= 10 * d * n * U * kB
    # x0 vs oracle x0 (both within Wedin of the exact sketched solution)
    xs = x0o
    rs = np.linalg.norm(Sb - Bm @ xs)
    wedin = 2.23 * kB * (np.linalg.norm(xs) + kB * rs / nB) * (10 * d * n * U)
    assert np.linalg.norm(x0g - x0o) <= 2 * wedin
    # estimates
    assert info.normest == pytest.approx(ne, rel=1e-10)
    assert info.condest == pytest.approx(ce, rel=1e-6)


def test_factor_rank_deficient_reports_erank(env):
    torch, ls, ctx = env
    d, n = 64, 4
    Bo = np.random.default_rng(0).standard_normal((d, n + 1))
    Bo[:, 2] = 0.0          # exactly rank deficient: R[2,2] is exactly zero
    with pytest.raises(ls.LsError) as e:
        run_factor(env, Bo)
    assert e.value.status == ls.LS_ERANK


def test_factor_deterministic(env):
    P = problems.make_problem(4000, 50, 1e10, 1e-6, 0)
    Bo = oracle.sketch(P["A"], P["b"], 1000, 8, 0)
    R1, x1, i1 = run_factor(env, Bo)
    R2, x2, i2 = run_factor(env, Bo)
    assert np.array_equal(R1, R2) and np.array_equal(x1, x2)
    assert i1.normest == i2.normest and i1.condest == i2.condest
