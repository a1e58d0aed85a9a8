"""Pins for the oracle's least-squares pieces: the residual/gradient pass, the
two substitutions, one refinement step (Eq. (3.2)), the direct Householder
solve (the yardstick of every forward-error rule), and the whole iteration
(Algorithm 2 with the Sec. 3.3 stopping rule).

Independent references: exact rational arithmetic (fractions) on tiny
problems, closed-form generated problems with known x and r (Sec. 1.1.1),
Wedin's bound (Fact 2.1), the sketch-and-solve bound (Fact 2.4), the
convergence rate of Thm. 3.1, and the paper's negative control ("bad
residual", Sec. 3.2).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import problems

U = 2.0 ** -53


def exact_solve(M, v):
    """Gaussian elimination over the rationals (M square, nonsingular)."""
    n = len(v)
    a = [[Fr(M[i][j]) for j in range(n)] + [Fr(v[i])] for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col] / a[col][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return [a[i][n] / a[i][i] for i in range(n)]


def exact_ls(A, b):
    m, n = A.shape
    Af = [[Fr(float(A[i, j])) for j in range(n)] for i in range(m)]
    bf = [Fr(float(v)) for v in b]
    AtA = [[sum(Af[k][i] * Af[k][j] for k in range(m)) for j in range(n)] for i in range(n)]
    Atb = [sum(Af[k][i] * bf[k] for k in range(m)) for i in range(n)]
    return np.array([float(v) for v in exact_solve(AtA, Atb)])


@pytest.mark.parametrize("m,n,seed", [(6, 2, 0), (9, 3, 1), (12, 4, 2), (5, 5, 3), (1, 1, 4)])
def test_qr_solve_vs_exact_rationals(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    x = oracle.qr_solve(A, b)
    xs = exact_ls(A, b)
    k = np.linalg.cond(A)
    r = b - A @ xs
    bound = 2.23 * k * (np.linalg.norm(xs) + k * np.linalg.norm(r) / np.linalg.norm(A, 2)) * (10 * m * n * U)
    assert np.linalg.norm(x - xs) <= bound


@pytest.mark.parametrize("kappa,res", [(1e2, 1e-10), (1e6, 1e-4), (1e10, 1e-6)])
def test_qr_solve_forward_stable_on_closed_form(kappa, res):
    P = problems.make_problem(2000, 30, kappa, res, 3)
    x = oracle.qr_solve(P["A"], P["b"])
    wedin = 2.23 * kappa * (1.0 + kappa * res) * U
    fe = oracle.forward_error(x, P["x"])
    assert fe <= 100 * wedin, (fe, wedin)
    # LAPACK's least-squares solver lands in the same error class
    fl = oracle.forward_error(np.linalg.lstsq(P["A"], P["b"], rcond=None)[0], P["x"])
    assert fe <= 100 * max(fl, wedin)


def test_residual_gradient_rounding_bound():
    rng = np.random.default_rng(0)
    m, n = 700, 23
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-3, 3, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    r, c = oracle.residual_gradient(A, b, x)
    L = np.longdouble
    rl = b.astype(L) - A.astype(L) @ x.astype(L)
    absr = np.abs(b) + np.abs(A) @ np.abs(x)
    g = (n + 1) * U / (1 - (n + 1) * U)
    assert np.all(np.abs(r - rl) <= g * absr * 1.01)
    # c = A^T r for the computed r: error of one m-term dot product per entry
    cl = A.astype(L).T @ r.astype(L)
    gm = m * U / (1 - m * U)
    assert np.all(np.abs(c - cl) <= gm * (np.abs(A).T @ np.abs(r)) * 1.01)
    # a transposed or sign-flipped implementation would fail these:
    assert np.abs(c - cl).max() < 1e-8 * np.abs(c).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_residual_and_gradient_vs_rationals(seed):
    """residual_exact / gradient_exact are the correctly rounded r = b - A x
    and c = A^T r: checked against exact rational sums (entries spread over
    many binades, cancellation in b - A x)."""
    rng = np.random.default_rng(seed)
    m, n = 23, 9
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-20, 20, (m, n)))
    x = rng.standard_normal(n) * np.exp(rng.uniform(-10, 10, n))
    b = A @ x * (1 + 1e-12 * rng.standard_normal(m))
    r = oracle.residual_exact(A, b, x)
    for j in range(m):
        ex = Fr(float(b[j])) - sum(Fr(float(A[j, k])) * Fr(float(x[k])) for k in range(n))
        assert r[j] == float(ex), j                  # float(Fraction) rounds to nearest
    c = oracle.gradient_exact(A, r)
    for k in range(n):
        ex = sum(Fr(float(A[j, k])) * Fr(float(r[j])) for j in range(m))
        assert c[k] == float(ex), k
    # and the plain FP64 pass is within its rounding bound of them
    ro, co = oracle.residual_gradient(A, b, x)
    g = (n + 1) * U / (1 - (n + 1) * U)
    assert np.all(np.abs(ro - r) <= 2 * g * (np.abs(b) + np.abs(A) @ np.abs(x)))


def test_substitutions_backward_stable():
    rng = np.random.default_rng(2)
    n = 60
    R = np.triu(rng.standard_normal((n, n))) + np.diag(np.sign(rng.standard_normal(n)) * 2)
    z = rng.standard_normal(n)
    x = oracle.trsv_upper(R, z)
    y = oracle.trsv_upper_T(R, z)
    L = np.longdouble
    g = n * U / (1 - n * U)
    res1 = np.abs(R.astype(L) @ x.astype(L) - z)
    res2 = np.abs(R.T.astype(L) @ y.astype(L) - z)
    assert np.all(res1 <= 2 * g * (np.abs(R) @ np.abs(x)))
    assert np.all(res2 <= 2 * g * (np.abs(R.T) @ np.abs(y)))


def test_one_refinement_step_vs_exact_rationals():
    """x1 = x0 + R^{-1} R^{-T} A^T (b - A x0) (Eq. (3.2)), checked against the
    same update carried out exactly over the rationals."""
    rng = np.random.default_rng(4)
    m, n = 10, 3
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    R = np.linalg.qr(A + 0.05 * rng.standard_normal((m, n)), mode="r")
    x0 = rng.standard_normal(n)
    x1, info = oracle.iterate(A, b, R, x0, q=1, normest_value=1.0, condest_value=1.0, use_stop=False)
    assert info["iters"] == 1
    Af = [[Fr(float(A[i, j])) for j in range(n)] for i in range(m)]
    Rf = [[Fr(float(R[i, j])) for j in range(n)] for i in range(n)]
    rr = [Fr(float(b[i])) - sum(Af[i][k] * Fr(float(x0[k])) for k in range(n)) for i in range(m)]
    c = [sum(Af[i][k] * rr[i] for i in range(m)) for k in range(n)]
    RtR = [[sum(Rf[k][i] * Rf[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    dlt = exact_solve(RtR, c)
    want = np.array([float(Fr(float(x0[k])) + dlt[k]) for k in range(n)])
    kR = np.linalg.cond(R)
    assert np.linalg.norm(x1 - want) <= 50 * n * m * U * kR ** 2 * np.linalg.norm(want)


@pytest.mark.parametrize("alpha,beta", [(0.75, 0.0), (0.9, 0.05), (1.0, 0.3)])
def test_two_damped_momentum_steps_vs_exact_rationals(alpha, beta):
    """App. B, Eq. (B.1): x_{i+1} = x_i + alpha d_i + beta (x_i - x_{i-1}) with
    d_i = R^{-1} R^{-T} A^T (b - A x_i) and x_{-1} = x_0 (the first step has no
    momentum).  Two steps against the same recurrence over the rationals."""
    rng = np.random.default_rng(9)
    m, n = 12, 3
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    R = np.linalg.qr(A + 0.05 * rng.standard_normal((m, n)), mode="r")
    x0 = rng.standard_normal(n)
    x2, info = oracle.iterate(A, b, R, x0, q=2, normest_value=1.0, condest_value=1.0, use_stop=False,
                              alpha=alpha, beta=beta)
    assert info["iters"] == 2
    Af = [[Fr(float(A[i, j])) for j in range(n)] for i in range(m)]
    Rf = [[Fr(float(R[i, j])) for j in range(n)] for i in range(n)]
    RtR = [[sum(Rf[k][i] * Rf[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    a, bt = Fr(alpha), Fr(beta)
    xp = [Fr(float(v)) for v in x0]
    xc = list(xp)
    for _ in range(2):
        rr = [Fr(float(b[i])) - sum(Af[i][k] * xc[k] for k in range(n)) for i in range(m)]
        c = [sum(Af[i][k] * rr[i] for i in range(m)) for k in range(n)]
        dl = exact_solve(RtR, c)
        xn = [xc[k] + a * dl[k] + bt * (xc[k] - xp[k]) for k in range(n)]
        xp, xc = xc, xn
    want = np.array([float(v) for v in xc])
    kR = np.linalg.cond(R)
    assert np.linalg.norm(x2 - want) <= 100 * n * m * U * kR ** 2 * np.linalg.norm(want)
    # the momentum term is really there: beta = 0 gives a different second step
    if beta:
        x2b, _ = oracle.iterate(A, b, R, x0, q=2, normest_value=1.0, condest_value=1.0, use_stop=False,
                                alpha=alpha, beta=0.0)
        assert np.linalg.norm(x2b - want) > 1e3 * np.linalg.norm(x2 - want) + 1e-14


def halving_problem(m=8, n=2):
    """A = [I_n; 0], b = e_1, R = I: with alpha = 1/2 the iterates from x_0 = 0
    are x_i = (1 - 2^-i) e_1 and r(x_i) = 2^-i e_1 EXACTLY in FP64, so
    ||r(x_i) - r(x_{i-1})|| = 2^-i and ||r(x_i)|| = 2^-i."""
    A = np.zeros((m, n))
    A[:n, :n] = np.eye(n)
    b = np.zeros(m)
    b[0] = 1.0
    return A, b, np.eye(n)


@pytest.mark.parametrize("extra", [0, 1, 3])
def test_stopping_rule_normest_term_fires_at_the_predicted_step(extra):
    """Sec. 3.3 rule ||r(x_{i+1}) - r(x_i)|| <= u (gamma normest ||x_{i+1}|| +
    rho condest ||r(x_{i+1})||) with gamma = 1, normest = 2^10, rho = 0: on the
    halving problem it first holds at i = 44 (2^-44 <= 2^-43 (1 - 2^-44), while
    2^-43 > 2^-43 (1 - 2^-43)), and x_44 is returned after `extra` more
    updates."""
    A, b, R = halving_problem()
    x, info = oracle.iterate(A, b, R, np.zeros(2), 100, 1024.0, 1.0, use_stop=True, extra=extra,
                             gamma=1.0, rho=0.0, alpha=0.5)
    assert info["converged"] and info["iters"] == 44 + extra
    assert x[0] == 1.0 - 2.0 ** -(44 + extra) and x[1] == 0.0
    # the rule compares the change of residual (2^-i), not the residual of x_0
    assert info["step_norm"] == 2.0 ** -(44 + extra)


def test_stopping_rule_condest_term_uses_the_new_residual():
    """gamma = 0: the rule reads 2^-i <= u rho condest 2^-i, i.e. it holds at
    the first test (i = 1) exactly when rho condest >= 2^53 and never when it
    is below: the condest term is rho condest ||r(x_{i+1})|| with the current
    residual."""
    A, b, R = halving_problem()
    rho = 0.04
    ce_hi = 2.0 ** 53 / rho * (1 + 1e-9)
    ce_lo = 2.0 ** 53 / rho * (1 - 1e-9)
    x, info = oracle.iterate(A, b, R, np.zeros(2), 30, 1.0, ce_hi, use_stop=True, gamma=0.0, rho=rho, alpha=0.5)
    assert info["converged"] and info["iters"] == 1 and x[0] == 0.5
    x, info = oracle.iterate(A, b, R, np.zeros(2), 30, 1.0, ce_lo, use_stop=True, gamma=0.0, rho=rho, alpha=0.5)
    assert not info["converged"] and info["iters"] == 30


def _setup(P, d=1000, zeta=8, seed=0):
    B = oracle.sketch(P["A"], P["b"], d, zeta, seed)
    R, x0, ne, ce, rc = oracle.factor(B, seed)
    assert rc == 0
    return R, x0, ne, ce


def test_sketch_and_solve_bound_fact_2_4():
    P = problems.make_problem(4000, 50, 1e4, 1e-3, 6)
    # Fact 2.4 needs S to embed range([A b]); measure eps on that subspace
    Ab = np.column_stack([P["A"], P["b"]])
    Qab = np.linalg.qr(Ab)[0]
    Bq = oracle.sketch(Qab, np.zeros(4000), 1000, 8, 0)[:, :51]
    sv = np.linalg.svd(Bq, compute_uv=False)
    eps = max(sv.max() - 1, 1 - sv.min())
    R, x0, ne, ce = _setup(P)
    rx = np.linalg.norm(P["r"])
    r0 = P["b"] - P["A"] @ x0
    assert np.linalg.norm(r0) <= (1 + eps) / (1 - eps) * rx * (1 + 1e-9)
    assert np.linalg.norm(P["r"] - r0) <= 2 * np.sqrt(eps) / (1 - eps) * rx * (1 + 1e-6)
    assert np.linalg.norm(P["x"] - x0) <= 2 * np.sqrt(eps) / (1 - eps) * 1e4 * rx * (1 + 1e-6)


def test_convergence_rate_theorem_3_1():
    """||R(x - x_i)|| contracts at least by g_IS(eps) per step (proof of Thm.
    3.1), eps measured as the distortion of S on range(A)."""
    P = problems.make_problem(4000, 50, 1e3, 1e-2, 7)
    R, x0, ne, ce = _setup(P)
    Bu = oracle.sketch(P["U"], np.zeros(4000), 1000, 8, 0)[:, :50]
    sv = np.linalg.svd(Bu, compute_uv=False)
    eps = max(sv.max() - 1, 1 - sv.min())
    g = (2 - eps) * eps / (1 - eps) ** 2
    assert g < 1
    x = x0.copy()
    errs = [np.linalg.norm(R @ (P["x"] - x))]
    for _ in range(8):
        x, _ = oracle.iterate(P["A"], P["b"], R, x, 1, ne, ce, use_stop=False)
        errs.append(np.linalg.norm(R @ (P["x"] - x)))
    floor = 1e3 * 1e-2 * 1e3 * U * 100    # well above rounding level
    for e0, e1 in zip(errs, errs[1:]):
        if e0 > floor:
            assert e1 <= g * e0 * (1 + 1e-6), (e0, e1, g)


@pytest.mark.parametrize("kappa,res", [(1e10, 1e-6), (10.0, 1e-12), (1e10, 1e-12), (1e8, 1e-4), (1e10, 1e-3)])
def test_iterative_sketching_forward_stable(kappa, res):
    """Sec. 1.1.3 / Thm. 4.1: FE reaches the Householder-QR level; the Sec. 3.3
    stopping rule fires before q = 100."""
    P = problems.make_problem(4000, 50, kappa, res, 0)
    x, info = oracle.solve(P["A"], P["b"], 1000, 8, 100, 0)
    fe = oracle.forward_error(x, P["x"])
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    assert info["converged"], info
    assert info["iters"] < 60
    assert fe <= 10 * fe_qr, (fe, fe_qr)
    # residual error also at the QR level
    rq = P["b"] - P["A"] @ oracle.qr_solve(P["A"], P["b"])
    ri = P["b"] - P["A"] @ x
    re_qr = np.linalg.norm(P["r"] - rq) / res
    re_is = np.linalg.norm(P["r"] - ri) / res
    assert re_is <= 10 * max(re_qr, 2.23 * (1 + kappa * res) * U / res)


def test_bad_residual_is_worse():
    """Negative control of Sec. 3.2: A^T b - A^T (A x) in place of
    A^T (b - A x) loses accuracy at kappa = 1e10, ||r|| = 1e-6."""
    P = problems.make_problem(4000, 50, 1e10, 1e-6, 0)
    R, x0, ne, ce = _setup(P)
    xs, _ = oracle.iterate(P["A"], P["b"], R, x0, 60, ne, ce, use_stop=False)
    xb, _ = oracle.iterate(P["A"], P["b"], R, x0, 60, ne, ce, use_stop=False, variant=1)
    assert oracle.forward_error(xb, P["x"]) > 10 * oracle.forward_error(xs, P["x"])


def test_damping_and_momentum_accelerate():
    """App. B, Eqs. (B.2)-(B.3) with eps = sqrt(n/d): faster contraction than
    the basic method."""
    P = problems.make_problem(4000, 50, 1e4, 1e-6, 1)
    R, x0, ne, ce = _setup(P)
    eps = np.sqrt(50 / 1000)
    runs = {"basic": (1.0, 0.0),
            "damping": ((1 - eps ** 2) ** 2 / (1 + eps ** 2), 0.0),
            "momentum": ((1 - eps ** 2) ** 2, eps ** 2)}
    err = {}
    for k, (a, bt) in runs.items():
        x, _ = oracle.iterate(P["A"], P["b"], R, x0, 6, ne, ce, use_stop=False, alpha=a, beta=bt)
        err[k] = oracle.forward_error(x, P["x"])
    assert err["damping"] < err["basic"]
    assert err["momentum"] < err["basic"]


def test_zero_start_still_converges():
    """'Bad initialization' of Sec. 3.2 is stable, only slower."""
    P = problems.make_problem(4000, 50, 1e6, 1e-6, 2)
    R, x0, ne, ce = _setup(P)
    x, info = oracle.iterate(P["A"], P["b"], R, np.zeros(50), 100, ne, ce)
    x1, info1 = oracle.iterate(P["A"], P["b"], R, x0, 100, ne, ce)
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    assert oracle.forward_error(x, P["x"]) <= 10 * fe_qr
    assert info["iters"] >= info1["iters"]


def test_lapack_householder_solve_same_class_as_plain():
    """The LAPACK-backed Householder solve (used for very tall problems) lands
    in the same forward-error class as the plain-loop oracle solve."""
    for kappa, res in [(1e8, 1e-4), (1e10, 1e-6), (1e3, 1e-10)]:
        P = problems.make_problem(3000, 40, kappa, res, 11)
        fe_plain = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
        fe_lapack = oracle.forward_error(oracle.qr_solve_lapack(P["A"], P["b"]), P["x"])
        wedin = 2.23 * kappa * (1.0 + kappa * res) * U
        assert fe_lapack <= 100 * wedin
        assert 0.05 * fe_plain <= fe_lapack <= 20 * fe_plain
