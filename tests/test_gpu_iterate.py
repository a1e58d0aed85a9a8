"""GPU parity of the iteration (a6 fused residual/gradient pass, a7 the two
triangular solves and update) and of the whole method, through the C ABI.

Tolerances:
 * fused pass, element-wise, from the rounding analysis of dot products
   (any summation order): |r_gpu - r_or| <= 2 gamma_{n+1} (|b| + |A||x|);
   |c_gpu - c_or| <= 2 gamma_m |A|^T |r| + |A|^T |r_gpu - r_or|.
 * substitutions: componentwise backward error |R^T y - c| <= 2 gamma_n |R^T||y|
   and |R d - y| <= 2 gamma_n |R||d| (substitution is componentwise backward
   stable in any blocking).
 * whole method: forward error <= 10x the forward error of the oracle's
   Householder-QR solution on the same problem (the acceptance rule).
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import DEFAULT_EXTRA, U, dev, gamma, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


PASS_CASES = [(4000, 50, 50), (1, 1, 2), (7, 3, 4), (1000, 17, 18), (999, 31, 32), (1003, 32, 32),
              (1001, 33, 34), (2049, 64, 64), (3000, 100, 100), (5001, 257, 258), (4000, 300, 300),
              (3007, 1000, 1000), (2000, 513, 514), (2100, 2048, 2048), (300, 255, 256), (130, 128, 128),
              # many tiles per CTA (the launch geometry of the large workload): at m = 200,000 every CTA
              # of the persistent pass takes 11 (n = 50), 55 (n = 200) or 164 (n = 1000) tiles, so the
              # tile ring and the r hand-off ring wrap many times and partials accumulate over tiles
              (200_000, 50, 50), (200_000, 200, 200), (200_001, 1000, 1000)]


@pytest.mark.parametrize("m,n,lda", PASS_CASES)
def test_fused_pass_elementwise(env, m, n, lda):
    torch, ls, ctx = env
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-4, 4, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    rp = b - A @ x + 1e-6 * rng.standard_normal(m)
    Ad, bd, xd = dev(torch, padded_rowmajor(A, lda)), dev(torch, b), dev(torch, x)
    rprev = dev(torch, rp)
    r = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(n, dtype=torch.float64, device="cuda")
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.ls_residual_gradient(Ad, m, n, lda, bd, xd, rprev, r, c, norms)
    rg, cg, ng = host(r), host(c), host(norms)
    ro, co = oracle.residual_gradient(A, b, x)
    absr = np.abs(b) + np.abs(A) @ np.abs(x)
    assert np.all(np.abs(rg - ro) <= 2 * gamma(n + 1) * absr)
    bound_c = 2 * gamma(m) * (np.abs(A).T @ np.abs(ro)) + np.abs(A).T @ np.abs(rg - ro) * 1.01
    assert np.all(np.abs(cg - co) <= bound_c + 1e-300)
    # squared norms: entries carry the r error e_j, plus summation error
    e = 2 * gamma(n + 1) * absr
    for got, v in [(ng[0], ro), (ng[1], ro - rp)]:
        e_v = e + U * np.abs(v)
        bound = np.sum(2 * np.abs(v) * e_v + e_v ** 2) + 2 * gamma(m) * np.sum((np.abs(v) + e_v) ** 2)
        assert abs(got - np.dot(v, v)) <= bound
    # deterministic: bit-identical on a second call
    c2 = torch.empty_like(c)
    n2 = torch.empty_like(norms)
    ctx.ls_residual_gradient(Ad, m, n, lda, bd, xd, rprev, None, c2, n2)
    assert np.array_equal(host(c2), cg) and np.array_equal(host(n2), ng)


def test_fused_pass_inplace_rprev(env):
    """r_prev == r_out: each entry read before it is overwritten."""
    torch, ls, ctx = env
    P = problems.make_problem(5000, 40, 1e4, 1e-3, 1)
    A, b = P["A"], P["b"]
    x = P["x"] + 1e-3
    rp = np.full(5000, 0.25)
    buf = dev(torch, rp)
    c = torch.empty(40, dtype=torch.float64, device="cuda")
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.ls_residual_gradient(dev(torch, A), 5000, 40, 40, dev(torch, b), dev(torch, x), buf, buf, c, norms)
    ro, _ = oracle.residual_gradient(A, b, x)
    assert np.allclose(host(buf), ro, rtol=0, atol=1e-14)
    assert host(norms)[1] == pytest.approx(np.sum((ro - rp) ** 2), rel=1e-10)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 50, 64, 100, 257, 1000, 1025, 2048])
def test_correct_backward_stable(env, n):
    torch, ls, ctx = env
    rng = np.random.default_rng(n)
    M = rng.standard_normal((3 * n + 5, n)) @ np.diag(np.exp(rng.uniform(-6, 0, n)))
    R = np.linalg.qr(M, mode="r")
    c = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    Rd = dev(torch, np.asfortranarray(R).ravel(order="F"))
    xd = dev(torch, x0)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    dd = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.ls_correct(Rd, n, n, dev(torch, c), xd, y, dd)
    yg, dg, xg = host(y), host(dd), host(xd)
    L = np.longdouble
    g = gamma(n)
    assert np.all(np.abs(R.T.astype(L) @ yg.astype(L) - c) <= 2 * g * (np.abs(R.T) @ np.abs(yg)) + 1e-300)
    assert np.all(np.abs(R.astype(L) @ dg.astype(L) - yg) <= 2 * g * (np.abs(R) @ np.abs(dg)) + 1e-300)
    assert np.array_equal(xg, x0 + dg)
    # against the oracle's substitutions
    yo = oracle.trsv_upper_T(R, c)
    do = oracle.trsv_upper(R, yo)
    k = np.linalg.cond(R)
    assert np.linalg.norm(dg - do) <= 4 * n * U * k * k * np.linalg.norm(do) + 1e-300


def _factor_on_gpu(torch, ctx, Bo):
    d, n1 = Bo.shape
    n = n1 - 1
    B = dev(torch, np.asfortranarray(Bo).ravel(order="F"))
    R = torch.empty(n * n, dtype=torch.float64, device="cuda")
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    info = ctx.ls_factor(B, d, n, d, R, n, x0, 0)
    return R, x0, info


def test_iterate_fixed_steps_matches_oracle(env):
    torch, ls, ctx = env
    P = problems.make_problem(4000, 50, 1e6, 1e-4, 3)
    Bo = oracle.sketch(P["A"], P["b"], 1000, 8, 0)
    R, x0, info = _factor_on_gpu(torch, ctx, Bo)
    Rh = host(R).reshape(50, 50).T
    x = x0.clone()
    opts = ls.default_opts()
    opts.use_stop = 0
    st, it = ctx.ls_iterate(dev(torch, P["A"]), 4000, 50, 50, dev(torch, P["b"]), R, 50, x, 6, opts, info)
    assert it.iters == 6 and it.stop_reason == 2
    xo, _ = oracle.iterate(P["A"], P["b"], Rh, host(x0), 6, info.normest, info.condest, use_stop=False)
    tol = 100 * 1e6 * (1 + 1e6 * 1e-4) * U
    assert np.linalg.norm(host(x) - xo) <= tol * np.linalg.norm(xo)


def test_iterate_resumable(env):
    torch, ls, ctx = env
    P = problems.make_problem(3000, 20, 1e4, 1e-6, 4)
    Bo = oracle.sketch(P["A"], P["b"], 400, 8, 0)
    R, x0, info = _factor_on_gpu(torch, ctx, Bo)
    Ad, bd = dev(torch, P["A"]), dev(torch, P["b"])
    opts = ls.default_opts()
    opts.use_stop = 0
    xa = x0.clone()
    ctx.ls_iterate(Ad, 3000, 20, 20, bd, R, 20, xa, 7, opts, info)
    xb = x0.clone()
    ctx.ls_iterate(Ad, 3000, 20, 20, bd, R, 20, xb, 3, opts, info)
    ctx.ls_iterate(Ad, 3000, 20, 20, bd, R, 20, xb, 4, opts, info)
    assert np.array_equal(host(xa), host(xb))


@pytest.mark.parametrize("kappa,res", [(1e10, 1e-6), (10.0, 1e-12), (1e10, 1e-12), (1e8, 1e-4), (1e10, 1e-3)])
def test_solve_small_config_forward_error(env, kappa, res):
    """The small configuration (m = 4000, n = 50, d = 20n, zeta = 8, seed 0)
    over the paper's Fig. 1 condition/residual grid."""
    torch, ls, ctx = env
    P = problems.make_problem(4000, 50, kappa, res, 0)
    x = torch.empty(50, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(dev(torch, P["A"]), dev(torch, P["b"]), 4000, 50, 50, 1000, 8, 100, 0, x)
    fe = oracle.forward_error(host(x), P["x"])
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    xo, io = oracle.solve(P["A"], P["b"], 1000, 8, 100, 0, extra=DEFAULT_EXTRA)
    assert st == ls.LS_OK and info.stop_reason == 0
    assert fe <= 10 * fe_qr, (fe, fe_qr)
    assert abs(info.iters - io["iters"]) <= 5
    assert info.normest == pytest.approx(io["normest"], rel=1e-10)
    assert info.condest == pytest.approx(io["condest"], rel=1e-6)


@pytest.mark.parametrize("extra", [0, 2])
def test_stopping_rule_fires_at_the_predicted_step(env, extra):
    """The Sec. 3.3 rule on a problem whose iterates are exact in FP64: A =
    [I_2; 0], b = e_1, R = I, alpha = 1/2 from x_0 = 0 gives r(x_i) = 2^-i e_1.
    With gamma = 1, normest = 2^10, rho = 0 the rule first holds at i = 44
    (the oracle's pin, tests/test_oracle_lsq.py), and x_44 is returned after
    `extra` more updates -- the same step and bits on the GPU."""
    torch, ls, ctx = env
    m, n = 8, 2
    A = np.zeros((m, n)); A[:n, :n] = np.eye(n)
    b = np.zeros(m); b[0] = 1.0
    R = dev(torch, np.eye(n).ravel(order="F"))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    opts = ls.default_opts()
    opts.gamma, opts.rho, opts.alpha, opts.extra_iters = 1.0, 0.0, 0.5, extra
    info = ls.ls_info()
    info.normest, info.condest = 1024.0, 1.0
    st, it = ctx.ls_iterate(dev(torch, A), m, n, n, dev(torch, b), R, n, x, 100, opts, info)
    assert st == ls.LS_OK and it.stop_reason == 0 and it.iters == 44 + extra, (st, it.iters)
    xh = host(x)
    assert xh[0] == 1.0 - 2.0 ** -(44 + extra) and xh[1] == 0.0
    assert it.step_norm == 2.0 ** -(44 + extra)


def test_solve_headline_shape_forward_error(env):
    """The whole method at the large workload's shape and launch configuration
    (n = 1000, d = 20 n, zeta = 8, kappa = 1e8, ||r|| = 1e-4) on m = 200,000
    rows: the rule held, and the forward error is within 10x that of a
    Householder-QR solve of the same problem (the acceptance rule; Thm 4.1)."""
    torch, ls, ctx = env
    m, n, d = 200_000, 1000, 20_000
    P = problems.make_problem_torch(m, n, 1e8, 1e-4, 11, device="cuda")
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(P["A"], P["b"], m, n, n, d, 8, 100, 0, x)
    xt = host(P["x"])
    fe = oracle.forward_error(host(x), xt)
    fe_qr = oracle.forward_error(oracle.qr_solve_lapack(host(P["A"]), host(P["b"])), xt)
    assert st == ls.LS_OK and info.stop_reason == 0, (st, info.stop_reason, info.iters)
    assert fe <= 10 * fe_qr, (fe, fe_qr, info.iters)


def test_solve_deterministic_and_host_pointers(env):
    torch, ls, ctx = env
    P = problems.make_problem(4000, 50, 1e10, 1e-6, 0)
    Ad, bd = dev(torch, P["A"]), dev(torch, P["b"])
    x1 = torch.empty(50, dtype=torch.float64, device="cuda")
    x2 = torch.empty(50, dtype=torch.float64, device="cuda")
    ctx.ls_solve(Ad, bd, 4000, 50, 50, 1000, 8, 100, 0, x1)
    ctx.ls_solve(Ad, bd, 4000, 50, 50, 1000, 8, 100, 0, x2)
    assert np.array_equal(host(x1), host(x2))
    xh = np.zeros(50)
    ctx.ls_solve(np.ascontiguousarray(P["A"]), np.ascontiguousarray(P["b"]), 4000, 50, 50, 1000, 8, 100, 0, xh)
    assert np.array_equal(xh, host(x1))


def test_solve_odd_n_padded_lda(env):
    torch, ls, ctx = env
    P = problems.make_problem(3000, 37, 1e6, 1e-5, 9)
    Ap = padded_rowmajor(P["A"], 38)
    x = torch.empty(37, dtype=torch.float64, device="cuda")
    st, info = ctx.ls_solve(dev(torch, Ap), dev(torch, P["b"]), 3000, 37, 38, 740, 8, 100, 0, x)
    fe = oracle.forward_error(host(x), P["x"])
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    assert fe <= 10 * fe_qr


def test_invalid_arguments(env):
    torch, ls, ctx = env
    A = torch.zeros(10 * 4, dtype=torch.float64, device="cuda")
    b = torch.zeros(10, dtype=torch.float64, device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ls.LsError) as e:
        ctx.ls_solve(A, b, 10, 3, 3, 20, 8, 10, 0, x)       # odd lda
    assert e.value.status == ls.LS_EINVAL
    with pytest.raises(ls.LsError):
        ctx.ls_solve(A, b, 10, 4, 4, 3, 2, 10, 0, x)        # d < n
    with pytest.raises(ls.LsError):
        ctx.ls_solve(A, b, 10, 4, 4, 20, 33, 10, 0, x)      # zeta > 32
    with pytest.raises(ls.LsError):
        ctx.ls_solve(A, b, 3, 4, 4, 20, 8, 10, 0, x)        # n > m


@pytest.mark.parametrize("variant", ["damping", "momentum"])
def test_damping_momentum_fixed_steps_match_oracle(env, variant):
    """App. B, Eq. (B.1) update x+ = x + alpha d + beta (x - x_prev) with the
    Eq. (B.2) / (B.3) weights, against the oracle's same update."""
    torch, ls, ctx = env
    P = problems.make_problem(4000, 50, 1e6, 1e-4, 8)
    Bo = oracle.sketch(P["A"], P["b"], 1000, 8, 0)
    R, x0, info = _factor_on_gpu(torch, ctx, Bo)
    Rh = host(R).reshape(50, 50).T
    opts = ls.damping_opts(50, 1000) if variant == "damping" else ls.momentum_opts(50, 1000)
    opts.use_stop = 0
    x = x0.clone()
    ctx.ls_iterate(dev(torch, P["A"]), 4000, 50, 50, dev(torch, P["b"]), R, 50, x, 6, opts, info)
    xo, _ = oracle.iterate(P["A"], P["b"], Rh, host(x0), 6, info.normest, info.condest, use_stop=False,
                           alpha=opts.alpha, beta=opts.beta)
    tol = 100 * 1e6 * (1 + 1e6 * 1e-4) * U
    assert np.linalg.norm(host(x) - xo) <= tol * np.linalg.norm(xo)


def test_damping_momentum_solve_faster_and_accurate(env):
    """Whole solve with the stopping rule: both variants meet the forward-error
    rule and need fewer updates than Algorithm 2 (App. B: faster rate)."""
    torch, ls, ctx = env
    P = problems.make_problem(4000, 50, 1e10, 1e-6, 0)
    Ad, bd = dev(torch, P["A"]), dev(torch, P["b"])
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    iters = {}
    for name, opts in [("basic", ls.default_opts()), ("damping", ls.damping_opts(50, 1000)),
                       ("momentum", ls.momentum_opts(50, 1000))]:
        x = torch.empty(50, dtype=torch.float64, device="cuda")
        st, info = ctx.ls_solve_ex(Ad, bd, 4000, 50, 50, 1000, 8, 100, 0, opts, x)
        assert st == ls.LS_OK
        assert oracle.forward_error(host(x), P["x"]) <= 10 * fe_qr
        iters[name] = info.iters
    assert iters["momentum"] < iters["basic"]
    assert iters["damping"] < iters["basic"]
