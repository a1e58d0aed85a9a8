"""GPU parity of the fixed-point fused pass (a6 as ls_iterate runs it for
n <= 1024): ls_fixed_point and ls_residual_gradient_fx through the C ABI.

Checks:
 * the fixed-point form of A is its definition: a_jk = round(A_jk 2^(1077-e_j))
   (ties to even) with e_j the largest biased exponent field of row j;
 * r and c against the oracle's plain FP64 pass with the FP64 element-wise
   rounding bounds of the other pass tests (any summation order);
 * r and c against the correctly rounded exact values (oracle.residual_exact /
   gradient_exact) with the bound of the fixed-point arithmetic: one rounding
   of A x and of b - A x, the rounding of A and x to 55 bits, and half a unit
   of the per-CTA fixed point of r_j 2^(e_j - 1077) -- far tighter than FP64
   dot products;
 * many tiles per CTA (rings wrap), ragged last tiles, the edge shapes, and
   bit-identical repeats;
 * non-finite input: NaN in x gives NaN c and norms; Inf in A is LS_ENONFINITE.
"""
import numpy as np
import pytest

import oracle
from gpu_common import U, dev, gamma, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


def exp_field(v):
    e = (np.asarray(v, dtype=np.float64).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    return np.maximum(e.astype(np.int64), 1)


def to_fixed(env, A, lda=None):
    torch, ls, ctx = env
    m, n = A.shape
    lda = lda or n + (n & 1)
    ldf = n + (n & 1)
    Ad = dev(torch, padded_rowmajor(A, lda))
    Af = torch.empty(m * ldf * 2, dtype=torch.int32, device="cuda")
    ex = torch.empty(m, dtype=torch.int32, device="cuda")
    ctx.ls_fixed_point(Ad, m, n, lda, Af, ldf, ex)
    return Af, ex, ldf


def run_fx(env, A, b, x, rp=None):
    torch, ls, ctx = env
    m, n = A.shape
    Af, ex, ldf = to_fixed(env, A)
    r = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(n, dtype=torch.float64, device="cuda")
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    rpd = dev(torch, rp) if rp is not None else None
    ctx.ls_residual_gradient_fx(Af, ex, m, n, ldf, dev(torch, b), dev(torch, x), rpd, r, c, norms)
    return (Af, ex, ldf), host(r), host(c), host(norms)


def test_fixed_point_form_is_its_definition(env):
    torch, ls, ctx = env
    rng = np.random.default_rng(3)
    m, n = 300, 37
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-30, 30, (m, n)))
    A[5] = 0.0
    A[6, :3] = [5e-324, -1e-310, 2.5e-320]          # subnormals
    A[7] *= 1e-300
    (Af, ex, ldf), = [to_fixed(env, A)]
    a = host(Af).reshape(m, ldf, 2)[:, :n].astype(np.int64)
    fx = a[:, :, 1] * (1 << 28) + a[:, :, 0]
    e = np.array([exp_field(A[j]).max() for j in range(m)])
    assert np.array_equal(host(ex), e)
    want = np.rint(np.ldexp(A, (1077 - e)[:, None])).astype(np.int64)   # rint: ties to even
    assert np.array_equal(fx, want)
    assert np.all((a[:, :, 0] >= 0) & (a[:, :, 0] < (1 << 28)))
    assert np.all(np.abs(fx) < (1 << 55))


PASS_CASES = [(4000, 50), (1, 1), (7, 3), (1000, 17), (999, 31), (1003, 32), (1001, 33), (2049, 64),
              (3000, 100), (300, 255), (300, 256), (5001, 257), (4000, 300), (2000, 512), (2000, 513),
              (3007, 1000), (2100, 1024),
              # many tiles per CTA: rings wrap (every stage in use), sums cross
              # tiles and fold points; three boxes of 256 columns (n in (512, 768])
              # and a ragged last box
              (200_000, 50), (200_000, 200), (150_001, 300), (200_000, 520), (200_003, 700), (200_001, 1000)]


@pytest.mark.parametrize("m,n", PASS_CASES)
def test_fx_pass_elementwise(env, m, n):
    torch, ls, ctx = env
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-4, 4, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    rp = b - A @ x + 1e-6 * rng.standard_normal(m)
    fxA, rg, cg, ng = run_fx(env, A, b, x, rp)
    # (1) within the FP64 pass's element-wise bounds of the oracle's plain loops
    ro, co = oracle.residual_gradient(A, b, x)
    absr = np.abs(b) + np.abs(A) @ np.abs(x)
    assert np.all(np.abs(rg - ro) <= 2 * gamma(n + 1) * absr)
    bound_c = 2 * gamma(m) * (np.abs(A).T @ np.abs(ro)) + np.abs(A).T @ np.abs(rg - ro) * 1.01
    assert np.all(np.abs(cg - co) <= bound_c + 1e-300)
    e = 2 * gamma(n + 1) * absr
    for got, v in [(ng[0], ro), (ng[1], ro - rp)]:
        e_v = e + U * np.abs(v)
        bound = np.sum(2 * np.abs(v) * e_v + e_v ** 2) + 2 * gamma(m) * np.sum((np.abs(v) + e_v) ** 2)
        assert abs(got - np.dot(v, v)) <= bound
    # (2) against the exact values, with the fixed-point arithmetic's own bound
    rows = np.unique(np.linspace(0, m - 1, min(m, 400)).astype(np.int64))
    rx = oracle.residual_exact(A, b, x, rows)
    ej = np.array([exp_field(A[j]).max() for j in rows])
    xt = exp_field(x).max()
    ax = np.abs(A[rows]) @ np.abs(x)
    rep = np.ldexp(np.abs(x).sum(), ej - 1078) + np.ldexp(np.abs(A[rows]).sum(axis=1), xt - 1078)
    bnd_r = 4 * U * (np.abs(b[rows]) + ax) + rep     # conversion of the 128-bit dot, then b - Ax
    assert np.all(np.abs(rg[rows] - rx) <= bnd_r), np.max(np.abs(rg[rows] - rx) / bnd_r)
    cols = np.unique(np.linspace(0, n - 1, min(n, 64)).astype(np.int64))
    cx = oracle.gradient_exact(A, rg, cols)
    e_all = np.array([exp_field(A[j]).max() for j in range(m)])
    nz = rg != 0
    Q = (exp_field(rg)[nz] + e_all[nz]).max() if nz.any() else 0
    half_p = np.ldexp(1.0, Q - 1078 - e_all)                     # half a unit of P_j, as r_j
    bnd_c = (4 * U * np.abs(cx) + np.ldexp(np.abs(rg), e_all - 1078).sum()
             + np.abs(A[:, cols]).T @ half_p)
    assert np.all(np.abs(cg[cols] - cx) <= bnd_c), np.max(np.abs(cg[cols] - cx) / bnd_c)
    # (3) bit-identical repeat
    Af, ex, ldf = fxA
    c2 = torch.empty(n, dtype=torch.float64, device="cuda")
    n2 = torch.empty(2, dtype=torch.float64, device="cuda")
    r2 = torch.empty(m, dtype=torch.float64, device="cuda")
    ctx.ls_residual_gradient_fx(Af, ex, m, n, ldf, dev(torch, b), dev(torch, x), dev(torch, rp), r2, c2, n2)
    assert np.array_equal(host(c2), cg) and np.array_equal(host(n2), ng) and np.array_equal(host(r2), rg)


def test_fx_pass_wide_dynamic_range(env):
    """Rows and columns spread over 60 binades, x over 40: the errors stay
    within the fixed-point bound (normwise in each row / column)."""
    torch, ls, ctx = env
    rng = np.random.default_rng(11)
    m, n = 5000, 300
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-20, 20, m))[:, None] * np.exp(rng.uniform(-20, 20, n))
    x = rng.standard_normal(n) * np.exp(rng.uniform(-14, 14, n))
    b = A @ x * (1 + 1e-9 * rng.standard_normal(m))
    _, rg, cg, _ = run_fx(env, A, b, x)
    rows = np.arange(0, m, 13)
    rx = oracle.residual_exact(A, b, x, rows)
    ej = np.array([exp_field(A[j]).max() for j in rows])
    xt = exp_field(x).max()
    rep = np.ldexp(np.abs(x).sum(), ej - 1078) + np.ldexp(np.abs(A[rows]).sum(axis=1), xt - 1078)
    bnd = 4 * U * (np.abs(b[rows]) + np.abs(A[rows]) @ np.abs(x)) + rep
    assert np.all(np.abs(rg[rows] - rx) <= bnd)
    # the residual of the FP64 loops, by contrast, carries sqrt(n)-sized summation error
    assert np.all(np.isfinite(cg))


def test_fx_pass_r_prev_none_and_inplace(env):
    torch, ls, ctx = env
    rng = np.random.default_rng(5)
    m, n = 7001, 120
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-2 * rng.standard_normal(m)
    Af, ex, ldf = to_fixed(env, A)
    c = torch.empty(n, dtype=torch.float64, device="cuda")
    norms = torch.empty(2, dtype=torch.float64, device="cuda").fill_(7.0)
    ctx.ls_residual_gradient_fx(Af, ex, m, n, ldf, dev(torch, b), dev(torch, x), None, None, c, norms)
    assert host(norms)[1] == 0.0
    buf = dev(torch, np.full(m, 0.25))
    c2 = torch.empty(n, dtype=torch.float64, device="cuda")
    n2 = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.ls_residual_gradient_fx(Af, ex, m, n, ldf, dev(torch, b), dev(torch, x), buf, buf, c2, n2)
    rnew = host(buf)
    assert np.array_equal(host(c2), host(c))
    assert host(n2)[1] == pytest.approx(np.sum((rnew - 0.25) ** 2), rel=1e-12)


def test_fx_pass_nonfinite(env):
    torch, ls, ctx = env
    rng = np.random.default_rng(6)
    m, n = 1000, 40
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    b = rng.standard_normal(m)
    xb = x.copy()
    xb[7] = np.nan
    _, _, cg, ng = run_fx(env, A, b, xb)
    assert np.all(np.isnan(cg)) and np.isnan(ng[0])   # norms[1] is 0 by definition without r_prev
    bb = b.copy()
    bb[123] = np.inf
    _, _, cg, ng = run_fx(env, A, bb, x)
    assert np.all(np.isnan(cg))
    Ab = A.copy()
    Ab[17, 3] = np.inf
    with pytest.raises(ls.LsError) as e:
        to_fixed(env, Ab)
    assert e.value.status == ls.LS_ENONFINITE


def test_fx_pass_zero_x_and_zero_rows(env):
    torch, ls, ctx = env
    rng = np.random.default_rng(8)
    m, n = 3000, 64
    A = rng.standard_normal((m, n))
    A[100:200] = 0.0
    b = rng.standard_normal(m)
    _, rg, cg, ng = run_fx(env, A, b, np.zeros(n))
    assert np.array_equal(rg, b)
    cx = oracle.gradient_exact(A, b)
    assert np.all(np.abs(cg - cx) <= 4 * U * np.abs(A).T @ np.abs(b))
    assert ng[0] == pytest.approx(np.dot(b, b), rel=1e-13)
