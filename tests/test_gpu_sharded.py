"""The row-sharded iteration on one GPU (ls_iterate_rows): the rows of A and
b split into P parts, one partial per part per iteration, the partials
reduced in part order, the step shared.  Checked: the forward-error rule
(<= 10x Householder QR) on the split problem, bit-identical repeats, and
the same result as the unsplit ls_iterate for P = 1."""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import dev, host, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


@pytest.fixture(scope="module")
def prob(env):
    torch, ls, ctx = env
    m, n, d = 60_000, 200, 4000
    P = problems.make_problem(m, n, 1e6, 1e-6, 21)
    Ad, bd = dev(torch, P["A"]), dev(torch, P["b"])
    B = torch.empty(d * (n + 1), dtype=torch.float64, device="cuda")
    ctx.ls_sketch(Ad, m, n, n, bd, d, 8, 0, B, d)
    R = torch.empty(n * n, dtype=torch.float64, device="cuda")
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    info = ctx.ls_factor(B, d, n, d, R, n, x0, 0)
    fe_qr = oracle.forward_error(oracle.qr_solve_lapack(P["A"], P["b"]), P["x"])
    return P, Ad, bd, R, x0, info, fe_qr


def _split(m, parts):
    cuts = np.linspace(0, m, parts + 1).astype(np.int64)
    cuts[1:-1] += np.arange(1, parts) * 7          # uneven parts
    return cuts


@pytest.mark.parametrize("parts", [2, 3, 7])
def test_row_sharded_meets_forward_error_rule_and_repeats(env, prob, parts):
    torch, ls, ctx = env
    P, Ad, bd, R, x0, info, fe_qr = prob
    m, n = P["A"].shape
    cuts = _split(m, parts)
    A_parts = [Ad[int(cuts[p]):] for p in range(parts)]          # row views (Ad is m x n)
    b_parts = [bd[int(cuts[p]):] for p in range(parts)]
    m_parts = [int(cuts[p + 1] - cuts[p]) for p in range(parts)]
    xs = []
    for _ in range(2):
        x = x0.clone()
        st, it = ctx.ls_iterate_rows(A_parts, m_parts, n, n, b_parts, R, n, x, 100, None, info)
        assert st == ls.LS_OK and it.stop_reason == 0, (st, it.iters)
        xs.append(host(x))
    assert np.array_equal(xs[0], xs[1])
    fe = oracle.forward_error(xs[0], P["x"])
    assert fe <= 10 * fe_qr, (fe, fe_qr)
    # and the unsplit iteration on the same start
    xu = x0.clone()
    st, itu = ctx.ls_iterate(Ad, m, n, n, bd, R, n, xu, 100, None, info)
    assert abs(itu.iters - it.iters) <= 3
    assert oracle.forward_error(host(xu), P["x"]) <= 10 * fe_qr


def test_one_part_equals_ls_iterate(env, prob):
    torch, ls, ctx = env
    P, Ad, bd, R, x0, info, fe_qr = prob
    m, n = P["A"].shape
    x1 = x0.clone()
    ctx.ls_iterate_rows([Ad], [m], n, n, [bd], R, n, x1, 100, None, info)
    x2 = x0.clone()
    ctx.ls_iterate(Ad, m, n, n, bd, R, n, x2, 100, None, info)
    assert np.array_equal(host(x1), host(x2))
