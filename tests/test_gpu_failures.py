"""Failure detection on the GPU without a GPU fault: every failure is made on
the host side of the library and travels back as a status.

 * A tile that never arrives: ls_inject_fault(LS_FAULT_SKIP_TILE) makes CTA
   0's producer skip one tile of the next fixed-point pass; with a 1 ms wait
   limit the consumers' bounded waits run out, the kernel returns, and the
   call reports LS_ETIMEOUT.  The next call on the same context succeeds and
   gives the same bits as a clean context.
 * An allocation that fails: LS_FAULT_ALLOC makes the next device scratch
   allocation fail (LS_ENOMEM); the context stays usable.
 * A non-finite input: NaN in b reaches the iterate, which the step kernel
   reports as LS_ENONFINITE.
"""
import numpy as np
import pytest

import problems
from gpu_common import dev, host, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture()
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


def _fx_inputs(torch, ctx, m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    ldf = n + (n & 1)
    Af = torch.empty(m * ldf * 2, dtype=torch.int32, device="cuda")
    ex = torch.empty(m, dtype=torch.int32, device="cuda")
    ctx.ls_fixed_point(dev(torch, A), m, n, n, Af, ldf, ex)
    return Af, ex, ldf, dev(torch, b), dev(torch, x)


@pytest.mark.parametrize("m,n,tile", [(100_000, 1000, 0), (40_000, 200, 3), (500, 50, 0)])
def test_skipped_tile_times_out_and_context_recovers(env, m, n, tile):
    torch, ls, ctx = env
    Af, ex, ldf, b, x = _fx_inputs(torch, ctx, m, n, m + n)
    c = torch.empty(n, dtype=torch.float64, device="cuda")
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.ls_set_wait_limit(1_000_000)                  # 1 ms
    ctx.ls_inject_fault(ls.LS_FAULT_SKIP_TILE, tile)
    with pytest.raises(ls.LsError) as e:
        ctx.ls_residual_gradient_fx(Af, ex, m, n, ldf, b, x, None, None, c, norms)
    assert e.value.status == ls.LS_ETIMEOUT
    ctx.ls_set_wait_limit(0)                          # back to the default
    ctx.ls_residual_gradient_fx(Af, ex, m, n, ldf, b, x, None, None, c, norms)
    with ls.Context(0, torch.cuda.current_stream()) as clean:
        c2 = torch.empty(n, dtype=torch.float64, device="cuda")
        n2 = torch.empty(2, dtype=torch.float64, device="cuda")
        clean.ls_residual_gradient_fx(Af, ex, m, n, ldf, b, x, None, None, c2, n2)
    assert np.array_equal(host(c), host(c2)) and np.array_equal(host(norms), host(n2))


def test_injected_allocation_failure_is_enomem(env):
    torch, ls, ctx = env
    P = problems.make_problem(4000, 50, 1e6, 1e-6, 0)
    A, b = dev(torch, P["A"]), dev(torch, P["b"])
    x = torch.empty(50, dtype=torch.float64, device="cuda")
    ctx.ls_inject_fault(ls.LS_FAULT_ALLOC)
    with pytest.raises(ls.LsError) as e:
        ctx.ls_solve(A, b, 4000, 50, 50, 1000, 8, 100, 0, x)
    assert e.value.status == ls.LS_ENOMEM
    st, info = ctx.ls_solve(A, b, 4000, 50, 50, 1000, 8, 100, 0, x)
    assert st == ls.LS_OK and info.stop_reason == 0


@pytest.mark.parametrize("n", [50, 1000, 1500])
def test_nan_in_b_is_enonfinite(env, n):
    torch, ls, ctx = env
    m = 20 * n + 1000
    P = problems.make_problem(m, n, 1e4, 1e-6, 1)
    b = P["b"].copy()
    b[m // 3] = np.nan
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ls.LsError) as e:
        ctx.ls_solve(dev(torch, P["A"]), dev(torch, b), m, n, n, 20 * n, 8, 100, 0, x)
    assert e.value.status == ls.LS_ENONFINITE
    # the same context then solves the clean problem
    st, info = ctx.ls_solve(dev(torch, P["A"]), dev(torch, P["b"]), m, n, n, 20 * n, 8, 100, 0, x)
    assert st == ls.LS_OK
