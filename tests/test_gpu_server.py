"""GPU tests of the continuous-batching server (ls_server_*).

Each admitted request is sketched, factored and iterated exactly as
ls_solve_batched does it and never reads another request's data, so the
checks are exact: a request's x and iteration count are bit-identical
 * to the same problem solved by ls_solve_batched alone,
 * whether it ran alone on a server or among other requests, admitted early
   or late, under a tight admission budget or a loose one.
Accuracy is that of the batched solver (checked against the oracle in
test_gpu_batched.py); here the forward error is rechecked against the
oracle's Householder-QR solution with the same acceptance rule.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import U, dev, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


def _mix(count=14, seed=11):
    sh = problems.batch_shapes(count=count, m_lo=500, m_hi=6000, n_lo=8, n_hi=80, kappa_lo=1e2, kappa_hi=1e10,
                               res_lo=1e-8, res_hi=1e-2, d_over_n=20, seed=seed)
    sh.append(dict(m=3000, n=300, d=6000, kappa=1e4, resnorm=1e-5, data_seed=77))     # n above 256
    sh.append(dict(m=2001, n=37, d=740, kappa=1e6, resnorm=1e-6, data_seed=78))       # odd n
    for i, s in enumerate(sh):
        s["index"] = i
    return sh


def _upload(torch, shapes):
    out = []
    for s in shapes:
        P = problems.make_problem(s["m"], s["n"], s["kappa"], s["resnorm"], s["data_seed"])
        n = s["n"]
        lda = n + (n % 2)
        out.append((dict(A=dev(torch, padded_rowmajor(P["A"], lda)), b=dev(torch, P["b"]),
                         x=torch.empty(n, dtype=torch.float64, device="cuda"), m=s["m"], n=n, lda=lda, d=s["d"],
                         seed=s["index"]), P))
    return out


def _serve(ls, ctx, reqs, *, max_inflight=64, workspace=1 << 30, admit=0, stagger=0, max_steps=2000):
    """Run requests through a fresh server; with stagger > 0 request i is
    submitted before step i * stagger.  Returns {index: info}, the largest
    in-flight count and admitted bytes seen, and the final stats."""
    srv = ls.Server(ctx, max_inflight, 512, workspace, admit, 8, 100)
    tick = {}
    out = {}
    peak = 0
    peak_bytes = 0
    pending = list(range(len(reqs)))
    step = 0
    try:
        while len(out) < len(reqs):
            while pending and (stagger == 0 or pending[0] * stagger <= step):
                i = pending.pop(0)
                tick[srv.ls_server_submit(reqs[i])] = i
            srv.ls_server_step()
            step += 1
            st = srv.ls_server_get_stats()
            peak = max(peak, st["inflight"])
            peak_bytes = max(peak_bytes, st["admitted_bytes"])
            for t, info in srv.ls_server_poll():
                out[tick[t]] = info
            assert step < max_steps
        stats = srv.ls_server_get_stats()
    finally:
        srv.close()
    return out, (peak, peak_bytes), stats


def test_server_matches_batched_bit_for_bit(env):
    torch, ls, ctx = env
    up = _upload(torch, _mix())
    reqs = [r for r, _ in up]
    res, _, stats = _serve(ls, ctx, reqs)
    xs = [host(r["x"]).copy() for r in reqs]
    assert stats["inflight"] == 0 and stats["queued"] == 0 and stats["completed"] == len(reqs)
    assert stats["workspace_bytes_used"] == 0 and stats["admitted_bytes"] == 0
    # the same problems through ls_solve_batched
    ref = [dict(r, x=torch.empty_like(r["x"])) for r in reqs]
    infos = ctx.ls_solve_batched(ref, 8, 100)
    for i, (r, P) in enumerate(up):
        assert np.array_equal(xs[i], host(ref[i]["x"])), i
        assert res[i].iters == infos[i].iters and res[i].stop_reason == infos[i].stop_reason
        assert res[i].normest == infos[i].normest and res[i].condest == infos[i].condest
        fe = oracle.forward_error(xs[i], P["x"])
        fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
        wedin = 10 * U * P["kappa"] * (1 + P["kappa"] * P["resnorm"])
        assert fe <= max(10 * fe_qr, wedin), (i, fe, fe_qr)


def test_server_alone_equals_in_mix_and_staggered(env):
    torch, ls, ctx = env
    up = _upload(torch, _mix(count=10, seed=12))
    reqs = [r for r, _ in up]
    _serve(ls, ctx, reqs)
    mixed = [host(r["x"]).copy() for r in reqs]
    for k in (0, 5, len(reqs) - 1):
        alone = dict(reqs[k], x=torch.empty_like(reqs[k]["x"]))
        _serve(ls, ctx, [alone])
        assert np.array_equal(host(alone["x"]), mixed[k]), k
    # arrivals spread over steps: requests join while others iterate
    stag = [dict(r, x=torch.empty_like(r["x"])) for r in reqs]
    _serve(ls, ctx, stag, stagger=3)
    for k, r in enumerate(stag):
        assert np.array_equal(host(r["x"]), mixed[k]), k


def test_server_admission_budget_and_slot_reuse(env):
    torch, ls, ctx = env
    up = _upload(torch, _mix(count=12, seed=13))
    reqs = [r for r, _ in up]
    need = [ls.server_request_bytes(r["m"], r["n"], r["lda"], r["d"]) for r in reqs]
    budget = max(need) + min(need)            # the largest request plus at most a small one
    res, (peak, peak_bytes), stats = _serve(ls, ctx, reqs, admit=budget)
    loose = [host(r["x"]).copy() for r in reqs]
    assert peak_bytes <= budget and peak < len(reqs) and len(res) == len(reqs)
    # few slots: slots are reused many times
    few = [dict(r, x=torch.empty_like(r["x"])) for r in reqs]
    res2, (peak2, _), _ = _serve(ls, ctx, few, max_inflight=2)
    assert peak2 <= 2
    for k, r in enumerate(few):
        assert np.array_equal(host(r["x"]), loose[k])
        assert res2[k].iters == res[k].iters


def test_server_rank_deficient_request(env):
    torch, ls, ctx = env
    up = _upload(torch, _mix(count=3, seed=14)[:3])
    reqs = [r for r, _ in up]
    reqs[1]["A"].view(reqs[1]["m"], reqs[1]["lda"])[:, 1] = 0.0
    res, _, stats = _serve(ls, ctx, reqs)
    assert res[1].stop_reason == 4
    for k in (0, 2):
        assert res[k].stop_reason == 0
        P = up[k][1]
        fe = oracle.forward_error(host(reqs[k]["x"]), P["x"])
        assert fe <= max(10 * oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"]),
                         10 * U * P["kappa"] * (1 + P["kappa"] * P["resnorm"]))
    assert stats["workspace_bytes_used"] == 0


def test_server_rejects_bad_requests(env):
    torch, ls, ctx = env
    srv = ls.Server(ctx, 4, 64, 1 << 20, 0, 8, 100)
    A = torch.zeros(4000 * 128, dtype=torch.float64, device="cuda")
    b = torch.zeros(4000, dtype=torch.float64, device="cuda")
    x = torch.zeros(128, dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(ls.LsError) as e:
            srv.ls_server_submit(dict(A=A, b=b, x=x, m=4000, n=100, lda=100, d=2000))      # n above max_n
        assert e.value.status == ls.LS_EINVAL
        with pytest.raises(ls.LsError) as e:
            srv.ls_server_submit(dict(A=A, b=b, x=x, m=4000, n=64, lda=64, d=20000))       # d above 12288
        assert e.value.status == ls.LS_EINVAL
        with pytest.raises(ls.LsError) as e:                                              # above the arena
            srv.ls_server_submit(dict(A=A, b=b, x=x, m=4000, n=64, lda=64, d=1280))
        assert e.value.status == ls.LS_ENOMEM
        assert srv.ls_server_step() == 0                                                  # idle step
        assert srv.ls_server_poll() == []
    finally:
        srv.close()
