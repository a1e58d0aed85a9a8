"""GPU checks of the batched-pass autotuner (ls_tune_batched): it writes one
choice per class of n present, solutions under the tuned table still meet
the acceptance rule and are deterministic, a server made from the tuned
context gives the batched solver's bits, and ls_reset_tuning restores the
default table exactly."""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import U, dev, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    yield torch, ls


def _batch(torch, count=16, seed=21):
    sh = problems.batch_shapes(count=count, m_lo=500, m_hi=5000, n_lo=10, n_hi=300, kappa_lo=1e2, kappa_hi=1e8,
                               res_lo=1e-8, res_hi=1e-3, d_over_n=20, seed=seed)
    probs, hps = [], []
    for i, s in enumerate(sh):
        P = problems.make_problem(s["m"], s["n"], s["kappa"], s["resnorm"], s["data_seed"])
        n = s["n"]
        lda = n + (n % 2)
        probs.append(dict(A=dev(torch, padded_rowmajor(P["A"], lda)), b=dev(torch, P["b"]),
                          x=torch.empty(n, dtype=torch.float64, device="cuda"), m=s["m"], n=n, lda=lda, d=s["d"],
                          seed=i))
        hps.append(P)
    return probs, hps


def test_tune_then_solve(env):
    torch, ls = env
    probs, hps = _batch(torch)
    with ls.Context(0, torch.cuda.current_stream()) as ctx:
        default = [dict(p, x=torch.empty_like(p["x"])) for p in probs]
        ctx.ls_solve_batched(default, 8, 100)
        report = ctx.ls_tune_batched(probs, reps=2)
        classes = {problems_class(p["n"]) for p in probs}
        assert len([ln for ln in report.splitlines() if ln.startswith("n<")]) == len(classes), report
        infos = ctx.ls_solve_batched(probs, 8, 100)
        x1 = [host(p["x"]).copy() for p in probs]
        for p, P, inf in zip(probs, hps, infos):
            fe = oracle.forward_error(host(p["x"]), P["x"])
            fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
            wedin = 10 * U * P["kappa"] * (1 + P["kappa"] * P["resnorm"])
            assert inf.stop_reason in (0, 1) and fe <= max(10 * fe_qr, wedin), (p["n"], fe, fe_qr)
        again = [dict(p, x=torch.empty_like(p["x"])) for p in probs]
        ctx.ls_solve_batched(again, 8, 100)
        assert all(np.array_equal(host(a["x"]), b) for a, b in zip(again, x1))
        # a server made from the tuned context: the batched solver's bits
        served = [dict(p, x=torch.empty_like(p["x"])) for p in probs]
        srv = ls.Server(ctx, 64, 512, 1 << 30, 0, 8, 100)
        try:
            for p in served:
                srv.ls_server_submit(p)
            got = 0
            while got < len(served):
                srv.ls_server_step()
                got += len(srv.ls_server_poll())
        finally:
            srv.close()
        assert all(np.array_equal(host(a["x"]), b) for a, b in zip(served, x1))
        # back to the defaults: the untuned bits
        ctx.ls_reset_tuning()
        reset = [dict(p, x=torch.empty_like(p["x"])) for p in probs]
        ctx.ls_solve_batched(reset, 8, 100)
        assert all(np.array_equal(host(a["x"]), host(b["x"])) for a, b in zip(reset, default))


def problems_class(n):
    b = 0
    while b < 5 and n >= (32 << b):
        b += 1
    return b
