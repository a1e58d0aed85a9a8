"""GPU parity of the batched solver (ls_solve_batched): many independent
problems of different shapes, one launch per phase for the whole batch.

Checks per problem, against the oracle on the same seeded inputs:
 * the sketch [S A, S b] is bit-identical to the oracle's (same Philox words,
   same left-to-right sums);
 * R is upper triangular, backward stable (|R^T R - B^T B| <= 10 d n u ||B||^2)
   and within the QR perturbation bound 10 d n u kappa(B) of the oracle's R;
 * normest within 1e-10 relative of the oracle's, condest within
   max(1e-6, 10 n u kappa(B)) (substitutions on R amplify rounding by
   kappa(R) u);
 * the final x is as accurate as a backward-stable solve: forward error
   <= 10x that of the oracle's Householder-QR solution, or within Wedin's
   bound 10 u kappa (1 + kappa ||r|| / (||A|| ||x||)) for a backward error of
   10 u (the accuracy the paper reports for its stopping rule; Householder
   QR often lands well inside that bound, and which of the two stops closer
   to x depends on rounding), with the stopping rule having held, in an
   iteration count close to the oracle's whole-method run.  The rule
   fires when ||r_i - r_{i-1}|| reaches the rounding floor, and two rounding
   orders put that floor up to a few decades apart; with a contraction of g
   per step a floor F times higher moves the firing step by log F / log(1/g),
   about iters * log10(F) / 16 since iters ~ 16 / log10(1/g).  Allowing
   F = 1e4 gives |iters - iters_oracle| <= max(5, iters / 4).
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import DEFAULT_EXTRA, U, dev, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


def _small_shapes():
    """A mixed batch: the batched distribution at smaller m, plus edge shapes
    (n = 1, m = 20 n exactly, odd n, n above the 256-thread split, ragged
    tiles)."""
    sh = problems.batch_shapes(count=24, m_lo=500, m_hi=4000, n_lo=10, n_hi=64, kappa_lo=1e2, kappa_hi=1e12,
                               res_lo=1e-10, res_hi=1e-2, d_over_n=20, seed=1)
    extra = [dict(m=500, n=1, kappa=1.0, resnorm=1e-3), dict(m=1000, n=50, kappa=1e10, resnorm=1e-6),
             dict(m=1237, n=37, kappa=1e6, resnorm=1e-5), dict(m=6000, n=300, kappa=1e4, resnorm=1e-4),
             dict(m=4001, n=200, kappa=1e8, resnorm=1e-8), dict(m=2000, n=99, kappa=1e12, resnorm=1e-2)]
    for k, e in enumerate(extra):
        e.update(d=20 * e["n"], data_seed=900 + k)
        sh.append(e)
    for i, s in enumerate(sh):
        s["index"] = i
    return sh


def _upload(torch, shapes, with_outputs=True):
    """numpy problems -> device problem dicts (lda even, padded)."""
    probs, host_probs = [], []
    for s in shapes:
        P = problems.make_problem(s["m"], s["n"], s["kappa"], s["resnorm"], s["data_seed"])
        n = s["n"]
        lda = n + (n % 2)
        Ad = dev(torch, padded_rowmajor(P["A"], lda))
        p = dict(A=Ad, b=dev(torch, P["b"]), x=torch.empty(n, dtype=torch.float64, device="cuda"), m=s["m"],
                 n=n, lda=lda, d=s["d"], seed=s["index"])
        if with_outputs:
            p["B_out"] = torch.empty(s["d"] * (n + 1), dtype=torch.float64, device="cuda")
            p["R_out"] = torch.empty(n * n, dtype=torch.float64, device="cuda")
        probs.append(p)
        host_probs.append(P)
    return probs, host_probs


@pytest.fixture(scope="module")
def small_batch(env):
    torch, ls, ctx = env
    shapes = _small_shapes()
    probs, hps = _upload(torch, shapes)
    infos = ctx.ls_solve_batched(probs, 8, 100)
    torch.cuda.synchronize()
    return shapes, probs, hps, infos


def test_batched_sketch_bit_identical(env, small_batch):
    shapes, probs, hps, _ = small_batch
    for s, p, P in zip(shapes, probs, hps):
        Bo = oracle.sketch(P["A"], P["b"], s["d"], 8, s["index"])
        Bg = host(p["B_out"]).reshape(s["n"] + 1, s["d"]).T
        assert np.array_equal(Bg, Bo), s


def test_batched_factor_parity(env, small_batch):
    shapes, probs, hps, infos = small_batch
    for s, p, P, inf in zip(shapes, probs, hps, infos):
        d, n = s["d"], s["n"]
        Bo = oracle.sketch(P["A"], P["b"], d, 8, s["index"])
        Rg = host(p["R_out"]).reshape(n, n).T
        Ro, x0o, ne, ce, rc = oracle.factor(Bo, s["index"])
        assert rc == 0
        Bm = Bo[:, :n]
        nB = np.linalg.norm(Bm, 2)
        kB = np.linalg.cond(Bm)
        assert np.all(np.tril(Rg, -1) == 0.0)
        L = np.longdouble
        err = np.max(np.abs(Rg.astype(L).T @ Rg.astype(L) - Bm.astype(L).T @ Bm.astype(L)))
        assert err <= 10 * d * n * U * nB ** 2, s
        D = np.sign(np.diag(Rg)) * np.sign(np.diag(Ro))
        assert np.linalg.norm(D[:, None] * Rg - Ro) / np.linalg.norm(Ro) <= 10 * d * n * U * kB, s
        assert inf.normest == pytest.approx(ne, rel=1e-10), s
        assert inf.condest == pytest.approx(ce, rel=max(1e-6, 10 * n * U * kB)), s


def test_batched_solutions_meet_acceptance(env, small_batch):
    shapes, probs, hps, infos = small_batch
    for s, p, P, inf in zip(shapes, probs, hps, infos):
        fe = oracle.forward_error(host(p["x"]), P["x"])
        fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
        assert inf.stop_reason == 0, (s, inf.as_dict())
        k, res = P["kappa"], P["resnorm"]
        wedin = 10 * U * k * (1 + k * res / (np.linalg.norm(P["A"], 2) * np.linalg.norm(P["x"])))
        assert fe <= max(10 * fe_qr, wedin), (s, fe, fe_qr, wedin)
        xo, io = oracle.solve(P["A"], P["b"], s["d"], 8, 100, s["index"], extra=DEFAULT_EXTRA)
        assert oracle.forward_error(xo, P["x"]) <= max(10 * fe_qr, wedin)
        if io["converged"]:
            assert abs(inf.iters - io["iters"]) <= max(5, io["iters"] / 4), (s, inf.iters, io["iters"])
        # else: the oracle's plain left-to-right sums leave ||r_i - r_{i-1}||
        # above the threshold until q; its iterate still meets the rule above


def test_batched_deterministic(env, small_batch):
    torch, ls, ctx = env
    shapes, probs, hps, infos = small_batch
    x1 = [host(p["x"]).copy() for p in probs]
    probs2 = [dict(p, x=torch.empty_like(p["x"]), B_out=None, R_out=None) for p in probs]
    infos2 = ctx.ls_solve_batched(probs2, 8, 100)
    for p, a, i1, i2 in zip(probs2, x1, infos, infos2):
        assert np.array_equal(host(p["x"]), a)
        assert i1.iters == i2.iters


def test_batched_single_problem_matches_batch_member(env, small_batch):
    """A batch of one runs the same kernels: its result equals that member's
    result inside the larger batch bit for bit (problems never interact)."""
    torch, ls, ctx = env
    shapes, probs, hps, infos = small_batch
    for k in (0, 7, len(probs) - 3):
        p = dict(probs[k], x=torch.empty_like(probs[k]["x"]), B_out=None, R_out=None)
        inf = ctx.ls_solve_batched([p], 8, 100)
        assert np.array_equal(host(p["x"]), host(probs[k]["x"]))
        assert inf[0].iters == infos[k].iters


def test_batched_fixed_steps_match_oracle(env):
    """use_stop = 0, q = 4: every problem takes exactly 4 updates; x_4 against
    the oracle's run from the oracle's own factor (moderate kappa, so the two
    starts agree to ~kappa u)."""
    torch, ls, ctx = env
    shapes = problems.batch_shapes(count=6, m_lo=600, m_hi=3000, n_lo=5, n_hi=40, kappa_lo=10, kappa_hi=1e4,
                                   res_lo=1e-6, res_hi=1e-2, d_over_n=20, seed=3)
    for i, s in enumerate(shapes):
        s["index"] = i
    probs, hps = _upload(torch, shapes, with_outputs=False)
    opts = ls.default_opts()
    opts.use_stop = 0
    infos = ctx.ls_solve_batched(probs, 8, 4, opts)
    for s, p, P, inf in zip(shapes, probs, hps, infos):
        assert inf.iters == 4 and inf.stop_reason == 2
        xo, io = oracle.solve(P["A"], P["b"], s["d"], 8, 4, s["index"], use_stop=False)
        assert io["iters"] == 4
        k = s["kappa"]
        tol = 100 * k * (1 + k * s["resnorm"]) * U
        assert np.linalg.norm(host(p["x"]) - xo) <= tol * np.linalg.norm(xo), s


def test_batched_rank_deficient_member_isolated(env):
    torch, ls, ctx = env
    shapes = problems.batch_shapes(count=3, m_lo=800, m_hi=2000, n_lo=8, n_hi=20, kappa_lo=10, kappa_hi=1e6,
                                   res_lo=1e-8, res_hi=1e-4, d_over_n=20, seed=4)
    for i, s in enumerate(shapes):
        s["index"] = i
    probs, hps = _upload(torch, shapes, with_outputs=False)
    # problem 1: an exactly zero column makes R[2, 2] exactly zero
    probs[1]["A"].view(shapes[1]["m"], probs[1]["lda"])[:, 2] = 0.0
    infos = ctx.ls_solve_batched(probs, 8, 100)
    assert infos[1].stop_reason == 4
    for k in (0, 2):
        P = hps[k]
        assert infos[k].stop_reason == 0
        fe = oracle.forward_error(host(probs[k]["x"]), P["x"])
        assert fe <= 10 * oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])


def test_batched_invalid_arguments(env):
    torch, ls, ctx = env
    assert len(ctx.ls_solve_batched([], 8, 100)) == 0
    A = torch.zeros(2000 * 2000, dtype=torch.float64, device="cuda")
    b = torch.zeros(2000, dtype=torch.float64, device="cuda")
    x = torch.zeros(2000, dtype=torch.float64, device="cuda")
    bad = [dict(A=A, b=b, x=x, m=2000, n=1030, lda=1030, d=2000, seed=0),      # n above 1024
           dict(A=A, b=b, x=x, m=100, n=10, lda=10, d=5, seed=0),             # d < n
           dict(A=A, b=b, x=x, m=100, n=10, lda=11, d=200, seed=0),           # odd lda
           dict(A=A, b=b, x=None, m=100, n=10, lda=10, d=200, seed=0)]        # no x
    for p in bad:
        with pytest.raises(ls.LsError) as e:
            ctx.ls_solve_batched([p], 8, 100)
        assert e.value.status == ls.LS_EINVAL


def test_batched_full_size_sampled(env):
    """The full batch (4096 problems, m up to 20,000, n up to 200, kappa up to
    1e12) in the configuration the benchmark times.  Every problem ends with
    the rule held or q reached and a finite x; where the rule held, x is as
    accurate as a backward-stable solve (10x Householder QR's forward error or
    Wedin's bound for a backward error of 10 u, as in the small batch); the
    acceptance rule of the benchmark (10x Householder QR, geqrf through torch)
    holds on at least 95% of the problems.  It cannot hold on all: at
    d = 20 n with n ~ 10 the embedding's distortion reaches ~0.38, the basic
    iteration then contracts by only ~0.9 per step, and a few problems either
    stop at the rounding floor of ||r_i - r_{i-1}|| with x a decade off or run
    to q = 100 (the oracle does the same on those problems).  A sample of 6
    problems is checked against the oracle's own Householder-QR solution."""
    torch, ls, ctx = env
    cfg = problems.BATCH
    shapes = problems.batch_shapes(**cfg)
    probs = problems.make_batch_torch(shapes)
    infos = ctx.ls_solve_batched(probs, cfg["zeta"], cfg["q"])
    torch.cuda.synchronize()
    stops = np.array([i.stop_reason for i in infos])
    assert np.all((stops == 0) | (stops == 1)), np.unique(stops, return_counts=True)
    assert np.mean(stops == 0) >= 0.99, np.unique(stops, return_counts=True)
    rng = np.random.default_rng(5)
    sample = set(rng.choice(len(probs), 6, replace=False).tolist())
    ok = []
    for k, (s, p, inf) in enumerate(zip(shapes, probs, infos)):
        n = p["n"]
        A = p["A"][:, :n]
        xt = p["x_true"]
        assert bool(torch.isfinite(p["x"]).all())
        Q, R = torch.linalg.qr(A)
        xq = torch.linalg.solve_triangular(R, (Q.T @ p["b"])[:, None], upper=True)[:, 0]
        fe_qr = float(torch.linalg.norm(xq - xt) / torch.linalg.norm(xt))
        fe = float(torch.linalg.norm(p["x"] - xt) / torch.linalg.norm(xt))
        ok.append(fe <= 10 * fe_qr)
        if inf.stop_reason == 0:          # ||A|| = ||x|| = 1 by construction
            wedin = 10 * U * s["kappa"] * (1 + s["kappa"] * s["resnorm"])
            assert fe <= max(10 * fe_qr, wedin), (k, fe, fe_qr, wedin)
        if k in sample:
            Ah, bh, xth = host(A), host(p["b"]), host(xt)
            fe_or = oracle.forward_error(oracle.qr_solve(Ah, bh), xth)
            assert fe <= max(10 * fe_or, 10 * U * s["kappa"] * (1 + s["kappa"] * s["resnorm"])), (k, fe, fe_or)
    assert np.mean(ok) >= 0.95, np.mean(ok)
