"""The seeded input generators (problems/) against the recipe they state:
the paper's construction A = U diag(sigma) V^T with log-spaced sigma, a unit
x, a residual of the stated norm orthogonal to range(A), b = A x + r (numpy
and torch forms); the batched and serving shape distributions; the sparse
workload's rows; the Poisson arrivals.  No GPU."""
import numpy as np
import pytest

import problems

U = 2.0 ** -53


def test_sigmas_log_spaced():
    s = problems.sigmas(11, 1e10)
    assert s[0] == 1.0 and s[-1] == pytest.approx(1e-10, rel=1e-14)
    assert np.allclose(np.diff(np.log10(s)), -1.0, rtol=0, atol=1e-12)
    assert np.array_equal(problems.sigmas(1, 1e8), np.ones(1))


@pytest.mark.parametrize("m,n,kappa,res", [(800, 20, 1e2, 1e-3), (2000, 50, 1e10, 1e-6), (500, 25, 1e8, 1e-10)])
def test_numpy_problem_is_the_stated_construction(m, n, kappa, res):
    P = problems.make_problem(m, n, kappa, res, 7)
    A, b, x, r = P["A"], P["b"], P["x"], P["r"]
    assert A.shape == (m, n) and A.flags["C_CONTIGUOUS"]
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.abs(sv - problems.sigmas(n, kappa)) <= 1e-13), np.max(np.abs(sv - problems.sigmas(n, kappa)))
    assert np.linalg.norm(x) == pytest.approx(1.0, rel=1e-14)
    assert np.linalg.norm(r) == pytest.approx(res, rel=1e-12)
    # r is orthogonal to range(A): ||A^T r|| at the rounding level of forming it
    assert np.linalg.norm(A.T @ r) <= 50 * U * np.sqrt(m) * res
    assert np.allclose(b, A @ x + r, rtol=0, atol=4 * U * (1 + res))
    # x and r are the solution and residual of min ||A x - b||
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(xs - x) <= 1e3 * kappa * U * (1 + kappa * res)


def test_problems_are_seeded():
    a = problems.make_problem(300, 10, 1e4, 1e-3, 3)
    b = problems.make_problem(300, 10, 1e4, 1e-3, 3)
    c = problems.make_problem(300, 10, 1e4, 1e-3, 4)
    assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["b"], b["b"])
    assert not np.array_equal(a["A"], c["A"])


def test_torch_problem_is_the_stated_construction():
    torch = pytest.importorskip("torch")
    m, n, kappa, res = 1500, 30, 1e8, 1e-4
    P = problems.make_problem_torch(m, n, kappa, res, 2, device="cpu")
    A, b, x, r = (P[k].numpy() for k in ("A", "b", "x", "r"))
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.abs(sv - problems.sigmas(n, kappa)) <= 1e-13)
    assert np.linalg.norm(x) == pytest.approx(1.0, rel=1e-14)
    assert np.linalg.norm(r) == pytest.approx(res, rel=1e-12)
    assert np.linalg.norm(A.T @ r) <= 50 * U * np.sqrt(m) * res
    assert np.allclose(b, A @ x + r, rtol=0, atol=4 * U * (1 + res))
    Q = problems.make_problem_torch(m, n, kappa, res, 2, device="cpu")
    assert torch.equal(P["A"], Q["A"]) and torch.equal(P["b"], Q["b"])


def test_batch_shapes_follow_the_recipe():
    cfg = problems.BATCH
    sh = problems.batch_shapes(**cfg)
    assert len(sh) == cfg["count"] == 4096
    n = np.array([s["n"] for s in sh]); m = np.array([s["m"] for s in sh])
    kap = np.array([s["kappa"] for s in sh]); res = np.array([s["resnorm"] for s in sh])
    assert n.min() >= 10 and n.max() <= 200
    assert np.all(m >= np.maximum(500, 20 * n)) and m.max() <= 20_000
    assert all(s["d"] == 20 * s["n"] for s in sh)
    assert kap.min() >= 1e2 and kap.max() <= 1e12 and res.min() >= 1e-10 and res.max() <= 1e-2
    # log-uniform: the logs' means sit at the middle of their ranges
    assert np.mean(np.log10(kap)) == pytest.approx(7.0, abs=0.15)
    assert np.mean(np.log10(res)) == pytest.approx(-6.0, abs=0.15)
    assert np.mean(np.log(n)) == pytest.approx(0.5 * (np.log(10) + np.log(200)), abs=0.05)
    assert [s["index"] for s in sh] == list(range(4096))
    assert sh == problems.batch_shapes(**cfg)


def test_serving_pool_and_arrivals():
    cfg = problems.SERVE
    sh = problems.batch_shapes(**cfg)
    n = np.array([s["n"] for s in sh]); m = np.array([s["m"] for s in sh])
    assert n.min() >= 20 and n.max() <= 500
    assert np.all(m >= np.maximum(1000, 20 * n)) and m.max() <= 500_000
    t = problems.poisson_arrivals(200, 4000, 1)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.mean(gaps) == pytest.approx(1 / 200, rel=0.05)
    assert np.std(gaps) == pytest.approx(1 / 200, rel=0.08)      # exponential: std = mean


def test_sparse_rows():
    S = problems.make_sparse(20_000, 50, 3)
    col = S["col"].reshape(-1, 3)
    assert np.all(np.diff(col, axis=1) > 0)                       # distinct, ascending
    assert col.min() >= 0 and col.max() < 50
    assert set(np.unique(S["val"])) == {-1.0, 1.0}
    assert np.array_equal(S["row_ptr"], np.arange(0, 3 * 20_000 + 1, 3))
    counts = np.bincount(col.ravel(), minlength=50)               # columns uniform
    exp = 3 * 20_000 / 50
    chi2 = np.sum((counts - exp) ** 2 / exp)
    assert chi2 < 100                                              # 49 degrees of freedom
    A = problems.sparse_to_dense(S)
    assert np.count_nonzero(A) == 3 * 20_000
    T = problems.make_sparse(20_000, 50, 3)
    assert np.array_equal(T["col"], S["col"]) and np.array_equal(T["b"], S["b"])
