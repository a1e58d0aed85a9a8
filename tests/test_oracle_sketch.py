"""Pins for the oracle's counting sort and sketch B = S [A b] (Algorithm 2,
sketch step; Sec. 2.2, Eq. (2.4)).

The CSR is checked against Python's stable sort; B against the explicit
dense S built from the index table and an exactly rounded sum (math.fsum),
within the bound of recursive summation; special cases A = I (B is S itself,
entries exactly +-1/sqrt(zeta)) and the subspace-embedding property.
"""
import math

import numpy as np
import pytest

import oracle

U = 2.0 ** -53


def dense_S(rows, signs, d, zeta):
    m = rows.shape[0]
    S = np.zeros((d, m))
    for j in range(m):
        for k in range(zeta):
            S[rows[j, k], j] = -1.0 if (signs[j] >> k) & 1 else 1.0
    return S


@pytest.mark.parametrize("m,d,zeta,seed", [(1, 1, 1, 0), (37, 8, 3, 5), (500, 40, 8, 1), (1000, 1000, 8, 2)])
def test_csr_is_stable_bucket_sort(m, d, zeta, seed):
    rows, signs = oracle.sketch_indices(m, d, zeta, seed)
    row_ptr, ent = oracle.sketch_csr(m, d, zeta, rows, signs)
    triples = [(int(rows[j, k]), j, (int(signs[j]) >> k) & 1) for j in range(m) for k in range(zeta)]
    triples.sort(key=lambda t: t[0])          # stable: keeps ascending j within a row
    want = np.array([(j << 1) | neg for (_, j, neg) in triples], dtype=np.uint32)
    assert np.array_equal(ent, want)
    counts = np.bincount(rows.ravel(), minlength=d)
    assert np.array_equal(np.diff(row_ptr), counts)
    assert row_ptr[0] == 0 and row_ptr[-1] == m * zeta


@pytest.mark.parametrize("m,n,d,zeta", [(60, 5, 12, 3), (300, 7, 40, 8), (1000, 1, 100, 8)])
def test_sketch_apply_vs_dense_S(m, n, d, zeta):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-5, 5, (m, 1)))
    b = rng.standard_normal(m)
    seed = 9
    rows, signs = oracle.sketch_indices(m, d, zeta, seed)
    row_ptr, ent = oracle.sketch_csr(m, d, zeta, rows, signs)
    s = oracle.sketch_scale(zeta)
    B = oracle.sketch_apply(A, b, d, row_ptr, ent, s)
    S = dense_S(rows, signs, d, zeta)
    Ab = np.column_stack([A, b])
    for t in range(d):
        nz = np.nonzero(S[t])[0]
        for c in range(n + 1):
            terms = [S[t, j] * Ab[j, c] for j in nz]      # exact (+-1 times a double)
            exact = math.fsum(terms)
            k = len(terms)
            bound = (k * U) * sum(abs(v) for v in terms) * abs(s) + U * abs(s * exact) + 1e-300
            assert abs(B[t, c] - s * exact) <= 2 * bound, (t, c)


def test_identity_gives_S_exactly():
    m, d, zeta = 64, 16, 4
    A = np.eye(m)
    b = np.zeros(m)
    rows, signs = oracle.sketch_indices(m, d, zeta, 4)
    row_ptr, ent = oracle.sketch_csr(m, d, zeta, rows, signs)
    s = oracle.sketch_scale(zeta)
    B = oracle.sketch_apply(A, b, d, row_ptr, ent, s)
    S = dense_S(rows, signs, d, zeta) * s
    assert np.array_equal(B[:, :m], S)
    assert np.all(B[:, m] == 0.0)
    assert np.all(np.count_nonzero(B[:, :m], axis=0) == zeta)
    assert set(np.unique(np.abs(B[:, :m]))) == {0.0, 0.5}


def test_scale_is_correctly_rounded():
    for zeta in range(1, 33):
        s = oracle.sketch_scale(zeta)
        assert s == 1.0 / math.sqrt(zeta)


def test_subspace_embedding_distortion():
    """||S v|| ~ ||v|| over range(A) with distortion well below 1 - 1/sqrt(2)
    at d = 20 n (Sec. 2.2; Thm. 3.1 needs eps < 0.29)."""
    import problems
    P = problems.make_problem(4000, 50, 1.0, 1e-3, 0)
    B = oracle.sketch(P["U"], np.zeros(4000), 1000, 8, 0)[:, :50]
    sv = np.linalg.svd(B, compute_uv=False)
    eps = max(sv.max() - 1, 1 - sv.min())
    assert eps < 0.29, eps
