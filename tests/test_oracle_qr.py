"""Pins for the oracle's Householder QR, sketch-and-solve start and the two
estimates (Algorithm 2 QR step; Sec. 3.2, Eq. (3.4); Sec. 2.3, Eq. (2.5);
Sec. 3.3).

Checks: R^T R = B^T B in extended precision to the backward-error bound of
Householder QR; |diag R| against LAPACK (numpy.linalg.qr, an independent
implementation); Q^T Q = I from the stored reflectors; an upper-triangular
input comes back as itself up to row signs; a zero column is reported; the
start x0 solves the sketched problem to Wedin's bound; normest <= ||R||_2;
condest equals the exact kappa_1 on small matrices where the estimator is
exact and never exceeds it.
"""
import numpy as np
import pytest

import oracle
import problems

U = 2.0 ** -53


def q_from_reflectors(F, tau):
    rows, _ = F.shape
    k = len(tau)
    Q = np.eye(rows)[:, :k].copy()
    for j in reversed(range(k)):
        v = np.zeros(rows)
        v[j] = 1.0
        v[j + 1:] = F[j + 1:, j]
        Q -= tau[j] * np.outer(v, v @ Q)
    return Q


@pytest.mark.parametrize("d,n,kappa", [(30, 5, 1e2), (200, 20, 1e8), (1000, 51, 1e10)])
def test_householder_backward_error(d, n, kappa):
    rng = np.random.default_rng(d)
    P = problems.make_problem(d, n, kappa, 0.0, d)
    B = P["A"] * rng.uniform(0.5, 2.0)
    F, tau, rc = oracle.householder_qr(B)
    assert rc == 0
    R = np.triu(F[:n, :n])
    BtB = B.astype(np.longdouble).T @ B.astype(np.longdouble)
    RtR = R.astype(np.longdouble).T @ R.astype(np.longdouble)
    err = float(np.max(np.abs(RtR - BtB)))
    nb = float(np.linalg.norm(B, 2))
    assert err <= 10 * d * n * U * nb * nb, err
    Q = q_from_reflectors(F, tau)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) < 10 * d * U
    assert np.max(np.abs(Q @ R - B)) < 10 * d * n * U * nb
    # |diag R| against LAPACK's Householder QR (independent code)
    Rl = np.linalg.qr(B, mode="r")
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-10 * kappa, atol=0)


def test_upper_triangular_input_is_fixed_point():
    rng = np.random.default_rng(0)
    T = np.triu(rng.standard_normal((8, 8))) + 4 * np.eye(8)
    F, tau, rc = oracle.householder_qr(T)
    R = np.triu(F)
    D = np.sign(np.diag(R))
    np.testing.assert_allclose(D[:, None] * R, np.sign(np.diag(T))[:, None] * T, rtol=0, atol=1e-14)


def test_zero_column_is_rank_error():
    B = np.ones((10, 3))
    B[:, 1] = 0.0
    _, _, rc = oracle.householder_qr(B)
    assert rc == 2
    B = np.ones((10, 3))       # rank 1: R[1,1] == 0
    _, _, rc = oracle.householder_qr(B)
    assert rc == 2


def test_factor_start_is_sketched_ls_solution():
    P = problems.make_problem(4000, 50, 1e6, 1e-4, 2)
    B = oracle.sketch(P["A"], P["b"], 1000, 8, 0)
    R, x0, ne, ce, rc = oracle.factor(B, 0)
    assert rc == 0
    Bm, Sb = B[:, :50], B[:, 50]
    ref = np.linalg.lstsq(Bm, Sb, rcond=None)[0]       # LAPACK, independent
    kB = np.linalg.cond(Bm)
    nB = np.linalg.norm(Bm, 2)
    rs = np.linalg.norm(Sb - Bm @ ref)
    wedin = 2.23 * kB * (np.linalg.norm(ref) + kB * rs / nB) * (10 * 1000 * U)
    assert np.linalg.norm(x0 - ref) <= 2 * wedin
    # R^T R = B^T B
    err = np.max(np.abs(R.T @ R - Bm.T @ Bm))
    assert err <= 10 * 1000 * 50 * U * nB ** 2


def test_normest_bounds_and_exact_cases():
    rng = np.random.default_rng(5)
    for n in [1, 2, 5, 50, 200]:
        R = np.triu(rng.standard_normal((n, n))) + np.eye(n) * 3
        ne = oracle.normest(R, seed=0)
        s = np.linalg.norm(R, 2)
        assert ne <= s * (1 + 1e-12)
        assert ne >= 0.3 * s
    # c * I: every unit vector is a top singular vector
    for c in [0.5, 3.0, 1e-7]:
        assert oracle.normest(c * np.eye(40), seed=1) == pytest.approx(c, rel=1e-14)
    assert oracle.power_steps(1) == 1
    assert oracle.power_steps(3) == 2         # ceil(ln 3) = 2
    assert oracle.power_steps(1000) == 7      # ceil(ln 1000) = 7
    assert oracle.power_steps(50) == 4


def test_condest_is_kappa1_lower_bound():
    rng = np.random.default_rng(7)
    for n in [1, 2, 3, 10, 50]:
        for _ in range(5):
            R = np.triu(rng.standard_normal((n, n)))
            R[np.diag_indices(n)] += np.sign(np.diag(R)) * 0.1 + (np.diag(R) == 0)
            k1 = np.linalg.norm(R, 1) * np.linalg.norm(np.linalg.inv(R), 1)
            ce = oracle.condest(R)
            assert ce <= k1 * (1 + 1e-9)
            assert ce >= k1 / 3.0
    # diagonal R: estimator is exact
    D = np.diag([1.0, 1e-3, 10.0, 1e-6])
    assert oracle.condest(D) == pytest.approx(10.0 / 1e-6, rel=1e-12)
    assert oracle.norm1_upper(D) == 10.0
    assert oracle.inv_norm1_est(D) == pytest.approx(1e6, rel=1e-12)


@pytest.mark.parametrize("R", [
    [[-1.0, -4.0, -8.0], [0.0, -2.0, -5.0], [0.0, 0.0, -2.0]],
    [[-0.5, 3.0, -2.0, 0.0], [0.0, -1.0, 0.0, -8.0], [0.0, 0.0, 0.5, 9.0], [0.0, 0.0, 0.0, 2.0]],
    [[2.0, 5.0, -1.0], [0.0, -0.5, -1.0], [0.0, 0.0, -1.0]],
])
def test_inverse_norm_estimator_needs_more_than_one_step(R):
    """Small triangular matrices on which the first sign-vector step of
    Hager's method lands on a column that is not the largest; the later
    steps reach the exact ||R^{-1}||_1."""
    R = np.array(R)
    exact = np.linalg.norm(np.linalg.inv(R), 1)
    assert oracle.inv_norm1_est(R) == pytest.approx(exact, rel=1e-12)
