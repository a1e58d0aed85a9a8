"""Pins for the oracle's random source (Philox4x32-10, Lemire, Floyd).

Philox is checked against Triton's independent Philox4x32 implementation,
run on the CPU through Triton's interpreter (outputs only).  Lemire's
bounded draw and Floyd's subset sampling are checked against the properties
that define them: range, exact uniformity in distribution (chi-square), and
distinctness of the zeta rows of every column (Sec. 2.2, Eq. (2.4): "exactly
zeta nonzero entries ... in uniformly random positions").
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle


def _triton_philox(cases):
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def kern(c_ptr, k_ptr, out_ptr):
        i = tl.program_id(0)
        c0 = tl.load(c_ptr + 4 * i + 0)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        klo = tl.load(k_ptr + 2 * i + 0).to(tl.uint64)
        khi = tl.load(k_ptr + 2 * i + 1).to(tl.uint64)
        seed = klo | (khi << 32)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a)
        tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c)
        tl.store(out_ptr + 4 * i + 3, d)

    ctr = torch.tensor([c for c, _ in cases], dtype=torch.int64).to(torch.uint32)
    key = torch.tensor([k for _, k in cases], dtype=torch.int64).to(torch.uint32)
    out = torch.zeros(len(cases), 4, dtype=torch.uint32)
    kern[(len(cases),)](ctr, key, out)
    return out.to(torch.int64).numpy().astype(np.uint32)


def test_philox_matches_triton_interpreter():
    rng = np.random.default_rng(1)
    cases = [([0, 0, 0, 0], [0, 0]),
             ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2),
             ([1, 0, 0, 0], [0, 0]),
             ([0, 0, 0, 1], [0, 0]),
             ([5, 7, 3, 0], [123, 456])]
    for _ in range(11):
        cases.append((list(rng.integers(0, 2**32, 4)), list(rng.integers(0, 2**32, 2))))
    ref = _triton_philox(cases)
    for (ctr, key), want in zip(cases, ref):
        got = oracle.philox4x32_10(ctr, key)
        assert np.array_equal(got, want), (ctr, key, got, want)


def test_philox_is_a_bijection_on_sampled_counters():
    # distinct counters under one key give distinct 128-bit outputs
    seen = set()
    for c in range(2000):
        seen.add(tuple(oracle.philox4x32_10([c, 0, 0, 0], [7, 9])))
    assert len(seen) == 2000


@pytest.mark.parametrize("rng_size", [1, 2, 3, 7, 10, 1000, 20001])
def test_bounded_draw_range_and_uniformity(rng_size):
    n = 60000
    draws = oracle.bounded_draws(seed=11, j=rng_size, rng=rng_size, ndraws=n)
    assert draws.max() < rng_size
    if rng_size == 1:
        assert np.all(draws == 0)
        return
    if rng_size <= 1000:
        counts = np.bincount(draws, minlength=rng_size)
        expected = n / rng_size
        chi2 = float(((counts - expected) ** 2 / expected).sum())
        dof = rng_size - 1
        # 6-sigma bound of the chi-square statistic
        assert chi2 < dof + 6 * math.sqrt(2 * dof), chi2
    else:
        # mean and variance of the discrete uniform law
        mu = (rng_size - 1) / 2
        assert abs(draws.mean() - mu) < 6 * rng_size / math.sqrt(12 * n)


@pytest.mark.parametrize("d,zeta", [(4, 2), (5, 3), (6, 1), (7, 4), (6, 6)])
def test_floyd_subsets_exactly_uniform(d, zeta):
    """All C(d, zeta) row subsets equally likely (chi-square over 40k columns)."""
    ncols = 40000
    rows, signs = oracle.sketch_indices(ncols, d, zeta, seed=3)
    subsets = list(itertools.combinations(range(d), zeta))
    index = {s: i for i, s in enumerate(subsets)}
    counts = np.zeros(len(subsets))
    for r in rows:
        t = tuple(int(v) for v in r)
        assert list(t) == sorted(set(t)), t          # distinct and ascending
        counts[index[t]] += 1
    if len(subsets) == 1:
        assert counts[0] == ncols
        return
    expected = ncols / len(subsets)
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    dof = len(subsets) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


def test_signs_balanced_and_independent_of_rows():
    rows, signs = oracle.sketch_indices(20000, 1000, 8, seed=0)
    bits = ((signs[:, None] >> np.arange(8)[None, :]) & 1).astype(np.float64)
    # each of the 8 used sign bits is a fair coin
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 6 * 0.5 / math.sqrt(20000))
    # rows are distinct, ascending and in range for every column
    assert rows.min() >= 0 and rows.max() < 1000
    assert np.all(np.diff(rows, axis=1) > 0)


def test_seed_changes_stream():
    r0, s0 = oracle.sketch_indices(500, 200, 8, seed=0)
    r1, s1 = oracle.sketch_indices(500, 200, 8, seed=1)
    r0b, s0b = oracle.sketch_indices(500, 200, 8, seed=0)
    assert np.array_equal(r0, r0b) and np.array_equal(s0, s0b)
    assert not np.array_equal(r0, r1)


def test_invalid_zeta_rejected():
    with pytest.raises(ValueError):
        oracle.sketch_indices(10, 4, 5, seed=0)   # zeta > d
    with pytest.raises(ValueError):
        oracle.sketch_indices(10, 64, 33, seed=0)  # zeta > 32
