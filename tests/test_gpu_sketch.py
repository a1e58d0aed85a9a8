"""GPU parity of the sketch steps (a1 indices, a2 CSR, a3 B = S[A b]) against
the oracle, through the C ABI.

Bar (stated for the sketch): indices, signs and CSR bit-exact; B within 1e-13
relative Frobenius error -- and, since the kernel keeps the oracle's
summation order (ascending j, left to right from +0.0, one final multiply),
bit-exact as well.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_common import dev, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, ls = require_gpu()
    ctx = ls.Context(0, torch.cuda.current_stream())
    yield torch, ls, ctx
    ctx.close()


INDEX_CASES = [(4000, 1000, 8, 0), (1, 1, 1, 0), (37, 8, 3, 5), (1000, 32, 32, 7), (5000, 64, 1, 2**40 + 5),
               (33, 2, 2, 9), (20001, 4000, 8, 123)]


@pytest.mark.parametrize("m,d,zeta,seed", INDEX_CASES)
def test_indices_bit_exact(env, m, d, zeta, seed):
    torch, ls, ctx = env
    rows = torch.empty(m * zeta, dtype=torch.int32, device="cuda")
    signs = torch.empty(m, dtype=torch.int32, device="cuda")
    ctx.ls_sketch_indices(m, d, zeta, seed, rows, signs)
    torch.cuda.synchronize()
    r_or, s_or = oracle.sketch_indices(m, d, zeta, seed)
    assert np.array_equal(host(rows).reshape(m, zeta), r_or)
    assert np.array_equal(host(signs).view(np.uint32), s_or)


def test_indices_full_size_bit_exact(env):
    """The large configuration's index table (m = 2e6, d = 20000, zeta = 8)."""
    torch, ls, ctx = env
    m, d, zeta = 2_000_000, 20_000, 8
    rows = torch.empty(m * zeta, dtype=torch.int32, device="cuda")
    signs = torch.empty(m, dtype=torch.int32, device="cuda")
    ctx.ls_sketch_indices(m, d, zeta, 0, rows, signs)
    r_or, s_or = oracle.sketch_indices(m, d, zeta, 0)
    assert np.array_equal(host(rows).reshape(m, zeta), r_or)
    assert np.array_equal(host(signs).view(np.uint32), s_or)


@pytest.mark.parametrize("m,d,zeta,seed", [(4000, 1000, 8, 0), (37, 8, 3, 5), (1, 1, 1, 0),
                                           (200_000, 100, 8, 1),     # buckets ~16000 > shared-memory sort
                                           (100_000, 20_000, 8, 3)])
def test_csr_bit_exact(env, m, d, zeta, seed):
    torch, ls, ctx = env
    r_or, s_or = oracle.sketch_indices(m, d, zeta, seed)
    rows = dev(torch, r_or.ravel())
    signs = dev(torch, s_or.view(np.int32))
    row_ptr = torch.empty(d + 1, dtype=torch.int64, device="cuda")
    ent = torch.empty(m * zeta, dtype=torch.int32, device="cuda")
    ctx.ls_sketch_csr(m, d, zeta, rows, signs, row_ptr, ent)
    rp_or, ent_or = oracle.sketch_csr(m, d, zeta, r_or, s_or)
    assert np.array_equal(host(row_ptr), rp_or)
    assert np.array_equal(host(ent).view(np.uint32), ent_or)


SKETCH_CASES = [(4000, 50, 50, 1000, 8, 0), (4000, 51, 52, 1000, 8, 1), (300, 1, 2, 20, 8, 2),
                (3000, 300, 300, 6000, 8, 3), (999, 7, 10, 140, 5, 4), (64, 64, 64, 64, 32, 5),
                (2500, 130, 132, 2600, 8, 6)]


@pytest.mark.parametrize("m,n,lda,d,zeta,seed", SKETCH_CASES)
def test_sketch_bit_exact(env, m, n, lda, d, zeta, seed):
    torch, ls, ctx = env
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-20, 20, (m, 1)))
    b = rng.standard_normal(m)
    Ad = dev(torch, padded_rowmajor(A, lda))
    bd = dev(torch, b)
    B = torch.empty((n + 1) * d, dtype=torch.float64, device="cuda")
    ctx.ls_sketch(Ad, m, n, lda, bd, d, zeta, seed, B, d)
    Bg = host(B).reshape(n + 1, d).T
    Bo = oracle.sketch(A, b, d, zeta, seed)
    rel = np.linalg.norm(Bg - Bo) / np.linalg.norm(Bo)
    assert rel <= 1e-13
    assert np.array_equal(Bg, Bo)


def test_sketch_ldb_padding(env):
    torch, ls, ctx = env
    P = problems.make_problem(1000, 10, 1e3, 1e-3, 4)
    d, ldb = 200, 203
    B = torch.full(((10 + 1) * ldb,), 7.0, dtype=torch.float64, device="cuda")
    ctx.ls_sketch(dev(torch, P["A"]), 1000, 10, 10, dev(torch, P["b"]), d, 8, 0, B, ldb)
    Bg = host(B).reshape(11, ldb).T
    assert np.array_equal(Bg[:d], oracle.sketch(P["A"], P["b"], d, 8, 0))
    assert np.all(Bg[d:] == 7.0)    # padding rows untouched


def test_sketch_full_size_sampled_rows(env):
    """Large configuration (m = 2e6, n = 1000, d = 20000): 12 sampled sketch
    rows recomputed by the oracle from their bucket rows of A."""
    torch, ls, ctx = env
    cfg = problems.LARGE
    m, n, d, zeta = cfg["m"], cfg["n"], cfg["d"], cfg["zeta"]
    P = problems.make_problem_torch(m, n, cfg["kappa"], cfg["resnorm"], cfg["seed"], device="cuda")
    A, b = P["A"], P["b"]
    B = torch.empty((n + 1) * d, dtype=torch.float64, device="cuda")
    ctx.ls_sketch(A, m, n, n, b, d, zeta, 0, B, d)
    Bg = host(B).reshape(n + 1, d).T
    r_or, s_or = oracle.sketch_indices(m, d, zeta, 0)
    rp, ent = oracle.sketch_csr(m, d, zeta, r_or, s_or)
    s = oracle.sketch_scale(zeta)
    for t in [0, 1, 777, 5000, 9999, 10000, 12345, 15000, 17777, 19998, 19999, 3]:
        e = ent[rp[t]:rp[t + 1]]
        js = (e >> 1).astype(np.int64)
        sub = host(A[torch.from_numpy(js).cuda()])
        bsub = host(b[torch.from_numpy(js).cuda()])
        local = ((np.arange(len(js), dtype=np.uint32) << 1) | (e & 1)).astype(np.uint32)
        row = oracle.sketch_apply(sub, bsub, 1, np.array([0, len(js)], dtype=np.int64), local, s)[0]
        assert np.array_equal(Bg[t], row), t
