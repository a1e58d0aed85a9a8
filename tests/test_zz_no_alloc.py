"""ls_residual_gradient_noalloc: the fused pass for callers that cannot
allocate device memory (they run inside a pool or arena they do not own, or
under a framework that forbids cudaMalloc on its hot path).  Checked through
the C ABI against the allocating entry point, ls_residual_gradient, on two
calls in a row: the same kernels and summation order give the same bits, and
the element-wise rounding bound of the parity tests is the message when they
do not.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import U, dev, gamma, host, padded_rowmajor, require_gpu

pytestmark = pytest.mark.gpu


def _outputs(torch, m, n):
    return (torch.empty(m, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"),
            torch.empty(2, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("m,n,lda", [(4000, 50, 50), (3007, 1000, 1000), (5001, 257, 258), (130, 128, 128)])
def test_noalloc_matches_allocating_pass(m, n, lda):
    torch, ls = require_gpu()
    L = ls.lib()
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-4, 4, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-3 * rng.standard_normal(m)
    rp = b - A @ x + 1e-6 * rng.standard_normal(m)
    Ad, bd, xd, rpd = dev(torch, padded_rowmajor(A, lda)), dev(torch, b), dev(torch, x), dev(torch, rp)
    stream = torch.cuda.current_stream()
    with ls.Context(0, stream) as ctx:
        r0, c0, n0 = _outputs(torch, m, n)
        ctx.ls_residual_gradient(Ad, m, n, lda, bd, xd, rpd, r0, c0, n0)
    ref_r, ref_c, ref_n = host(r0), host(c0), host(n0)
    absr = np.abs(b) + np.abs(A) @ np.abs(x)
    for call in range(2):                      # two calls in a row share the scratch
        r1, c1, n1 = _outputs(torch, m, n)
        st = L.ls_residual_gradient_noalloc(C.c_void_p(stream.cuda_stream), Ad.data_ptr(), m, n, lda,
                                            bd.data_ptr(), xd.data_ptr(), rpd.data_ptr(), r1.data_ptr(),
                                            c1.data_ptr(), n1.data_ptr())
        assert st == ls.LS_OK, (call, st)
        rg, cg, ng = host(r1), host(c1), host(n1)
        bound_r = np.max(np.abs(rg - ref_r) / (2 * gamma(n + 1) * absr))
        bound_c = np.max(np.abs(cg - ref_c) / (2 * gamma(m) * (np.abs(A).T @ np.abs(ref_r)) + 1e-300))
        assert np.array_equal(rg, ref_r), (call, "r differs", bound_r)
        assert np.array_equal(cg, ref_c), (call, "c differs", bound_c)
        assert np.array_equal(ng, ref_n), (call, "norms differ", ng, ref_n)


def test_noalloc_without_previous_residual_or_residual_output():
    """r_prev = NULL (the call zeroes norms[1] itself) and r_out = NULL."""
    torch, ls = require_gpu()
    L = ls.lib()
    m, n = 6001, 300
    rng = np.random.default_rng(7)
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-2 * rng.standard_normal(m)
    Ad, bd, xd = dev(torch, A), dev(torch, b), dev(torch, x)
    stream = torch.cuda.current_stream()
    with ls.Context(0, stream) as ctx:
        _, c0, n0 = _outputs(torch, m, n)
        ctx.ls_residual_gradient(Ad, m, n, n, bd, xd, None, None, c0, n0)
    for call in range(2):
        _, c1, n1 = _outputs(torch, m, n)
        n1.fill_(123.0)                        # norms[1] must be written even without r_prev
        st = L.ls_residual_gradient_noalloc(C.c_void_p(stream.cuda_stream), Ad.data_ptr(), m, n, n,
                                            bd.data_ptr(), xd.data_ptr(), None, None, c1.data_ptr(),
                                            n1.data_ptr())
        assert st == ls.LS_OK, (call, st)
        assert np.array_equal(host(c1), host(c0)), call
        ng = host(n1)
        assert ng[0] == host(n0)[0] and ng[1] == 0.0, (call, ng)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, ls = require_gpu()
    L = ls.lib()
    m, n = 2000, 1026
    A = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    b = torch.zeros(m, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    c = torch.empty(n, dtype=torch.float64, device="cuda")
    nr = torch.empty(2, dtype=torch.float64, device="cuda")
    st = L.ls_residual_gradient_noalloc(C.c_void_p(torch.cuda.current_stream().cuda_stream), A.data_ptr(), m, n, n,
                                        b.data_ptr(), x.data_ptr(), None, None, c.data_ptr(), nr.data_ptr())
    assert st == ls.LS_EINVAL
