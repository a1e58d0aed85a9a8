"""CPU-side checks of the C-ABI library: it builds, loads, and exports every
entry point declared in include/ls.h (no compute calls: there is no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ls.h")).read()
    return sorted(set(re.findall(r"^LS_API\s+[\w\s\*]+?\b(ls_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_04362_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["ls_create", "ls_destroy", "ls_last_error", "ls_workspace_bytes", "ls_sketch_indices", "ls_solve_ex",
              "ls_sketch_csr", "ls_sketch", "ls_factor", "ls_residual_gradient", "ls_correct",
              "ls_iterate", "ls_solve", "ls_default_opts"]:
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    import ctypes
    import paper_2311_04362_gb300 as ls
    L = ls.lib()
    for s in declared_symbols():
        assert hasattr(L, s)
    o = ls.default_opts()
    assert (o.gamma, o.rho, o.extra_iters, o.use_stop, o.alpha, o.beta) == (1.0, 0.04, 3, 1, 1.0, 0.0)
    # no GPU here: creating a context must fail with a status, not crash
    h = ctypes.c_void_p()
    st = L.ls_create(ctypes.byref(h), 0, None)
    assert st != ls.LS_OK or h.value
    if st == ls.LS_OK:
        L.ls_destroy(h)
    assert L.ls_last_error(None) == b"null context"


def test_damping_and_momentum_weights(libpath):
    """App. B, Eqs. (B.2)-(B.3) with e = sqrt(n/d)."""
    import paper_2311_04362_gb300 as ls
    n, d = 50, 1000
    e2 = n / d
    o = ls.damping_opts(n, d)
    assert o.alpha == pytest.approx((1 - e2) ** 2 / (1 + e2), rel=1e-15) and o.beta == 0.0
    o = ls.momentum_opts(n, d)
    assert o.alpha == pytest.approx((1 - e2) ** 2, rel=1e-15) and o.beta == pytest.approx(e2, rel=1e-15)
    assert o.use_stop == 1 and o.rho == 0.04


def test_header_declares_the_next_rows():
    syms = declared_symbols()
    for s in ["ls_solve_batched", "ls_solve_batched_mixed", "ls_tune_batched", "ls_reset_tuning", "ls_server_create",
              "ls_server_submit", "ls_server_step", "ls_server_poll", "ls_server_get_stats", "ls_server_destroy",
              "ls_server_request_bytes", "ls_sketch_sparse", "ls_solve_sparse", "ls_opts_damping",
              "ls_opts_momentum", "ls_residual_gradient_noalloc"]:
        assert s in syms, s


def test_server_request_bytes_accounting(libpath):
    """Host-only: a request counts its resident A, b, x plus the workspace
    (sketch d (n+1), R and R^T 2 n^2, eight n-vectors, pass partials, r_prev),
    each rounded up to 256 bytes."""
    import paper_2311_04362_gb300 as ls

    def al(x):
        return (x + 255) // 256 * 256

    for m, n, lda, d in [(1000, 10, 10, 200), (50000, 123, 124, 2460), (500000, 500, 500, 10000)]:
        got = ls.server_request_bytes(m, n, lda, d)
        resident = al(8 * m * lda) + al(8 * m) + al(8 * n)
        fixed = al(8 * d * (n + 1)) + al(16 * n * n) + al(64 * n) + al(8 * m)
        assert got > resident + fixed                       # plus the pass partials
        partials = got - resident - fixed
        assert 0 < partials <= al(8 * (n + 2) * m)          # at most one partial per row
    assert ls.server_request_bytes(0, 10, 10, 200) == 0
    assert ls.server_request_bytes(100, 10, 8, 200) == 0    # lda < n
    assert ls.server_request_bytes(2000, 20, 20, 400) < ls.server_request_bytes(4000, 20, 20, 400)
    assert ls.server_request_bytes(4000, 20, 20, 400) < ls.server_request_bytes(4000, 40, 40, 800)


def test_api_rejects_without_a_context(libpath):
    """Host-only argument checks: a null context is LS_EINVAL everywhere."""
    import ctypes as C
    import paper_2311_04362_gb300 as ls
    L = ls.lib()
    assert L.ls_solve_batched(None, None, 0, 8, 100, None, None) == ls.LS_EINVAL
    assert L.ls_tune_batched(None, None, 0, 1, None, 0) == ls.LS_EINVAL
    assert L.ls_server_destroy(None) == ls.LS_EINVAL
    assert L.ls_solve_sparse(None, None, None, None, 10, 2, 20, None, 4, 8, 10, 0, None, None, None) == ls.LS_EINVAL
    n_out = C.c_int()
    assert L.ls_server_poll(None, None, None, 0, C.byref(n_out)) == ls.LS_EINVAL


def test_workspace_bytes_covers_the_solve(libpath):
    """ls_workspace_bytes (no GPU here: the host path assumes 152 SMs) is 0 for
    an invalid shape, grows with every dimension, and covers at least the
    arrays a solve of that shape must hold at once: the sketch B_aug (d x
    (n+1) doubles) and R (n x n) beside the sketch's bucket entries (m zeta
    4-byte words, twice: the hash output and the sorted CSR)."""
    import paper_2311_04362_gb300 as ls
    L = ls.lib()
    assert L.ls_workspace_bytes(0, 10, 20, 8) == 0 and L.ls_workspace_bytes(100, 10, 20, 0) == 0
    m, n, d, z = 200_000, 100, 2000, 8
    w = L.ls_workspace_bytes(m, n, d, z)
    assert w >= 8 * d * (n + 1) + 8 * n * n + 2 * 4 * m * z
    for args in [(2 * m, n, d, z), (m, 2 * n, 2 * d, z), (m, n, 2 * d, z), (m, n, d, 2 * z)]:
        assert L.ls_workspace_bytes(*args) >= w, args
