"""Multi-rank host logic on CPU (gloo, world size 2): bench.py's timing is
the max over ranks and its value the whole-job throughput; under torchrun
only rank 0 prints the reference arm; and the row-sharded iteration (each
rank forms the partial A^T r and squared norms of its own rows with the
oracle's pass, the partials are all-gathered and summed in rank order, the
step is shared) reaches the same iterate on both ranks, bit for bit, and
the forward-error rule."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    local_ms = [120.0, 180.0][rank]
    ms_max = bench.max_over_ranks(local_ms, dist, "cpu")
    out.put((rank, ms_max, bench.job_throughput(world, 5, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [180.0, 180.0]
    assert res[0][2] == pytest.approx(2 * 5 / 0.18)


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 4, 2000.0) == pytest.approx(2.0)


def test_reference_arm_nonzero_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert res.returncode == 0
    assert res.stdout.strip() == ""


def _sharded_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    import problems
    m, n, d = 4000, 50, 1000
    P = problems.make_problem(m, n, 1e6, 1e-6, 5)            # every rank draws the same problem
    B = oracle.sketch(P["A"], P["b"], d, 8, 0)
    R, x, ne, ce, rc = oracle.factor(B, 0)
    lo, hi = [0, 1700, m][rank], [1700, m][rank]               # uneven split of the rows
    A_p, b_p = P["A"][lo:hi], P["b"][lo:hi]
    rp = None
    u = 2.0 ** -53
    xn = float(np.linalg.norm(x))
    iters = 0
    for i in range(100):
        r, c = oracle.residual_gradient(A_p, b_p, x)
        local = np.concatenate([c, [r @ r, 0.0 if rp is None else (r - rp) @ (r - rp)]])
        parts = [torch.zeros(n + 2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(local))
        tot = np.zeros(n + 2)
        for p in range(world):                                  # fixed rank order
            tot = tot + parts[p].numpy()
        rn, dn = np.sqrt(tot[n]), np.sqrt(tot[n + 1])
        if rp is not None and dn <= u * (1.0 * ne * xn + 0.04 * ce * rn):
            break
        y = oracle.trsv_upper_T(R, tot[:n])
        x = x + oracle.trsv_upper(R, y)
        xn = float(np.linalg.norm(x))
        rp = r
        iters += 1
    fe = oracle.forward_error(x, P["x"])
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    out.put((rank, x.tobytes(), iters, fe, fe_qr))
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_iteration_gloo():
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29531
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, x0, it0, fe0, fq0), (_, x1, it1, fe1, fq1) = res
    assert x0 == x1 and it0 == it1                              # same iterate on both ranks
    assert it0 < 100 and fe0 <= 10 * fq0, (it0, fe0, fq0)
