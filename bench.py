#!/usr/bin/env python3
"""Benchmark: iterative-sketching least-squares solves/s on GB300.

Workload (one "step" = one whole solve: sketch, Householder QR of the sketch,
sketch-and-solve start, refinement with the Sec. 3.3 stopping rule): the
large single FP64 problem m = 2,000,000, n = 1000 (A is 16 GB, so inputs
exceed L2 every step), A = U diag(sigma) V^T with sigma log-spaced over
[1e-8, 1], ||r|| = 1e-4, d = 20 n = 20000, zeta = 8, seed 0, q <= 100.
Synthetic data, generated on the device (problems.make_problem_torch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  With N > 1 (torchrun), every rank solves its own
replica (independent problems: "replicas only", weak scaling) and the time is
the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LS solves/s at ≤10× QR fwd error"
UNIT = "solves/s"
CFG = dict(m=2_000_000, n=1000, kappa=1e8, resnorm=1e-4, d=20_000, zeta=8, seed=0, q=100)
WORKLOAD = ("large single FP64 problem: m=2,000,000, n=1000, kappa=1e8, ||r||=1e-4, d=20n=20000, "
            "zeta=8, Philox seed 0, q<=100 with the Sec. 3.3 stopping rule")

# HBM copy bandwidth when MEASURED_PEAKS.json is absent (one earlier GB300
# measurement, the profiling recipe's fallback).
HBM_FALLBACK_GBS = 6800.0
EXTRA_ITERS = 3        # updates after the stopping rule first holds, as ls_default_opts sets

# ncu DRAM traffic (read + write bytes) of one fixed-point pass launch on this
# workload, keyed by the hash of the kernel source it was taken on (a stale
# hash reports null): the capture is at m = 200,000 rows, scaled x10 to the
# m = 2,000,000 launch (the pass reads every row once, so traffic is linear in m).
NCU_TRAFFIC = {"911ff398312fa250": 16.0866e9}   # (1.604089 GB read + 4.6 MB written) x 10


def _code_only(text: str) -> str:
    """C/CUDA source with comments and blank space removed, so that a comment
    edit does not change the hash (string literals here hold no comment
    markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the fixed-point pass kernel's code (the k_fx_pass part of
    fxpass.cu, the integer arithmetic of fxarith.cuh and the shared device
    helpers of ls_internal.cuh), comments excluded."""
    csrc = os.path.join(ROOT, "paper_2311_04362_gb300", "csrc")
    with open(os.path.join(csrc, "fxpass.cu")) as fh:
        text = fh.read()
    h = hashlib.sha256(_code_only(text[text.index("namespace {"):text.index("// Sum the per-CTA fixed-point")]).encode())
    with open(os.path.join(csrc, "ls_internal.cuh")) as fh:
        helpers = fh.read()
    h.update(_code_only(helpers[:helpers.index("// -------------------------------------------------------------------- context")]).encode())
    with open(os.path.join(csrc, "fxarith.cuh")) as fh:
        h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def config_dict(world: int) -> dict:
    """The workload's config, the same in both arms."""
    return {"workload": WORKLOAD, **{k: CFG[k] for k in ("m", "n", "d", "zeta", "kappa", "resnorm", "q")},
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (A is 16 GB per step)"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------ multi-rank
def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (one all-reduce; identity without a group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, ms_max: float) -> float:
    """Whole-job solves/s: every rank solved `steps` problems; the job took the
    slowest rank's time."""
    return world * steps / (ms_max / 1e3)


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- oracle timing
_SAMPLE_CACHE: dict = {}


def _oracle_sample(iters_hint):
    """One bounded sample of the oracle on the large workload (single thread):
      sketch     : oracle sketch of the first m_s = 50,000 rows (d = 20000), x m/m_s
      QR         : oracle Householder QR + start + estimates of a 2000 x 1001
                   sketch, x d/2000 (cost linear in d for d >> n)
      iteration  : 2 oracle refinement steps on the m_s rows, per step x m/m_s
      iterations : the oracle's own count on a shape-matched small problem
                   (m = 20000, n = 100, d = 20n, same kappa and ||r||), unless
                   the GPU run's count is given.
    Returns (estimated seconds per full solve, wall seconds of the sample,
    description, details)."""
    import oracle
    import problems

    oracle.build()
    w0 = time.perf_counter()
    m, n, d, zeta = CFG["m"], CFG["n"], CFG["d"], CFG["zeta"]
    ms_rows, dq = 50_000, 2000
    # the sample's inputs (and the oracle's iteration count) are drawn once
    # per process; only the oracle's own work below is timed
    if "P" not in _SAMPLE_CACHE:
        _SAMPLE_CACHE["P"] = problems.make_problem(ms_rows, n, CFG["kappa"], CFG["resnorm"], 1)
    P = _SAMPLE_CACHE["P"]
    A, b = P["A"], P["b"]
    t0 = time.perf_counter()
    oracle.sketch(A, b, d, zeta, 0)
    t_sk = time.perf_counter() - t0
    Bq = oracle.sketch(A, b, dq, zeta, 0)
    t0 = time.perf_counter()
    R, x0, ne, ce, rc = oracle.factor(Bq, 0)
    t_qr = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.iterate(A, b, R, x0, 2, ne, ce, use_stop=False)
    t_it = (time.perf_counter() - t0) / 2
    if iters_hint is None:
        if "iters" not in _SAMPLE_CACHE:
            Ps = problems.make_problem(20000, 100, CFG["kappa"], CFG["resnorm"], 2)
            _, info = oracle.solve(Ps["A"], Ps["b"], 2000, zeta, CFG["q"], 0, extra=EXTRA_ITERS)
            _SAMPLE_CACHE["iters"] = info["iters"] + 1
        iters = _SAMPLE_CACHE["iters"]
        how = "oracle count on m=20000, n=100"
    else:
        iters = iters_hint + 1
        how = "GPU run's count"
    scale_m = m / ms_rows
    est = t_sk * scale_m + t_qr * (d / dq) + t_it * scale_m * iters
    desc = (f"oracle on a bounded sample: sketch of {ms_rows} rows (x{scale_m:.0f}), QR of a {dq}x{n + 1} "
            f"sketch (x{d / dq:.0f}), 2 passes over {ms_rows} rows (x{scale_m:.0f} x {iters} passes, {how})")
    return est, time.perf_counter() - w0, desc, {"t_sketch_s": t_sk, "t_qr_s": t_qr, "t_pass_s": t_it,
                                                   "passes": iters}


def _one_thread():
    """Pool initializer: one BLAS / OpenMP thread per worker process (the
    workers run one per core; numpy's QR in the input generator would
    otherwise start a thread per core in every worker)."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_sample_worker(iters_hint):
    est, wall, _, _ = _oracle_sample(iters_hint)
    return est, wall


def cpu_baseline(iters_hint: int | None):
    """Time the oracle (plain single-threaded C, as it stands) on a bounded
    sample of the workload and scale it to seconds per full solve, on one core
    and then on every core of this host (one independent sample per core, all
    at once, in spawned processes; the throughput is the sum of their rates).
    Returns a cpu_baseline dict: value = all-core solves/s, cores = the
    processes used, one_core = the single-core figures."""
    import multiprocessing as mp

    est1, wall1, desc, det = _oracle_sample(iters_hint)
    cores = len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores, initializer=_one_thread) as pool:
        res = pool.map(_oracle_sample_worker, [iters_hint] * cores)
    wall_all = time.perf_counter() - t0
    rate_all = sum(1.0 / e for e, _ in res)
    return {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": desc + f"; estimated {est1:.1f} s per solve on one core; the all-core value runs "
                             f"{cores} such samples at once and sums their rates",
            "one_core": {"value": 1.0 / est1, "est_s_per_solve": est1, "sample_wall_s": wall1, **det},
            "all_cores": {"value": rate_all, "est_s_per_solve_median": statistics.median(e for e, _ in res),
                          "wall_s": wall_all}}


# --------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the damping / momentum timings")
    ap.add_argument("--check-qr", action="store_true",
                    help="also the forward error of LAPACK's Householder QR on the host (slow)")
    ap.add_argument("--no-qr-check", action="store_true", help="skip the device Householder-QR forward error")
    ap.add_argument("--no-small", action="store_true", help="skip the small-configuration line")
    ap.add_argument("--count", type=int, default=None, help="problems for --case batched / serve")
    ap.add_argument("--q", type=int, default=None, help="iterations for --case batched (stopping rule off)")
    ap.add_argument("--case", choices=["solve", "pass", "sketch", "factor", "batched", "serve"], default="solve",
                    help="pass / sketch: only the fused residual/gradient pass, or only the sketch B = S[A b], "
                         "on an m x 1000 problem (for ncu captures)")
    ap.add_argument("--m", type=int, default=200_000, help="rows for --case pass")
    ap.add_argument("--n", type=int, default=1000, help="columns for --case pass")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched uneven-problems timing")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (continuous batching) sweep")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    ap.add_argument("--no-sparse", action="store_true", help="skip the sparse-A workload")
    ap.add_argument("--rates", action="store_true",
                    help="only the instruction-rate probe (librates.so): sustained thread-ops per SM clock of the "
                         "FP64 / FP32 / integer forms the fused pass can be built from")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, world, rank)
    if args.rates:
        return rates_case()
    if args.case == "pass":
        return pass_case(args)
    if args.case == "factor":
        return factor_case(args)
    if args.case == "sketch":
        return sketch_case(args)
    if args.case == "batched":
        return batched_profile_case(args)
    if args.case == "serve":
        return serve_profile_case(args)

    import numpy as np
    import torch

    import paper_2311_04362_gb300 as ls
    import problems

    torch.cuda.set_device(local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        pg = dist

    def barrier():
        if pg:
            pg.barrier()

    from paper_2311_04362_gb300 import build
    build.build()
    m, n, d, zeta, seed, q = CFG["m"], CFG["n"], CFG["d"], CFG["zeta"], CFG["seed"], CFG["q"]
    P = problems.make_problem_torch(m, n, CFG["kappa"], CFG["resnorm"], CFG["seed"] + rank, device="cuda")
    A, b, xtrue = P["A"], P["b"], P["x"]
    stream = torch.cuda.current_stream()
    ctx = ls.Context(local_rank, stream)
    x = torch.empty(n, dtype=torch.float64, device="cuda")

    for _ in range(args.warmup):
        ctx.ls_solve(A, b, m, n, n, d, zeta, q, seed, x)
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        st, info = ctx.ls_solve(A, b, m, n, n, d, zeta, q, seed, x)
        infos.append((st, ls.ls_info.from_buffer_copy(info)))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
    value = job_throughput(world, args.steps, ms_max)

    fe = float(torch.linalg.norm(x - xtrue) / torch.linalg.norm(xtrue))
    statuses = sorted({ls.STATUS_NAMES[s] for s, _ in infos})
    iters = [i.iters for _, i in infos]
    pass_ms = sum(i.ms_pass for _, i in infos) / max(1, sum(i.n_pass for _, i in infos))
    launches = sum(i.launches for _, i in infos)
    alg_bytes = 8.0 * m * (n + 3)       # A once, b, r_prev read, r written
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    if not hbm_peak:
        hbm_peak, peak_src = HBM_FALLBACK_GBS, "profiling recipe fallback 6.8 TB/s (of fallback)"
    achieved_gbs = alg_bytes / (pass_ms / 1e3) / 1e9
    khash = kernel_source_hash()
    traffic = NCU_TRAFFIC.get(khash)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A)
        bh = torch.empty(m, dtype=torch.float64, pin_memory=True)
        bh.copy_(b)
        xh = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ctx.ls_solve(Ah, bh, m, n, n, d, zeta, q, seed, xh)    # warm the staging buffer
        k2 = args.e2e_steps or max(1, args.steps // 2)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k2):
            _, einfo = ctx.ls_solve(Ah, bh, m, n, n, d, zeta, q, seed, xh)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms2 = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
        # context: the same bytes copied by torch alone (one copy from the pinned buffer)
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        A.copy_(Ah, non_blocking=True)
        u1.record(stream)
        torch.cuda.synchronize()
        upload_ms = u0.elapsed_time(u1)
        e2e = {"value": job_throughput(world, k2, ms2), "unit": UNIT, "ms_per_solve": ms2 / k2,
               "phase_ms": {"sketch_incl_upload_wait": einfo.ms_sketch, "factor": einfo.ms_factor,
                            "iterate": einfo.ms_iterate},
               "torch_upload_ms": upload_ms,
               "h2d_bytes_per_step": 8 * m * n + 8 * m, "d2h_bytes_per_step": 8 * n, "steps": k2,
               "fe": float(np.linalg.norm(xh.numpy() - xtrue.cpu().numpy()) / np.linalg.norm(xtrue.cpu().numpy()))}
        del Ah, bh

    # App. B variants on the same problem (reported beside the Algorithm 2 headline)
    variants = {}
    if not args.no_variants:
        for vname, vopts in (("damping", ls.damping_opts(n, d)), ("momentum", ls.momentum_opts(n, d))):
            xv = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.ls_solve_ex(A, b, m, n, n, d, zeta, q, seed, vopts, xv)   # warm
            barrier()
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            vinfo = None
            for _ in range(args.steps):
                st_v, vinfo = ctx.ls_solve_ex(A, b, m, n, n, d, zeta, q, seed, vopts, xv)
            v1.record(stream)
            torch.cuda.synchronize()
            vms = max_over_ranks(v0.elapsed_time(v1), pg, "cuda")
            variants[vname] = {"value": job_throughput(world, args.steps, vms), "unit": UNIT,
                               "iters": vinfo.iters, "alpha": vopts.alpha, "beta": vopts.beta,
                               "fe": float(torch.linalg.norm(xv - xtrue) / torch.linalg.norm(xtrue)),
                               "status": ls.STATUS_NAMES[st_v]}

    batched = None
    if not args.no_batched:
        batched = batched_case(ctx, stream, args, pg, world, rank)

    serving = None
    if not args.no_serving:
        serving = serving_case(ctx, args)

    mixed = None
    if not args.no_mixed:
        mixed = mixed_case(ctx, stream, args, pg, world)

    sparse = None
    if not args.no_sparse:
        sparse = sparse_case(ctx, stream, args, pg, world)

    # the forward-error rule on the headline problem, outside the timed region:
    # a Householder-QR solve of the same A, b on the device (LAPACK-style gels)
    acc_qr = {}
    if rank == 0 and not args.no_qr_check:
        t0 = time.perf_counter()
        xq = householder_tsqr_solve(A, b)
        fq = float(torch.linalg.norm(xq - xtrue) / torch.linalg.norm(xtrue))
        acc_qr = {"fe_qr": fq, "fe_over_qr": fe / fq, "qr": "Householder QR of the same A on the device "
                  "(torch.linalg.qr, tall-skinny: 500,000-row blocks, then the stacked R factors)",
                  "qr_seconds": time.perf_counter() - t0}
        del xq
        torch.cuda.empty_cache()
    if args.check_qr and rank == 0:
        import oracle
        t0 = time.perf_counter()
        xq = oracle.qr_solve_lapack(A.cpu().numpy(), b.cpu().numpy())
        acc_qr["fe_qr_lapack_host"] = oracle.forward_error(xq, xtrue.cpu().numpy())
        acc_qr["lapack_seconds"] = time.perf_counter() - t0

    small = None
    if rank == 0 and world == 1 and not args.no_small:
        small = small_case(ctx, stream, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(int(statistics.median(iters)))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(world),
            "roofline": {"bound": "hbm", "kernel": "k_fx_pass", "achieved": achieved_gbs, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved_gbs / hbm_peak, "peak_source": peak_src,
                         "traffic": traffic, "algorithmic_bytes": alg_bytes,
                         "algorithmic_bytes_rule": "8 m (n + 3): A once, b, r_prev read, r written",
                         "pass_ms": pass_ms, "kernel_source_hash": khash},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "accuracy": {"fe": fe, "status": statuses, "iters": iters, **acc_qr},
            "small_config": small,
            "variants_app_b": variants,
            "batched": batched,
            "serving": serving,
            "mixed_precision": mixed,
            "sparse": sparse,
            "phase_ms": {"sketch": statistics.mean(i.ms_sketch for _, i in infos),
                         "factor": statistics.mean(i.ms_factor for _, i in infos),
                         "iterate": statistics.mean(i.ms_iterate for _, i in infos)},
            "latency_ms": {"p50": statistics.median([i.ms_sketch + i.ms_factor + i.ms_iterate for _, i in infos]),
                           "max": max(i.ms_sketch + i.ms_factor + i.ms_iterate for _, i in infos)},
        }
        print(json.dumps(line))
    ctx.close()
    if pg:
        pg.destroy_process_group()


def householder_tsqr_solve(A, b, block: int = 500_000):
    """x = argmin ||b - A y|| by Householder QR on the device, as a
    tall-skinny QR: each block of rows is factored (torch.linalg.qr, LAPACK-
    style Householder through cuSOLVER, whose 32-bit sizes limit one call to
    2^31 entries), the R factors are stacked and factored again, and Q^T b is
    carried along.  Backward stable like one Householder QR of A."""
    import torch

    m, n = A.shape
    Rs, zs = [], []
    for r0 in range(0, m, block):
        Q, R = torch.linalg.qr(A[r0:r0 + block], mode="reduced")
        zs.append(Q.T @ b[r0:r0 + block])
        Rs.append(R)
        del Q
    Q2, R2 = torch.linalg.qr(torch.cat(Rs, 0), mode="reduced")
    z = Q2.T @ torch.cat(zs, 0)
    return torch.linalg.solve_triangular(R2, z.unsqueeze(1), upper=True)[:, 0]


def _oracle_small_solve_worker(_):
    import oracle
    import problems
    c = problems.SMALL
    P = problems.make_problem(c["m"], c["n"], c["kappa"], c["resnorm"], c["seed"])
    t0 = time.perf_counter()
    oracle.solve(P["A"], P["b"], c["d"], c["zeta"], c["q"], c["seed"], extra=EXTRA_ITERS)
    return time.perf_counter() - t0


def small_case(ctx, stream, args):
    """The small configuration (m = 4000, n = 50, kappa = 1e10, ||r|| = 1e-6,
    d = 20 n, zeta = 8, seed 0): GPU solves/s through ls_solve (device
    inputs, CUDA events over `steps` solves) beside the oracle's whole solve,
    fully timed -- on one core, and on every core at once (one solve per core,
    spawned processes; rates summed)."""
    import multiprocessing as mp

    import numpy as np
    import torch

    import oracle
    import problems

    c = problems.SMALL
    m, n, d = c["m"], c["n"], c["d"]
    P = problems.make_problem(m, n, c["kappa"], c["resnorm"], c["seed"])
    A, b = torch.from_numpy(P["A"]).cuda(), torch.from_numpy(P["b"]).cuda()
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.ls_solve(A, b, m, n, n, d, c["zeta"], c["q"], c["seed"], x)
    steps = max(10, 4 * args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        st, info = ctx.ls_solve(A, b, m, n, n, d, c["zeta"], c["q"], c["seed"], x)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fe = oracle.forward_error(x.cpu().numpy(), P["x"])
    fe_qr = oracle.forward_error(oracle.qr_solve(P["A"], P["b"]), P["x"])
    t0 = time.perf_counter()
    xo, io = oracle.solve(P["A"], P["b"], d, c["zeta"], c["q"], c["seed"], extra=EXTRA_ITERS)
    t_or = time.perf_counter() - t0
    # throughput: the same problem as `copies` members of one ls_solve_batched
    # call (embedding seed = member index; A and b shared, x per member)
    copies = 2048
    xs_b = torch.empty((copies, n), dtype=torch.float64, device="cuda")
    members = [dict(A=A, b=b, x=xs_b[i], m=m, n=n, lda=n, d=d, seed=i) for i in range(copies)]
    ctx.ls_solve_batched(members, c["zeta"], c["q"])
    bsteps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(bsteps):
        binf = ctx.ls_solve_batched(members, c["zeta"], c["q"])
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / bsteps
    fe_b = [oracle.forward_error(xs_b[i].cpu().numpy(), P["x"]) for i in range(0, copies, copies // 16)]
    batched = {"copies": copies, "value": copies * 1e3 / bms, "unit": UNIT, "ms_per_call": bms,
               "iters_mean": float(np.mean([binf[i].iters for i in range(copies)])),
               "fe_over_qr_max_of_16": max(fe_b) / fe_qr,
               "kind": "one ls_solve_batched call of the problem repeated, embedding seeds 0..copies-1"}
    cores = len(os.sched_getaffinity(0))
    with mp.get_context("spawn").Pool(cores, initializer=_one_thread) as pool:
        ts = pool.map(_oracle_small_solve_worker, range(cores))
    return {"workload": "small single FP64 problem: m=4000, n=50, kappa=1e10, ||r||=1e-6, d=20n=1000, zeta=8, "
                        "seed 0, q<=100",
            "batched": batched,
            "value": 1e3 / ms, "unit": UNIT, "ms_per_solve": ms, "iters": info.iters, "fe": fe, "fe_qr": fe_qr,
            "phase_ms": {"sketch": info.ms_sketch, "factor": info.ms_factor, "iterate": info.ms_iterate},
            "launches": info.launches,
            "fe_over_qr": fe / fe_qr,
            "oracle": {"value": 1.0 / t_or, "unit": UNIT, "seconds_per_solve": t_or, "cores": 1,
                       "iters": io["iters"], "fe": oracle.forward_error(xo, P["x"]), "kind": "oracle, fully timed"},
            "oracle_all_cores": {"value": sum(1.0 / t for t in ts), "unit": UNIT, "cores": cores,
                                 "kind": "oracle, one fully timed solve per core at once"}}


def rates_case():
    """Instruction-rate probe: one JSON line with, per instruction form, the
    sustained rate in thread-operations per SM clock and per ns on the GPU."""
    import ctypes

    import torch

    from paper_2311_04362_gb300 import build
    build.build()
    torch.cuda.init()
    L = ctypes.CDLL(build.RATES_LIB)
    L.ls_probe_rates.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
    buf = ctypes.create_string_buffer(8192)
    rc = L.ls_probe_rates(buf, len(buf), 4096)
    out = json.loads(buf.value.decode())
    out["rc"] = rc
    out["device"] = torch.cuda.get_device_name(0)
    print(json.dumps(out))
    return rc


def batched_case(ctx, stream, args, pg, world, rank):
    """4096 independent uneven problems (problems.BATCH) solved by one
    ls_solve_batched call per step; solves/s over the whole batch, timed with
    CUDA events on the launching stream.  Acceptance: the fraction of problems
    whose forward error is within 10x that of a Householder-QR solve (geqrf
    through torch) -- Algorithm 2 as stated and with the App. B momentum
    weights (e = sqrt(n/d) = sqrt(1/20) for every problem).  The basic
    method is timed with the default pass tiles and after ls_tune_batched
    (whose time and table are reported); momentum with the tuned table."""
    import torch

    import paper_2311_04362_gb300 as ls
    import problems

    cfg = problems.BATCH
    shapes = problems.batch_shapes(**cfg)
    probs = problems.make_batch_torch(shapes)
    nprob = len(probs)
    fe_qr = []
    for p in probs:
        n = p["n"]
        Q, R = torch.linalg.qr(p["A"][:, :n])
        xq = torch.linalg.solve_triangular(R, (Q.T @ p["b"])[:, None], upper=True)[:, 0]
        fe_qr.append(float(torch.linalg.norm(xq - p["x_true"]) / torch.linalg.norm(p["x_true"])))
        del Q, R
    out = {"workload": "4096 uneven FP64 problems: m log-uniform in [500, 20000], n log-uniform in [10, 200], "
                       "m >= 20n, kappa log-uniform in [1e2, 1e12], ||r|| log-uniform in [1e-10, 1e-2], d = 20n, "
                       "zeta = 8, Philox seed = problem index, q <= 100 with the Sec. 3.3 stopping rule",
           "problems": nprob, "sum_m": int(sum(s["m"] for s in shapes)),
           "A_bytes": int(sum(8 * p["m"] * p["lda"] for p in probs))}
    steps = max(1, args.steps // 2)
    runs = [("basic_default_tiles", ls.default_opts(), False), ("basic", ls.default_opts(), True),
            ("momentum", ls.momentum_opts(1, 20), True)]
    for name, opts, tuned in runs:
        if tuned and "tuning" not in out:
            t0 = time.perf_counter()
            report = ctx.ls_tune_batched(probs, reps=2)
            out["tuning"] = {"seconds": time.perf_counter() - t0, "table": report.strip().splitlines()}
        ctx.ls_solve_batched(probs, cfg["zeta"], cfg["q"], opts)      # warm
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            infos = ctx.ls_solve_batched(probs, cfg["zeta"], cfg["q"], opts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
        fe = [float(torch.linalg.norm(p["x"] - p["x_true"]) / torch.linalg.norm(p["x_true"])) for p in probs]
        ok = sum(1 for a, q_ in zip(fe, fe_qr) if a <= 10 * q_)
        held = sum(1 for i in infos if i.stop_reason == 0)
        its = [i.iters for i in infos]
        out[name] = {"value": job_throughput(world, steps * nprob, ms), "unit": UNIT,
                     "ms_per_batch": ms / steps, "steps": steps, "alpha": opts.alpha, "beta": opts.beta,
                     "accept_10x_qr": ok / nprob, "rule_held": held / nprob,
                     "iters_mean": sum(its) / nprob, "iters_max": max(its),
                     "phase_ms": {"sketch": infos[0].ms_sketch, "factor": infos[0].ms_factor,
                                  "iterate": infos[0].ms_iterate},
                     "gpu_launches_per_batch": infos[0].launches}
    ctx.ls_reset_tuning()
    del probs
    torch.cuda.empty_cache()
    return out


def serving_case(ctx, args):
    """Continuous batching (ls_server_*): Poisson arrival streams at each rate
    of problems.SERVE, requests drawn from a pool of problems resident in HBM,
    admission within a 150 GB budget (each request counts its A, b, x and
    workspace).  Per rate: completed solves/s over the span from the first
    arrival to the last completion, p50/p99 latency from arrival (host clock)
    to the poll that returned the request, and the fraction of requests whose
    forward error is within 10x that of a Householder-QR solve of their
    problem."""
    import numpy as np
    import torch

    import paper_2311_04362_gb300 as ls
    import problems

    cfg = problems.SERVE
    shapes = problems.batch_shapes(**cfg)
    pool = problems.make_batch_torch(shapes)
    fe_qr = []
    for p in pool:
        n = p["n"]
        Q, R = torch.linalg.qr(p["A"][:, :n])
        xq = torch.linalg.solve_triangular(R, (Q.T @ p["b"])[:, None], upper=True)[:, 0]
        fe_qr.append(float(torch.linalg.norm(xq - p["x_true"]) / torch.linalg.norm(p["x_true"])))
        del Q, R
    torch.cuda.synchronize()
    nreq = cfg["requests_per_rate"]
    xbuf = torch.empty((nreq, max(p["n"] for p in pool)), dtype=torch.float64, device="cuda")
    srv = ls.Server(ctx, 2048, 512, 48 * 2**30, cfg["budget_bytes"], cfg["zeta"], cfg["q"])
    out = {"workload": "Poisson arrivals of FP64 requests drawn from a pool of 96 problems: n log-uniform in "
                       "[20, 500], m log-uniform in [max(1000, 20n), 5e5], kappa log-uniform in [1e2, 1e10], "
                       "||r|| log-uniform in [1e-8, 1e-2], d = 20n, zeta = 8, q <= 100; 150 GB admission budget",
           "pool_A_bytes": int(sum(8 * p["m"] * p["lda"] for p in pool)), "rates": []}
    try:
        for rate in cfg["rates"]:
            arr = problems.poisson_arrivals(rate, nreq, cfg["seed"])
            rng = np.random.default_rng(np.random.SeedSequence([cfg["seed"], int(rate), 0x9001]))
            pick = rng.integers(0, len(pool), nreq)
            tick = {}
            done_t = {}
            infos = {}
            i = 0
            peak = 0
            steps = 0
            t0 = time.perf_counter()
            while len(done_t) < nreq:
                now = time.perf_counter() - t0
                while i < nreq and arr[i] <= now:
                    p = pool[pick[i]]
                    req = dict(p, x=xbuf[i, :p["n"]], seed=i)
                    tick[srv.ls_server_submit(req)] = i
                    i += 1
                st = srv.ls_server_get_stats()
                if st["inflight"] + st["queued"] == 0:
                    if i < nreq:
                        while time.perf_counter() - t0 < arr[i]:
                            pass
                    continue
                srv.ls_server_step()
                steps += 1
                peak = max(peak, st["inflight"])
                tnow = time.perf_counter() - t0
                for t, info in srv.ls_server_poll():
                    done_t[tick[t]] = tnow
                    infos[tick[t]] = info
            lat = np.array([done_t[k] - arr[k] for k in range(nreq)]) * 1e3
            span = max(done_t.values()) - arr[0]
            ok = 0
            for k in range(nreq):
                p = pool[pick[k]]
                fe = float(torch.linalg.norm(xbuf[k, :p["n"]] - p["x_true"]) / torch.linalg.norm(p["x_true"]))
                ok += fe <= 10 * fe_qr[pick[k]]
            out["rates"].append({"rate": rate, "requests": nreq, "solves_per_s": nreq / span,
                                 "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                 "accept_10x_qr": ok / nreq,
                                 "rule_held": sum(1 for v in infos.values() if v.stop_reason == 0) / nreq,
                                 "peak_inflight": peak, "steps": steps})
    finally:
        srv.close()
    del pool, xbuf
    torch.cuda.empty_cache()
    return out


def mixed_case(ctx, stream, args, pg, world):
    """FP32 sketch and QR (ls_solve_batched_mixed) against all-FP64 on the
    mixed-precision problem (problems.MIXED): solves/s, iterations, forward
    error against a Householder-QR solve (geqrf through torch), and the error
    of each FP32 stage against the FP64 one (relative Frobenius norms)."""
    import torch

    import paper_2311_04362_gb300 as ls
    import problems

    cfg = problems.MIXED
    m, n, d = cfg["m"], cfg["n"], cfg["d"]
    P = problems.make_problem_torch(m, n, cfg["kappa"], cfg["resnorm"], cfg["seed"] + 7, device="cuda")
    xt = P["x"]
    Q, R = torch.linalg.qr(P["A"])
    xq = torch.linalg.solve_triangular(R, (Q.T @ P["b"])[:, None], upper=True)[:, 0]
    fe_qr = float(torch.linalg.norm(xq - xt) / torch.linalg.norm(xt))
    del Q, R
    out = {"workload": f"m=1,000,000, n=200, kappa=1e4, ||r||=1e-3, d=4000, zeta=8, data seed {cfg['seed'] + 7}, "
                       f"embedding seed {cfg['seed']}, q <= 100",
           "fe_qr": fe_qr}
    stages = {}
    steps = max(1, args.steps)
    for name, mixed in (("fp64", False), ("mixed", True)):
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        Bo = torch.empty(d * (n + 1), dtype=torch.float64, device="cuda")
        Ro = torch.empty(n * n, dtype=torch.float64, device="cuda")
        prob = dict(A=P["A"], b=P["b"], x=x, m=m, n=n, lda=n, d=d, seed=cfg["seed"], B_out=Bo, R_out=Ro)
        ctx.ls_solve_batched([prob], cfg["zeta"], cfg["q"], mixed=mixed)       # warm, and the stage outputs
        stages[name] = (Bo, Ro)
        run = dict(prob, B_out=None, R_out=None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            inf = ctx.ls_solve_batched([run], cfg["zeta"], cfg["q"], mixed=mixed)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
        fe = float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt))
        out[name] = {"value": job_throughput(world, steps, ms), "unit": UNIT, "iters": inf.iters,
                     "stop_reason": inf.stop_reason, "fe": fe, "fe_over_qr": fe / fe_qr,
                     "phase_ms": {"sketch": inf.ms_sketch, "factor": inf.ms_factor, "iterate": inf.ms_iterate}}
    # the single-problem FP64 path (multi-CTA QR, TMA-fed pass) on the same problem
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.ls_solve(P["A"], P["b"], m, n, n, d, cfg["zeta"], cfg["q"], cfg["seed"], x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st, inf = ctx.ls_solve(P["A"], P["b"], m, n, n, d, cfg["zeta"], cfg["q"], cfg["seed"], x)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
    fe = float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt))
    out["fp64_single_path"] = {"value": job_throughput(world, steps, ms), "unit": UNIT, "iters": inf.iters,
                               "fe": fe, "fe_over_qr": fe / fe_qr,
                               "phase_ms": {"sketch": inf.ms_sketch, "factor": inf.ms_factor,
                                            "iterate": inf.ms_iterate}}
    B64, R64 = stages["fp64"]
    B32, R32 = stages["mixed"]
    R64m, R32m = R64.view(n, n), R32.view(n, n)          # column-major n x n: rows of the view are columns
    sgn = torch.sign(torch.diagonal(R64m)) * torch.sign(torch.diagonal(R32m))
    out["stage_error"] = {
        "sketch_rel_fro": float(torch.linalg.norm(B32 - B64) / torch.linalg.norm(B64)),
        "R_rel_fro": float(torch.linalg.norm(R32m * sgn[None, :] - R64m) / torch.linalg.norm(R64m)),
    }
    return out


def batched_profile_case(args):
    """One ls_solve_batched call on problems.BATCH (--count problems, default
    4096) with the stopping rule off for --q iterations (default 3): a fixed
    amount of work per kernel, for launch lists and ncu captures."""
    import torch

    import paper_2311_04362_gb300 as ls
    import problems
    from paper_2311_04362_gb300 import build

    build.build()
    cfg = dict(problems.BATCH, count=args.count or problems.BATCH["count"])
    probs = problems.make_batch_torch(problems.batch_shapes(**cfg))
    o = ls.default_opts()
    o.use_stop = 0
    with ls.Context(0, torch.cuda.current_stream()) as ctx:
        infos = ctx.ls_solve_batched(probs, cfg["zeta"], args.q or 3, o)
        torch.cuda.synchronize()
    print(json.dumps({"case": "batched", "problems": len(probs), "q": args.q or 3, "ms_sketch": infos[0].ms_sketch,
                      "ms_factor": infos[0].ms_factor, "ms_iterate": infos[0].ms_iterate,
                      "launches": infos[0].launches}))


def serve_profile_case(args):
    """--count problems of problems.SERVE (default 48) submitted at once to a
    server, stepped until all finish: one admission batch, then the
    iteration steps.  Prints the step times (host clock)."""
    import numpy as np
    import torch

    import paper_2311_04362_gb300 as ls
    import problems
    from paper_2311_04362_gb300 import build

    build.build()
    cfg = dict(problems.SERVE, count=args.count or 48)
    pool = problems.make_batch_torch(problems.batch_shapes(**cfg))
    torch.cuda.synchronize()
    with ls.Context(0, torch.cuda.current_stream()) as ctx:
        srv = ls.Server(ctx, 1024, 512, 16 * 2**30, cfg["budget_bytes"], cfg["zeta"], cfg["q"])
        t0 = time.perf_counter()
        for p in pool:
            srv.ls_server_submit(p)
        done, steps = 0, []
        while done < len(pool):
            a = time.perf_counter()
            srv.ls_server_step()
            steps.append(time.perf_counter() - a)
            done += len(srv.ls_server_poll())
        total = time.perf_counter() - t0
        srv.close()
    print(json.dumps({"case": "serve", "requests": len(pool), "total_s": total, "steps": len(steps),
                      "first_step_ms": 1e3 * steps[0], "median_step_ms": 1e3 * float(np.median(steps))}))


def sparse_case(ctx, stream, args, pg, world):
    """The sparse workload of Sec. 3.5 (problems.SPARSE: m = 3e6, 3 nonzeros
    per row, n = 500, d = 30 n) through ls_solve_sparse: solves/s, phases,
    and the distance to a Householder-QR solution of the densified matrix
    (geqrf through torch)."""
    import torch

    import paper_2311_04362_gb300 as ls
    import problems

    cfg = problems.SPARSE
    m, n = cfg["m"], cfg["n"]
    d = cfg["d_over_n"] * n
    S = problems.make_sparse(m, n, cfg["seed"], cfg["nnz_per_row"])
    rp, col, val, b = (torch.from_numpy(S[k]).cuda() for k in ("row_ptr", "col", "val", "b"))
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.ls_solve_sparse(rp, col, val, m, n, S["nnz"], b, d, cfg["zeta"], cfg["q"], cfg["seed"], x)   # warm
    torch.cuda.synchronize()
    steps = max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st, inf = ctx.ls_solve_sparse(rp, col, val, m, n, S["nnz"], b, d, cfg["zeta"], cfg["q"], cfg["seed"], x)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, "cuda")
    A = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    rows = torch.repeat_interleave(torch.arange(m, device="cuda"), torch.diff(rp))
    A[rows, col.long()] = val
    t0 = time.perf_counter()
    Q, R = torch.linalg.qr(A)
    xq = torch.linalg.solve_triangular(R, (Q.T @ b)[:, None], upper=True)[:, 0]
    torch.cuda.synchronize()
    tq = time.perf_counter() - t0
    rel = float(torch.linalg.norm(x - xq) / torch.linalg.norm(xq))
    del A, Q, R
    torch.cuda.empty_cache()
    return {"workload": "m=3,000,000, 3 nonzeros per row in random columns, values +-1, Gaussian b, n=500, "
                        "d=30n=15000, zeta=8, seed 0, q <= 100",
            "value": job_throughput(world, steps, ms), "unit": UNIT, "iters": inf.iters,
            "stop_reason": inf.stop_reason, "rel_diff_to_qr": rel,
            "phase_ms": {"sketch": inf.ms_sketch, "factor": inf.ms_factor, "iterate": inf.ms_iterate},
            "dense_qr_solve_s": tq}


def pass_case(args):
    """Fused residual/gradient passes on an m x n row-major A (default
    m = 200,000, n = 1000: 1.6 GB, larger than L2; n even) inside ls_iterate
    (R = s I, a stable Richardson step, stopping rule off).  Each pass is
    timed by CUDA events on its stream inside the library.  Used for
    small-case ncu captures of k_fused_pass."""
    import torch

    import paper_2311_04362_gb300 as ls
    from paper_2311_04362_gb300 import build

    build.build()
    m, n = args.m, args.n
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    A = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)
    b = torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    R = torch.eye(n, dtype=torch.float64, device="cuda") * (m ** 0.5 + n ** 0.5 + 1.0)
    stream = torch.cuda.current_stream()
    opts = ls.default_opts()
    opts.use_stop = 0
    with ls.Context(0, stream) as ctx:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = ls.ls_info()
        info.normest, info.condest = 1.0, 1.0
        ctx.ls_iterate(A, m, n, n, b, R, n, x, args.warmup + args.steps, opts, info)
    ms = info.ms_pass / max(1, info.n_pass)
    print(json.dumps({"case": "fused pass in ls_iterate", "m": m, "n": n, "ms_per_pass": ms, "passes": info.n_pass,
                      "tflops": 4.0 * m * n / (ms / 1e3) / 1e12, "gbs": 8.0 * m * (n + 3) / (ms / 1e3) / 1e9}))


def sketch_case(args):
    """The sketch B = S [A b] alone (ls_sketch) on an m x 1000 row-major A
    (default m = 200,000: 1.6 GB) with d = 20,000, zeta = 8, timed with CUDA
    events on the launching stream.  Used for small-case ncu captures."""
    import torch

    import paper_2311_04362_gb300 as ls
    from paper_2311_04362_gb300 import build

    build.build()
    m, n, d, zeta = args.m, 1000, 20_000, 8
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    A = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)
    b = torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    B = torch.empty((n + 1) * d, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    with ls.Context(0, stream) as ctx:
        for _ in range(args.warmup):
            ctx.ls_sketch(A, m, n, n, b, d, zeta, 0, B, d)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.ls_sketch(A, m, n, n, b, d, zeta, 0, B, d)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": "sketch", "m": m, "n": n, "d": d, "zeta": zeta, "ms_per_call": ms,
                      "alg_gbs": (8.0 * m * (n + 1) + 8.0 * d * (n + 1)) / (ms / 1e3) / 1e9}))


def factor_case(args):
    """The factor step alone (ls_factor: Householder QR, start x0, estimates)
    on a d x (n + 1) column-major matrix of the large workload's sketch shape
    (d = 20,000, n = --n, default 1000: 160 MB), timed with CUDA events on the
    launching stream; B is restored from a copy before each call (the copy is
    outside the timed interval).  Used for small-case ncu captures of the QR."""
    import torch

    import paper_2311_04362_gb300 as ls
    from paper_2311_04362_gb300 import build

    build.build()
    n = args.n
    d = 20 * n
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    B0 = torch.randn((n + 1) * d, dtype=torch.float64, device="cuda", generator=g)
    B = torch.empty_like(B0)
    R = torch.empty(n * n, dtype=torch.float64, device="cuda")
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    times = []
    with ls.Context(0, stream) as ctx:
        for it in range(args.warmup + args.steps):
            B.copy_(B0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.ls_factor(B, d, n, d, R, n, x0, 0)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    flops = 2.0 * d * (n + 1) ** 2 - 2.0 / 3.0 * (n + 1) ** 3
    print(json.dumps({"case": "factor", "d": d, "n": n, "ms_per_call": ms, "qr_tflops": flops / (ms / 1e3) / 1e12}))


def reference_arm(args, world, rank):
    """The oracle (CPU, as it stands) on this arm's workload and config: each
    step is one bounded sample per host core, all at once (see cpu_baseline);
    the value is the summed rate in solves/s, ms_per_step the measured wall
    time of a step."""
    if rank != 0:
        return
    import multiprocessing as mp

    cores = len(os.sched_getaffinity(0))
    vals, walls = [], []
    desc, det = None, None
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_one_thread) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_sample_worker, [None] * cores)
            wall = time.perf_counter() - t0
            if i >= args.warmup:
                vals.append(sum(1.0 / e for e, _ in res))
                walls.append(wall)
    est1, _, desc, det = _oracle_sample(None)
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc + f"; {cores} samples at once per step, rates summed; one core alone: "
                                              f"{est1:.1f} s per solve", **det},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
