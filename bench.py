"""Benchmark: TNrSVD solves/s on one GB300 (or N replicas), with roofline and CPU-oracle baseline.

Workload (one step = one full TNrSVD solve: merge check, Omega, every MPO product, every
QR/rounding sweep and the final MPO-SVD): the 2^20 x 2^20 MPO with prescribed singular values
sigma_j = 0.7^j (j < 32), built as U diag(sigma) V^T from orthogonal rank-5 MPOs in the merged
layout (site dims 64, 4 x 7), k = 16, p = 16, q = 2 (the shape of the paper's Section 6.3
prescribed-sigma experiment). Synthetic, seeded inputs.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision fp64]
Under torchrun (WORLD_SIZE > 1) every rank runs an independent replica of the same workload
(a single solve does not shard); value = solves of all ranks / max time over ranks.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "TNrSVD solves/s (2^20 x 2^20 MPO, sigma_j = 0.7^j, k=16 p=16 q=2)"
DTYPES = {"mixed": "bf16x3/f64", "fp64": "f64"}
KERNELS = {
    "qr": "k_site1_cholqr2 (site-1 CholeskyQR2, one cooperative launch) / k_qr_coop (Householder fallback)",
    "qr_small": "k_qr_small / k_qr_small_tpc (one-CTA FP64 Householder QR, explicit Q)",
    "qr_piv": "k_compress (cooperative exact compression sweep: pivoted FP64 QR per bond on an 8-CTA thread-block "
              "cluster (DSMEM exchange) + grid-wide absorb, then the fused rounding sweeps / certificate on CTA 0)",
    "svd": "k_svd_step / k_jacobi (FP64 truncated SVD step, one-sided Jacobi)",
    "gemm": "k_gemm / k_gemm_tiny (FP64 GEMM)",
    "contract": "k_contract (per-site MPO product)",
}
UNIT = "solves/s"
# DRAM bytes (read + write) per launch from one ncu capture of the named kernel, as recorded in
# profiles/; reported only while that kernel is unchanged (empty: not yet re-captured).
TRAFFIC_BYTES = {"qr_piv": 2.80e6}
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 FP64 (no tensor-core boost), nominal from the platform table


C1_METRIC = "TNrSVD solves/s (4096 x 4096 MPO, d=6, I=J=4, ranks 3, k=10 p=10 q=1, plain FP64)"


def workload_config(precision="mixed", which="prescribed"):
    if which == "c1":
        c = W.c1_plain_fp64()
        cfg = {"workload": "Gaussian MPO 4096 x 4096, d=6, I=J=4, ranks 3, N(0,1)/sqrt(12), k=10 p=10 q=1, seed 0",
               "precision": "all FP64", "tol": c["tol"], "max_rank": c["max_rank"],
               "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}
        return c, cfg
    c = W.c2_prescribed()
    cfg = {
        "workload": "prescribed-sigma MPO 2^20 x 2^20 (merged sites 64,4^7; A ranks 25), k=16 p=16 q=2, seed 2",
        "precision": ("products BF16 x3 on tcgen05 / FP32 accumulate, sweeps + SVD + B in FP64"
                      if precision == "mixed" else "all FP64"),
        "tol": c["tol"],
        "max_rank": c["max_rank"],
        "l2": "flushed between timed steps (256 MiB write)",
        "parallelism": "replicas",
    }
    return c, cfg


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (their summary goes into the JSON line): TNR_BENCH_OUT, else the temp dir
        out = os.environ.get("TNR_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_bench_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def run_oracle_sample(c, budget_s):
    """Time the CPU oracle (as it stands) on the same workload: whole solves until ~budget_s."""
    from oracle import tnrsvd as ot

    n, t0 = 0, time.perf_counter()
    S = None
    while True:
        _, S, _ = ot.tnrsvd(c["A"], c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"])
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 50:
            break
    return n / el, n, el, S


def replicas_rate(total_ms, steps, world, dev, dist=None):
    """Whole-job rate of `world` independent replicas, each having run `steps` steps in its own
    `total_ms`: the slowest rank (all_reduce MAX) bounds the job. Returns (steps/s, max ms)."""
    import torch

    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return world * steps / (max_ms / 1000.0), max_ms


def reference_arm(args):
    """--impl reference: the CPU oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    c, cfg = workload_config()
    for _ in range(args.warmup):
        run_oracle_sample(c, 0.0)
    t0 = time.perf_counter()
    steps = 0
    for _ in range(args.steps):
        run_oracle_sample(c, 0.0)
        steps += 1
    el = time.perf_counter() - t0
    v = steps / el
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} whole solves of the same workload (numpy/LAPACK FP64 oracle)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batched_metric(d, ranks, ks):
    return (f"TNrSVD solves/s, batch of independent Gaussian-core MPOs (d {d[0]}-{d[1]}, I=J in {{2,4}}, "
            f"ranks {ranks[0]}-{ranks[1]}, k in {set(ks)}, p=k, q=1)")


def batched_config(n, d=None, ranks=None, ks=None, zipup=True):
    d, ranks, ks = d or BATCH_D, ranks or BATCH_RANKS, ks or BATCH_KS
    probs = W.batched_gaussian(0, n, d_range=d, rank_range=ranks, ks=ks)
    cfg = {"workload": f"{n} independent Gaussian-core MPOs, d uniform {d[0]}-{d[1]}, I=J in {{2,4}}, "
                       f"ranks uniform {ranks[0]}-{ranks[1]}, k in {set(ks)}, p=k, q=1, "
                       "max_rank=K, tol 1e-12, seed 0",
           "rounding": ("zip-up: every product rounded while it is formed, then the Alg. 5.2/5.3 sweeps"
                        if zipup else "two-sweep: full products, exact compression, Alg. 5.2/5.3 sweeps"),
           "problems": n, "l2": "flushed between timed steps (256 MiB write)"}
    return probs, cfg


# Batched workload sizes: the stated distribution. Gaussian cores do not compress, so the products
# carry R K-wide bonds (up to 2048); the zip-up rounding never forms them.
BATCH_D = (8, 20)
BATCH_RANKS = (4, 32)
BATCH_KS = (8, 16, 32)


def batched_main(args):
    """--workload batched: one step = one solve of the whole batch (persistent kernel by default).
    Under torchrun the batch is split over the ranks by greedy LPT on each problem's estimated work
    (no collective on the data path); every rank solves its share in one persistent launch, the
    singular values are gathered on rank 0 in batch order, value = problems / max time over ranks."""
    import torch
    import torch.distributed as dist

    from paper_1707_07803_gb300 import shard
    from paper_1707_07803_gb300 import tnrsvd as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    bd, br, bk = tuple(args.batch_d), tuple(args.batch_ranks), tuple(args.batch_ks)
    zipup = args.batch_rounding == "zipup"
    all_probs, cfg = batched_config(args.batch, bd, br, bk, zipup)
    costs = []
    for pr in all_probs:
        I = [c.shape[1] for c in pr["A"]]
        J = [c.shape[2] for c in pr["A"]]
        R = [1] + [c.shape[3] for c in pr["A"]]
        costs.append(shard.problem_cost(I, J, R, pr["k"], pr["p"], pr["q"], pr["max_rank"], zipup))
    parts, loads = shard.lpt_partition(costs, world)
    probs = [all_probs[i] for i in parts[rank]]
    rounding = T.TNR_ROUND_ZIPUP if zipup else T.TNR_ROUND_TWO_SWEEP
    dprobs = [dict(pr, A=T.Mpo.from_numpy(pr["A"], device=dev), rounding=rounding) for pr in probs]
    persistent = args.batch_impl == "persistent"
    if world > 1:
        cfg["parallelism"] = (f"batch split over {world} GPUs by greedy LPT on estimated work (max/mean load "
                              f"{max(loads) / (sum(loads) / world):.3f}), one process per GPU, no collective on "
                              "the data path, singular values gathered on rank 0")
    if persistent:
        plan = T.PersistentBatch(dprobs, precision=T.TNR_MIXED, autotune=True, graph=True, stream=stream)
        run = lambda: plan.launch(stream)  # noqa: E731
        pc = plan.config()
        cfg["kernel"] = (f"persistent kernel: one CTA per problem from a device work queue, grid {pc['grid']} "
                         f"({pc['ctas_per_sm']} CTAs/SM autotuned, {pc['smem_bytes'] // 1024} KB shared "
                         "memory each), one CUDA-graph launch per batch")
        cfg["precision"] = ("products of the power iteration with FP32 operands / FP32 accumulation (FP32 pipe), "
                            "roundings, QR, SVD and B in FP64")
    else:
        plan = T.BatchPlan(dprobs, workers=args.workers, precision=T.TNR_MIXED)
        run = plan.run  # noqa: E731
        cfg["workers"] = plan.workers
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        run()
    torch.cuda.synchronize()
    classes = T.stats_classes()
    T.stats_reset()
    T.stats_enable(0)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches, _ = T.stats(-1)
    if persistent:
        T.stats_reset()
        ok = plan.collect(stream, check=False) == 0  # records one launch's algorithmic FP64 flops
        fp64_flops_per_batch = T.stats_work(classes.index("batch"))
        launches_per_step = 1.0
    else:
        fp64_counted = ("gemm", "qr", "qr_small", "qr_piv")
        fp64_flops_per_batch = sum(T.stats_work(classes.index(c)) for c in fp64_counted) / max(args.steps, 1)
        launches_per_step = launches / max(args.steps, 1)
        ok = all(s == 0 for s in plan.statuses())
    # end to end through the public API: H2D of every problem's cores from pinned memory, the
    # batch, D2H of every S and of every U and V core
    host = [[torch.from_numpy(np.ascontiguousarray(np.asarray(x).reshape(-1, order="F"))).pin_memory()
             for x in pr["A"]] for pr in probs]
    h2d = sum(x.numel() * 8 for hc in host for x in hc)
    e2e_ms = 0.0
    d2h = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pr, hc in zip(dprobs, host):
            for dst, src in zip(pr["A"].cores, hc):
                dst.copy_(src, non_blocking=True)
        run()
        if persistent:
            plan.collect(stream, check=False)
        outs = []
        d2h = 0
        for i in range(plan.n):
            U, S, V = plan.outputs(i)
            outs.append(S.to("cpu", non_blocking=True))
            d2h += S.numel() * 8
            for M in (U, V):
                for kk, core in enumerate(M.cores):
                    n_el = M.R[kk] * M.I[kk] * M.J[kk] * M.R[kk + 1]
                    outs.append(core[:n_el].to("cpu", non_blocking=True))
                    d2h += n_el * 8
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    n = args.batch
    # the slowest rank bounds the job; all problems of the batch over that time
    _, max_ms = replicas_rate(total_ms, args.steps, world, dev, dist)
    value = n * args.steps / (max_ms / 1000.0)
    ms_step = max_ms / args.steps
    _, e2e_max = replicas_rate(e2e_ms, args.steps, world, dev, dist)
    S_all = shard.gather_in_order([plan.outputs(i)[1].cpu().numpy().tolist() for i in range(plan.n)], parts, rank,
                                  world, dist)
    achieved = fp64_flops_per_batch / (ms_step * 1e-3) / 1e9
    line = {
        "metric": batched_metric(bd, br, bk), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic", "config": cfg,
        "e2e": {"value": n * args.steps / (e2e_max / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "launches_per_step": launches_per_step,
        "roofline": {"kernel": ("k_batch_solve (persistent, one CTA per problem)" if persistent
                                else "whole batch (all FP64 classes together)"),
                     "bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
                     "peak_source": "FP64 nominal 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json)",
                     "frac": achieved / FP64_NOMINAL_GFLOPS, "traffic": None,
                     "note": ("algorithmic FP64 flops of the batch (products, merges, QRs, compression, "
                              "absorbs, SVD-step QRs; Jacobi sweeps and the FP32 products of mixed mode not counted) / batch time")},
        "clocks": clocks,
        "statuses_ok": bool(ok),
    }
    if rank == 0:
        line["gathered_problems"] = len(S_all)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


SPARSE_METRIC = "sparse TNrSVD solves/s (2^20 x 2^20 banded, 8 nnz/row, band 64, ten 4x4 sites; k=20 p=10 q=1)"


def sparse_main(args):
    """--workload sparse: one step = Alg. 4.1 conversion + TNrSVD through the block form."""
    import torch

    from paper_1707_07803_gb300 import tnrsvd as T

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = 1 << 20
    I = J = [4] * 10
    k, p, q, seed = 20, 10, 1, 5
    r, c, v = W.banded_coo(0, n, 8, 64)
    rd = torch.from_numpy(r).to(dev)
    cd = torch.from_numpy(c).to(dev)
    vd = torch.from_numpy(v).to(dev)
    precision = T.TNR_MIXED if args.precision == "mixed" else T.TNR_FP64
    classes = T.stats_classes()

    def step():
        R, X, digits = T.sparse_to_mpo(n, n, rd, cd, vd, I, J)
        return R, T.tnr_sparse_solve(n, n, R, X, digits, I, J, k, p, q, seed, precision=precision)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    T.stats_reset()
    T.stats_enable(sum(1 << classes.index(c) for c in ("contract", "gemm", "qr")))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(local)
    sampler.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R, (U, S, V) = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    clocks = sampler.stop()
    sp_launches, sp_ms = T.stats(classes.index("contract"))
    sp_bytes = T.stats_work(classes.index("contract"))
    fp64 = {c: (T.stats(classes.index(c)), T.stats_work(classes.index(c))) for c in ("gemm", "qr")}
    T.stats_enable(0)
    peaks = read_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    achieved = (sp_bytes / max(sp_launches, 1)) / (sp_ms / max(sp_launches, 1) * 1e-3) / 1e9 if sp_launches else 0.0
    spmm = {"kernel": "k_spmm_rows (products over the compact lists of the block form)", "bound": "hbm",
            "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "peak_source": "hbm_gbs of MEASURED_PEAKS.json" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s",
            "frac": achieved / hbm, "traffic": None,
            "launches_per_step": sp_launches / args.steps, "avg_launch_us": 1000 * sp_ms / max(sp_launches, 1),
            "share_of_step": sp_ms / max(total_ms, 1e-9),
            "note": "algorithmic bytes per product: 12 B per nonzero (index + value) + 4 B per row "
                    "pointer + 8 B per right-hand-side element read once + 8 B per output element written"}
    # the dominant class: the FP64 symmetric Grams of the tall CholeskyQR2 (GEMM class)
    (g_launches, g_ms), g_flops = fp64["gemm"]
    g_rate = g_flops / (g_ms * 1e-3) / 1e9 if g_ms > 0 else 0.0
    gram = {"kernel": "k_gram_rm + k_gemm (symmetric Grams of the 2^20 x K CholeskyQR2, FP64 GEMMs)", "class": "gemm",
            "bound": "alu", "achieved": g_rate, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
            "peak_source": "FP64 nominal 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json)",
            "frac": g_rate / FP64_NOMINAL_GFLOPS, "traffic": None,
            "launches_per_step": g_launches / args.steps, "avg_launch_us": 1000 * g_ms / max(g_launches, 1),
            "share_of_step": g_ms / max(total_ms, 1e-9),
            "note": "algorithmic FP64 flops recorded per launch (n K (K+1) per symmetric Gram, 2mnk per GEMM)"}
    line = {
        "metric": SPARSE_METRIC, "value": args.steps / (total_ms / 1000.0), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": f"banded 2^20 x 2^20, 8 nnz/row in [i-64, i+64], N(0,1), {R} blocks of 4x4; "
                               f"conversion (Alg. 4.1) + TNrSVD k={k} p={p} q={q} via the block form",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "clocks": clocks,
        "roofline": gram if g_ms >= sp_ms else spmm,
        "spmm": spmm,
    }
    print(json.dumps(line))
    return 0


CONV_METRIC = "sparse->MPO conversions/s (Alg. 4.1; 2^20 x 2^20 banded, 8 nnz/row, band 64, ten 4x4 sites)"


def conversion_main(args):
    """--workload conversion: one step = Alg. 4.1 on the device (tnr_sparse_count + tnr_sparse_fill
    into preallocated outputs; the count synchronises once to read R)."""
    import torch

    from paper_1707_07803_gb300 import tnrsvd as T

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = 1 << 20
    I = J = [4] * 10
    d = len(I)
    r, c, v = W.banded_coo(0, n, 8, 64)
    nnz = int(r.size)
    rd, cd, vd = (torch.from_numpy(x).to(dev) for x in (r, c, v))
    ws = torch.empty(max(T.tnr_sparse_workspace(n, n, nnz, I, J), 1), dtype=torch.uint8, device=dev)
    R = T.tnr_sparse_count(n, n, rd, cd, I, J, ws)
    X = torch.empty(R * 16, dtype=torch.float64, device=dev)
    digits = torch.empty(R * 2 * (d - 1), dtype=torch.uint8, device=dev)

    def step():
        Rs = T.tnr_sparse_count(n, n, rd, cd, I, J, ws)
        T.tnr_sparse_fill(n, n, rd, cd, vd, I, J, Rs, X, digits, ws)
        return Rs

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    classes = T.stats_classes()
    names = ("conv_flags", "conv_scan", "conv_fill")
    T.stats_reset()
    T.stats_enable(sum(1 << classes.index(x) for x in names))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(local)
    sampler.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    clocks = sampler.stop()
    per = {x: T.stats(classes.index(x)) for x in names}
    launches, _ = T.stats(-1)
    T.stats_enable(0)
    peaks = read_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    src = "hbm_gbs of MEASURED_PEAKS.json (measured copy)" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"
    out_bytes = R * (8.0 * I[0] * J[0] + 2.0 * (d - 1))
    # algorithmic bytes: the count pass reads row and col (16 B per nonzero); the fill pass reads
    # row, col and val (24 B per nonzero) and writes every block's values and digits once
    alg = {"conv_flags": 16.0 * nnz, "conv_fill": 24.0 * nnz + out_bytes}
    fill_l, fill_ms = per["conv_fill"]
    fill_ms_step = fill_ms / args.steps
    fill_gbs = alg["conv_fill"] / (fill_ms_step * 1e-3) / 1e9
    flags_l, flags_ms = per["conv_flags"]
    step_ms = total_ms / args.steps
    whole_gbs = (alg["conv_flags"] + alg["conv_fill"]) / (step_ms * 1e-3) / 1e9
    # end to end: H2D of the COO triplets from pinned memory, conversion, D2H of X and digits
    hr, hc, hv = (torch.from_numpy(x).pin_memory() for x in (r, c, v))
    hX = torch.empty(X.numel(), dtype=torch.float64).pin_memory()
    hD = torch.empty(digits.numel(), dtype=torch.uint8).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rd.copy_(hr, non_blocking=True)
        cd.copy_(hc, non_blocking=True)
        vd.copy_(hv, non_blocking=True)
        step()
        hX.copy_(X, non_blocking=True)
        hD.copy_(digits, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    line = {
        "metric": CONV_METRIC, "value": args.steps / (total_ms / 1000.0), "unit": "conversions/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64 (copy only)", "data": "synthetic",
        "config": {"workload": f"banded 2^20 x 2^20, 8 nnz/row in [i-64, i+64], N(0,1), int64 COO sorted, "
                               f"ten 4x4 sites; R = {R} blocks", "nnz": nnz,
                   "l2": "flushed between timed steps (256 MiB write); inputs 201 MB, outputs "
                         f"{out_bytes / 1e6:.0f} MB"},
        "e2e": {"value": args.steps / (e2e_ms / 1000.0), "unit": "conversions/s", "h2d_bytes_per_step": 24 * nnz,
                "d2h_bytes_per_step": int(X.numel() * 8 + digits.numel())},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_zero + k_fill_w (block zeroing and warp-window fill of Alg. 4.1)", "class": "conv_fill",
                     "bound": "hbm", "achieved": fill_gbs, "peak": hbm, "unit": "GB/s", "peak_source": src,
                     "frac": fill_gbs / hbm, "traffic": None, "launches_per_step": fill_l / args.steps,
                     "avg_launch_us": 1000 * fill_ms / max(fill_l, 1), "share_of_step": fill_ms / max(total_ms, 1e-9),
                     "note": "algorithmic bytes 24 B per nonzero read + R (8 I1 J1 + 2 (d-1)) B written"},
        "count_pass": {"kernel": "k_first_scan (first-occurrence flags and per-tile counts)",
                       "achieved_gbs": alg["conv_flags"] / (flags_ms / args.steps * 1e-3) / 1e9 if flags_ms else None,
                       "share_of_step": flags_ms / max(total_ms, 1e-9)},
        "whole_conversion_gbs": whole_gbs,
        "clocks": clocks,
    }
    from oracle import convert as oc  # the CPU baseline: the oracle of Alg. 4.1 as it stands

    t0 = time.perf_counter()
    k_cpu = 0
    while True:
        oc.convert(r, c, v, n, n, I, J)
        k_cpu += 1
        el = time.perf_counter() - t0
        if el > args.cpu_budget or k_cpu >= 5:
            break
    line["cpu_baseline"] = {"value": k_cpu / el, "unit": "conversions/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"{k_cpu} whole conversions of the same matrix in {el:.1f} s (numpy)"}
    print(json.dumps(line))
    return 0


PAPER_METRIC = ("TNrSVD solves/s, Section 6.3 prescribed-sigma matrix 2^15 x 2^15 (50 values 0.5^k, MPO rank 25, "
                "rank-50 approximation K=100, q=1, tol 1e-6), with the N = 10..50 sweep and the Hilbert submatrix")
PAPER_N15_SECONDS = 2.13  # the paper's TNrSVD runtime at N = 15 (MATLAB, i7-6700; other hardware, context)


def paper_main(args):
    """--workload paper: the paper's Section 6.3 workloads, one FP64 solve per step at each size."""
    import torch

    from paper_1707_07803_gb300 import tnrsvd as T

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(local)

    def timed(c, exact):
        A = T.Mpo.from_numpy(c["A"], device=dev)
        plan = T.SolvePlan(A, c["k"], c["p"], tol=c["tol"], max_rank=c["max_rank"], precision=T.TNR_FP64)
        for _ in range(max(3, args.warmup)):
            plan.run(c["q"], c["seed"])
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run(c["q"], c["seed"])
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        S = plan.S.cpu().numpy()
        return tot / args.steps, float(np.linalg.norm(S - exact) / np.linalg.norm(exact))

    sampler.start()
    sweep, hil = [], []
    for N in sorted(W.PAPER_SIGMA_TOLS):
        c = W.paper_prescribed(N)
        ms, err = timed(c, c["sigma"])
        sweep.append({"N": N, "tol": c["tol"], "ms_per_solve": ms, "solves_per_s": 1000.0 / ms,
                      "sv_rel_err_vs_exact": err})
    for N in (10, 12):
        c = W.paper_hilbert(N)
        s_true = np.linalg.svd(c["dense"], compute_uv=False)[: c["k"]]
        ms, err = timed(c, s_true)
        hil.append({"N": N, "ms_per_solve": ms, "solves_per_s": 1000.0 / ms, "sv_rel_err_vs_dense_lapack": err,
                    "mpo_ranks": [int(x.shape[3]) for x in c["A"]][:-1]})
    clocks = sampler.stop()
    n15 = next(x for x in sweep if x["N"] == 15)
    line = {
        "metric": PAPER_METRIC, "value": n15["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": n15["ms_per_solve"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": n15["solves_per_s"] * PAPER_N15_SECONDS, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "Section 6.3: A = U diag(0.5^k) V^T (k < 50), U, V orthogonal rank-5 MPOs (QR'd "
                               "Gaussian cores; the paper used TT_RAND), 2^N x 2^N with N sites of 2 x 2, first 7 "
                               "merged; k=50 p=50 q=1; rounding tolerance per N as in the paper",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "baseline_note": "vs_baseline = the paper's 2.13 s at N = 15 (MATLAB on an i7-6700) / ours"},
        "sweep": sweep, "hilbert": hil, "clocks": clocks,
    }
    print(json.dumps(line))
    return 0


ADJ_METRIC = ("gradient evaluations/s of L = sum of the top-16 TNrSVD singular values "
              "(4^12 x 4^12 MPO, rank 16, k=16 p=16 q=2, FP64 forward + adjoint)")


def adjoint_main(args):
    """--workload adjoint: one step = tnr_diff_forward + tnr_diff_backward on the d=12 workload."""
    import torch

    from paper_1707_07803_gb300 import tnrsvd as T

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    d, rank, k, p, q, seed, n_sv = 12, 16, 16, 16, 2, 3, 16
    A_host = W.gaussian_mpo(0, [4] * d, [4] * d, [1] + [rank] * (d - 1) + [1],
                            scale=lambda kk, sh: 1.0 / np.sqrt(sh[1] * sh[0]))
    A_host = [c.astype(np.float32).astype(np.float64) for c in A_host]  # FP32 Gaussian cores (values)
    A = T.Mpo.from_numpy(A_host, device=dev, dtype=np.float32)  # passed as float32 (TNR_F32)
    for c in A.cores:
        c.requires_grad_(True)

    def step():
        S = T.tnrsvd_values(A, k, p, q, seed)
        return torch.autograd.grad(S[:n_sv].sum(), A.cores)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g = step()
    e1.record(stream)
    e1.synchronize()
    total_ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    grads = [x.cpu().numpy() for x in g]
    # central differences of the GPU forward (h = 1e-6) on sampled core entries
    rng = np.random.default_rng(1)
    h = 1e-6
    got, fd = [], []
    for _ in range(args.fd_entries):
        c = int(rng.integers(0, d))
        e = int(rng.integers(0, A_host[c].size))
        vals = []
        for sgn in (1, -1):
            Ap = [x.copy() for x in A_host]
            f = Ap[c].reshape(-1, order="F")
            f[e] += sgn * h
            Ap[c] = f.reshape(A_host[c].shape, order="F")
            with torch.no_grad():
                vals.append(float(T.tnrsvd_values(T.Mpo.from_numpy(Ap, device=dev), k, p, q, seed)[:n_sv].sum()))
        fd.append((vals[0] - vals[1]) / (2 * h))
        got.append(grads[c][e])
    got, fd = np.array(got), np.array(fd)
    line = {
        "metric": ADJ_METRIC, "value": args.steps / (total_ms / 1000.0), "unit": "gradients/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"Gaussian MPO d={d}, I=J=4, rank {rank}, FP32-valued cores, k={k} p={p} q={q}, "
                               f"loss = sum of the top {n_sv} singular values",
                   "l2": "working set above L2 (products of 512-wide bonds)"},
        "clocks": clocks,
        "gradient_check": {"entries": args.fd_entries, "h": h,
                           "normwise_rel_err_vs_gpu_central_differences":
                               float(np.linalg.norm(got - fd) / max(np.linalg.norm(fd), 1e-300))},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default per workload: prescribed 200, sparse 20, batched 20, adjoint 2)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--workload", default="prescribed",
                    choices=["prescribed", "c1", "batched", "adjoint", "sparse", "conversion", "paper"],
                    help="prescribed: one 2^20 x 2^20 solve per step (default); c1: the plain FP64 4096 x 4096 "
                         "solve; batched: a batch of independent Gaussian-core MPOs per step (persistent "
                         "kernel); adjoint: forward and backward of the differentiable solve per step; sparse: "
                         "Alg. 4.1 conversion and the block-sparse TNrSVD per step; conversion: Alg. 4.1 alone; "
                         "paper: the Section 6.3 sweeps (prescribed sigma N=10..50, Hilbert N=10,12)")
    ap.add_argument("--fd-entries", type=int, default=16)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--batch-impl", default="persistent", choices=["persistent", "pool"],
                    help="batched workload: persistent kernel (default) or the host worker pool")
    ap.add_argument("--batch-d", type=int, nargs=2, default=list(BATCH_D), help="batched: range of d")
    ap.add_argument("--batch-ranks", type=int, nargs=2, default=list(BATCH_RANKS), help="batched: range of ranks")
    ap.add_argument("--batch-ks", type=int, nargs="+", default=list(BATCH_KS), help="batched: set of k")
    ap.add_argument("--batch-rounding", default="zipup", choices=["zipup", "two_sweep"],
                    help="batched: rounding of the products (zip-up by default)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"prescribed": 200, "c1": 200, "sparse": 20, "batched": 5, "adjoint": 2,
                      "conversion": 50, "paper": 5}[args.workload]
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batched":
        return batched_main(args)
    if args.workload == "adjoint":
        return adjoint_main(args)
    if args.workload == "sparse":
        return sparse_main(args)
    if args.workload == "conversion":
        return conversion_main(args)
    if args.workload == "paper":
        return paper_main(args)
    if args.workload == "c1":
        args.precision = "fp64"  # the plain FP64 configuration

    import torch
    import torch.distributed as dist

    from paper_1707_07803_gb300 import tnrsvd as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    c, cfg = workload_config(args.precision, args.workload)
    metric = C1_METRIC if args.workload == "c1" else METRIC
    A = T.Mpo.from_numpy(c["A"], device=dev, flat=True)
    precision = T.TNR_MIXED if args.precision == "mixed" else T.TNR_FP64
    plan = T.SolvePlan(A, c["k"], c["p"], tol=c["tol"], max_rank=c["max_rank"], precision=precision)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    for _ in range(max(3, args.warmup)):
        plan.run(c["q"], c["seed"])
    torch.cuda.synchronize()

    # dominant kernel class for the roofline: time every class on one warm-up solve, keep the
    # largest FP64 class (the tensor-core contraction is reported separately)
    classes = T.stats_classes()
    T.stats_reset()
    T.stats_enable((1 << len(classes)) - 1)
    plan.run(c["q"], c["seed"])
    torch.cuda.synchronize()
    per_class = {n: T.stats(i)[1] for i, n in enumerate(classes)}
    T.stats_enable(0)
    fp64_classes = [n for n in ("qr", "qr_small", "qr_piv", "svd", "gemm", "contract") if n in per_class]
    dom = max(fp64_classes, key=lambda n: per_class[n])
    qr_cls = classes.index(dom)
    tc_cls = classes.index("contract_tc")
    T.stats_reset()
    T.stats_enable((1 << qr_cls) | (1 << tc_cls))
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(c["q"], c["seed"])
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches, _ = T.stats(-1)
    qr_launches, qr_ms = T.stats(qr_cls)
    qr_flops = T.stats_work(qr_cls)
    tc_launches, tc_ms = T.stats(tc_cls)
    tc_flops = T.stats_work(tc_cls)
    T.stats_enable(0)
    value, max_ms = replicas_rate(total_ms, args.steps, world, dev, dist)

    # accuracy of this run against the exact singular values (prescribed workload)
    S = plan.S.cpu().numpy()
    sv_err = (float(np.linalg.norm(S - c["sigma"][: c["k"]]) / np.linalg.norm(c["sigma"][: c["k"]]))
              if "sigma" in c else None)

    # end to end through the public API with host buffers (SolvePlan.run_host): one H2D copy of the
    # cores from pinned memory, the solve, one D2H copy of S, U and V (the output buffer at its
    # capacities) into pinned memory
    host_in = T.Mpo.host_flat(c["A"])
    host_out = torch.empty(plan.out_flat.numel(), dtype=torch.float64).pin_memory()
    h2d = host_in.numel() * 8
    d2h = host_out.numel() * 8
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run_host(host_in, host_out, c["q"], c["seed"])
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_value, e2e_ms = replicas_rate(e2e_ms, args.steps, world, dev, dist)
    # the host copy is the result: its singular values equal the device ones
    if "sigma" in c:
        assert np.array_equal(host_out[: c["k"]].numpy(), plan.S.cpu().numpy())
    qr_avg_ms = qr_ms / max(qr_launches, 1)
    achieved_gflops = (qr_flops / max(qr_launches, 1)) / (qr_avg_ms * 1e-3) / 1e9 if qr_launches else 0.0
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic", "config": cfg,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"kernel": KERNELS.get(dom, dom), "class": dom, "bound": "alu",
                     "achieved": achieved_gflops, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
                     "peak_source": "FP64 nominal 1.25 TFLOP/s (no FP64 entry in MEASURED_PEAKS.json)",
                     "frac": achieved_gflops / FP64_NOMINAL_GFLOPS, "traffic": TRAFFIC_BYTES.get(dom),
                     "launches_per_step": qr_launches / args.steps, "avg_launch_us": 1000 * qr_avg_ms,
                     "share_of_step": qr_ms / max(total_ms, 1e-9),
                     "class_ms_one_solve": {k: round(v, 4) for k, v in per_class.items() if v > 0}},
        "contraction": ({"kernel": "k_tc_gemm_tma (TMA-staged FP64 boxes via cp.async.bulk.tensor, tcgen05 BF16 x3, FP32 accumulate in TMEM)", "bound": "tensor",
                         "launches_per_step": tc_launches / args.steps,
                         "avg_launch_us": 1000 * tc_ms / max(tc_launches, 1),
                         "achieved": (tc_flops / max(tc_launches, 1)) / (tc_ms / max(tc_launches, 1) * 1e-3) / 1e12
                         if tc_launches else 0.0,
                         "peak": read_peaks().get("bf16_tflops"), "unit": "TFLOP/s",
                         "peak_source": "bf16_tflops of MEASURED_PEAKS.json (measured burst)",
                         "share_of_step": tc_ms / max(total_ms, 1e-9)} if tc_launches else None),
        "accuracy": {"sv_rel_err_vs_exact": sv_err},
        "clocks": clocks,
    }
    if line["contraction"] and line["contraction"]["peak"]:
        line["contraction"]["frac"] = line["contraction"]["achieved"] / line["contraction"]["peak"]
    if rank == 0:
        rate, n, el, So = run_oracle_sample(c, args.cpu_budget)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{n} whole solves of the same workload in {el:.1f} s (numpy/LAPACK FP64)"}
        line["accuracy"]["sv_rel_err_vs_oracle"] = float(np.linalg.norm(S - So) / np.linalg.norm(So))
        if args.workload == "c1":  # information: against the dense 4096 x 4096 LAPACK SVD (no bound holds)
            from oracle import mpo as om

            s_true = np.linalg.svd(om.dense(c["A"]), compute_uv=False)[: c["k"]]
            line["accuracy"]["sv_rel_err_vs_dense_lapack"] = float(np.linalg.norm(S - s_true) / np.linalg.norm(s_true))
            line["accuracy"]["max_rel_err_vs_dense_lapack"] = float(np.max(np.abs(S - s_true) / s_true))
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
