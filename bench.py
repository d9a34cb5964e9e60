#!/usr/bin/env python3
"""Benchmark: adaptive s-step CG on one GB300, through the libascg C ABI.

One step = one full solve of the 3D Poisson 7-point problem on a 128^3 grid
(n = 2,097,152, nnz = 14,581,760), adaptive s-step CG with the Chebyshev basis
on the closed-form eigenvalue bounds, s_max = 16, relative target 1e-12,
x_1 = 0. Each step runs every row of the hot path: residual setup, matrix
powers, Gram, condition estimates and choice of s_k, coordinate CG steps,
recovery, and the final true residual.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0. For N > 1 (torchrun), every rank solves its
own replica: a single solve does not shard across GPUs here, so the job is
replicas only, with weak scaling.
"""
from __future__ import annotations

import os

# the oracle (CPU baseline) runs single-threaded; set before numpy is imported
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import math
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG iters/s and HBM GB/s vs classical CG at 1e-10; served p50/p99 solve latency"
SINGLE_WORKLOADS = {
    # the headline workload: one large solve timed against classical CG on the same GPU
    "poisson3d_128": dict(
        desc=("3D Poisson 7-point 128^3 (n=2097152, nnz=14581760), equilibrated, b~U[-1,1] normalised "
              "(seed 1002), x1=0; adaptive s-step CG, Chebyshev basis on closed-form bounds, s_max=16, s0=f=16, "
              "c=1, eps*=1e-12; one full solve per step"),
        make="poisson3d_128", eps=1e-12, basis="chebyshev", s_max=16, newton_warmup=0, flush_l2=False,
        l2="inputs larger than L2: A 183 MB, basis 554 MB, vectors 16.8 MB each"),
    # 2D variable-coefficient diffusion, the largest single solve, at 1e-10
    "diffusion2048": dict(
        desc=("2D FV diffusion 2048^2 (n=4194304, nnz=20963328), log-normal sigma=2 cell coefficients, harmonic "
              "faces, equilibrated, b~U[-1,1] normalised (seed 1003), x1=0; adaptive s-step CG, Newton basis on "
              "Leja-ordered Ritz values of 24 classical warm-up iterations, s_max=12, c=1, eps*=1e-10; one full "
              "solve per step"),
        make="diffusion2d_2048", eps=1e-10, basis="newton", s_max=12, newton_warmup=24, flush_l2=False,
        l2="inputs larger than L2: A 252 MB, basis 840 MB, vectors 33.6 MB each"),
    # the small 2D Poisson problem at 1e-10 (fits in L2: flushed between steps)
    "poisson2d_32": dict(
        desc=("2D Poisson 5-point 32^2 (n=1024, nnz=4992), equilibrated, b~U[-1,1] normalised (seed 1001), x1=0; "
              "adaptive s-step CG, monomial basis, s_max=8, s0=f=8, c=1, eps*=1e-10; one full solve per step"),
        make="poisson2d_32", eps=1e-10, basis="monomial", s_max=8, newton_warmup=0, flush_l2=True,
        l2="inputs smaller than L2: a 256 MB buffer is written between timed steps, outside the timed region"),
}
WORKLOAD = SINGLE_WORKLOADS["poisson3d_128"]["desc"]
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_FMA_PER_CLK_SM = 2.0   # nominal: 1.25 TFLOP/s FP64 = 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2


def _measured_peak(key, fallback):
    """A peak from MEASURED_PEAKS.json (driver-written), else the fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


BF16_PEAK_TF, BF16_PEAK_SRC = _measured_peak("bf16_tflops", 1900.0)
HBM_PEAK_GBS, HBM_PEAK_SRC = _measured_peak("hbm_gbs", 6800.0)


def hbm_view(nbytes, ms):
    """Algorithmic bytes over a kernel's device time against the HBM copy peak:
    the bandwidth side of a kernel that another unit bounds."""
    if not ms or ms <= 0:
        return None
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": gbs / HBM_PEAK_GBS,
            "peak_source": f"{HBM_PEAK_SRC} copy bandwidth"}


def fp64_dgemm_tflops(torch, size=4096, reps=5):
    """FP64 rate of cuBLAS DGEMM (torch.matmul in float64) on this GPU, best of
    `reps`: a measured companion to the derived FP64 peak (DGEMM on GB300 uses
    the same FP64 units as DFMA)."""
    a = torch.randn(size, size, dtype=torch.float64, device="cuda")
    b = torch.randn(size, size, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return 2.0 * size ** 3 / (best * 1e-3) / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default="adaptive", choices=["adaptive", "classical"],
                    help="solver timed as the step (classical CG is the comparison baseline)")
    ap.add_argument("--no-classical", action="store_true", help="skip the classical-CG comparison solves")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sequential", action="store_true",
                    help="batch workload: skip the one-by-one adaptive solves of the same systems")
    ap.add_argument("--no-all-cores", action="store_true",
                    help="skip the all-host-cores oracle baseline (one replica per core)")
    ap.add_argument("--autotune", action="store_true",
                    help="batch workload: measure the Gram schedule threshold first (ascg_tune_gram_schedule)")
    ap.add_argument("--moment-gram", action="store_true",
                    help="batch and served workloads: G from the monomial basis' moments (a variant)")
    ap.add_argument("--requests", type=int, default=200, help="served workload: requests in the open-loop run")
    ap.add_argument("--load", type=float, default=0.7, help="served workload: arrival rate / saturation throughput")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served workload: device-memory budget (GB)")
    ap.add_argument("--policy", default="sjf", choices=["fifo", "sjf"],
                    help="served workload: admission order (submission order, or shortest estimated work first)")
    ap.add_argument("--large-cap", type=int, default=1,
                    help="served workload: most systems of >= 2^19 rows running at once (0: no cap)")
    ap.add_argument("--no-yield", dest="yield_large", action="store_false",
                    help="served workload: the largest size class does not wait for the smaller ones")
    ap.add_argument("--workload", default="poisson3d_128",
                    choices=list(SINGLE_WORKLOADS) + ["batch", "serve"],
                    help="a single-solve workload, or batch: 256 uneven systems solved by ascg_solve_batch (one "
                         "step = one batched call), or serve: the solve server on a Poisson-arrival stream")
    ap.add_argument("--gram-fp64", action="store_true",
                    help="form the Gram matrix with FP64 FMAs (CUDA cores) instead of the tensor-core digit split")
    return ap.parse_args()


def job_totals(elapsed, units, world, device):
    """Whole-job figures over the ranks (replicas): the slowest rank's elapsed
    time and the sum of all ranks' units of work."""
    if world == 1:
        return float(elapsed), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed), float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# roofline traffic from a committed ncu summary (bytes per launch), if current
# ---------------------------------------------------------------------------

MPK_KERNEL_TEXT = ("template <int SIG, bool R>", "// col_emax[c] = max over the warp entries")


def kernel_source_hash(name="kernels_mpk.cu", span=MPK_KERNEL_TEXT, text=None):
    """Hash of a kernel's own source text (from span[0] up to span[1]), so that
    edits elsewhere in the file keep a committed ncu figure valid."""
    if text is None:
        with open(os.path.join(ROOT, "paper_1701_03989_gb300", "csrc", name)) as f:
            text = f.read()
    a = text.index(span[0])
    b = text.index(span[1], a)
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per launch of the matrix powers kernel from profiles/, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "mpk_split_poisson3d_128.txt")
    if not os.path.exists(path):
        return None, None
    vals = {}
    for line in open(path):
        if ":" in line and line.split(":", 1)[0].strip() in ("source_hash", "dram_bytes_per_launch_full"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    try:
        return float(vals["dram_bytes_per_launch_full"]), None
    except (KeyError, ValueError):
        return None, "no traffic figure"


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the workload
# ---------------------------------------------------------------------------

def oracle_sample(spec, cfg, seconds: float):
    """Times whole oracle blocks of the workload's adaptive solve (sbar = s_max).

    p and r come from untimed classical oracle iterations (the Newton
    basis' 24 warm-up iterations, else 24), so the timed blocks are
    steady-state blocks with the workload's basis. Each block runs the
    oracle's matrix powers, Gram, block controller and recovery. Returns
    (iterations, seconds, blocks)."""
    from oracle import ascg_oracle as O
    A = O.Operator.from_csr(cfg["A"])
    b = cfg["b"]
    s = spec["s_max"]
    warm = O.classical_cg(A, b, np.zeros(A.n), eps_target=0.0, max_iters=spec["newton_warmup"] or 24)
    x, r, p = warm.x, warm.r, warm.p
    if spec["basis"] == "chebyshev":
        bp = O.chebyshev_params(cfg["lam"][0], cfg["lam"][1], s)
    elif spec["basis"] == "newton":
        bp = O.newton_params(O.leja_order(O.ritz_values(warm.alphas, warm.betas)), s)
    else:
        bp = O.monomial_params(s)
    eps_star = spec["eps"] * O.norm2(b)
    iters, blocks = 0, 0
    t0 = time.perf_counter()
    while True:
        Y = O.matrix_powers(A, p, r, s, bp)
        G = O.gram(Y)
        blk, inner, idx = O.adaptive_block(G, s, bp, eps_star, 1.0, A.n, True, 10 ** 6)
        if inner.steps == 0:   # a tiny problem may converge inside the sample: start again from the warm-up
            x, r, p = warm.x, warm.r, warm.p
            continue
        x, r, p = O.recover(Y[:, idx], x, inner.xc, inner.rc, inner.pc)
        iters += inner.steps
        blocks += 1
        if inner.stop == "converged":
            x, r, p = warm.x, warm.r, warm.p
        el = time.perf_counter() - t0
        if el >= seconds:
            return iters, el, blocks


def _oracle_sample_worker(args):
    """One replica of the oracle sample in a process of its own (all-cores baseline)."""
    name, seconds = args
    import workloads as W
    spec = SINGLE_WORKLOADS[name]
    cfg = getattr(W, spec["make"])()
    return oracle_sample(spec, cfg, seconds)


def oracle_all_cores(name, seconds, procs):
    """The oracle as it stands, one independent replica per host core, in
    processes started with spawn (safe beside a CUDA context). Returns
    (iterations per second summed over the replicas, processes, the slowest
    replica's seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        outs = pool.map(_oracle_sample_worker, [(name, seconds)] * procs)
    return sum(i / s for i, s, _b in outs), procs, max(s for _i, s, _b in outs)


def _sample_text(spec, ci, cs, cb):
    return (f"{cb} whole steady-state oracle blocks (sbar={spec['s_max']}, {spec['basis']}, {ci} iterations) after "
            f"{spec['newton_warmup'] or 24} untimed classical iterations, {cs:.1f} s")


def reference_arm(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import workloads as W
    name = args.workload if args.workload in SINGLE_WORKLOADS else "poisson3d_128"
    spec = SINGLE_WORKLOADS[name]
    cfg = getattr(W, spec["make"])()
    for _ in range(args.warmup):
        oracle_sample(spec, cfg, 1.0)
    its, secs = 0, 0.0
    for _ in range(args.steps):
        i, s, _b = oracle_sample(spec, cfg, 10.0)
        its += i
        secs += s
    v = its / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": spec["desc"], "parallelism": "replicas only"},
        "cpu_baseline": {"value": v, "unit": "iters/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: >=10 s of whole steady-state oracle blocks (sbar={spec['s_max']}, "
                                   f"{spec['basis']}) after {spec['newton_warmup'] or 24} untimed classical "
                                   f"iterations"},
        "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def untimed(P, o):
    """A copy of the options with the library's per-phase timing off."""
    c = P.ascg_options.from_buffer_copy(o)
    c.flags = o.flags & ~P.ASCG_FLAG_TIMING
    return c


def _timed_solves(P, torch, op, bd, xd, o, steps, stream, flush=None):
    """Solves `steps` times; each solve bracketed by CUDA events on the solve
    stream, with the L2 flush (if any) outside the brackets. Returns (total
    device ms, results)."""
    evs, res = [], []
    for _ in range(steps):
        xd.zero_()
        if flush is not None:
            flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res.append(P.ascg_solve(op, bd, xd, o, stream=stream))
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs), res


def our_arm(args):
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    import workloads as W

    spec = SINGLE_WORKLOADS[args.workload]
    cfg = getattr(W, spec["make"])()
    A, b = cfg["A"], cfg["b"]
    n = A.n
    eps = spec["eps"]
    op = P.ascg_op_create_csr(n, A.nnz, A.rowptr, A.colind, A.val, 0)
    stream = torch.cuda.current_stream()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    max_it = 60000
    lam = cfg["lam"] if spec["basis"] == "chebyshev" else None
    o_adaptive = P.make_options(method="adaptive", basis=spec["basis"], s_max=spec["s_max"], eps_target=eps, lam=lam,
                                newton_warmup=spec["newton_warmup"], max_iters=max_it, timing=True,
                                gram_fp64=args.gram_fp64)
    o_classical = P.make_options(method="classical", eps_target=eps, max_iters=max_it, timing=True)
    o_phases = o_classical if args.method == "classical" else o_adaptive
    # the timed solves run as a user runs them: the library's per-phase CUDA
    # events (five per block, each a break in the chain of dependent launches)
    # stay off there, and a second set of solves takes the phase split
    o = untimed(P, o_phases)
    flush = None
    if spec["flush_l2"]:
        scrub = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def flush():
            scrub.fill_(1)

    for _ in range(args.warmup):
        xd.zero_()
        P.ascg_solve(op, bd, xd, o, stream=stream)
    torch.cuda.synchronize()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if world == 1 else local
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms, results = _timed_solves(P, torch, op, bd, xd, o, args.steps, stream, flush)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    iters = sum(r.iters for r in results)
    ms_job, iters_job = job_totals(ms, iters, world, "cuda")
    value = iters_job / (ms_job * 1e-3)
    ok = all(r.status == P.ASCG_OK for r in results)

    # per-kernel device times recorded by the library with CUDA events on this
    # stream, from the same solves run again with the phase events on
    pms, presults = _timed_solves(P, torch, op, bd, xd, o_phases, args.steps, stream, flush)
    ok = ok and all(r.status == P.ASCG_OK for r in presults)
    t_gram = sum(r.t_gram_ms for r in presults)
    n_gram = sum(r.gram_launches for r in presults)
    f_gram = sum(r.gram_flops for r in presults)
    t_mpk = sum(r.t_mpk_ms for r in presults)
    t_ctrl = sum(r.t_ctrl_ms for r in presults)
    t_rec = sum(r.t_recover_ms for r in presults)
    t_cg = sum(r.t_cg_ms for r in presults)
    bytes_alg = sum(r.mpk_bytes + r.gram_bytes + r.recover_bytes for r in presults)
    flops_alg = sum(r.mpk_flops + r.gram_flops + r.recover_flops for r in presults)
    peak_tf = FP64_FMA_PER_CLK_SM * 2 * SMS * SM_MAX_MHZ * 1e6 / 1e12
    achieved_tf = f_gram / (t_gram * 1e-3) / 1e12 if t_gram > 0 else None   # FP64 flops of G = Y^T Y
    traffic_full, traffic_note = committed_traffic() if args.workload == "poisson3d_128" else (
        None, "no ncu traffic capture of this workload")
    f_mpk = sum(r.mpk_flops for r in presults)
    n_mpk = sum(r.mpk_launches for r in presults)
    achieved_mpk = f_mpk / (t_mpk * 1e-3) / 1e12 if t_mpk > 0 else None
    per_launch_mpk = f_mpk / n_mpk if n_mpk else None
    # the tensor-core Gram: its multiply-adds per launch (tiles of 128 x 240 and
    # 128 x 16 per row of Y) against the measured dense bf16/fp16 peak
    tc_flops = 2.0 * 128 * (240 + 16) * n * n_gram
    achieved_tc = tc_flops / (t_gram * 1e-3) / 1e12 if t_gram > 0 else None

    # end to end: host buffers through ascg_solve_host, copies inside the timed region
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    o_e2e = untimed(P, o)   # the same solve
    P.ascg_solve_host(op, bh, xh, o_e2e, stream=stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_s, e2e_iters = 0.0, 0
    for _ in range(args.steps):
        xh.zero_()
        if flush is not None:
            flush()
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.ascg_solve_host(op, bh, xh, o_e2e, stream=stream)
        e2e_s += time.perf_counter() - t0
        e2e_iters += r.iters
    e2e_s, e2e_iters = job_totals(e2e_s, e2e_iters, world, "cuda")
    e2e_value = e2e_iters / e2e_s

    # classical CG on the same GPU, same problem, same target (and fixed s on the small problem)
    classical = None
    if not args.no_classical:
        oc = untimed(P, o_classical)
        xd.zero_()
        P.ascg_solve(op, bd, xd, oc, stream=stream)
        torch.cuda.synchronize()
        cms, cres = _timed_solves(P, torch, op, bd, xd, oc, args.steps, stream, flush)
        cms /= args.steps
        cit = sum(r.iters for r in cres) / args.steps
        ams = ms / args.steps
        # classical CG's own floor per iteration: max(FP64 instructions, HBM bytes) of
        # its three kernels (SpMV + p^T A p; r and r^T r; x += alpha p and p = r + beta p)
        c_flops = 2.0 * (A.nnz + n) + 2.0 * 3 * n + 2.0 * n
        c_bytes = 12.0 * A.nnz + 4.0 * (n + 1) + 8.0 * n * (2 + 3 + 5)
        floor_us = 1e6 * max(c_flops / (peak_tf * 1e12), c_bytes / (HBM_PEAK_GBS * 1e9))
        per_it_us = 1e3 * cms / max(cit, 1)
        classical = {"iters_per_s": cit / (cms * 1e-3), "iters_per_solve": cit, "ms_per_solve": cms,
                     "adaptive_ms_per_solve": ams, "adaptive_iters_per_solve": iters / args.steps,
                     "time_to_solution_speedup": cms / ams,
                     "syncs_classical": sum(r.grid_reductions for r in cres) / args.steps,
                     "syncs_adaptive": sum(r.grid_reductions for r in results) / args.steps,
                     "true_res_classical": cres[-1].rel_res_true,
                     "us_per_iteration": per_it_us,
                     "floor_us_per_iteration": floor_us,
                     "roofline_frac": floor_us / per_it_us,
                     "floor_note": "max(FP64: 2(nnz+n) SpMV + 2n p^T A p + 4n r update + 4n x and p update "
                                   "flops at the FP64 peak; HBM: 12 nnz + 4(n+1) bytes of A + 10 vector passes of "
                                   "8n bytes at the measured copy peak)"}
        if args.workload == "poisson2d_32":
            of = P.make_options(method="fixed", basis="monomial", s_max=4, eps_target=eps, max_iters=max_it)
            fms, fres = _timed_solves(P, torch, op, bd, xd, of, args.steps, stream, flush)
            classical["fixed_s4_ms_per_solve"] = fms / args.steps
            classical["fixed_s4_iters_per_solve"] = sum(r.iters for r in fres) / args.steps

    dgemm_tf = fp64_dgemm_tflops(torch)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ci, cs, cb = oracle_sample(spec, cfg, 12.0)
        cpu = {"value": ci / cs, "unit": "iters/s", "cores": 1, "kind": "oracle",
               "sample": _sample_text(spec, ci, cs, cb)}
        if not args.no_all_cores:
            procs = os.cpu_count() or 1
            try:
                v_all, used, slowest = oracle_all_cores(args.workload, 10.0, procs)
                cpu["all_cores"] = {"value": v_all, "unit": "iters/s", "cores": used, "kind": "oracle replicas",
                                    "sample": f"{used} independent oracle replicas, one process per host core "
                                              f"(spawned), each >= 10 s of whole blocks as above; slowest "
                                              f"{slowest:.1f} s; iterations/s summed"}
            except Exception as e:   # the 1-core figure stands on its own
                cpu["all_cores"] = {"unavailable": str(e)[:200]}

    if rank == 0:
        desc = spec["desc"]
        if args.method == "classical":
            desc = desc.split("; adaptive s-step CG")[0] + f"; classical CG (Alg. 1), eps*={eps:g}; one full solve per step"
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_job / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc,
                       "method": args.method,
                       "parallelism": "replicas only" if world > 1 else "single GPU",
                       "gram": ("FP64 FMAs on the CUDA cores" if args.gram_fp64 else
                                "tensor cores: exact split of Y into fp16 digits, integer sums "
                                "(FP64-level normwise error); FP64 kernel with --gram-fp64"),
                       "l2": spec["l2"]},
            "status_ok": ok,
            "iters_per_solve": iters / args.steps,
            "blocks_per_solve": sum(r.blocks for r in results) / args.steps,
            "true_rel_res": results[-1].rel_res_true,
            # algorithmic bytes and flops over the headline device time
            "hbm_gbs_algorithmic": bytes_alg / (ms * 1e-3) / 1e9,
            "fp64_tflops_algorithmic": flops_alg / (ms * 1e-3) / 1e12,
            "phase_ms_per_solve": {"matrix_powers": t_mpk / args.steps, "gram": t_gram / args.steps,
                                   "controller": t_ctrl / args.steps, "recovery": t_rec / args.steps,
                                   "classical_iterations": t_cg / args.steps,
                                   "ms_per_solve_with_phase_events": pms / args.steps},
            "roofline": {"bound": "alu", "kernel": "mpk_split_step_kernel", "achieved": achieved_mpk,
                         "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": (achieved_mpk / peak_tf) if achieved_mpk else None,
                         "traffic": traffic_full, "traffic_note": traffic_note,
                         "flops_per_launch": per_launch_mpk,
                         "peak_source": "derived: FP64 DFMA 2 per clock per SM (nominal 1.25 TFLOP/s) x 152 SMs x "
                                        "2070 MHz max clock; FP64 is the binding unit (not HBM); the MEASURED_PEAKS "
                                        "file has no FP64 figure",
                         "fp64_dgemm_measured_tflops": dgemm_tf,
                         "frac_of_dgemm": (achieved_mpk / dgemm_tf) if achieved_mpk and dgemm_tf else None,
                         "hbm": hbm_view(sum(r.mpk_bytes for r in presults), t_mpk)},
            "roofline_gram": {"bound": "tensor", "kernel": "gram_tc_kernel (+ column exponents)",
                              "achieved": achieved_tc, "peak": BF16_PEAK_TF, "unit": "TFLOP/s",
                              "frac": (achieved_tc / BF16_PEAK_TF) if achieved_tc and BF16_PEAK_TF else None,
                              "flops_per_launch": 2.0 * 128 * (240 + 16) * n,
                              "fp64_equiv_tflops": achieved_tf,
                              "peak_source": f"{BF16_PEAK_SRC} dense bf16 burst (fp16 runs at the same rate)",
                              "hbm": hbm_view(sum(r.gram_bytes for r in presults), t_gram)},
            # the recovery of x, r and p (on the tensor cores where the Gram took them):
            # its algorithmic bytes, 8 w n + 32 n per block (r and p only, 8 w n + 16 n,
            # on the FP64 path), against the measured copy peak
            "roofline_recovery": (lambda h: dict(h, bound="hbm", kernel="recover_tc_kernel") if h else None)(
                hbm_view(sum(r.recover_bytes for r in presults), t_rec)),
            "vs_classical": classical,
            "e2e": {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 8 * n},
            "gpu_launches": sum(r.launches for r in results),
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    P.ascg_op_destroy(op)
    if world > 1:
        dist.destroy_process_group()
    return 0


def batch_arm(args):
    """256 independent SPD systems (2D/3D Poisson and banded, n log-uniform in
    [1e3, 2e5], targets 1e-8 or 1e-12), adaptive monomial s_max = 10, solved by
    one ascg_solve_batch call per step; beside it, the same systems solved one
    by one with ascg_solve (one pass)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    import workloads as W
    t_gen = time.perf_counter()
    systems = W.batch_systems(256)
    ops = [P.ascg_op_create_csr(s["A"].n, s["A"].nnz, s["A"].rowptr, s["A"].colind, s["A"].val, 0) for s in systems]
    t_gen = time.perf_counter() - t_gen
    bs = [torch.from_numpy(s["b"]).cuda() for s in systems]
    xs = [torch.zeros(s["A"].n, dtype=torch.float64, device="cuda") for s in systems]
    eps = [s["eps"] for s in systems]
    tuned = None
    if args.autotune:
        thr, table = P.ascg_tune_gram_schedule(10)
        tuned = {"tc_lane_rows": thr, "table_us": [[int(r[0]), round(r[1], 1), round(r[2], 1)] for r in table]}
    o = P.make_options(method="adaptive", basis="monomial", s_max=10, eps_target=1e-10, max_iters=20000,
                       moment_gram=args.moment_gram, tc_lane_rows=tuned["tc_lane_rows"] if tuned else 0)
    stream = torch.cuda.current_stream()

    def batch_once():
        for x in xs:
            x.zero_()
        return P.ascg_solve_batch(ops, bs, xs, o, eps_targets=eps, stream=stream)

    for _ in range(args.warmup):
        batch_once()
    torch.cuda.synchronize()
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs = [batch_once() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    res, st = outs[-1]
    iters = sum(r.iters for r in res)
    value = iters * args.steps / (ms * 1e-3)
    ok = all(r.status == P.ASCG_OK for r in res)
    worst_true = max(r.rel_res_true / e for r, e in zip(res, eps))
    def one_by_one(opts):
        """The same systems solved one by one through ascg_solve with opts."""
        its = 0
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for q in range(len(systems)):
            xs[q].zero_()
            oq = P.ascg_options.from_buffer_copy(opts)
            oq.eps_target = eps[q]
            r = P.ascg_solve(ops[q], bs[q], xs[q], oq, stream=stream)
            its += r.iters
        s1.record(stream)
        torch.cuda.synchronize()
        return s0.elapsed_time(s1), its

    seq_ms = seq_iters = None
    classical = None
    if not args.no_sequential:
        # the same systems one by one through ascg_solve (tensor-core Gram where w >= 9)
        seq_ms, seq_iters = one_by_one(o)
    if not args.no_classical:
        # classical CG (Alg. 1) on the same systems and targets: one by one through
        # ascg_solve, and batched in the same lockstep engine as s-step CG with
        # s = 1 (Alg. 2 with s = 1 equals classical CG in exact arithmetic, one
        # global reduction per iteration)
        oc = P.make_options(method="classical", eps_target=1e-10, max_iters=200000)
        c_ms, c_its = one_by_one(oc)
        o1 = P.make_options(method="fixed", basis="monomial", s_max=1, eps_target=1e-10, max_iters=200000)
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        r1, _st1 = P.ascg_solve_batch(ops, bs, xs, o1, eps_targets=eps, stream=stream)
        b1.record(stream)
        torch.cuda.synchronize()
        s1_ms = b0.elapsed_time(b1)
        classical = {"one_by_one_ms": c_ms, "one_by_one_iters": c_its,
                     "s1_batched_ms": s1_ms, "s1_batched_iters": sum(r.iters for r in r1),
                     "s1_batched_ok": all(r.status == P.ASCG_OK for r in r1),
                     "adaptive_batched_ms": ms / args.steps,
                     "speedup_vs_classical_one_by_one": c_ms / (ms / args.steps),
                     "speedup_vs_s1_batched": s1_ms / (ms / args.steps)}
    line = {
        "metric": "batched CG iters/s (256 uneven SPD systems, one ascg_solve_batch call per step)",
        "value": value, "unit": "iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "256 SPD systems: 2D Poisson / 3D Poisson / banded (hbw 8..64) uniform, n log-uniform "
                               "in [1e3, 2e5], eps* 1e-8 or 1e-12 at p = 1/2, seed 1004; adaptive monomial s_max=10",
                   "rows_total": int(sum(s["A"].n for s in systems)),
                   "nnz_total": int(sum(s["A"].nnz for s in systems)),
                   "gram": ("Hankel moments of the monomial basis, FP64 (a variant)" if args.moment_gram else
                            "tensor cores for lanes of tc_lane_rows rows or more (whole 1024-row chunks, one launch), "
                            "FP64 FMAs on per-system row items below")},
        "status_ok": ok, "iters_per_batch": iters, "lockstep_blocks": res[0].launches,
        "worst_true_res_over_target": worst_true,
        "sequential": None if seq_ms is None else {
            "ms": seq_ms, "iters": seq_iters, "iters_per_s": seq_iters / (seq_ms * 1e-3),
            "batch_speedup": seq_ms / (ms / args.steps)},
        "vs_classical": classical,
        "setup_s": t_gen, "clocks": clocks, "gram_schedule": tuned or {"tc_lane_rows": 1 << 10, "source": "default"},
    }
    print(json.dumps(line), flush=True)
    for op in ops:
        P.ascg_op_destroy(op)
    return 0


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v, dtype=float), q)) if len(v) else None


def serve_arm(args):
    """Served workload: requests drawn from a pool of 12 SPD operators (2D/3D
    Poisson and banded, sizes at log-uniform quantiles of [1e4, 4e6]), targets
    uniform over {1e-6, 1e-8, 1e-10, 1e-12}, fresh seeded right-hand sides,
    arriving as a Poisson process. The solve server (continuous batching,
    adaptive monomial s_max = 10) serves them under a device-memory budget.
    Steps: (1) saturation throughput: the same requests, all submitted at
    once, served to the end (a smaller sample's mix is too far from the
    stream's for a stable figure); (2) the open-loop run at `load` x
    saturation, latency from each request's
    arrival to the step that completed it; (3) the same arrivals through a
    FIFO queue served one request at a time by classical CG (ascg_solve),
    from measured service times per (operator, target); (4) an end-to-end
    sample with right-hand sides copied from pinned host memory at submission
    and solutions copied back at completion."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    import workloads as W
    t_gen = time.perf_counter()
    pool = W.serve_pool()
    ops = [P.ascg_op_create_csr(p["A"].n, p["A"].nnz, p["A"].rowptr, p["A"].colind, p["A"].val, 0) for p in pool]
    nop = [p["A"].n for p in pool]
    nreq = max(int(args.requests), 8)
    nwarm = max(4, min(nreq // 10, 40))
    ne2e = max(8, min(nreq // 4, 100))
    nsat = min(nreq, 300)   # the saturation sample: the first requests of the stream
    req = W.serve_requests(nreq)
    t_gen = time.perf_counter() - t_gen

    def rhs(i):
        g = torch.Generator(device="cuda")
        g.manual_seed(int(req["rhs_seed"][i]) % (2 ** 63))
        b = torch.rand(nop[req["op"][i]], dtype=torch.float64, device="cuda", generator=g).mul_(2.0).sub_(1.0)
        return b.div_(torch.linalg.vector_norm(b))

    bs = [rhs(i) for i in range(nreq)]
    xs = [torch.zeros_like(b) for b in bs]
    o = P.make_options(method="adaptive", basis="monomial", s_max=10, eps_target=1e-10, max_iters=60000,
                       moment_gram=args.moment_gram)
    stream = torch.cuda.current_stream()
    budget = int(args.budget_gb * 1e9)
    slots = 256
    srv = P.ascg_server_create(o, budget, slots, stream)
    order = P.ASCG_ADMIT_SHORTEST_FIRST if args.policy == "sjf" else P.ASCG_ADMIT_FIFO
    P.ascg_server_set_policy(srv, order, args.large_cap, args.yield_large)

    def run(idx, arrivals, host_io=False):
        """Serves requests idx arriving at `arrivals` (seconds from the start).
        Returns per-request latency (s), completions, wall seconds, peak
        systems running and the server steps taken."""
        for i in idx:
            xs[i].zero_()
        hb = hx = None
        if host_io:
            hb = {i: bs[i].cpu().pin_memory() for i in idx}
            hx = {i: torch.zeros(bs[i].numel(), dtype=torch.float64).pin_memory() for i in idx}
            db = {i: torch.empty_like(bs[i]) for i in idx}
        torch.cuda.synchronize()
        order = np.argsort(arrivals, kind="stable")
        arr = {int(idx[k]): float(arrivals[k]) for k in range(len(idx))}
        lat, comp = {}, {}
        pos, peak = 0, 0
        steps0 = P.ascg_server_info(srv).steps
        t0 = time.perf_counter()
        while len(lat) < len(idx):
            now = time.perf_counter() - t0
            while pos < len(idx) and arrivals[order[pos]] <= now:
                i = int(idx[order[pos]])
                if host_io:
                    db[i].copy_(hb[i], non_blocking=True)
                    P.ascg_server_submit(srv, ops[req["op"][i]], db[i], xs[i], float(req["eps"][i]), i)
                else:
                    P.ascg_server_submit(srv, ops[req["op"][i]], bs[i], xs[i], float(req["eps"][i]), i)
                pos += 1
            comps, nact, npend = P.ascg_server_step(srv, cap=slots)
            peak = max(peak, nact + len(comps))
            if host_io and comps:
                for c in comps:
                    hx[c.tag].copy_(xs[c.tag], non_blocking=True)
                stream.synchronize()
            t = time.perf_counter() - t0
            for c in comps:
                lat[c.tag] = t - arr[c.tag]
                comp[c.tag] = c
            if nact == 0 and npend == 0 and pos < len(idx):
                wait = arrivals[order[pos]] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
        wall = time.perf_counter() - t0
        return lat, comp, wall, peak, P.ascg_server_info(srv).steps - steps0

    # (1) saturation: the stream's first requests, all submitted at once
    run(np.arange(nwarm), np.zeros(nwarm))  # warm-up
    _, _, sat_wall, sat_peak, _ = run(np.arange(nsat), np.zeros(nsat))
    mu = nsat / sat_wall
    lam = args.load * mu
    # (2) open loop at load x saturation
    idx = np.arange(nreq)
    arrivals = np.cumsum(req["gap"][:nreq]) / lam
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat, comp, wall, peak, steps = run(idx, arrivals)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    gpu_ms = e0.elapsed_time(e1)
    lat_ms = [1e3 * lat[i] for i in range(nreq)]
    iters = sum(comp[i].result.iters for i in range(nreq))
    ok = all(comp[i].result.status == P.ASCG_OK for i in range(nreq))
    worst = max(comp[i].result.rel_res_true / req["eps"][i] for i in range(nreq))
    # latency by request size (rows): thirds of the log-uniform range
    edges = [0, 1e5, 1e6, float("inf")]
    by_size = {}
    for lo_, hi_ in zip(edges[:-1], edges[1:]):
        sel = [lat_ms[i] for i in range(nreq) if lo_ <= nop[req["op"][i]] < hi_]
        by_size[f"n<{hi_:g}"] = {"count": len(sel), "p50_ms": _pct(sel, 50), "p99_ms": _pct(sel, 99)}
    # (3) FIFO sequential classical CG on the same arrivals, from measured service times
    oc = P.make_options(method="classical", eps_target=1e-10, max_iters=200000)
    service = {}
    for key in sorted({(int(req["op"][i]), float(req["eps"][i])) for i in range(nreq)}):
        i = next(i for i in range(nreq) if (int(req["op"][i]), float(req["eps"][i])) == key)
        x = torch.zeros_like(bs[i])
        oq = P.ascg_options.from_buffer_copy(oc)
        oq.eps_target = key[1]
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        P.ascg_solve(ops[key[0]], bs[i], x, oq, stream=stream)
        c1.record(stream)
        torch.cuda.synchronize()
        service[key] = c0.elapsed_time(c1) * 1e-3
    fin, fifo, fifo_of = 0.0, [], {}
    for k in np.argsort(arrivals, kind="stable"):
        fin = max(arrivals[k], fin) + service[(int(req["op"][k]), float(req["eps"][k]))]
        fifo.append(1e3 * (fin - arrivals[k]))
        fifo_of[int(k)] = fifo[-1]
    fifo_wall = fin - arrivals.min()
    for lo_, hi_ in zip(edges[:-1], edges[1:]):
        sel = [fifo_of[i] for i in range(nreq) if lo_ <= nop[req["op"][i]] < hi_]
        by_size[f"n<{hi_:g}"].update({"classical_fifo_p50_ms": _pct(sel, 50), "classical_fifo_p99_ms": _pct(sel, 99)})
    # (4) end to end: host right-hand sides in, solutions out
    e_idx = np.arange(ne2e)
    elat, _, ewall, _, _ = run(e_idx, arrivals[:ne2e], host_io=True)
    elat_ms = [1e3 * elat[i] for i in range(ne2e)]
    P.ascg_server_destroy(srv)
    h2d = sum(8 * nop[req["op"][i]] for i in range(ne2e)) / ne2e
    line = {
        "metric": "served solve latency p50 (ms), Poisson arrivals at %.2fx saturation throughput" % args.load,
        "value": _pct(lat_ms, 50), "unit": "ms", "n_gpus": 1, "steps": nreq, "warmup": nwarm,
        "ms_per_step": gpu_ms / nreq, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "solve server: %d requests from a pool of 12 SPD operators (2D/3D Poisson, banded hbw "
                               "8..64; n at log-uniform quantiles of [1e4, 4e6]), eps* uniform over {1e-6, 1e-8, "
                               "1e-10, 1e-12}, Poisson arrivals, seed 1005; adaptive monomial s_max=10; budget "
                               "%.0f GB, %d slots" % (nreq, args.budget_gb, slots),
                   "pool_n": nop, "pool_nnz": [int(p["A"].nnz) for p in pool],
                   "gram": "Hankel moments (a variant)" if args.moment_gram else "Y^T Y"},
        "p50_ms": _pct(lat_ms, 50), "p99_ms": _pct(lat_ms, 99), "max_ms": max(lat_ms),
        "policy": {"admit": args.policy, "large_class_cap": args.large_cap, "yield_large": args.yield_large},
        "by_size": by_size,
        "saturation_sample": nsat,
        "throughput_rps": nreq / wall, "arrival_rps": lam, "saturation_rps": mu,
        "saturation_wall_s": sat_wall, "saturation_peak_running": sat_peak, "peak_running": peak,
        "server_steps": steps, "iters_per_s": iters / wall, "status_ok": ok, "worst_true_res_over_target": worst,
        "classical_fifo": {"p50_ms": _pct(fifo, 50), "p99_ms": _pct(fifo, 99), "max_ms": max(fifo),
                           "throughput_rps": nreq / fifo_wall, "service_pairs": len(service),
                           "note": "FIFO queue, one request at a time, ascg_solve classical CG; service time "
                                   "measured once per (operator, target)"},
        "e2e": {"value": _pct(elat_ms, 50), "unit": "ms", "p99_ms": _pct(elat_ms, 99), "requests": ne2e,
                "throughput_rps": ne2e / ewall, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d},
        "setup_s": t_gen, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for op in ops:
        P.ascg_op_destroy(op)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch":
        return batch_arm(args)
    if args.workload == "serve":
        return serve_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
