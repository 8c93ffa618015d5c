#!/usr/bin/env python3
"""Benchmark: s-step BDCD for kernel ridge regression on one GB300.

Workload (default): dense K-RR, m = 50000 samples, n = 512 features, A ~
N(0,1)/sqrt(n) stored FP32, y = sin(A w) + 0.1 N(0,1), RBF with bandwidth
sigma = 1 (gamma = 1/(2 sigma^2) = 0.5), lambda = 1e-4, block size b = 16,
s = 64 inner steps per outer step, fp16 tensor-core kernel block (the matrix
scaled by one power of two, 11 significant bits, one MMA per k-step) with
the FP64 recurrence and FP64 gradient accumulation; the split-bf16 form
(bf16x3, three MMAs per k-step) is measured beside it in the time-to-
tolerance and error records.  Synthetic data stand in for the paper's
LIBSVM sets.

One "step" is one outer s-step (sample, gather, Gram, FP64 recurrence, fused
kernel-block gradient update, alpha update) = s*b coordinate updates.  The
metric is coordinate updates per second.  L2 (129 MB) could hold the packed
operand, so a buffer larger than L2 is written before every timed step and
each step is timed alone with CUDA events on the solver's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--s S] [--prec fp16|bf16x3|bf16|tf32|fp64]
  python bench.py --impl reference   # the FP64 CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coordinate updates/s and time-to-duality-gap 1e-6 (mixed vs FP64 s=1, 1 GB300)"
UNIT = "coordinate updates/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one fused-block launch from
# an ncu capture: (prec, m, n, b, s, first 16 hex digits of the sha256 of
# csrc/block_tc.cu when it was taken) -> bytes.  A changed kernel source
# matches no entry, so its traffic reads null until it is captured again.
NCU_TRAFFIC = {("fp16", 50000, 512, 16, 64, "2bec218b23016340"): 53.15e6,
               ("bf16x3", 50000, 512, 16, 64, "2bec218b23016340"): 109.09e6}
WORKLOAD = "K-RR BDCD dense m=50000 n=512 RBF sigma=1 lambda=1e-4 b=16"


def emit(out, args):
    """Prints a workload's JSON line, or collects it (the side summaries of
    the default line)."""
    if getattr(args, "collect", None) is not None:
        args.collect.append(out)
    else:
        print(json.dumps(out), flush=True)


def kernel_source_sha16():
    import hashlib
    path = os.path.join(ROOT, "paper_2406_18001_gb300", "csrc", "block_tc.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def oracle_threads():
    """All host cores for the oracle's parallel row loops (results do not
    depend on the count); returns the count in effect."""
    import oracle
    oracle.build()
    return oracle.set_threads(os.cpu_count() or 1)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained"), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_problem(m, n, seed=0):
    from paper_2406_18001_gb300 import inputs
    return inputs.krr_dense(m=m, n=n, seed=seed, dtype=np.float32)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_max(x, ws, device):
    """The maximum of x over the ranks of the job (x itself at one rank): the
    job's time is its slowest replica's.  Joins the default process group
    (NCCL on a GPU device, gloo on the CPU) if none is up yet."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        if device.type == "cuda":
            dist.init_process_group("nccl", device_id=device)
        else:
            dist.init_process_group("gloo")
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ms, ws):
    """Whole-job throughput of ws replicas that each processed units_per_rank
    units, the job taking ms milliseconds (the max over ranks)."""
    return ws * units_per_rank / (ms * 1e-3)


# ----------------------------------------------------------- reference ----
def run_reference(args):
    """The FP64 CPU oracle (s-step BDCD, Algorithm 4 as printed, the same s
    and b as this bench's arm) timed on the host, its row loops on every core.
    Each step is one outer s-step of the workload restricted to its first
    m_sub rows, m_sub sized so the whole run stays within ~150 s; the rate is
    scaled to the full m (the oracle's cost per step is linear in m)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    nt = oracle_threads()
    p = make_problem(args.m, args.n)
    A64 = p.A.astype(np.float64)
    k = oracle.kernel("rbf", gamma=args.gamma)
    s = args.s
    cal = min(args.m, 2000)
    t0 = time.perf_counter()
    oracle.sstep_bdcd_krr(A64[:cal], p.y[:cal], k, args.lam, args.b, s, s, seed=0)
    per_row = (time.perf_counter() - t0) / cal
    budget = 150.0 / (args.steps + args.warmup)
    m_sub = int(max(args.b, min(args.m, budget / max(per_row, 1e-9))))
    As, ys = np.ascontiguousarray(A64[:m_sub]), p.y[:m_sub].copy()
    alpha = np.zeros(m_sub)
    for w in range(args.warmup):
        alpha = oracle.sstep_bdcd_krr(As, ys, k, args.lam, args.b, s, s, seed=0, first_block=w * s, alpha0=alpha)
    t0 = time.perf_counter()
    for i in range(args.steps):
        alpha = oracle.sstep_bdcd_krr(As, ys, k, args.lam, args.b, s, s, seed=0, first_block=(args.warmup + i) * s,
                                      alpha0=alpha)
    dt = time.perf_counter() - t0
    v = args.steps * s * args.b / dt * (m_sub / args.m)
    sample = (f"{args.steps} outer s-steps (s={s}, b={args.b}) on the first {m_sub} of {args.m} rows "
              f"(n={args.n}), rate scaled by {m_sub}/{args.m}; plain FP64 C, row loops on {nt} threads")
    out = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "s": s, "b": args.b, "m": args.m, "n": args.n, "m_sample": m_sub},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(args, budget_s=12.0):
    """Oracle throughput on a bounded sample: block updates (Algorithm 3,
    s = 1) of the full workload until ~budget_s, its row loops on every host
    core."""
    import oracle
    p = make_problem(args.m, args.n)
    A64 = p.A.astype(np.float64)
    k = oracle.kernel("rbf", gamma=args.gamma)
    nt = oracle_threads()
    alpha = np.zeros(args.m)
    t0 = time.perf_counter()
    blocks = 0
    while time.perf_counter() - t0 < budget_s and blocks < 512:
        alpha = oracle.sstep_bdcd_krr(A64, p.y, k, args.lam, args.b, 1, 1, seed=0, first_block=blocks,
                                      alpha0=alpha)
        blocks += 1
    dt = time.perf_counter() - t0
    return {"value": blocks * args.b / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{blocks} BDCD block updates (b={args.b}) of the full {args.m}x{args.n} workload "
                      f"({dt:.1f} s, plain FP64 C, row loops of U_k on {nt} threads)"}


# ------------------------------------------------------ time to tolerance --
def fp64_residual(B, torch, A, y, alpha, k, lam):
    """||(K/lambda + m I) alpha - y|| / ||y|| over all m rows: K alpha by the
    FP64 CUDA-core kernel block (RBF distances from coordinate differences),
    one pass over every column."""
    m = alpha.numel()
    g = torch.zeros(m, dtype=torch.float64, device=alpha.device)
    cols = torch.arange(m, dtype=torch.int32, device=alpha.device)
    B.kernel_block_apply(A, k, "fp64", cols, alpha / lam, g)
    r = g + m * alpha - y
    return float(torch.linalg.norm(r) / torch.linalg.norm(y))


def solve_to_tol(B, torch, A, y, k, lam, b, s, prec, tol, budget, seed):
    """One solve to relative residual tol: the mixed forms check the cached
    gradient every ~256 block updates and confirm on a recomputed gradient
    (DCD_FLAG_REFRESH); the FP64 form's cached gradient is exact to rounding."""
    ce = max(1, 256 // s)
    flags = B.FLAG_REFRESH if prec != "fp64" else 0
    plan = B.Plan(1, A, y, k, lam, b, s, budget, seed=seed, prec=prec, tol=tol, check_every=ce, flags=flags)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, _ = plan.run(-1)
    wall = time.perf_counter() - t0
    alpha = plan.alpha.clone()
    plan.close()
    out = {"prec": prec, "s": s, "converged": bool(st["converged"]), "block_updates": st["iters_done"],
           "coordinate_updates": st["iters_done"] * b, "ms": st["ms_total"], "wall_s": wall,
           "resid_solver": st["final_metric"], "refreshes": st["refreshes"], "ms_refresh": st["ms_refresh"],
           "check_every_outer_steps": ce}
    out["resid_fp64"] = fp64_residual(B, torch, A, y, alpha, k, lam)
    out["reached_tol_fp64"] = bool(out["converged"] and out["resid_fp64"] <= tol)
    return out, alpha


def time_to_tol(args, torch, B, A, y, k, seed):
    """Time to relative residual ||(K/lambda + mI) a - y|| / ||y|| <= tol:
    the mixed forms (this bench's precision, and split bf16 whose iterates
    track the FP64 ones) against the plain FP64 s = 1 form, on the same index
    stream.  The mixed forms recompute the gradient from alpha (sliced exact
    products, accurate epilogue) before accepting convergence.  Every
    result's residual is re-evaluated over all rows with the FP64 kernel
    block; a form counts only where it meets tol there.
      full:  the workload itself.  A FP64 s = 1 run to tol takes minutes
             here, so its time is ESTIMATED: its measured time per block
             update times the block updates the split-bf16 solve needed (the
             same iteration up to rounding).
      small: the first ttt_small_m rows of the same workload, every form run
             to tol and timed (a measured ratio), and each result compared
             with the closed form alpha* = (K/lambda + m I)^-1 y (kernel block
             from the FP64 oracle, dense solve)."""
    b, m = args.b, args.m
    forms = list(dict.fromkeys((args.prec, "bf16x3")))

    def best(runs, base_ms):
        ok = {f: r["ms"] for f, r in runs.items() if r["reached_tol_fp64"]}
        if not ok or base_ms is None:
            return None, None
        f = min(ok, key=ok.get)
        return base_ms / ok[f], f

    mixed = {f: solve_to_tol(B, torch, A, y, k, args.lam, b, args.s, f, args.tol, args.ttt_budget, seed)[0]
             for f in forms}
    # FP64 s = 1: time per block update over a bounded run
    n64 = args.ttt_fp64_steps
    p64 = B.Plan(1, A, y, k, args.lam, b, 1, n64 + 8, seed=seed, prec="fp64")
    p64.run(8)
    base, _ = p64.run(0)
    torch.cuda.synchronize()
    p64.run(n64)
    st64, _ = p64.run(0)
    p64.close()
    ms_blk = (st64["ms_total"] - base["ms_total"]) / n64
    twin = mixed["bf16x3"]
    fp64 = {"prec": "fp64", "s": 1, "estimated": True, "ms_per_block_update": ms_blk, "blocks_timed": n64,
            "block_updates_basis": twin["block_updates"],
            "ms_estimated": ms_blk * twin["block_updates"] if twin["converged"] else None,
            "how": "measured ms per block update x the split-bf16 solve's block updates (same index stream)"}
    sp, form = best(mixed, fp64["ms_estimated"])
    full = {"mixed": mixed, "fp64_s1": fp64, "speedup_estimated": sp, "speedup_form": form}
    out = {"tol": args.tol, "metric": "relative residual ||(K/lambda + m I) alpha - y|| / ||y||", "full": full}
    if args.ttt_small_m > 0:
        ms_ = min(args.ttt_small_m, m)
        As, ys = A[:ms_].contiguous(), y[:ms_].contiguous()
        runs, alphas = {}, {}
        for f in forms:
            runs[f], alphas[f] = solve_to_tol(B, torch, As, ys, k, args.lam, b, args.s, f, args.tol, args.ttt_budget,
                                              seed)
        f6, alphas["fp64_s1"] = solve_to_tol(B, torch, As, ys, k, args.lam, b, 1, "fp64", args.tol, args.ttt_budget,
                                             seed)
        sp, form = best(runs, f6["ms"] if f6["reached_tol_fp64"] else None)
        small = {"m": ms_, "mixed": runs, "fp64_s1": f6, "speedup_measured": sp, "speedup_form": form}
        if not args.no_cpu:
            import oracle
            oracle_threads()
            A64 = As.double().cpu().numpy()
            ko = oracle.kernel("rbf", gamma=args.gamma)
            t0 = time.perf_counter()
            Kf = oracle.kernel_block(ko, A64, np.arange(ms_))
            star = np.linalg.solve(Kf / args.lam + ms_ * np.eye(ms_), ys.cpu().numpy())
            small["closed_form_s"] = time.perf_counter() - t0
            del Kf
            small["alpha_vs_closed_form"] = {
                f: float(np.linalg.norm(a.cpu().numpy() - star) / np.linalg.norm(star)) for f, a in alphas.items()}
        out["small"] = small
    return out


# ------------------------------------------- headline error vs the oracle --
def krr_objective_on_support(oracle, A64, y, ko, lam, alpha):
    """1/2 a^T (K/lambda + m I) a - y^T a for an alpha with few nonzeros: only
    the support's kernel entries (from the oracle) enter."""
    supp = np.nonzero(alpha)[0]
    Kss = oracle.kernel_block(ko, A64, supp, rows=supp)
    a = alpha[supp]
    return 0.5 * (a @ (Kss @ a) / lam + len(alpha) * (a @ a)) - y[supp] @ a


def headline_error(args, torch, B, A, y, k, p, seed):
    """Error of the headline configuration against the FP64 oracle (Algorithm
    4 as printed) on the same index stream: err_steps outer steps from
    alpha = 0 of the full workload, alpha's relative 2-norm error and the dual
    objective's relative error, for this bench's precision and for bf16x3."""
    import oracle
    H = args.err_steps * args.s
    nt = oracle_threads()
    A64 = p.A.astype(np.float64)
    ko = oracle.kernel("rbf", gamma=args.gamma)
    t0 = time.perf_counter()
    want = oracle.sstep_bdcd_krr(A64, p.y, ko, args.lam, args.b, args.s, H, seed=seed)
    t_or = time.perf_counter() - t0
    f_want = krr_objective_on_support(oracle, A64, p.y, ko, args.lam, want)
    out = {"H_block_updates": H, "outer_steps": args.err_steps, "seed": seed, "oracle_s": t_or,
           "oracle_threads": nt, "oracle": "sstep_bdcd_krr (Algorithm 4, FP64, Q_k materialised)"}
    for prec in dict.fromkeys((args.prec, "bf16x3")):
        al = B.krr_solve(A, y, k, args.lam, args.b, args.s, H, seed=seed, prec=prec)[0].cpu().numpy()
        f = krr_objective_on_support(oracle, A64, p.y, ko, args.lam, al)
        out[prec] = {"alpha_rel_err": float(np.linalg.norm(al - want) / np.linalg.norm(want)),
                     "objective_rel_err": float(abs(f - f_want) / abs(f_want))}
    return out


def dense_roofline(prec, m, n, b, s, t_block, bf16_peak, hbm_peak, src, traffic=None):
    """Roofline of one fused kernel-block launch (a5) on the method's own
    work: 2 m n sb flops (the paper's sbfmn of Thm 2 with f = 2n) and one read
    of the packed operand plus the gradient.  The split precisions issue 3
    MMAs per k-step; that tensor-pipe work is reported apart (mma_pipe) and is
    not what frac measures."""
    sb = s * b
    esz = {"bf16": 2, "tf32": 4, "bf16x3": 4, "tf32x3": 8, "fp8": 1, "fp64": 8, "fp16": 2}[prec]
    mma_mult = 3 if prec in ("bf16x3", "tf32x3") else 1  # MMAs per k-step
    flops = 2.0 * m * n * sb
    bytes_ = m * n * esz + sb * n * esz + m * (8 + 8 + 4)
    ridge = bf16_peak * 1e12 / (hbm_peak * 1e9)
    # a contraction's peak is its own dtype's: the measured bf16 figure times the nominal ratio
    tc_peak = {"bf16": 1.0, "bf16x3": 1.0, "fp16": 1.0, "fp8": 2.0, "tf32": 1.1 / 2.25,
               "tf32x3": 1.1 / 2.25}.get(prec, 0.0) * bf16_peak
    if tc_peak and flops * mma_mult / bytes_ >= ridge:
        roof = {"bound": "tensor", "achieved": flops / t_block / 1e12, "peak": tc_peak, "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_ / t_block / 1e9, "peak": hbm_peak, "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if traffic is None:
        traffic = NCU_TRAFFIC.get((prec, m, n, b, s, kernel_source_sha16()))
    roof["traffic"] = traffic
    roof["peak_source"] = f"{src} (MEASURED_PEAKS.json bf16 burst; HBM copy)"
    roof["kernel"] = ("block_tc2_kernel (fused kernel block + gradient update, CTA pairs)" if prec != "fp64"
                      else "block_simt_f64_kernel")
    roof["algorithmic"] = {"flops_per_launch": flops, "bytes_per_launch": bytes_,
                           "flops_rule": "2*m*n*s*b (method flops; split MMA passes not counted)"}
    if tc_peak:
        roof["mma_pipe"] = {"mma_per_k_step": mma_mult, "flops_per_launch": flops * mma_mult,
                            "achieved": flops * mma_mult / t_block / 1e12, "unit": "TFLOP/s",
                            "frac": flops * mma_mult / t_block / 1e12 / tc_peak}
    return roof


# ---------------------------------------------------------------- GPU -----
def run_gpu(args):
    import torch
    from paper_2406_18001_gb300 import binding as B

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    # a non-default stream: full outer steps then replay as one CUDA graph
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        return _run_gpu(args, torch, B, ws, rank, local, dev, stream)


def _run_gpu(args, torch, B, ws, rank, local, dev, stream):
    p = make_problem(args.m, args.n, seed=rank)
    A = torch.from_numpy(p.A).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    k = B.kernel("rbf", gamma=args.gamma)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2
    upd_per_step = args.s * args.b
    H = (args.warmup + args.steps + 8) * args.s
    plan = B.Plan(1, A, y, k, args.lam, args.b, args.s, H, seed=rank, prec=args.prec,
                  flags=B.FLAG_NO_DEFER if args.no_defer else 0)
    for _ in range(args.warmup):
        plan.run(1)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            plan.enqueue(1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_steps = sorted(a.elapsed_time(b) for a, b in ev)
    st, _ = plan.run(0)
    launches = st["gpu_launches_per_step"] * args.steps
    plan.close()
    ms = rank_max(ms, ws, dev)

    # dominant kernel (fused kernel block) duration, measured live: per-phase
    # CUDA events on the solver's stream, L2 flushed before every step
    plan2 = B.Plan(1, A, y, k, args.lam, args.b, args.s, (args.roof_steps + 4) * args.s, seed=rank + 1,
                   prec=args.prec, flags=B.FLAG_PHASE_TIMERS)
    plan2.run(2)
    base, _ = plan2.run(0)
    for _ in range(args.roof_steps):
        flush.zero_()
        plan2.run(1)
    st2, _ = plan2.run(0)
    plan2.close()
    nsteps2 = args.roof_steps
    phase = {ph: (st2[f"ms_{ph}"] - base[f"ms_{ph}"]) / nsteps2 for ph in
             ("sample", "gram", "recur", "block", "update")}
    t_block = phase["block"] * 1e-3
    hbm_peak, bf16_peak, bf16_sus, src = peaks()
    roof = dense_roofline(args.prec, args.m, args.n, args.b, args.s, t_block, bf16_peak, hbm_peak, src,
                          args.traffic)
    roof["algorithmic"]["launch_ms"] = phase["block"]

    # end to end through the C ABI with host buffers (pinned), copies timed
    if True:
        A_h = torch.from_numpy(p.A).pin_memory()
        y_h = torch.from_numpy(p.y).pin_memory()
        al_h = torch.zeros(args.m, dtype=torch.float64).pin_memory()
        gr_h = torch.zeros(args.m, dtype=torch.float64).pin_memory()
        Hh = args.steps * args.s
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.krr_solve(A_h.numpy(), y_h.numpy(), k, args.lam, args.b, args.s, Hh, seed=rank, prec=args.prec,
                    alpha=al_h.numpy(), grad=gr_h.numpy(), flags=B.FLAG_HOST_IO,
                    stream=torch.cuda.current_stream().cuda_stream)
        dt = time.perf_counter() - t0
        h2d = p.A.nbytes + p.y.nbytes + args.m * 8
        d2h = args.m * 8 * 2
        e2e = {"value": Hh * args.b / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps, "steps": args.steps, "wall_s": dt}

    # the literal order (Algorithms 2 / 4 as printed: the m x sb block stored, U^T alpha read back from
    # it) beside the fused step: time per outer step (one-stream steps, L2 flushed) and bytes moved
    lit = None
    if args.literal_steps > 0:
        def one_stream_ms(flags):
            pl = B.Plan(1, A, y, k, args.lam, args.b, args.s, (args.literal_steps + 4) * args.s, seed=rank,
                        prec=args.prec, flags=flags)
            pl.run(2)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.literal_steps)]
            for e0, e1 in evs:
                flush.zero_()
                e0.record(stream)
                pl.enqueue(1)
                e1.record(stream)
            torch.cuda.synchronize()
            pl.close()
            return sorted(a.elapsed_time(b_) for a, b_ in evs)[len(evs) // 2]
        esz = {"bf16": 2, "tf32": 4, "bf16x3": 4, "tf32x3": 8, "fp8": 1, "fp64": 8, "fp16": 2}[args.prec]
        qsz = 8 if args.prec == "fp64" else 4
        sb = args.s * args.b
        lit = {"ms_per_step_median": one_stream_ms(B.FLAG_LITERAL | B.FLAG_NO_GRAPH),
               "fused_ms_per_step_median_one_stream": one_stream_ms(B.FLAG_NO_GRAPH),
               "bytes_per_step": args.m * args.n * esz + 2 * args.m * sb * qsz + args.m * 16,
               "fused_bytes_per_step": args.m * args.n * esz + args.m * 24,
               "bytes_rule": "literal: A once + the m x sb block written and read back + alpha, g; fused: A once + g, "
                             "alpha, row terms"}
    ttt = None
    if not args.no_ttt:
        ttt = time_to_tol(args, torch, B, A, y, k, rank)
    herr = None
    if rank == 0 and not args.no_cpu and args.err_steps > 0:
        herr = headline_error(args, torch, B, A, y, k, p, rank)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args)

    if rank == 0:
        value = job_rate(args.steps * upd_per_step, ms, ws)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
               "config": {"workload": WORKLOAD, "m": args.m, "n": args.n, "s": args.s, "b": args.b,
                          "gamma": args.gamma, "lambda": args.lam, "precision": args.prec,
                          "step": ("look-ahead, in-order gradient" if args.no_defer
                                   else "look-ahead, deferred gradient (step k+1's recurrence beside step k's block)"),
                          "l2": "256 MB buffer written before every timed step; steps timed alone",
                          "parallelism": "replicas" if ws > 1 else "single"},
               "step_ms": {"min": ms_steps[0], "median": ms_steps[len(ms_steps) // 2], "max": ms_steps[-1]},
               "phase_ms": phase,
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(), "time_to_tol": ttt, "error_vs_oracle": herr, "literal_order": lit}
        if ws == 1 and not args.no_also:
            out["also"] = side_summaries(args)
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------- one kernel block --
def side_summaries(args):
    """The other workloads, measured after the headline's timed region at the
    same --steps (at least 4) with their throughput and roofline only (no CPU
    baseline, no time-to-tolerance, FP8 without its subproblem errors and
    end-to-end run): config 1 (K-SVM blobs, FP64 s = 8), config 3 (K-SVM on
    CSR, block through the transposed copy, the full pass beside it), config 4
    (batched sweep at a fixed budget) and config 5 (FP8 stress).  A workload
    that fails reports its error instead."""
    import copy
    out = {}
    for name, fn, extra in (("ksvm_blobs_fp64", run_gpu_svm, {}),
                            ("ksvm_csr", run_gpu_csr, {"prec": "bf16x3"}),
                            ("krr_sweep", run_gpu_sweep, {"sweep_tol": 0.0}),
                            ("krr_fp8", run_gpu_fp8, {})):
        a = copy.copy(args)
        a.no_cpu, a.no_ttt, a.summary, a.collect, a.s_set = True, True, True, [], False
        a.steps = max(4, args.steps)
        for key, v in extra.items():
            setattr(a, key, v)
        try:
            fn(a)
            line = a.collect[-1]
        except Exception as e:  # keep the headline line whatever happens here
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
            continue
        roof = line.get("roofline") or {}
        ent = {"workload": line["config"]["workload"], "value": line["value"], "unit": line["unit"],
               "ms_per_step": line["ms_per_step"], "dtype": line["dtype"],
               "block_ms": (line.get("phase_ms") or {}).get("block"),
               "roofline": {k: roof.get(k) for k in ("bound", "achieved", "peak", "unit", "frac")},
               "clocks": line.get("clocks")}
        if "moved" in roof:
            ent["roofline"]["moved"] = roof["moved"]
            ent["roofline"]["full_pass"] = roof["full_pass"]
        if "bf16_storage" in line:
            ent["bf16_storage_value"] = line["bf16_storage"]["value"]
        out[name] = ent
    return out


def run_block(args):
    """A few fused kernel-block launches (dcd_kernel_block_apply) at the
    headline shape (m rows, n features, s*b sampled columns, RBF) in one
    precision, "refresh" included: the launch the profiles capture.  Reports
    the launch time (CUDA events, median) against the method's 2 m n s b flops.
    A diagnostic line, not the headline."""
    import torch
    from paper_2406_18001_gb300 import binding as B
    dev = torch.device("cuda", 0)
    p = make_problem(args.m, args.n)
    A = torch.from_numpy(p.A).to(dev)
    g = np.random.default_rng(1)
    nc = args.s * args.b
    cols = torch.from_numpy(g.integers(0, args.m, nc).astype(np.int32)).to(dev)
    w = torch.from_numpy(g.standard_normal(nc)).to(dev)
    gd = torch.zeros(args.m, dtype=torch.float64, device=dev)
    k = B.kernel("rbf", gamma=args.gamma)
    ms = []
    for _ in range(args.block_launches):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.kernel_block_apply(A, k, args.prec, cols, w, gd)  # packs A, then the block: the call, not the kernel
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    flops = 2.0 * args.m * args.n * nc
    med = sorted(ms)[len(ms) // 2]
    print(json.dumps({"metric": "kernel block apply call (pack + block)", "value": flops / (med * 1e-3) / 1e12,
                      "unit": "TFLOP/s (method flops over the whole call)", "prec": args.prec,
                      "config": {"m": args.m, "n": args.n, "ncols": nc}, "ms_per_call": ms}), flush=True)


# --------------------------------------------------------------- K-SVM -----
WORKLOAD_SVM = ("K-SVM-L1 DCD on two Gaussian blobs: m=2000, n=64 (means +-0.5 per coordinate, unit variance), "
                "labels +-1, RBF sigma=8 (gamma=1/128), C=1, FP64 kernel block")


def svm_true_gap(oracle, A64, y, ko, loss, C_, alpha):
    ob = oracle.svm_objectives(A64, y, ko, loss, C_, alpha)
    return (ob["primal"] - ob["dual"]) / abs(ob["primal"])


def svm_time_to_gap(args, torch, B, A, y, k, A64, seed):
    """Time to relative duality gap (P - D) / |P| <= tol (Section 5.1 reading:
    P from w = sum_j alpha_j y_j phi(a_j)): the mixed forms (tensor-core block,
    gradient recomputed by the exact-slice arithmetic before accepting) at
    s = 8 and 64 against the plain FP64 s = 1 form, every solve run to the
    tolerance and timed, each result's gap re-evaluated by the FP64 oracle."""
    import oracle
    ko = oracle.kernel("rbf", gamma=args.svm_gamma)
    runs = {}
    for prec, s in (("fp64", 1), (args.svm_mixed_prec, 8), (args.svm_mixed_prec, 64)):
        flags = B.FLAG_REFRESH if prec != "fp64" else 0
        plan = B.Plan(0, A, y, k, 1.0, 1, s, args.svm_ttg_budget, seed=seed, prec=prec, tol=args.tol,
                      check_every=max(1, 1024 // s), flags=flags, loss=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, _ = plan.run(-1)
        wall = time.perf_counter() - t0
        alpha = plan.alpha.cpu().numpy()
        plan.close()
        gap = svm_true_gap(oracle, A64, y.cpu().numpy(), ko, 1, 1.0, alpha)
        runs[f"{prec}_s{s}"] = {"prec": prec, "s": s, "converged": bool(st["converged"]),
                                "coordinate_updates": st["iters_done"], "ms": st["ms_total"], "wall_s": wall,
                                "gap_solver": st["final_metric"], "gap_fp64": gap, "refreshes": st["refreshes"],
                                "reached_tol_fp64": bool(st["converged"] and gap <= args.tol)}
    base = runs["fp64_s1"]
    ok = {k_: r["ms"] for k_, r in runs.items() if k_ != "fp64_s1" and r["reached_tol_fp64"]}
    best = min(ok, key=ok.get) if ok and base["reached_tol_fp64"] else None
    return {"tol": args.tol, "metric": "relative duality gap (P - D) / |P|", "runs": runs,
            "speedup_measured": base["ms"] / ok[best] if best else None, "speedup_form": best}


def run_gpu_svm(args):
    """Config 1: s-step DCD for the K-SVM-L1 dual on the blobs, FP64, s = 1
    and s = 8 (value: the s = 8 form).  The block is m x s FP64 kernel entries
    per step, so a step is bound by kernel launches and their dependent chain,
    not by memory or arithmetic; the roofline is reported as latency (us per
    outer step against the launch-only floor of the same kernels)."""
    import torch
    from paper_2406_18001_gb300 import binding as B, inputs
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    m, n = args.svm_m, args.svm_n
    gam = args.svm_gamma
    res = {}
    with torch.cuda.stream(stream):
        p = inputs.blobs(m=m, n=n, seed=rank)
        A, y = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.y).to(dev)
        k = B.kernel("rbf", gamma=gam)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        with ClockSampler(local) as clk:
            for s in (1, 8):
                H = (args.warmup + args.steps + 4) * s
                plan = B.Plan(0, A, y, k, 1.0, 1, s, H, seed=rank, prec="fp64", loss=1)
                for _ in range(args.warmup):
                    plan.run(1)
                torch.cuda.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                for i in range(args.steps):
                    flush.zero_()
                    ev[i][0].record(stream)
                    plan.enqueue(1)
                    ev[i][1].record(stream)
                torch.cuda.synchronize()
                ms = rank_max(sum(a.elapsed_time(b_) for a, b_ in ev), ws, dev)
                st, _ = plan.run(0)
                plan.close()
                res[s] = {"ms_per_step": ms / args.steps, "us_per_update": 1e3 * ms / (args.steps * s),
                          "updates_per_s": job_rate(args.steps * s, ms, ws),
                          "kernels_per_step": st["gpu_launches_per_step"]}
        # end to end through the C ABI with host buffers, s = 8, the config's H
        Ah, yh = p.A.copy(), p.y.copy()
        al_h = np.zeros(m)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, st_e, _ = B.svm_solve(Ah, yh, k, 1, 1.0, 8, args.svm_H, seed=rank, prec="fp64", alpha=al_h,
                                    flags=B.FLAG_HOST_IO, stream=stream.cuda_stream)
        dt = time.perf_counter() - t0
        e2e = {"value": args.svm_H / dt, "unit": UNIT, "h2d_bytes_per_step": (Ah.nbytes + yh.nbytes + m * 8),
               "d2h_bytes_per_step": 2 * m * 8, "steps": 1, "wall_s": dt, "H": args.svm_H}
        ttg = None if args.no_ttt else svm_time_to_gap(args, torch, B, A, y, k, p.A, rank)
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        nt = oracle_threads()
        ko = oracle.kernel("rbf", gamma=gam)
        t0 = time.perf_counter()
        done, alpha = 0, np.zeros(m)
        while time.perf_counter() - t0 < 12.0 and done < args.svm_H:
            alpha = oracle.sstep_dcd_svm(p.A, p.y, ko, 1, 1.0, 8, 512, seed=rank, first=done, alpha0=alpha)
            done += 512
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
               "sample": f"{done} of the {args.svm_H} coordinate updates (Algorithm 2, s=8) of the full workload "
                         f"({dt:.1f} s, plain FP64 C, row loops of U_k on {nt} threads)"}
    if rank == 0:
        r8 = res[8]
        roof = {"bound": "latency", "achieved": 1e3 * r8["ms_per_step"], "unit": "us/outer step", "peak": None,
                "frac": None, "traffic": None, "kernels_per_step": r8["kernels_per_step"],
                "kernel": "whole outer step (sample, FP64 Gram, DCD chain, FP64 block, update)",
                "algorithmic": {"flops_per_update": 3.0 * m * n, "bytes_per_step": m * n * 8 + m * 16,
                                "note": "A (1 MB FP64) is L2-resident; the block is 2000 x 8 entries per step"}}
        out = {"metric": METRIC, "value": r8["updates_per_s"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": r8["ms_per_step"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD_SVM, "m": m, "n": n, "s": 8, "gamma": gam, "C": 1.0, "loss": 1,
                          "l2": "256 MB buffer written before every timed step; steps timed alone"},
               "forms": {"s1": res[1], "s8": res[8]}, "time_to_gap": ttg,
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": r8["kernels_per_step"] * args.steps,
               "clocks": clk.summary()}
        emit(out, args)


# ------------------------------------------------------------------ CSR -----
WORKLOAD_CSR = ("K-SVM squared hinge DCD, CSR m=200000 n=50000 50 nnz/row U(0,1) rows unit-norm, "
                "poly (a.b+1)^3, C=0.5, b=1")


def csr_cpu_baseline(p, y, s, budget_s=12.0):
    """The FP64 oracle (s-step DCD, Algorithm 2) on the first m_sub rows, in
    dense form over the columns those rows touch (the oracle is dense); its
    per-update cost is linear in rows x columns, so the rate is scaled by
    (m_sub x n_sub) / (m x n)."""
    import oracle
    nt = oracle_threads()
    m_sub = min(p.m, 500)
    e1 = int(p.row_ptr[m_sub])
    used, col = np.unique(p.col_idx[:e1], return_inverse=True)
    D = np.zeros((m_sub, used.size))
    D[np.repeat(np.arange(m_sub), np.diff(p.row_ptr[:m_sub + 1])), col] = p.values[:e1]
    k = oracle.kernel("poly", coef0=1.0, degree=3)
    H = s
    t0 = time.perf_counter()
    done = 0
    alpha = np.zeros(m_sub)
    while time.perf_counter() - t0 < budget_s and done < 200000:
        alpha = oracle.sstep_dcd_svm(D, y[:m_sub], k, 2, 0.5, s, H, seed=0, first=done, alpha0=alpha)
        done += H
        H = min(4 * H, 4096)
    dt = time.perf_counter() - t0
    scale = (m_sub * used.size) / (p.m * p.n)
    return {"value": done / dt * scale, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{done} DCD updates (s={s}) on the first {m_sub} rows x their {used.size} columns in dense "
                      f"form ({dt:.1f} s, plain FP64 C, row loops on {nt} threads), rate scaled by rows x columns "
                      f"to the full matrix"}


def run_gpu_csr(args):
    """Config 3: throughput of s-step DCD (squared hinge) on the CSR matrix;
    the roofline is HBM bandwidth for the CSR block kernel."""
    import torch
    from paper_2406_18001_gb300 import binding as B, inputs
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    s = args.s if args.s_set else 32
    with torch.cuda.stream(stream):
        p = inputs.sparse_csr(m=args.csr_m, n=args.csr_n, nnz_per_row=args.csr_nnz, seed=rank)
        A = B.Csr(torch.from_numpy(p.row_ptr).to(dev), torch.from_numpy(p.col_idx).to(dev),
                  torch.from_numpy(p.values).to(dev), p.n)
        y = torch.from_numpy(p.y).to(dev)
        k = B.kernel("poly", coef0=1.0, degree=3)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        H = (args.warmup + args.steps + 8) * s
        plan = B.Plan(0, A, y, k, 0.5, 1, s, H, seed=rank, prec=args.prec, loss=2)
        for _ in range(args.warmup):
            plan.run(1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                plan.enqueue(1)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        ms = rank_max(ms, ws, dev)
        st, _ = plan.run(0)
        launches = st["gpu_launches_per_step"] * args.steps
        plan.close()
        def phases(flags):
            pl = B.Plan(0, A, y, k, 0.5, 1, s, (args.roof_steps + 4) * s, seed=rank + 1, prec=args.prec, loss=2,
                        flags=B.FLAG_PHASE_TIMERS | flags)
            pl.run(2)
            base, _ = pl.run(0)
            for _ in range(args.roof_steps):
                flush.zero_()
                pl.run(1)
            st2, _ = pl.run(0)
            pl.close()
            return {ph: (st2[f"ms_{ph}"] - base[f"ms_{ph}"]) / args.roof_steps for ph in
                    ("sample", "gram", "recur", "block", "update")}

        phase = phases(0)
        phase_full = phases(B.FLAG_CSR_FULL_PASS)
        fp64 = args.prec == "fp64"
        roof = csr_roofline(p, s, fp64, phase["block"], phase_full["block"])
        # end to end through the C ABI with host arrays
        Ah = B.Csr(p.row_ptr, p.col_idx, p.values, p.n)
        yh = p.y.copy()
        al_h = np.zeros(p.m)
        Hh = args.steps * s
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.svm_solve(Ah, yh, k, 2, 0.5, s, Hh, seed=rank, prec=args.prec, alpha=al_h, flags=B.FLAG_HOST_IO,
                    stream=stream.cuda_stream)
        dt = time.perf_counter() - t0
        h2d = p.row_ptr.nbytes + p.col_idx.nbytes + p.values.nbytes + p.y.nbytes + p.m * 8
        e2e = {"value": Hh / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": 2 * p.m * 8 / args.steps, "steps": args.steps, "wall_s": dt}
    cpu = None if args.no_cpu else csr_cpu_baseline(p, p.y, s)
    if rank == 0:
        value = job_rate(args.steps * s, ms, ws)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD_CSR, "m": p.m, "n": p.n, "nnz_per_row": args.csr_nnz, "s": s, "b": 1,
                          "precision": args.prec + (" (CSR block: FP64)" if fp64 else " (CSR block: FP32 CUDA cores)"),
                          "l2": "256 MB buffer written before every timed step; steps timed alone"},
               "phase_ms": phase, "phase_ms_full_pass": phase_full, "roofline": roof, "cpu_baseline": cpu,
               "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary()}
        emit(out, args)


def csr_roofline(p, s, fp64, t_block, t_full):
    """The CSR kernel block against HBM.  The full pass's algorithmic bytes
    per outer step are one read of every column index and value of A, its
    row offsets, and g read and written with y read (nnz (4 + 4|8) + (m + 1) 8
    + m 24).  The block runs through the transposed copy, which reads only the
    incidences: for each sampled row j and column c it holds, the entries of
    column c (expected s (nnz / m) sum_c nnz_c^2 / nnz of them); each costs
    its CSC row index twice (count, scatter), element index and value once,
    and its key and product written and read back (4 + 4 + 8 + v + 2 (8 + v)
    bytes), plus per row the offsets, g read and written and y (32 bytes).
    `achieved` is the full pass's bytes over the transposed block's time (the
    effective rate); `moved` is the transposed block's own bytes over its time;
    `full_pass` times the full pass (forced) on the same steps."""
    hbm_peak, _, _, src = peaks()
    nnz, m = int(p.row_ptr[-1]), p.m
    vb = 8 if fp64 else 4
    full_bytes = nnz * (4 + vb) + (m + 1) * 8 + m * 24
    cnt = np.bincount(p.col_idx, minlength=p.n).astype(np.float64)
    inc = min(s, 32) * (nnz / m) * float(np.sum(cnt * cnt)) / nnz * (-(-s // 32))
    moved = inc * (4 + 4 + 8 + vb + 2 * (8 + vb)) + m * 32
    eff = full_bytes / (t_block * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": eff, "peak": hbm_peak, "unit": "GB/s", "frac": eff / hbm_peak,
            "traffic": None, "peak_source": src,
            "kernel": "CSR kernel block + gradient update through the transposed copy (csc_count, csc_scatter, "
                      "csc_apply per 32 sampled columns)",
            "algorithmic": {"bytes_per_launch": full_bytes, "launch_ms": t_block,
                            "rule": "the full pass's bytes (every column index and value, offsets, g r/w, y) over "
                                    "the transposed block's time: its effective rate"},
            "moved": {"bytes_per_launch": moved, "expected_incidences": inc,
                      "achieved": moved / (t_block * 1e-3) / 1e9, "frac": moved / (t_block * 1e-3) / 1e9 / hbm_peak},
            "full_pass": {"launch_ms": t_full, "achieved": full_bytes / (t_full * 1e-3) / 1e9,
                          "frac": full_bytes / (t_full * 1e-3) / 1e9 / hbm_peak}}


# ------------------------------------------------------------ FP8 stress -----
WORKLOAD_FP8 = ("K-RR precision stress: m=400000, n=2048 dense, A = Z diag(sig) W^T (sig log-spaced, cond 1e4, "
                "E||a||^2 = 64) stored BF16 and as FP8 e4m3 with per-row scales, y = sin(A w) + 0.1 N(0,1), "
                "RBF sigma=8, lambda=1e-6, b=32, s=128")


def _fp8_arm(B, torch, A, y, k, lam, b, s, prec, args, stream, flush, seed):
    """Throughput of one storage / precision arm: K timed outer steps, then
    the per-phase device times from a second plan with phase timers."""
    H = (args.warmup + args.steps + 4) * s
    plan = B.Plan(1, A, y, k, lam, b, s, H, seed=seed, prec=prec)
    for _ in range(args.warmup):
        plan.run(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        plan.enqueue(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b_) for a, b_ in ev)
    ms = rank_max(ms, dist_env()[0], torch.device("cuda", torch.cuda.current_device()))
    st, _ = plan.run(0)
    plan.close()
    nroof = max(3, min(args.roof_steps, 10))
    plan2 = B.Plan(1, A, y, k, lam, b, s, (nroof + 3) * s, seed=seed + 1, prec=prec, flags=B.FLAG_PHASE_TIMERS)
    plan2.run(1)
    base, _ = plan2.run(0)
    for _ in range(nroof):
        flush.zero_()
        plan2.run(1)
    st2, _ = plan2.run(0)
    plan2.close()
    phase = {ph: (st2[f"ms_{ph}"] - base[f"ms_{ph}"]) / nroof for ph in ("sample", "gram", "recur", "block", "update")}
    return ms, st["gpu_launches_per_step"] * args.steps, phase


def run_gpu_fp8(args):
    """Config 5: the K-RR stress configuration.  Throughput of FP8 storage
    (kind::f8f6f4 block) and BF16 storage (kind::f16 block) at m = 400000,
    n = 2048, b = 32, s = 128; alpha error on rows 0..19999 against the FP64
    oracle (same index stream, fixed H) and against the FP64 GPU path."""
    import torch
    from paper_2406_18001_gb300 import binding as B, inputs
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    m, n, b = args.fp8_m, args.fp8_n, 32
    s = args.s if args.s_set else 128
    gam, lam = 1.0 / 128, 1e-6
    summary = getattr(args, "summary", False)  # a side summary of the default line: throughput only
    k = B.kernel("rbf", gamma=gam)
    with torch.cuda.stream(stream):
        # the stored matrices, generated on the device from the seeded recipe
        mix = torch.from_numpy(inputs.ill_conditioned_mixer(n, seed=rank)).to(dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(5000 + rank)
        w = torch.randn(n, generator=gen, device=dev, dtype=torch.float32) / 8.0  # A w ~ N(0, 1)
        A16 = torch.empty((m, n), dtype=torch.bfloat16, device=dev)
        y = torch.empty(m, dtype=torch.float64, device=dev)
        for r0 in range(0, m, 65536):
            r1 = min(m, r0 + 65536)
            Z = torch.randn((r1 - r0, n), generator=gen, device=dev, dtype=torch.float32)
            A16[r0:r1] = (Z @ mix).to(torch.bfloat16)
            y[r0:r1] = torch.sin(A16[r0:r1].float() @ w).double() + 0.1 * torch.randn(
                r1 - r0, generator=gen, device=dev, dtype=torch.float64)
        del Z
        F = B.quantize_e4m3(A16, stream=stream.cuda_stream)  # FP8 storage of the BF16 matrix
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ms8, launches, ph8 = _fp8_arm(B, torch, F, y, k, lam, b, s, "fp8", args, stream, flush, rank)
        ms16, _, ph16 = _fp8_arm(B, torch, A16, y, k, lam, b, s, "bf16", args, stream, flush, rank)

        e2e = None
        if not summary:
            # end to end through the C ABI with host buffers (FP8 codes, scales, y)
            q_h = F.codes.cpu().pin_memory()
            sc_h = F.scale.cpu().pin_memory()
            y_h = y.cpu().pin_memory()
            al_h = torch.zeros(m, dtype=torch.float64).pin_memory()
            gr_h = torch.zeros(m, dtype=torch.float64).pin_memory()
            Hh = args.steps * s
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.krr_solve(B.Fp8(q_h.numpy(), sc_h.numpy()), y_h.numpy(), k, lam, b, s, Hh, seed=rank, prec="fp8",
                        alpha=al_h.numpy(), grad=gr_h.numpy(), flags=B.FLAG_HOST_IO, stream=stream.cuda_stream)
            dt = time.perf_counter() - t0
            e2e = {"value": Hh * b / dt, "unit": UNIT, "h2d_bytes_per_step": (m * n + 4 * m + 16 * m) / args.steps,
                   "d2h_bytes_per_step": 16 * m / args.steps, "steps": args.steps, "wall_s": dt}
            del q_h, sc_h

        if not summary:
            # alpha error on the 20000-row subproblem (rows 0..19999 of the stored matrix)
            msub = min(m, args.fp8_sub)
            Asub16 = A16[:msub].contiguous()
            ysub = y[:msub].contiguous()
            Fsub = B.quantize_e4m3(Asub16, stream=stream.cuda_stream)
            Hs = args.fp8_oracle_blocks
            Hl = args.fp8_long_steps * s
            err = {}
            ref_long = {}
            for tag, Am, prec in (("fp64_on_bf16", Asub16, "fp64"), ("fp64_on_fp8", Fsub, "fp64")):
                ref_long[tag] = B.krr_solve(Am, ysub, k, lam, b, s, Hl, seed=7, prec="fp64")[0].cpu().numpy()
            arms = {}
            for tag, Am, prec in (("fp8", Fsub, "fp8"), ("bf16", Asub16, "bf16"), ("fp64_on_bf16", Asub16, "fp64"),
                                  ("fp64_on_fp8", Fsub, "fp64")):
                arms[tag] = (B.krr_solve(Am, ysub, k, lam, b, s, Hs, seed=7, prec=prec)[0].cpu().numpy(),
                             B.krr_solve(Am, ysub, k, lam, b, s, Hl, seed=7, prec=prec)[0].cpu().numpy())
            torch.cuda.synchronize()
            A_sub_h = Asub16.float().cpu().numpy().astype(np.float64)
            y_sub_h = ysub.cpu().numpy()

    def rel(a, b_):
        return float(np.linalg.norm(a - b_) / np.linalg.norm(b_))

    out_err = None
    cpu = None
    if rank == 0:
        if not summary:
            out_err = {"rows": msub, "seed": 7,
                       "long_H_blocks": Hl,
                       "vs_fp64_gpu_long": {"fp8_vs_fp64_on_fp8_data": rel(arms["fp8"][1], ref_long["fp64_on_fp8"]),
                                            "bf16_vs_fp64_on_bf16_data": rel(arms["bf16"][1], ref_long["fp64_on_bf16"]),
                                            "fp8_storage_vs_bf16_storage_fp64": rel(ref_long["fp64_on_fp8"],
                                                                                    ref_long["fp64_on_bf16"]),
                                            "fp8_vs_fp64_on_bf16_data": rel(arms["fp8"][1], ref_long["fp64_on_bf16"])}}
            if not args.no_cpu:
                import oracle
                nt = oracle_threads()
                ko = oracle.kernel("rbf", gamma=gam)
                t0 = time.perf_counter()
                want = oracle.bdcd_krr(A_sub_h, y_sub_h, ko, lam, b, Hs, seed=7)
                t_or = time.perf_counter() - t0
                out_err["oracle_H_blocks"] = Hs
                out_err["vs_oracle"] = {t: rel(arms[t][0], want) for t in arms}
                out_err["vs_oracle_note"] = ("oracle = FP64 BDCD (Algorithm 3) on the BF16-stored rows; fp64_on_fp8 and "
                                             "fp8 differ from it by the FP8 storage")
                upd = Hs * b
                cpu = {"value": upd / t_or * msub / m, "unit": UNIT, "cores": nt, "kind": "oracle",
                       "sample": f"{Hs} BDCD block updates (b={b}) on rows 0..{msub - 1} ({t_or:.1f} s, plain FP64 C, "
                                 f"row loops on {nt} threads), rate scaled by rows to m={m}"}
        hbm_peak, bf16_peak, bf16_sus, src = peaks()
        sb = s * b
        flops = 2.0 * m * n * sb
        fp8_peak = 2.0 * bf16_peak
        # DRAM bytes of one launch from the m = 65536 capture of the same kernel source, scaled by rows (the
        # 8.4 MB of sampled rows fixed); null once the kernel source has changed since the capture
        traffic = ((158.56e6 - 8.4e6) * m / 65536 + 8.4e6
                   if (n, s, b) == (2048, 128, 32) and kernel_source_sha16() == "2bec218b23016340" else None)
        roof = {"bound": "tensor", "achieved": flops / (ph8["block"] * 1e-3) / 1e12, "peak": fp8_peak,
                "unit": "TFLOP/s", "traffic": traffic,
                "peak_source": f"{src} bf16 burst x 2 (nominal fp8 / bf16 dense ratio 4.5 / 2.25)",
                "kernel": "block_tc2_kernel<MODE_FP8> (kind::f8f6f4 kernel block + gradient update, CTA pairs)",
                "algorithmic": {"flops_per_launch": flops, "launch_ms": ph8["block"]}}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof16 = {"achieved": flops / (ph16["block"] * 1e-3) / 1e12, "peak": bf16_peak, "unit": "TFLOP/s"}
        roof16["frac"] = roof16["achieved"] / bf16_peak
        value = job_rate(args.steps * s * b, ms8, ws)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms8 / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "fp8-e4m3", "data": "synthetic",
               "config": {"workload": WORKLOAD_FP8, "m": m, "n": n, "b": b, "s": s, "gamma": gam, "lambda": lam,
                          "precision": "fp8 (per-row-scaled e4m3, kind::f8f6f4, FP32 accumulation)",
                          "l2": "A (0.82 GB FP8 / 1.64 GB BF16) above L2; 256 MB buffer written before every step"},
               "phase_ms": ph8,
               "bf16_storage": {"value": job_rate(args.steps * s * b, ms16, ws), "ms_per_step": ms16 / args.steps,
                                "phase_ms": ph16, "roofline": roof16},
               "alpha_error": out_err,
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary()}
        emit(out, args)


# ---------------------------------------------------------------- sweep -----
WORKLOAD_SWEEP = ("batched K-RR sweep: 256 BDCD solves, m ~ U[1000, 20000], n=128, A, y ~ N(0,1), RBF sigma on a "
                  "log grid [0.1, 10] x lambda on a log grid [1e-6, 1e-1], b alternating 8 / 32, s autotuned")


def run_gpu_sweep(args):
    """Config 4: every problem runs a fixed budget of block updates in one
    bdcd_krr_solve_batched call (s from the autotuner, measured once in a
    first call); value = coordinate updates of all problems / wall time of
    the call, whose steps replay one CUDA graph over 16 streams."""
    import torch
    from paper_2406_18001_gb300 import binding as B, inputs
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    count = args.sweep_count
    grid = inputs.sweep_grid(count)
    with torch.cuda.stream(stream):
        probs = []
        for p in range(count):
            pr = inputs.sweep_problem(p + 1000 * rank)
            sig, lam = grid[p % len(grid)]
            probs.append(dict(A=torch.from_numpy(pr.A).to(dev), y=torch.from_numpy(pr.y).to(dev),
                              k=B.kernel("rbf", gamma=1.0 / (2 * sig * sig)), lam=lam, b=8 if p % 2 == 0 else 32,
                              s=args.sweep_s if args.sweep_s else 0, H=args.sweep_H, seed=p))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, st0, _ = B.krr_solve_batched(probs, prec=args.prec, stream=stream.cuda_stream)  # autotune + warm-up
        t_first = time.perf_counter() - t0
        for p, st in zip(probs, st0):
            p["s"] = int(st["s_used"])
            p.pop("alpha", None)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            _, _, sts, _ = B.krr_solve_batched(probs, prec=args.prec, streams=args.sweep_streams,
                                               stream=stream.cuda_stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        # the same solves one after another (bdcd_krr_solve each), for the batching gain
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p in probs:
            B.krr_solve(p["A"], p["y"], p["k"], p["lam"], p["b"], p["s"], p["H"], seed=p["seed"], prec=args.prec,
                        stream=stream.cuda_stream)
        torch.cuda.synchronize()
        wall_seq = time.perf_counter() - t0
        # end to end: pinned host inputs in, the batched call, every alpha back
        host = []
        for p in range(count):
            pr = inputs.sweep_problem(p + 1000 * rank)
            host.append((torch.from_numpy(pr.A).pin_memory(), torch.from_numpy(pr.y).pin_memory()))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p, (Ah, yh) in zip(probs, host):
            p["A"] = Ah.to(dev, non_blocking=True)
            p["y"] = yh.to(dev, non_blocking=True)
        al_e2e, _, _, _ = B.krr_solve_batched(probs, prec=args.prec, stream=stream.cuda_stream)
        al_h = [a.to("cpu", non_blocking=True) for a in al_e2e]
        torch.cuda.synchronize()
        wall_e2e = time.perf_counter() - t0
        h2d = sum(Ah.nbytes + yh.nbytes for Ah, yh in host)
        d2h = sum(a.numel() * 8 for a in al_h)
        # every problem to relative residual tol with an epoch cap, the gradient recomputed (exact-slice
        # products) before a problem is accepted; a sample of the results checked by an FP64 residual
        conv = None
        if args.sweep_tol > 0:
            cprobs = [dict(p, H=args.sweep_epochs * p["A"].shape[0] // p["b"]) for p in probs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cal, _, cst, _ = B.krr_solve_batched(cprobs, prec=args.prec, tol=args.sweep_tol, check_every=4,
                                                 flags=B.FLAG_REFRESH, streams=args.sweep_streams,
                                                 stream=stream.cuda_stream)
            torch.cuda.synchronize()
            wall_c = time.perf_counter() - t0
            chk = [i for i in range(count) if cst[i]["converged"]][:: max(1, count // 8)][:8]
            res = [fp64_residual(B, torch, cprobs[i]["A"], cprobs[i]["y"], cal[i], cprobs[i]["k"], cprobs[i]["lam"])
                   for i in chk]
            conv = {"tol": args.sweep_tol, "epoch_cap": args.sweep_epochs, "problems": count,
                    "converged": sum(int(x["converged"]) for x in cst), "wall_s": wall_c,
                    "coordinate_updates": sum(int(x["iters_done"]) * p["b"] for x, p in zip(cst, cprobs)),
                    "refreshes": sum(int(x["refreshes"]) for x in cst),
                    "unconverged": [{"sigma": grid[i % len(grid)][0], "lambda": grid[i % len(grid)][1],
                                     "m": cprobs[i]["A"].shape[0], "b": cprobs[i]["b"],
                                     "final_metric": cst[i]["final_metric"]}
                                    for i in range(count) if not cst[i]["converged"]][:16],
                    "fp64_resid_checked": {"problems": chk, "max": max(res) if res else None}}
    upd = sum(int(st["iters_done"]) * p["b"] for st, p in zip(sts, probs))
    wall = rank_max(wall, ws, dev)  # the job's times are its slowest replica's
    wall_e2e = rank_max(wall_e2e, ws, dev)
    launches = sum(int(st["gpu_launches_per_step"]) * int(st["outer_steps"]) for st in sts)
    # roofline of the whole call on the method's work: every outer step is one fused block of 2 m n sb
    # flops that reads its problem's packed operand once (the split forms' extra MMA passes apart)
    n_sw = 128
    esz = {"bf16": 2, "tf32": 4, "bf16x3": 4, "tf32x3": 8, "fp8": 1, "fp64": 8, "fp16": 2}[args.prec]
    mult = 3 if args.prec in ("bf16x3", "tf32x3") else 1
    flops = sum(int(st["outer_steps"]) * 2.0 * p["A"].shape[0] * n_sw * p["s"] * p["b"]
                for st, p in zip(sts, probs))
    bytes_ = sum(int(st["outer_steps"]) * (p["A"].shape[0] * (n_sw * esz + 20) + p["s"] * p["b"] * n_sw * esz)
                 for st, p in zip(sts, probs))
    hbm_peak, bf16_peak, _, src = peaks()
    tc_peak = {"bf16": 1.0, "bf16x3": 1.0, "fp16": 1.0, "fp8": 2.0, "tf32": 1.1 / 2.25,
               "tf32x3": 1.1 / 2.25}.get(args.prec, 0.0) * bf16_peak
    roof = {"bound": "tensor", "achieved": flops / wall / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
            "frac": flops / wall / 1e12 / tc_peak if tc_peak else None, "traffic": None, "peak_source": src,
            "kernel": "whole batched call (all problems' steps)",
            "algorithmic": {"flops": flops, "flops_rule": "sum over steps of 2*m*n*s*b (method flops)",
                            "bytes": bytes_, "hbm_gbs": bytes_ / wall / 1e9, "wall_s": wall},
            "mma_pipe": {"mma_per_k_step": mult, "flops": flops * mult,
                         "frac": flops * mult / wall / 1e12 / tc_peak if tc_peak else None}}
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = sweep_cpu_baseline(probs, upd)
    e2e = {"value": job_rate(upd, wall_e2e * 1e3, ws), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "steps": 1, "wall_s": wall_e2e}
    s_hist = {}
    for p in probs:
        s_hist[f"b{p['b']}_s{p['s']}"] = s_hist.get(f"b{p['b']}_s{p['s']}", 0) + 1
    if rank == 0:
        out = {"metric": METRIC, "value": job_rate(upd, wall * 1e3, ws), "unit": UNIT, "n_gpus": ws, "steps": 1,
               "warmup": 1, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
               "config": {"workload": WORKLOAD_SWEEP, "problems": count, "H_block_updates": args.sweep_H,
                          "precision": args.prec, "streams": args.sweep_streams, "rounds_per_graph": 8,
                          "l2": "problems total ~0.65 GB of A (above L2); one timed batched call"},
               "sweep": {"coordinate_updates": upd, "wall_s": wall, "sequential_single_solves_wall_s": wall_seq,
                         "first_call_with_autotune_s": t_first,
                         "s_chosen": s_hist, "to_tolerance": conv},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary()}
        emit(out, args)


def sweep_cpu_baseline(probs, upd_total, nsample=8, budget_s=15.0):
    """The FP64 oracle (Algorithm 3, one thread) on a few of the sweep's
    problems for a bounded time; a block update costs ~ m * n * b, so the
    rate is measured as m * coordinate updates per second and the whole
    sweep's time estimated from it."""
    import oracle
    nt = oracle_threads()
    idx = np.linspace(0, len(probs) - 1, nsample).astype(int)
    work = 0.0
    t0 = time.perf_counter()
    for i in idx:
        p = probs[i]
        A = p["A"].cpu().numpy().astype(np.float64)
        y = p["y"].cpu().numpy()
        k = oracle.kernel("rbf", gamma=p["k"].gamma)
        blocks = max(1, int(2.4e9 / (A.shape[0] * A.shape[1] * p["b"])))  # ~ the same work per sampled problem
        oracle.bdcd_krr(A, y, k, p["lam"], p["b"], blocks, seed=p["seed"])
        work += A.shape[0] * blocks * p["b"]
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    rate_mu = work / dt  # m * coordinate updates per second
    total_mu = sum(p["A"].shape[0] * p["H"] * p["b"] for p in probs)
    return {"value": upd_total / (total_mu / rate_mu), "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"Algorithm 3 on {len(idx)} of the {len(probs)} problems ({dt:.1f} s, plain FP64 C, row "
                      f"loops on {nt} threads); the whole sweep's time estimated from the measured m x updates "
                      f"per second"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=50000)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--s", type=int, default=None)
    ap.add_argument("--workload", default="krr", choices=["krr", "svm", "csr", "sweep", "fp8", "block"],
                    help="krr: dense K-RR BDCD (the headline); svm: K-SVM-L1 DCD on the blobs; csr: sparse K-SVM "
                         "DCD; sweep: batched K-RR; fp8: the FP8 / BF16 storage stress configuration")
    ap.add_argument("--block-launches", type=int, default=4, help="block workload: apply calls")
    ap.add_argument("--svm-m", type=int, default=2000)
    ap.add_argument("--svm-n", type=int, default=64)
    ap.add_argument("--svm-gamma", type=float, default=1.0 / 128, help="RBF gamma = 1/(2 sigma^2), sigma = 8")
    ap.add_argument("--svm-H", type=int, default=20000, help="coordinate updates of the end-to-end solve")
    ap.add_argument("--svm-ttg-budget", type=int, default=2000000, help="coordinate-update cap of the gap solves")
    ap.add_argument("--svm-mixed-prec", default="bf16x3")
    ap.add_argument("--sweep-count", type=int, default=256)
    ap.add_argument("--sweep-H", type=int, default=2048, help="block updates per problem")
    ap.add_argument("--sweep-s", type=int, default=0, help="fixed s for every problem (0: the autotuner's)")
    ap.add_argument("--sweep-streams", type=int, default=16, help="worker streams of the batched call")
    ap.add_argument("--sweep-tol", type=float, default=1e-6, help="relative residual of the converging sweep (0: skip)")
    ap.add_argument("--sweep-epochs", type=int, default=200, help="epoch cap per problem of the converging sweep")
    ap.add_argument("--fp8-m", type=int, default=400000)
    ap.add_argument("--fp8-n", type=int, default=2048)
    ap.add_argument("--fp8-sub", type=int, default=20000, help="rows of the alpha-error subproblem")
    ap.add_argument("--fp8-oracle-blocks", type=int, default=32, help="block updates the oracle runs (about 28 s of one core)")
    ap.add_argument("--fp8-long-steps", type=int, default=20, help="outer steps of the GPU-only comparison")
    ap.add_argument("--csr-m", type=int, default=200000)
    ap.add_argument("--csr-n", type=int, default=50000)
    ap.add_argument("--csr-nnz", type=int, default=50)
    ap.add_argument("--b", type=int, default=16)
    ap.add_argument("--gamma", type=float, default=0.5)
    ap.add_argument("--lam", type=float, default=1e-4)
    ap.add_argument("--prec", default="fp16",
                    choices=["bf16", "tf32", "bf16x3", "tf32x3", "fp8", "fp64", "refresh", "fp16"])
    ap.add_argument("--roof-steps", type=int, default=50)
    ap.add_argument("--traffic", type=float, default=None, help="dram bytes per launch from an ncu capture")
    ap.add_argument("--no-defer", action="store_true",
                    help="time the look-ahead steps with the in-order gradient (each recurrence after the "
                         "previous step's block)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance solves")
    ap.add_argument("--no-also", action="store_true",
                    help="default workload: skip the side summaries of the other configurations")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--ttt-budget", type=int, default=400000, help="block-update cap of the tolerance solve")
    ap.add_argument("--ttt-small-m", type=int, default=6000,
                    help="rows of the subproblem on which both forms run to tolerance (0: skip)")
    ap.add_argument("--literal-steps", type=int, default=10,
                    help="outer steps timed in the literal order beside the fused step (0: skip)")
    ap.add_argument("--err-steps", type=int, default=2,
                    help="outer steps of the headline compared with the oracle (0: skip)")
    ap.add_argument("--ttt-fp64-steps", type=int, default=200)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.s_set = args.s is not None
    if args.s is None:
        args.s = 64
    if args.impl != "reference":
        # a plan captures its step graphs in its first steps (one per buffer set, up to three, each
        # after one direct run of that set): the warm-up covers them
        args.warmup = max(args.warmup, 8)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "svm":
        run_gpu_svm(args)
    elif args.workload == "block":
        run_block(args)
    elif args.workload == "csr":
        run_gpu_csr(args)
    elif args.workload == "sweep":
        run_gpu_sweep(args)
    elif args.workload == "fp8":
        run_gpu_fp8(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
