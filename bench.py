#!/usr/bin/env python
"""Benchmark of the SpTRSV hot path on GB300.

Workload (one step): 512 independent lower-triangular CSR systems (n log-
uniform in [1e3, 2e5], band log-uniform in [16, 1024], 4-16 off-diagonals
per row, FP32 values, 1-32 right-hand sides, odd-indexed systems rewritten
by the narrowest-level rule with chunks of 8 levels); one step is the
batched forward solve x = L^{-1} (b [+ T b]) plus its adjoint: transpose
solve g_b' = L^{-T} w, T^T application and the value gradient on L's
pattern.  Analysis and rewriting are the preprocessing step of the method
(done once, timed and reported separately).

Printed (rank 0): ONE JSON line with value = algorithmic GB/s of the whole
step over all ranks, the dominant kernel's roofline, the plain level-set
baseline (one launch per level, per system, original DAG), a single-system
section (2D Laplacian 1024^2) and the CPU oracle timed on the host.
``--impl reference`` times the CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "SpTRSV GB/s & % HBM peak: batched fwd+adjoint vs plain level-set solve"
WORKLOAD = ("batch512: 512 banded lower-triangular CSR systems, n~logU[1e3,2e5], "
            "band~logU[16,1024], 4-16 offdiag/row, FP32, 1-32 RHS; odd systems rewritten "
            "(narrowest-level 1%, D=8); step = batched fwd solve + adjoint "
            "(transpose solve, T^T, value gradient)")
FALLBACK_HBM = 6800.0


def workload_name(args):
    """The workload string of the JSON line (the benchmark's, unless the
    batch was resized for a profiling run)."""
    w = WORKLOAD
    if args.nmat != 512:
        w = w.replace("batch512: 512 ", f"batch{args.nmat}: {args.nmat} ")
    if args.n_hi != 200_000:
        w = w.replace("n~logU[1e3,2e5]", f"n~logU[1e3,{args.n_hi}]")
    return w


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nmat", type=int, default=512)
    ap.add_argument("--n-hi", type=int, default=200_000,
                    help="largest system of the batch (rows); smaller values give a still contended "
                         "batch small enough for a full profiler capture")
    ap.add_argument("--split", action="store_true",
                    help="split ONE batch over the ranks (shard.partition, strong scaling) instead of "
                         "one batch per rank (weak scaling)")
    ap.add_argument("--no-extras", action="store_true", help="skip baseline/single/cpu legs")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--ncu", action="store_true", help="minimal run for a profiler launch list")
    ap.add_argument("--profile-single", type=int, default=0, metavar="N",
                    help="profiling run only: level analysis, level-persistent and sync-free solves "
                         "(FP64, 1 RHS) of the N x N 2D Laplacian, 3 times each; prints timings")
    return ap.parse_args()


def profile_single(N):
    """A small single-system case for a profiler: the kernels of the level
    analysis, the level-persistent, the sync-free and the hybrid solve on the
    N x N 2D Laplacian (2N-1 levels), each run 3 times after one warm-up."""
    import torch
    import paper_2609_40159_gb300 as P
    from paper_2609_40159_gb300 import autotune
    A = P.Matrix.from_host(S.lap2d(N))
    b = torch.as_tensor(S.rhs(A.n, 1, seed=1)).cuda()
    x = torch.empty_like(b)
    out = {"n": A.n, "levels": 2 * N - 1}
    out["analyze_ms"] = autotune.time_call(lambda: P.analyze(A), reps=3, warmup=1)
    plan = P.Plan(A)
    for mode in ("level", "syncfree", "hybrid"):
        plan.set(mode, 4 if mode == "hybrid" else 32, 1)
        ms = autotune.time_call(lambda: plan.solve(b, out=x), reps=3, warmup=1)
        out[mode] = {"ms": ms, "us_per_level": 1e3 * ms / (2 * N - 1)}
    if P.handle().status() != 0:
        raise RuntimeError("device status after the profiling run")
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ bytes
def bytes_fwd(n, nnz, k, wv, tn=0, tnnz=0):
    """Algorithmic bytes of one forward solve: L once (values + column
    indices + row pointers), b read, x written (x gathers assumed cached),
    plus T for a rewritten system."""
    b = nnz * (wv + 4) + (n + 1) * 4 + 2 * n * k * wv
    if tn:
        b += tnnz * (wv + 4) + (tn + 1) * 4
    return b


def bytes_bwd(n, nnz, k, wv, tn=0, tnnz=0):
    """Transpose solve (L^T once, g_x read, g_b' written), value gradient
    (column indices, row pointers, g_b' and x read, gradient written) and,
    for a rewritten system, T^T (T once, g_b' read, g_b written)."""
    b = nnz * (wv + 4) + (n + 1) * 4 + 2 * n * k * wv
    b += nnz * 4 + (n + 1) * 4 + 2 * n * k * wv + nnz * wv
    if tn:
        b += tnnz * (wv + 4) + (tn + 1) * 4 + 2 * n * k * wv
    return b


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_source_hash():
    """sha256 of the batched solve kernel's sources with comments and blank
    lines removed: the DRAM traffic recorded in profiles/traffic.json is used
    only while the code it was measured on is unchanged."""
    import hashlib
    import re
    h = hashlib.sha256()
    for fn in ("block.cuh", "batch.cu", "rows.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2609_40159_gb300", "csrc", fn)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()


# ----------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "yes", "1"):
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None,
                    sm_max_mhz=float(max(mx)) if mx else None,
                    samples=len(sm), reasons=sorted(reasons))


# ------------------------------------------------------------- reference
def run_reference(args, items, rank):
    """The CPU oracle on the same workload: every step is a bounded sample
    (a rotating slice of the systems) of fwd solve + adjoint in FP64."""
    import oracle
    nmat = len(items)
    per = max(1, nmat // 8)
    wv = 4
    prepared = []
    for m, it in enumerate(items):
        A = S.CSR(it.A.n, it.A.row_ptr, it.A.col_idx, it.A.vals.astype(np.float64))
        prepared.append(A)

    def step(s):
        ms = [(s * per + q) % nmat for q in range(per)]
        t0 = time.perf_counter()
        nb = 0
        for m in ms:
            A, it = prepared[m], items[m]
            x = oracle.solve(A, it.b)
            g = oracle.solve_transpose(A, it.b)
            oracle.grad_vals(A, g, x)
            nb += bytes_fwd(A.n, A.nnz, it.nrhs, wv) + bytes_bwd(A.n, A.nnz, it.nrhs, wv)
        return time.perf_counter() - t0, nb

    for s in range(args.warmup):
        step(s)
    tt, bb = 0.0, 0
    for s in range(args.steps):
        t, b = step(args.warmup + s)
        tt += t
        bb += b
    gbs = bb / tt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "reference": "CPU oracle (no reference code exists)"},
        "cpu_baseline": {"kind": "oracle", "value": gbs, "unit": "GB/s", "cores": 1,
                         "sample": f"{per} of {nmat} systems per step (rotating), fwd + transpose "
                                   "solve + value gradient, FP64 on widened FP32 values"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours
def build_batch(P, items, dev):
    """Device systems (rewrites of the marked ones), packed RHS."""
    import torch
    t_an = t_rw = 0.0
    mats, Ts, levels = [], [], []
    for it in items:
        A = P.Matrix.from_host(it.A, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        an = P.analyze(A)
        t_an += time.perf_counter() - t0
        lv = [an.nlevels, an.nlevels]
        T = None
        if it.rewritten:
            t0 = time.perf_counter()
            rows, tg = S.narrowest_levels_list(an.nlevels, an.level_ptr.cpu().numpy(),
                                               an.perm.cpu().numpy(), 0.01, 8)
            A2, T = P.rewrite(A, an.lev, rows, tg)
            t_rw += time.perf_counter() - t0
            lv[1] = P.analyze(A2).nlevels
            A = A2
        mats.append(A)
        Ts.append(T)
        levels.append(lv)
    return mats, Ts, levels, t_an, t_rw


def main():
    args = parse()
    if args.profile_single:
        profile_single(args.profile_single)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # inputs are drawn before CUDA is touched (spawned worker pool): one
    # batch per rank, or (--split) this rank's share of one batch under the
    # deterministic partition every rank computes alike
    if args.split:
        from paper_2609_40159_gb300 import shard
        items = S.batch_spec_parallel(nmat=args.nmat, seed=3, n_hi=args.n_hi)
        costs = [shard.system_cost(it.A.n, it.A.nnz, it.nrhs) for it in items]
        items = [items[m] for m in shard.local_share(costs, rank, world)]
    else:
        items = S.batch_spec_parallel(nmat=args.nmat, seed=3 + 1000 * rank, n_hi=args.n_hi)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, items, rank)
        return

    import torch
    import paper_2609_40159_gb300 as P
    from paper_2609_40159_gb300 import autotune

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    t0 = time.perf_counter()
    mats, Ts, levels, t_an, t_rw = build_batch(P, items, dev)
    nrhs = [it.nrhs for it in items]
    t1 = time.perf_counter()
    bplan = P.BatchPlan(mats, Ts, nrhs, transpose=True)
    t_plan = time.perf_counter() - t1
    t_prep = time.perf_counter() - t0

    b = torch.cat([torch.as_tensor(it.b).reshape(-1) for it in items]).to(dev)
    gen = torch.Generator(device=dev).manual_seed(5 + rank)
    w = torch.rand(b.numel(), generator=gen, device=dev, dtype=torch.float32) * 2 - 1
    x, gbp, gb = torch.empty_like(b), torch.empty_like(b), torch.empty_like(b)
    gv = torch.empty(bplan.total_nnz, dtype=torch.float32, device=dev)

    tune = None
    if not args.no_tune and not args.ncu:
        # each direction on its own timing: the transpose solve has its own geometry
        tune = {d: autotune.tune_batch(bplan, b, candidates=(8, 16, 32), tiles=(1, 2, 4, 8), reps=3, direction=d)
                for d in ("forward", "transpose")}

    # algorithmic bytes
    wv = 4
    bf = bb = 0
    for A, T, k in zip(mats, Ts, nrhs):
        tn, tnnz = (A.n, T.nnz) if T is not None else (0, 0)
        bf += bytes_fwd(A.n, A.nnz, k, wv, tn, tnnz)
        bb += bytes_bwd(A.n, A.nnz, k, wv, tn, tnnz)
    b_solveT = sum(A.nnz * (wv + 4) + (A.n + 1) * 4 + 2 * A.n * k * wv for A, k in zip(mats, nrhs))
    step_bytes = bf + bb

    # three graphs per step: forward, transpose solve, T^T + gradient
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        gplan = P.BatchPlan(mats, Ts, nrhs, transpose=True)
        if tune is not None:
            labels = autotune.batch_classes(gplan)
            for d, tr in tune.items():
                gplan.set_geometry([tr["choice"][l]["rows_per_warp"] for l in labels],
                                   [tr["choice"][l]["rhs_tile"] for l in labels], direction=d)
        for _ in range(2):
            gplan.solve(b, out=x)
            gplan.solve_transpose(w, out=gbp)
            gplan.tt_apply(gbp, out=gb)
            gplan.grad_vals(gbp, x, out=gv)
        torch.cuda.synchronize()
        g_f, g_t, g_r = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_f, stream=s):
            gplan.solve(b, out=x)
        with torch.cuda.graph(g_t, stream=s):
            gplan.solve_transpose(w, out=gbp)
        with torch.cuda.graph(g_r, stream=s):
            gplan.tt_apply(gbp, out=gb)
            gplan.grad_vals(gbp, x, out=gv)
    torch.cuda.synchronize()
    if P.handle().status() != 0:
        raise RuntimeError("device status after set-up")

    def step():
        g_f.replay()
        g_t.replay()
        g_r.replay()

    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    clk = Clocks(local)
    clk.start()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for k in range(K):
            ev[k][0].record(s)
            g_f.replay()
            ev[k][1].record(s)
            g_t.replay()
            ev[k][2].record(s)
            g_r.replay()
            ev[k][3].record(s)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist:
        dist.barrier()
    tot_ms = ev[0][0].elapsed_time(ev[K - 1][3])
    f_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    t_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    r_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in ev]))
    ms_step = tot_ms / K
    if dist:
        tm = torch.tensor([ms_step], device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms_step = float(tm.item())
    # bytes of the whole job: every rank's own (reported outside the timed region)
    job_bytes = world * step_bytes
    if dist and args.split:
        tb = torch.tensor([float(step_bytes)], device=dev, dtype=torch.float64)
        dist.all_reduce(tb, op=dist.ReduceOp.SUM)
        job_bytes = float(tb.item())
    value = job_bytes / (ms_step * 1e-3) / 1e9
    status = P.handle().status()

    # correctness spot check of the timed buffers on two systems (device only)
    if rank == 0 and status != 0:
        raise RuntimeError(f"device status {status} after timed region")

    # roofline of the dominant kernel (forward or transpose batched solve)
    peak, peak_kind = hbm_peak()
    if f_ms >= t_ms:
        dom, dom_bytes, dom_ms = "k_batch<float,false> (forward batched solve)", bf, f_ms
    else:
        dom, dom_bytes, dom_ms = "k_batch<float,true> (transpose batched solve)", b_solveT, t_ms
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tpath) as f:
            tj = json.load(f)
        key = "fwd" if f_ms >= t_ms else "trans"
        # the record is for the benchmark's own batch only
        default = args.nmat == 512 and args.n_hi == 200_000 and not args.split
        if default and tj.get("source_sha256") == kernel_source_hash() and key in tj:
            traffic = tj[key]["bytes_per_launch_full_scale"]
    except Exception:
        traffic = None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes": dom_bytes, "ms_per_launch": dom_ms}
    # the second bound: dependency latency.  One hop = the per-row time of a
    # 1-row-per-level chain through the same kernel (alone on the GPU, one
    # right-hand side); the batch cannot finish before its deepest system's
    # chain of levels has been walked at that rate.
    if rank == 0 and not args.ncu:
        hop_f, hop_t = chain_hop_ns(P, dev)
        depth = int(max(lv[1] for lv in levels))
        hop = hop_f if f_ms >= t_ms else hop_t
        bound_ms = depth * hop * 1e-6
        roofline["latency"] = {"t_hop_ns": hop, "t_hop_ns_fwd": hop_f, "t_hop_ns_transpose": hop_t,
                               "depth": depth, "bound_ms": bound_ms, "frac": bound_ms / dom_ms,
                               "probe": "chain of 131,072 rows (1 row per level), FP32, 1 RHS, "
                                        "batched kernel, CUDA events, median of 5"}

    # end to end through the C ABI with host buffers (sptrsv_batch_step_host):
    # every step copies its inputs from pinned host memory and its results
    # back; the library alternates two device buffer sets, so that one
    # step's copies overlap the neighbouring steps' solves.  Host wall clock
    # around Ke enqueued steps and the final wait.
    e2e = None
    if not args.ncu:
        pin = lambda t: torch.empty(t.numel(), dtype=t.dtype, pin_memory=True)
        hb, hw, hx, hgb, hgv = pin(b), pin(w), pin(x), pin(gb), pin(gv)
        hb.copy_(b.cpu())
        hw.copy_(w.cpu())
        gplan.step_host(hb, hw, hx, hgb, hgv)  # the first call allocates the device sets
        gplan.step_wait()
        Ke = max(4, min(K, 10))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(Ke):
            gplan.step_host(hb, hw, hx, hgb, hgv)
        gplan.step_wait()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / Ke
        if dist:
            tm = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(tm, op=dist.ReduceOp.MAX)  # the slowest rank bounds the job
            e2e_ms = float(tm.item())
        if P.handle().status() != 0:
            raise RuntimeError("device status after the end-to-end run")
        # the host results are the device path's (same kernels, same inputs)
        if not (torch.equal(hx[:1 << 20], x[:1 << 20].cpu()) and torch.equal(hgv[-(1 << 20):], gv[-(1 << 20):].cpu())):
            raise RuntimeError("end-to-end results differ from the device path")
        e2e = {"value": job_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
               "ms_per_step": e2e_ms, "steps": Ke,
               "how": "sptrsv_batch_step_host per step (H2D of b and w from pinned host memory, fwd + "
                      "transpose solve, T^T, value gradient, D2H of x, g_b and g_vals; two device buffer "
                      "sets inside the library so that copies overlap the neighbouring steps' solves), "
                      "sptrsv_batch_step_wait at the end; host wall clock",
               "h2d_bytes_per_step": int(hb.numel() * 4 + hw.numel() * 4),
               "d2h_bytes_per_step": int(hx.numel() * 4 + hgb.numel() * 4 + hgv.numel() * 4)}

    # one host-side gather of every rank's report (no collective in the data path)
    from paper_2609_40159_gb300 import shard
    reports = shard.gather_reports({"rank": rank, "systems": len(items), "status": int(status),
                                    "ms_per_step": tot_ms / K, "phase_ms": [f_ms, t_ms, r_ms]}, dist)

    extras = {}
    if rank == 0 and not args.no_extras and not args.ncu:
        extras = run_extras(P, items, mats, dev, bf)

    if rank == 0:
        nlev = np.array(levels)
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if args.split else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "systems_per_gpu": len(items),
                       "rows_per_gpu": int(sum(A.n for A in mats)),
                       "nnz_per_gpu": int(sum(A.nnz for A in mats)),
                       "rhs_per_gpu": int(sum(it.nrhs * it.A.n for it in items)),
                       "l2": f"inputs {bf / 1e9:.1f} GB per forward solve >> 129 MB L2; no flush needed",
                       "timing": "CUDA events on the launching stream around 3 CUDA-graph "
                                 "replays per step (fwd | transpose | T^T + gradient)",
                       "parallelism": (f"dp{world} (one batch split over the GPUs by greedy LPT, "
                                       f"shard.partition; no collective in the data path)" if args.split else
                                       f"dp{world} (independent batches per GPU, no collective)")},
            "gb_per_step": step_bytes / 1e9,
            "solves_per_s": (args.nmat if args.split else world * len(items)) / (ms_step * 1e-3),
            "phase_ms": {"fwd": f_ms, "transpose": t_ms, "tt_and_grad": r_ms},
            "fwd_only_gbs": bf / (f_ms * 1e-3) / 1e9,
            "algorithmic_bytes": {"fwd_solve": bf, "transpose_solve": b_solveT, "step": step_bytes},
            "levels": {"max_orig": int(nlev[:, 0].max()), "max_rewritten": int(nlev[1::2, 1].max()),
                       "sum_orig": int(nlev[:, 0].sum()), "sum_after": int(nlev[:, 1].sum())},
            "preprocess_s": {"analyze": t_an, "rewrite": t_rw, "plan": t_plan, "total": t_prep},
            "autotune": None if tune is None else {d: {"choice": tr["choice"], "ms": tr["ms"]}
                                                   for d, tr in tune.items()},
            "roofline": roofline,
            "clocks": clocks,
            "gpu_launches": 7 * K,
            "e2e": e2e,
        }
        if world > 1:
            line["per_rank"] = reports
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def chain_hop_ns(P, dev, n=1 << 17):
    """Nanoseconds per dependency hop of the batched kernel: a 1-row-per-level
    chain (row i depends on row i-1 only) solved alone, forward and
    transpose, per row."""
    import torch
    from paper_2609_40159_gb300 import autotune
    A = P.Matrix.from_host(S.chain(n, seed=1).astype(np.float32), device=dev)
    bp = P.BatchPlan([A], None, [1], transpose=True)
    bp.set_geometry(rhs_tile=1)
    b = torch.rand(n, device=dev, dtype=torch.float32)
    x = torch.empty_like(b)
    f = autotune.time_call(lambda: bp.solve(b, out=x), reps=5, warmup=2)
    t = autotune.time_call(lambda: bp.solve_transpose(b, out=x), reps=5, warmup=2)
    return f * 1e6 / n, t * 1e6 / n


def _host_ms(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, 1e3 * (time.perf_counter() - t0))
    return best


def _single_config(P, A_h, dev, k, autotune, modes_run=("level_launch", "level", "syncfree", "hybrid"),
                   modes=None):
    """Analysis, rewrite (narrowest-level 1 %, chunks of 8 levels) and the
    forward solve in every mode (or the given ones) on the original and the
    rewritten DAG."""
    modes_run = modes if modes is not None else modes_run
    import torch
    A = P.Matrix.from_host(A_h, device=dev)
    an = P.analyze(A)
    rows, tg = S.narrowest_levels_list(an.nlevels, an.level_ptr.cpu().numpy(), an.perm.cpu().numpy(), 0.01, 8)
    Lp, T = P.rewrite(A, an.lev, rows, tg)
    an2 = P.analyze(Lp, prev_lev=an.lev, first_row=int(np.min(rows)))
    res = {"n": A.n, "nnz": A.nnz, "levels_orig": an.nlevels, "levels_rewritten": an2.nlevels,
           "cv_cost_orig": float(an.stats[3]), "cv_cost_rewritten": float(an2.stats[3]),
           "rows_rewritten": int(len(rows)), "nnz_T": int(T.nnz), "nnz_Lp": int(Lp.nnz),
           "preprocess_ms": {"analyze": _host_ms(lambda: P.analyze(A)),
                             "rewrite_1pct": _host_ms(lambda: P.rewrite(A, an.lev, rows, tg)),
                             "analyze_incremental_after_rewrite":
                                 _host_ms(lambda: P.analyze(Lp, prev_lev=an.lev, first_row=int(np.min(rows))))}}
    b = torch.as_tensor(S.rhs(A_h.n, k, seed=1)).to(dev)
    x = torch.empty_like(b)
    modes = {}
    for name, (M, TT) in {"orig": (A, None), "rewritten": (Lp, T)}.items():
        p = P.Plan(M, TT)
        nb = bytes_fwd(M.n, M.nnz, k, 8, M.n if TT is not None else 0, TT.nnz if TT is not None else 0)
        for mode in modes_run:
            p.set(mode, 1 if mode == "hybrid" else 0, 0)
            ms = autotune.time_call(lambda: p.solve(b, out=x), reps=3, warmup=1)
            modes[f"{name}:{mode}"] = {"us": 1e3 * ms, "gbs": nb / (ms * 1e-3) / 1e9}
    res["fwd"] = modes
    return res


def _diff_config(P, A_h, dev, k, autotune):
    """Differentiated solve (autograd): forward + adjoint (transpose solve,
    value gradient, T^T for the rewritten system), original and rewritten."""
    import torch
    A = P.Matrix.from_host(A_h, device=dev)
    an = P.analyze(A)
    rows, tg = S.narrowest_levels_list(an.nlevels, an.level_ptr.cpu().numpy(), an.perm.cpu().numpy(), 0.01, 8)
    Lp, T = P.rewrite(A, an.lev, rows, tg)
    b = torch.as_tensor(S.rhs(A_h.n, k, seed=4)).to(dev)
    w = torch.as_tensor(S.rhs(A_h.n, k, seed=5)).to(dev)
    res = {"n": A.n, "nnz": A.nnz, "k": k, "levels_orig": an.nlevels}
    for name, (M, TT) in {"orig": (A, None), "rewritten": (Lp, T)}.items():
        p = P.Plan(M, TT, transpose=True)
        vals = M.vals.requires_grad_(True)  # the plan's own value tensor
        bb = b.clone().requires_grad_(True)

        def step():
            xx = P.solve(p, bb, vals)
            (xx * w).sum().backward()

        ms = autotune.time_call(step, reps=3, warmup=1)
        vals.requires_grad_(False)
        tn, tnnz = (M.n, TT.nnz) if TT is not None else (0, 0)
        nb = bytes_fwd(M.n, M.nnz, k, 8, tn, tnnz) + bytes_bwd(M.n, M.nnz, k, 8, tn, tnnz)
        res[name] = {"ms_fwd_bwd": ms, "gbs": nb / (ms * 1e-3) / 1e9,
                     "levels": P.analyze(M).nlevels}
    return res


def _time_cold(fn, reps, flush):
    """Median ms of fn() with L2 flushed before every call (a write of
    `flush`, twice the L2 size, between the calls; CUDA events)."""
    import torch
    fn()
    ts = []
    for _ in range(reps):
        flush.add_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _lap2d_config(P, dev, dt, autotune):
    """2D Laplacian 1024^2 in one value type: level analysis, rewrite of the
    narrowest 1 % of levels, every solve mode on the original and the
    rewritten DAG, warm (L2-resident: 59 MB FP64 / 38 MB FP32 fit in the
    L2) and cold (L2 flushed before every solve)."""
    import torch
    A_h = S.lap2d(1024, dtype=dt)
    A = P.Matrix.from_host(A_h, device=dev)
    an = P.analyze(A)
    rows, tg = S.narrowest_levels_list(an.nlevels, an.level_ptr.cpu().numpy(), an.perm.cpu().numpy(), 0.01, 8)
    Lp, T = P.rewrite(A, an.lev, rows, tg)
    an2 = P.analyze(Lp)
    wv = np.dtype(dt).itemsize
    b = torch.as_tensor(S.rhs(A_h.n, 1, seed=1, dtype=dt)).to(dev)
    x = torch.empty_like(b)
    l2 = getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 128 << 20) or (128 << 20)
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device=dev)
    res = {"levels_orig": an.nlevels, "levels_rewritten": an2.nlevels,
           "cv_cost_orig": float(an.stats[3]), "cv_cost_rewritten": float(an2.stats[3]),
           "rows_rewritten": int(len(rows)), "nnz_T": int(T.nnz), "nnz_Lp": int(Lp.nnz),
           "l2_flush_bytes": int(flush.numel() * 4)}
    modes = {}
    for name, (M, TT) in {"orig": (A, None), "rewritten": (Lp, T)}.items():
        p = P.Plan(M, TT)
        nb = bytes_fwd(M.n, M.nnz, 1, wv, M.n if TT is not None else 0, TT.nnz if TT is not None else 0)
        for mode in ("level_launch", "level", "syncfree", "block", "hybrid"):
            p.set(mode, 4 if mode == "hybrid" else 32, 1)
            ms = autotune.time_call(lambda: p.solve(b, out=x), reps=5, warmup=2)
            msc = _time_cold(lambda: p.solve(b, out=x), 3, flush)
            modes[f"{name}:{mode}"] = {"us": 1e3 * ms, "us_cold_l2": 1e3 * msc, "gbs": nb / (ms * 1e-3) / 1e9,
                                       "us_per_level": 1e3 * ms / (an.nlevels if TT is None else an2.nlevels)}
    res["fwd"] = modes
    # analysis, rewrite and the incremental re-analysis (host-timed, each call synchronises)
    an_ms = _host_ms(lambda: P.analyze(A))
    rw_ms = _host_ms(lambda: P.rewrite(A, an.lev, rows, tg))
    inc_ms = _host_ms(lambda: P.analyze(Lp, prev_lev=an.lev, first_row=int(np.min(rows))))
    res["preprocess_ms"] = {"analyze": an_ms, "rewrite_1pct": rw_ms, "analyze_incremental_after_rewrite": inc_ms,
                            "analyze_gbs": (A.nnz * (wv + 4) + (A.n + 1) * 4 + A.n * 4) / (an_ms * 1e-3) / 1e9}
    return res


def _env_config(P, A_h, dev, moves=30):
    """The paper's environment step on the GPU kernels (RewriteEnv): a
    scripted policy (highest source affinity, then fewest rows, then lowest
    level) makes `moves` moves; host-timed per move (every move rewrites the
    list, re-analyses incrementally from the moved row and reads the level
    summary back), then one move's calls timed apart."""
    import torch
    env = P.RewriteEnv(P.Matrix.from_host(A_h, device=dev))
    L0 = env.nlevels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    valid = collapses = done = 0
    per_move = []
    for _ in range(moves):
        if env.done():
            break
        tm = time.perf_counter()
        mask = env.valid_actions()
        cands = np.flatnonzero(mask)
        ls = int(min(cands, key=lambda l: (-env.src_aff[l], env.level_rows[l], l)))
        _, info = env.step(ls)
        per_move.append(1e3 * (time.perf_counter() - tm))
        valid += info["valid"]
        collapses += bool(info["valid"] and info["collapsed"] > 0)
        done += 1
    dt = time.perf_counter() - t0
    row = env.rows[-1] if env.rows else 0
    prev_lev = env.an.lev.clone()
    rw = _host_ms(lambda: P.rewrite(env.A, env.an0.lev, env.rows, env.targets))
    inc = _host_ms(lambda: P.analyze(env.Lp, prev_lev=prev_lev, first_row=row))
    summ = _host_ms(lambda: P.level_summary(env.Lp, env.an, env.threshold))
    full = _host_ms(lambda: P.analyze(env.Lp))
    return {"n": int(A_h.n), "moves": done, "valid": valid, "collapses": collapses,
            "levels": [int(L0), int(env.nlevels)], "ms_per_move": 1e3 * dt / max(done, 1),
            "ms_per_move_median": float(np.median(per_move)) if per_move else None,
            "ms_per_move_max": float(np.max(per_move)) if per_move else None,
            "last_move_ms": {"rewrite_list": rw, "analyze_incremental": inc, "level_summary": summ,
                             "analyze_full_for_comparison": full}}


def run_extras(P, items, mats, dev, bf_total):
    """Plain level-set baseline, a single-system comparison and the CPU
    oracle, all on rank 0."""
    import torch
    import oracle
    from paper_2609_40159_gb300 import autotune
    out = {}
    # --- plain level-set solve, one launch per level, original DAG, per system
    sub = list(range(0, len(items), 16))
    wv = 4
    plans, bs, nbytes = [], [], 0
    for m in sub:
        A = P.Matrix.from_host(items[m].A, device=dev)
        plans.append(P.Plan(A, mode="level_launch"))
        bs.append(torch.as_tensor(items[m].b).to(dev))
        nbytes += bytes_fwd(A.n, A.nnz, items[m].nrhs, wv)
    for p, bb in zip(plans[:2], bs[:2]):
        p.solve(bb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for p, bb in zip(plans, bs):
        p.solve(bb)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["baseline_plain_level_set"] = {
        "gbs": nbytes / (ms * 1e-3) / 1e9, "solves_per_s": len(sub) / (ms * 1e-3),
        "ms": ms, "sample": f"{len(sub)} of {len(items)} systems (every 16th), forward only, "
                            "original DAG, one kernel launch per level, host loop over systems",
        "levels_launched": int(sum(p.info()["nlevels"] for p in plans)),
        "frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak()[0], "frac_of": "HBM peak (same as roofline.peak)"}
    del plans
    # --- single system: 2D Laplacian 1024^2, FP64 and FP32, every mode, original and rewritten
    out["single_lap2d_1024_f64"] = _lap2d_config(P, dev, np.float64, autotune)
    out["single_lap2d_1024_f32"] = _lap2d_config(P, dev, np.float32, autotune)
    out["env_step_lap2d_1024"] = _env_config(P, S.lap2d(1024), dev, moves=30)
    out["powerlaw_4M_f64"] = _single_config(P, S.powerlaw(4_000_000, alpha=2.1, seed=2), dev, 1, autotune)
    # the nnz-matched variant of the power-law DAG (mean ~9 off-diagonals per row)
    out["powerlaw_4M_alpha1.7_f64"] = _single_config(P, S.powerlaw(4_000_000, alpha=1.7, seed=2), dev, 1, autotune,
                                                     modes=("level", "syncfree", "hybrid"))
    out["lap3d_128_f64_diff_k8"] = _diff_config(P, S.lap3d(128), dev, 8, autotune)
    # --- CPU oracle on the host cores (whole batch, fwd + adjoint, one pass)
    t0 = time.perf_counter()
    nb = 0
    for it in items:
        A64 = S.CSR(it.A.n, it.A.row_ptr, it.A.col_idx, it.A.vals.astype(np.float64))
        xx = oracle.solve(A64, it.b)
        g = oracle.solve_transpose(A64, it.b)
        oracle.grad_vals(A64, g, xx)
        nb += bytes_fwd(A64.n, A64.nnz, it.nrhs, 4) + bytes_bwd(A64.n, A64.nnz, it.nrhs, 4)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": 1,
                           "cores_available": os.cpu_count(), "kind": "oracle", "seconds": dt,
                           "sample": f"all {len(items)} systems, one fwd solve + transpose solve "
                                     "+ value gradient (no rewrite), FP64 on widened FP32 values"}
    return out


if __name__ == "__main__":
    main()
