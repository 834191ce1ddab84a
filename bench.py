"""Benchmark: periodic potential + gradient throughput on the 2D oblique clustered workload.

Workload: oblique cell a1 = (1, 0), a2 = (0.45, 0.85), N = 200,000 sources in 16 Gaussian
clusters (sigma log-uniform in [1e-4, 1e-2] of the cell), balanced +/-1 charges, eps = 1e-6,
evaluation at every source (self term excluded).  One step = one full evaluation
(far field: spread, FFT, scale, inverse FFT, interpolate; near field: plane-wave passes and
the residual direct sum; assembly) with the sources already set.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank evaluates its own replica of the workload (independent cells: weak
scaling, no collective on the data path); value = total points/s over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

EPS = 1e-6
N_POINTS = 200_000
WORKLOAD = "oblique2d_clusters: a1=(1,0) a2=(0.45,0.85), N=200000, 16 gaussian clusters sigma in [1e-4,1e-2], +/-1 charges"
METRIC = "points/s (potential+force) at 1e-6 rel err"
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        try:
            sm = [float(r[1]) for r in rows]
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = float(rows[0][2])
        except ValueError:
            pass
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(g, idx, nthreads=None):
    from oracle import ewald as E
    t0 = time.perf_counter()
    pot, grad = E.ewald(g["L"], g["y"], g["q"], x=g["y"][idx], self_idx=idx, nthreads=nthreads)
    return pot, grad, time.perf_counter() - t0


def stage_flops(info, d, leaf_folded, out_folded):
    """Algorithmic flops of each timed stage, from the plan's work counts and the fixed
    per-unit costs of each kernel's formula (documented with the kernels):
      spread      per point: w^d products + d*w window series of n_W terms (2 flops/term)
      interp      per target: 2 w^d FMAs (value, x-derivative) + d*w window series (value, derivative)
      nearfield   per visited pair 5 (2D) / 7 (3D); per pair inside the support two
                  residual series of n_A, n_B terms (2 flops/term) + 16 (2D) / 22 (3D)
      pw_upward   per (out box, source) pair: the p^d moment outer product (2 flops each) and
                  2 d p Chebyshev recurrence flops; per merge parent (generic path) 12 p^3 (2D)
                  or 8 * 3 * 2 p^{d+1} (3D separable re-expansion)
      pw_out      per box (2D parity form): 2 (K+1) p^2 + 4 (K+1)^2 p; credited to pw_upward
                  where the moments launch computes the outgoing waves itself
      pw_translate_in per box (2D parity form): ~100 (K+1)^2 (nine phased colleagues, both
                  k1 signs) + 4 (K+1)^2 p + 2 (K+1) p^2
      pw_downward per parent 12 p^3 (2D) or 8 * 3 * 2 p^{d+1} (3D), plus the leaf evaluation
                  (4 p^d per target) where the single-launch pass folds it in
      pw_leaf_eval per target 4 p^d
    """
    w, p, K = info["window_w"], info["n_proxy"], info["n_pw"]
    n1 = 2 * K + 1
    npw = (K + 1) * n1 ** (d - 1)
    nW = 15
    n = info["n"]
    out = {}
    out["spread"] = n * (2 * w ** d + 2 * d * w * nW)
    out["interp"] = n * (4 * w ** d + 2 * d * w * 2 * nW)
    visit, inside = (5, 2 * (12 + 14) + 16) if d == 2 else (7, 2 * (13 + 14) + 22)
    out["nearfield"] = info["near_pairs"] * visit + info["near_pairs_in"] * inside
    merge_unit = 12 * p ** 3 if d == 2 else 8 * 3 * 2 * p ** (d + 1)
    out["pw_upward"] = info["pw_moment_sources"] * (2 * p ** d + 2 * d * p) + info["pw_merge_parents"] * merge_unit
    if d == 2:
        out["pw_out"] = info["n_pw_boxes_out"] * (2 * (K + 1) * p ** 2 + 4 * (K + 1) ** 2 * p)
        out["pw_translate_in"] = info["n_pw_boxes_in"] * (100 * (K + 1) ** 2 + 4 * (K + 1) ** 2 * p
                                                          + 2 * (K + 1) * p ** 2)
    else:
        out["pw_out"] = info["n_pw_boxes_out"] * (2 * (K + 1) * p ** d + 8 * (K + 1) * n1 * p ** (d - 1) * (d - 1))
        out["pw_translate_in"] = info["n_pw_boxes_in"] * (3 ** d * 14 * npw + 8 * (K + 1) * n1 * p ** (d - 1) * (d - 1)
                                                          + 3 * (K + 1) * p ** d)
    if out_folded:
        out["pw_upward"] += out["pw_out"]
        out["pw_out"] = 0
    leaf = info["pw_eval_targets"] * 4 * p ** d
    out["pw_downward"] = info["pw_down_parents"] * merge_unit + (leaf if leaf_folded else 0)
    out["pw_leaf_eval"] = 0 if leaf_folded else leaf
    return out


# DRAM bytes (read + write) per launch of each stage's main kernel on this workload, from
# one `ncu --set full` capture of the kernel as it stands (profiles/ holds the summaries);
# None where no capture of the current kernel exists
STAGE_TRAFFIC = {"nearfield": 17922560, "pw_upward": 6190336, "pw_downward": 13728768}

STAGE_KERNELS = {
    "spread": "k_spread_halo + k_fold_whole", "interp": "k_interp_halo", "nearfield": "k_near_warp",
    "pw_upward": "k_moments_direct2d (outgoing waves folded in)", "pw_out": "k_pw_out",
    "pw_translate_in": "k_pw_in2d_p",
    "pw_downward": "k_down_persist2d (leaf evaluation folded in)", "pw_leaf_eval": "k_leaf_eval",
}


def replica_summary(t_local, n, steps, ws, pg, device):
    """Replicas (one independent cell per rank, no collective on the data path): the timed
    region is the slowest rank's, and the value is every rank's points over that time.
    Returns (points/s over all ranks, ms per step, the slowest rank's seconds)."""
    t_max = t_local
    if pg is not None and ws > 1:
        import torch
        tt = torch.tensor([t_local], device=device, dtype=torch.float64)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_max = float(tt.item())
    return ws * n * steps / t_max, 1e3 * t_max / steps, t_max


def batched_line(P, torch, stream, ncells=16, nmax=20_000, steps=20):
    """Batched cells (the 3D batched workload's shape, bounded to ncells cells of at most nmax
    sources so that the host tree builds stay short): points/s of one graph-replayed batch
    evaluation with device outputs, timed with CUDA events."""
    cells = W.batched_cells(ncells, nmax=nmax)
    b = P.Batch([(c["L"], EPS) for c in cells], precision="mixed", stream=stream.cuda_stream)
    t0 = time.perf_counter()
    b.set_sources([c["y"] for c in cells], [c["q"] for c in cells])
    t_set = time.perf_counter() - t0
    ntot = sum(len(c["q"]) for c in cells)
    bp = torch.empty(ntot, dtype=torch.float64, device="cuda")
    bg = torch.empty(3 * ntot, dtype=torch.float64, device="cuda")
    for _ in range(3):
        b.eval_device(bp, bg)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.eval_device(bp, bg)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    b.close()
    return {"cells": ncells, "points": ntot, "value": ntot / (ms * 1e-3), "unit": "points/s", "ms_per_eval": ms,
            "t_set_sources_s": t_set, "workload": f"batched_cells({ncells}, nmax={nmax}): 3D triclinic, edges U(1,4), "
                                                  "angles U(60,120), uniform or 4-cluster, +/-1 charges, eps 1e-6, mixed"}


def run_reference(args, ws, rank):
    """The oracle (plain FP64 Ewald on the host cores) on a bounded sample of targets."""
    if rank != 0:
        return
    g = W.oblique2d_clusters(N_POINTS)
    rng = np.random.default_rng(7)
    nsamp = 64
    times = []
    ncores = os.cpu_count() or 1
    for k in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(N_POINTS, nsamp, replace=False))
        _, _, dt = oracle_sample(g, idx, nthreads=ncores)
        if k >= args.warmup:
            times.append(dt)
    value = nsamp * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "eps": EPS},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": ncores, "kind": "oracle",
                             "sample": f"{nsamp} random targets per step, full-N structure factors"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: only the mixed plan, warm-up + steps evaluations, no other work")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import paper_2606_28608_b300 as P

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    g = W.oblique2d_clusters(N_POINTS)
    n, d = g["y"].shape
    peaks, peak_kind = load_peaks()

    def make(prec, profile=False):
        pl = P.Plan(g["L"], EPS, precision=prec, profile=profile, stream=stream.cuda_stream)
        pl.set_sources(g["y"], g["q"])
        return pl

    pot = torch.empty(n, dtype=torch.float64, device=dev)
    grad = torch.empty((n, d), dtype=torch.float64, device=dev)
    if args.ncu:
        plan = make("mixed")
        for _ in range(args.warmup + args.steps):
            plan.eval_device(pot, grad)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_run": True, "evals": args.warmup + args.steps, "launches_per_eval": plan.info()["launches"]}))
        return
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def timed(pl, steps, warmup):
        for _ in range(warmup):
            pl.eval_device(pot, grad)
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pl.eval_device(pot, grad)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3  # seconds

    t_set0 = time.perf_counter()
    plan = make("mixed")
    torch.cuda.synchronize()
    t_set_sources = time.perf_counter() - t_set0  # plan + host tree build + device layouts
    for _ in range(args.warmup):
        plan.eval_device(pot, grad)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    t_total = timed(plan, args.steps, 0)
    clocks = sampler.stop()
    value, ms_per_step, t_max = replica_summary(t_total, n, args.steps, ws, pg, dev)
    pot_m = pot.cpu().numpy().copy()
    grad_m = grad.cpu().numpy().copy()
    info = plan.info()

    # FP64 comparator (same workload, fewer steps)
    plan64 = make("fp64")
    t64 = timed(plan64, max(2, args.steps // 4), 2)
    pts64 = n * max(2, args.steps // 4) / t64
    pot_64 = pot.cpu().numpy().copy()
    del plan64

    # per-stage device times (CUDA events on the plan's stream) for the roofline
    pprof = make("mixed", profile=True)
    pprof.eval_device(pot, grad)  # counts pairs inside the support
    torch.cuda.synchronize()
    stage_acc = {}
    nprof = 5
    for _ in range(nprof):
        flush.fill_(1.0)
        pprof.eval_device(pot, grad)
        torch.cuda.synchronize()
        for k, v in pprof.stage_times().items():
            stage_acc[k] = stage_acc.get(k, 0.0) + v / nprof
    pinfo = pprof.info()
    del pprof

    # end-to-end through the C ABI with host buffers: charges in, potential+gradient out
    q_host = torch.from_numpy(g["q"]).pin_memory()
    pot_host = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    grad_host = torch.empty((n, d), dtype=torch.float64).pin_memory().numpy()
    reps = max(3, args.steps // 2)
    plan.set_charges(q_host.numpy())
    plan.eval(out=(pot_host, grad_host))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        plan.set_charges(q_host.numpy())
        plan.eval(out=(pot_host, grad_host))
    e2e_t = (time.perf_counter() - t0) / reps
    e2e = {"value": ws * n / e2e_t, "unit": "points/s", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n * (1 + d)}

    out = None
    if rank == 0:
        # accuracy against the oracle on sampled targets (full-N structure factors)
        rng = np.random.default_rng(11)
        idx = np.sort(rng.choice(n, 128, replace=False))
        cpu_line = None
        pref, gref, dt = oracle_sample(g, idx, nthreads=os.cpu_count())
        e_pot = float(np.linalg.norm(pot_m[idx] - pref) / np.linalg.norm(pref))
        e_grad = float(np.linalg.norm(grad_m[idx] - gref) / np.linalg.norm(gref))
        e_pot64 = float(np.linalg.norm(pot_64[idx] - pref) / np.linalg.norm(pref))
        if not args.no_cpu_baseline:
            cpu_line = {"value": len(idx) / dt, "unit": "points/s", "cores": os.cpu_count(),
                        "kind": "oracle",
                        "sample": f"{len(idx)} random targets of the workload, full-N structure factors"}
        # roofline: every timed stage is bound by the FP32 ALU pipes (tiny byte counts; the
        # working set stays in L2); report each and pick the dominant one
        sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
        fp32_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2 flops
        # the single-launch downward pass evaluates the leaves itself (its leaf stage is empty)
        leaf_folded = stage_acc.get("pw_leaf_eval", 0.0) < 0.05 * stage_acc.get("pw_downward", 0.0)
        # likewise the moments launch computes the outgoing waves (its outgoing stage is empty)
        out_folded = stage_acc.get("pw_out", 0.0) < 0.05 * stage_acc.get("pw_upward", 0.0)
        fl = stage_flops(pinfo, d, leaf_folded, out_folded)
        stages = {k: round(v, 4) for k, v in stage_acc.items()}
        per_stage = {}
        for k, f in fl.items():
            t = stage_acc.get(k, 0.0) / 1e3
            if t > 0:
                per_stage[k] = {"ms": round(1e3 * t, 4), "gflop": round(f / 1e9, 4),
                                "tflops": round(f / t / 1e12, 4), "frac": round(f / t / 1e12 / fp32_peak, 5),
                                "kernels": STAGE_KERNELS.get(k)}
        dominant = max(per_stage, key=lambda k: per_stage[k]["ms"]) if per_stage else None
        achieved = per_stage[dominant]["tflops"] if dominant else None
        out = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "eps": EPS, "precision": "mixed", "l2": "flushed (256 MB write) between steps",
                       "depth": info["depth"], "n_images": info["n_images"], "M": info["M"][:d],
                       "near_pairs": pinfo["near_pairs"], "near_pairs_in": pinfo["near_pairs_in"]},
            "accuracy": {"E_pot_mixed": e_pot, "E_grad_mixed": e_grad, "E_pot_fp64": e_pot64,
                         "sample": len(idx)},
            "fp64": {"value": pts64, "unit": "points/s"},
            "stages_ms": stages, "dominant_stage": dominant, "stage_roofline": per_stage,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": (achieved / fp32_peak) if achieved else None,
                         "traffic": STAGE_TRAFFIC.get(dominant),
                         "kernel": STAGE_KERNELS.get(dominant), "stage": dominant,
                         "peak_note": f"FP32 FMA pipes: 148 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz "
                                      "(recipe unit counts at the maximum clock; no measured FP32 peak exists)"},
            "cpu_baseline": cpu_line, "e2e": e2e,
            "gpu_launches": None, "clocks": clocks,
        }
        out["t_set_sources_s"] = t_set_sources
        out["batched"] = batched_line(P, torch, stream)
        out["gpu_launches"] = int(info["launches"]) * args.steps
        out["config"]["launches_per_step"] = int(info["launches"])
        print(json.dumps(out))
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
