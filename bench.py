"""Benchmark: periodic potential + gradient throughput, mixed precision against FP64.

Headline workload (the largest single-GPU configuration): 3D triclinic cell
a1 = (1, 0, 0), a2 = (0.3, 2, 0), a3 = (0.5, 0.7, 17) (longest edge ~17x the shortest),
N = 4,000,000 sources in 64 anisotropic Gaussian clusters (sigma 1e-4..1e-2 of the cell per
fractional axis, randomly rotated, wrapped), q ~ U(-1, 1) minus the mean, eps = 1e-6,
evaluation at every source (self term excluded).  One step = one full evaluation (far
field: spread, FFT, scale, inverse FFT, interpolate; near field: the plane-wave passes and
the residual direct sum; assembly) with the sources already set.

The line also carries: the same cell in FP64 (`fp64`), the end-to-end figure through the C
ABI with host buffers (`e2e`: positions and charges in, tree build, evaluation, potential and
gradient out, every step), the accuracy against stored oracle values, per-stage roofline
accounting, the oracle timed on the host cores (`cpu_baseline`), and secondary lines for
the 2D oblique 200k cell and a batch of 3D cells.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload triclinic3d_4m|oblique2d_200k]
Under torchrun each rank evaluates its own replica (independent cells: weak scaling, no
collective on the data path); value = total points/s over ranks.
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
METRIC = "points/s (potential+force) at 1e-6 rel err"
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

WORKLOADS = {
    "triclinic3d_4m": dict(
        make=lambda: W.triclinic3d_clusters(4_000_000), golden="triclinic3d_4m",
        desc="triclinic3d_clusters: a1=(1,0,0) a2=(0.3,2,0) a3=(0.5,0.7,17), N=4000000, 64 anisotropic "
             "gaussian clusters sigma in [1e-4,1e-2] of the cell, q~U(-1,1) minus mean"),
    "cube_2k": dict(
        make=lambda: W.cube_uniform(2000), golden=None,
        desc="cube_uniform: L = I, N=2000 uniform sources, q~N(0,1) minus mean"),
    "water_333k": dict(
        make=lambda: W.water_box(333_000), golden="water_333k",
        desc="water_box: triclinic cell edges (3.1,3.3,9.8) angles (85,95,100), 333000 rigid 3-site "
             "molecules (999000 charges -0.834/+0.417/+0.417)"),
    # the headline cell's shape at 1/8 of the points (profiling captures: a few GB on the device)
    "triclinic3d_500k": dict(
        make=lambda: W.triclinic3d_clusters(500_000), golden=None,
        desc="triclinic3d_clusters: a1=(1,0,0) a2=(0.3,2,0) a3=(0.5,0.7,17), N=500000, 64 anisotropic "
             "gaussian clusters sigma in [1e-4,1e-2] of the cell, q~U(-1,1) minus mean"),
    "oblique2d_200k": dict(
        make=lambda: W.oblique2d_clusters(200_000), golden=None,
        desc="oblique2d_clusters: a1=(1,0) a2=(0.45,0.85), N=200000, 16 gaussian clusters sigma in "
             "[1e-4,1e-2], +/-1 charges"),
}


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
    """The oracle (plain FP64 Ewald) at the sampled sources, one call: its reciprocal-space
    structure factors run over every source, whatever the sample size."""
    from oracle import ewald as E
    t0 = time.perf_counter()
    pot, grad = E.ewald(g["L"], g["y"], g["q"], x=g["y"][idx], self_idx=idx, nthreads=nthreads)
    return pot, grad, time.perf_counter() - t0


def golden_sample(name):
    """Stored oracle values at seeded targets of a full-size workload (written by the oracle
    alone, tests/golden/make_fullsize.py)."""
    with open(os.path.join(ROOT, "tests", "golden", f"fullsize_{name}.json")) as f:
        c = json.load(f)["cells"][0]
    return np.asarray(c["idx"]), np.asarray(c["pot"]), np.asarray(c["grad"])


def half_ball_counts(c, K):
    """Slices k0 >= 0, rows (k0, k1 >= 0) and modes (k0, k1, k2 >= 0) of the plane-wave ball
    |k| <= 3c/pi inside the (K+1)(2K+1)^2 half grid (the outgoing waves' support)."""
    kb = 3.0 * c / math.pi
    nk0 = nrows = nhalf = 0
    for k0 in range(K + 1):
        rows_k0 = 0
        for k1 in range(-K, K + 1):
            m = -1
            for k2 in range(K + 1):
                if math.sqrt(k0 * k0 + k1 * k1 + k2 * k2) <= kb:
                    m = k2
            nhalf += m + 1
            if k1 >= 0 and m >= 0:
                rows_k0 += 1
        nrows += rows_k0
        if rows_k0:
            nk0 = k0 + 1
    return nk0, nrows, nhalf


def stage_flops(info, d, leaf_folded, out_folded):
    """Algorithmic flops of each timed stage, from the plan's work counts and the fixed
    per-unit costs of each kernel's formula (documented with the kernels):
      spread      per point: w^d products + d*w window series of n_W terms (2 flops/term)
      interp      per target: 2 w^d FMAs (value, x-derivative) + d*w window series (value, derivative)
      nearfield   per visited pair 5 (2D) / 7 (3D); per pair inside the support two
                  residual series of n_A, n_B terms (2 flops/term) + 16 (2D) / 22 (3D)
      pw_moments  per (out box, source) pair: the p^d moment outer product (2 flops each) and
                  2 d p Chebyshev recurrence flops
      pw_merge    per merge parent 12 p^3 (2D generic) or 14 p^4 (3D: the eight children over
                  the triangular shift matrices axis by axis, 7 p^4 multiply-adds)
      pw_out      per box (2D parity form): 2 (K+1) p^2 + 4 (K+1)^2 p; credited to pw_moments
                  where the moments launch computes the outgoing waves itself;
                  3D over the ball |k| <= 3c/pi: 2 n_k0 p^3 + 4 n_rows p^2 + 4 n_half p (n_half
                  modes with k2 >= 0, n_rows rows (k0, k1 >= 0), n_k0 slices meeting the ball)
      pw_translate_in per box (2D parity form): ~100 (K+1)^2 + 4 (K+1)^2 p + 2 (K+1) p^2;
                  3D: 27 phased colleagues per half-ball mode (14 flops each) + the three
                  axis contractions (the transpose of pw_out's)
      pw_downward per parent 12 p^3 (2D) or 14 p^4 (3D, the eight children over the
                  triangular shift matrices), plus the leaf evaluation (4 p^d per target) where
                  the single-launch pass folds it in
      pw_leaf_eval per target 2 (p^d + 3 p^{d-1} ... ) ~ 4 p^d (value and three derivatives)
    """
    w, p, K = info["window_w"], info["n_proxy"], info["n_pw"]
    n1 = 2 * K + 1
    nW = 15
    n = info["n_targets"] or info["n"]
    out = {}
    out["spread"] = info["n"] * (2 * w ** d + 2 * d * w * nW)
    out["interp"] = n * (4 * w ** d + 2 * d * w * 2 * nW)
    visit, inside = (5, 2 * (12 + 14) + 16) if d == 2 else (7, 2 * (13 + 14) + 22)
    out["nearfield"] = info["near_pairs"] * visit + info["near_pairs_in"] * inside
    merge_unit = 12 * p ** 3 if d == 2 else 14 * p ** 4
    down_unit = 12 * p ** 3 if d == 2 else 14 * p ** 4
    out["pw_moments"] = info["pw_moment_sources"] * (2 * p ** d + 2 * d * p)
    out["pw_merge"] = info["pw_merge_parents"] * merge_unit
    if d == 2:
        out["pw_out"] = info["n_pw_boxes_out"] * (2 * (K + 1) * p ** 2 + 4 * (K + 1) ** 2 * p)
        out["pw_translate_in"] = info["n_pw_boxes_in"] * (100 * (K + 1) ** 2 + 4 * (K + 1) ** 2 * p
                                                          + 2 * (K + 1) * p ** 2)
    else:
        nk0, nrows, nhalf = half_ball_counts(info["c"], K)
        transforms = 2 * nk0 * p ** 3 + 4 * nrows * p ** 2 + 4 * nhalf * p
        out["pw_out"] = info["n_pw_boxes_out"] * transforms
        out["pw_translate_in"] = info["n_pw_boxes_in"] * (27 * 14 * nhalf + transforms)
    if out_folded:
        out["pw_moments"] += out["pw_out"]
        out["pw_out"] = 0
    leaf = info["pw_eval_targets"] * 4 * p ** d
    out["pw_downward"] = info["pw_down_parents"] * down_unit + (leaf if leaf_folded else 0)
    out["pw_leaf_eval"] = 0 if leaf_folded else leaf
    return out


# DRAM bytes (read + write) per launch of each stage's main kernel, per workload, from one
# `ncu` capture of the kernel as it stands (profiles/ holds the summaries); absent where no
# capture of the current kernel exists
STAGE_TRAFFIC = {
    "oblique2d_200k": {"nearfield": 17930000, "pw_moments": 6190336, "pw_downward": 13728768},
    "triclinic3d_4m": {"nearfield": 2306000000},  # 2.17 GB read + 0.136 GB written (k_near_warp)
}

STAGE_KERNELS = {
    2: {"spread": "k_spread_halo + k_fold_whole", "interp": "k_interp_halo", "nearfield": "k_near_warp",
        "pw_moments": "k_moments_direct2d (outgoing waves folded in)", "pw_merge": "k_merge2d_p",
        "pw_out": "k_pw_out", "pw_translate_in": "k_pw_in2d_p",
        "pw_downward": "k_down_persist2d (leaf evaluation folded in)", "pw_leaf_eval": "k_leaf_eval"},
    3: {"spread": "k_spread3d_reg + k_fold", "interp": "k_interp3d_w", "nearfield": "k_near_warp",
        "pw_moments": "k_leaf_moments3d_t", "pw_merge": "k_merge3d_r", "pw_out": "k_pw_out3d_h",
        "pw_translate_in": "k_pw_in3d_h", "pw_downward": "k_down3d_r",
        "pw_leaf_eval": "k_leaf_eval3d_tc (tcgen05 kind::tf32, split operands)"},
}


def fp32_peak_tflops(peaks):
    """FP32 FMA pipe peak of this device: SMs x 128 lanes x 2 flops x the maximum SM clock
    (no FP32 figure is measured; the SM count is the device's own)."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    return nsm * 128 * 2 * sm_mhz * 1e6 / 1e12, nsm, sm_mhz


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


def batched_line(P, torch, stream, ncells=16, nmax=20_000, steps=20, ws=1, rank=0, pg=None):
    """Batched cells (the 3D batched workload's shape; by default bounded to 16 cells of at most
    20,000 sources, --batch-cells 256 --batch-nmax 200000 for the full workload): points/s of one
    graph-replayed batch
    evaluation with device outputs, timed with CUDA events, mixed and FP64 on the same cells.
    With several ranks the cells are split by estimated work (pdmk_partition_cells, the same
    partition computed on every rank, no exchange); the value is all ranks' points over the
    slowest rank's time."""
    all_cells = W.batched_cells(ncells, nmax=nmax)
    work = [P.cell_work(c["L"], EPS, len(c["q"])) for c in all_cells]
    owner = P.partition_cells(work, ws)
    cells = [c for c, r in zip(all_cells, owner) if r == rank]
    out = {"cells": ncells, "workload": f"batched_cells({ncells}, nmax={nmax}): 3D triclinic, edges U(1,4), "
                                        "angles U(60,120), uniform or 4-cluster, +/-1 charges, eps 1e-6",
           "partition": "cells split over ranks by estimated work" if ws > 1 else "one rank"}
    if not cells:
        return out
    for prec in ("mixed", "fp64"):
        b = P.Batch([(c["L"], EPS) for c in cells], precision=prec, stream=stream.cuda_stream)
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
        ns = steps if prec == "mixed" else max(3, steps // 4)
        e0.record(stream)
        for _ in range(ns):
            b.eval_device(bp, bg)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / ns
        b.close()
        tot = float(ntot)
        if pg is not None and ws > 1:
            tt = torch.tensor([ms, tot], device="cuda", dtype=torch.float64)
            pg.all_reduce(tt[:1], op=pg.ReduceOp.MAX)
            pg.all_reduce(tt[1:], op=pg.ReduceOp.SUM)
            ms, tot = float(tt[0].item()), float(tt[1].item())
        out["points"] = int(tot)
        out[prec] = {"value": tot / (ms * 1e-3), "unit": "points/s", "ms_per_eval": ms, "t_set_sources_s": t_set}
    out["value"] = out["mixed"]["value"]
    out["unit"] = "points/s"
    return out


def run_reference(args, ws, rank):
    """The oracle (plain FP64 Ewald on the host cores) on the headline workload.  A step is a
    sample of `per_step` targets; each oracle call pays the reciprocal-space structure factors
    over all N sources once, so the warm-up steps run as one call and the K timed steps as one
    call over their K samples (a bounded run: two calls)."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    g = wl["make"]()
    n = len(g["q"])
    rng = np.random.default_rng(7)
    per_step = 2 if n > 1_000_000 else 16
    ncores = os.cpu_count() or 1
    idx_w = np.sort(rng.choice(n, per_step * args.warmup, replace=False))
    oracle_sample(g, idx_w, nthreads=ncores)
    idx = np.sort(rng.choice(n, per_step * args.steps, replace=False))
    _, _, dt = oracle_sample(g, idx, nthreads=ncores)
    value = len(idx) / dt
    sample = (f"{per_step} random targets per step, the {args.steps} timed steps in one oracle call "
              f"(its full-N reciprocal sums paid once per call)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "eps": EPS},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": ncores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def timed_device(pl, pot, grad, stream, flush, steps, warmup):
    """Seconds of `steps` device evaluations (CUDA events on the caller's stream around each,
    L2 flushed by a 256 MB write before each, outside the events)."""
    import torch
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
    return sum(a.elapsed_time(b) for a, b in evs) / 1e3


def stage_profile(P, g, prec, stream, pot, grad, flush, nprof=3):
    """Per-stage device times (CUDA events between the stages, which then run one after
    another on one stream) and the plan's work counts."""
    import torch
    pl = P.Plan(g["L"], EPS, precision=prec, profile=True, stream=stream.cuda_stream)
    pl.set_sources(g["y"], g["q"])
    pl.eval_device(pot, grad)  # counts the pairs inside the support
    torch.cuda.synchronize()
    acc = {}
    for _ in range(nprof):
        flush.fill_(1.0)
        pl.eval_device(pot, grad)
        torch.cuda.synchronize()
        for k, v in pl.stage_times().items():
            acc[k] = acc.get(k, 0.0) + v / nprof
    info = pl.info()
    pl.close()
    return acc, info


def stage_roofline(acc, info, d, peak):
    leaf_folded = acc.get("pw_leaf_eval", 0.0) < 0.05 * acc.get("pw_downward", 0.0)
    out_folded = acc.get("pw_out", 0.0) < 0.05 * acc.get("pw_moments", 0.0)
    fl = stage_flops(info, d, leaf_folded, out_folded)
    per = {}
    for k, f in fl.items():
        t = acc.get(k, 0.0) / 1e3
        if t > 0:
            per[k] = {"ms": round(1e3 * t, 4), "gflop": round(f / 1e9, 4), "tflops": round(f / t / 1e12, 4),
                      "frac": round(f / t / 1e12 / peak, 5), "kernels": STAGE_KERNELS[d].get(k)}
    return per


SWEEP_REGIMES = [
    ("ring2d_a1", lambda n: W.wavy_ring2d(n, aspect=1.0)),
    ("ring2d_a10", lambda n: W.wavy_ring2d(n, aspect=10.0)),
    ("ring2d_a100", lambda n: W.wavy_ring2d(n, aspect=100.0)),
    ("sphere3d_rect_iso", lambda n: W.wavy_sphere3d(n, (1, 1, 1), triclinic=False)),
    ("sphere3d_rect_rod", lambda n: W.wavy_sphere3d(n, (1, 1, 10), triclinic=False)),
    ("sphere3d_rect_slab", lambda n: W.wavy_sphere3d(n, (1, 10, 10), triclinic=False)),
    ("sphere3d_tri_iso", lambda n: W.wavy_sphere3d(n, (1, 1, 1), triclinic=True)),
    ("sphere3d_tri_rod", lambda n: W.wavy_sphere3d(n, (1, 1, 10), triclinic=True)),
    ("sphere3d_tri_slab", lambda n: W.wavy_sphere3d(n, (1, 10, 10), triclinic=True)),
]
SWEEP_RUNS = [("mixed", 1e-3), ("mixed", 1e-6), ("fp64", 1e-6), ("fp64", 1e-9), ("fp64", 1e-12)]


def run_sweep(args):
    """The paper's experiment grid (Sec. 6, Tables 2-4) on this GPU: wavy rings in oblique 2D
    cells of aspect 1, 10, 100 and wavy sphere shells in rectangular and triclinic 3D cells
    (iso / rod / slab), at eps 1e-3 .. 1e-12.  Per (regime, precision, eps): the set-up time
    (tree build and layouts: the paper's t_build), the evaluation time (device, potential and
    gradient at every source), points/s, and E_rel of the potential against the oracle on
    sampled targets.  One JSON line per run."""
    import torch
    import paper_2606_28608_b300 as P
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.sweep_n
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for name, make in SWEEP_REGIMES:
        g = make(n)
        d = g["y"].shape[1]
        rng = np.random.default_rng(31)
        idx = np.sort(rng.choice(n, args.sweep_samples, replace=False))
        pref, _, t_or = oracle_sample(g, idx, nthreads=os.cpu_count())
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        grad = torch.empty((n, d), dtype=torch.float64, device="cuda")
        for prec, eps in SWEEP_RUNS:
            t0 = time.perf_counter()
            pl = P.Plan(g["L"], eps, precision=prec, stream=stream.cuda_stream)
            pl.set_sources(g["y"], g["q"])
            torch.cuda.synchronize()
            t_build = time.perf_counter() - t0
            steps = 5 if prec == "mixed" else 2
            t = timed_device(pl, pot, grad, stream, flush, steps, 2)
            p = pot.cpu().numpy()
            info = pl.info()
            pl.close()
            e = float(np.linalg.norm(p[idx] - pref) / np.linalg.norm(pref))
            print(json.dumps({"sweep": name, "n": n, "precision": prec, "eps": eps, "t_build_s": round(t_build, 4),
                              "t_eval_s": t / steps, "points_per_s": n * steps / t, "E_pot": e,
                              "depth": info["depth"], "n_images": info["n_images"], "M": info["M"][:d],
                              "oracle_s": round(t_or, 2), "oracle_samples": len(idx)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="triclinic3d_4m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-cells", type=int, default=16, help="cells of the batched secondary line")
    ap.add_argument("--batch-nmax", type=int, default=20_000, help="largest cell of the batched line")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 2D and batched secondary lines")
    ap.add_argument("--sweep", action="store_true",
                    help="run the paper's wavy ring / sphere grid (Tables 2-4 shapes) instead of the benchmark")
    ap.add_argument("--sweep-n", type=int, default=1_000_000)
    ap.add_argument("--sweep-samples", type=int, default=32)
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: only the mixed plan, warm-up + steps evaluations, no other work")
    ap.add_argument("--ncu-setup", action="store_true",
                    help="profiling run: warm-up + steps set-ups (pdmk_set_sources) of the mixed plan, no evaluation")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
    if args.sweep:
        if rank == 0:
            run_sweep(args)
        return
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
    wl = WORKLOADS[args.workload]
    g = wl["make"]()
    n, d = g["y"].shape
    peaks, peak_kind = load_peaks()

    def make(prec, gg=g):
        pl = P.Plan(gg["L"], EPS, precision=prec, stream=stream.cuda_stream)
        pl.set_sources(gg["y"], gg["q"])
        return pl

    pot = torch.empty(n, dtype=torch.float64, device=dev)
    grad = torch.empty((n, d), dtype=torch.float64, device=dev)
    if args.ncu_setup:
        plan = P.Plan(g["L"], EPS, precision="mixed", stream=stream.cuda_stream)
        for _ in range(args.warmup + args.steps):
            plan.set_sources(g["y"], g["q"])
        torch.cuda.synchronize()
        print(json.dumps({"ncu_setup_run": True, "set_ups": args.warmup + args.steps,
                          "phases_ms_last": plan.setup_times()}))
        plan.close()
        return
    if args.ncu:
        plan = make("mixed")
        for _ in range(args.warmup + args.steps):
            plan.eval_device(pot, grad)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_run": True, "evals": args.warmup + args.steps,
                          "launches_per_eval": plan.info()["launches"]}))
        return
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    # ---- headline: mixed precision, device outputs, graph-replayed evaluations ----
    t_set0 = time.perf_counter()
    plan = make("mixed")
    torch.cuda.synchronize()
    t_set_sources = time.perf_counter() - t_set0  # plan + device tree build + layouts
    for _ in range(args.warmup):
        plan.eval_device(pot, grad)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    t_total = timed_device(plan, pot, grad, stream, flush, args.steps, 0)
    clocks = sampler.stop()
    value, ms_per_step, _ = replica_summary(t_total, n, args.steps, ws, pg, dev)
    pot_m = pot.cpu().numpy().copy()
    grad_m = grad.cpu().numpy().copy()
    info = plan.info()

    # ---- end to end through the C ABI with host buffers, every step: positions and charges
    # in (page-locked), tree build and layouts, evaluation, potential + gradient out
    y_host = torch.from_numpy(np.ascontiguousarray(g["y"])).pin_memory().numpy()
    q_host = torch.from_numpy(np.ascontiguousarray(g["q"])).pin_memory().numpy()
    pot_host = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    grad_host = torch.empty((n, d), dtype=torch.float64).pin_memory().numpy()
    reps = 5
    plan.set_sources(y_host, q_host)
    plan.eval(out=(pot_host, grad_host))
    t0 = time.perf_counter()
    for _ in range(reps):
        plan.set_sources(y_host, q_host)
        plan.eval(out=(pot_host, grad_host))
    e2e_t = (time.perf_counter() - t0) / reps
    setup_phases = {k: round(v, 2) for k, v in plan.setup_times().items()}
    e2e = {"value": ws * n / e2e_t, "unit": "points/s", "h2d_bytes_per_step": 8 * n * (d + 1),
           "d2h_bytes_per_step": 8 * n * (1 + d),
           "per_step": "pdmk_set_sources (positions + charges from pinned host memory, tree build and "
                       "layouts on the device, lists on the host) + pdmk_eval into pinned host arrays",
           "set_sources_phases_ms": setup_phases}
    # the same with fixed positions: charges in, potential + gradient out
    reps_c = max(3, args.steps // 2)
    plan.set_charges(q_host)
    plan.eval(out=(pot_host, grad_host))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps_c):
        plan.set_charges(q_host)
        plan.eval(out=(pot_host, grad_host))
    e2e_c = (time.perf_counter() - t0) / reps_c
    e2e_charges = {"value": ws * n / e2e_c, "unit": "points/s", "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": 8 * n * (1 + d),
                   "per_step": "pdmk_set_charges from pinned host memory + pdmk_eval into pinned host arrays"}
    plan.close()
    del plan

    # ---- FP64 comparator on the same workload ----
    plan64 = make("fp64")
    s64 = max(2, args.steps // 4)
    t64 = timed_device(plan64, pot, grad, stream, flush, s64, 2)
    pts64 = n * s64 / t64
    pot_64 = pot.cpu().numpy().copy()
    grad_64 = grad.cpu().numpy().copy()
    plan64.close()
    del plan64

    # ---- per-stage device times for the roofline ----
    stage_acc, pinfo = stage_profile(P, g, "mixed", stream, pot, grad, flush)

    out = None
    if rank == 0:
        # accuracy against the oracle: stored values at seeded targets (full-size workloads), or
        # a fresh oracle sample
        cpu_line = None
        if wl["golden"]:
            idx, pref, gref = golden_sample(wl["golden"])
            acc_sample = f"{len(idx)} seeded targets, stored oracle values (tests/golden/fullsize_{wl['golden']}.json)"
        else:
            rng = np.random.default_rng(11)
            idx = np.sort(rng.choice(n, 128, replace=False))
            pref, gref, _ = oracle_sample(g, idx, nthreads=os.cpu_count())
            acc_sample = f"{len(idx)} random targets, oracle with full-N structure factors"
        rel = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
        accuracy = {"E_pot_mixed": rel(pot_m[idx], pref), "E_grad_mixed": rel(grad_m[idx], gref),
                    "E_pot_fp64": rel(pot_64[idx], pref), "E_grad_fp64": rel(grad_64[idx], gref),
                    "sample": acc_sample}
        if not args.no_cpu_baseline:
            rng = np.random.default_rng(12)
            ns = 16 if n > 1_000_000 else 128
            cidx = np.sort(rng.choice(n, ns, replace=False))
            _, _, dt = oracle_sample(g, cidx, nthreads=os.cpu_count())
            cpu_line = {"value": ns / dt, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
                        "sample": f"{ns} random targets of the workload in one oracle call, including its "
                                  f"full-N reciprocal-space structure factors ({dt:.1f} s)"}
        fp32_peak, nsm, sm_mhz = fp32_peak_tflops(peaks)
        per_stage = stage_roofline(stage_acc, pinfo, d, fp32_peak)
        dominant = max(per_stage, key=lambda k: per_stage[k]["ms"]) if per_stage else None
        achieved = per_stage[dominant]["tflops"] if dominant else None
        out = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": wl["desc"], "eps": EPS, "precision": "mixed",
                       "l2": "flushed (256 MB write) between steps; inputs also exceed L2",
                       "depth": info["depth"], "n_images": info["n_images"], "M": info["M"][:d],
                       "near_pairs": pinfo["near_pairs"], "near_pairs_in": pinfo["near_pairs_in"],
                       "n_proxy": info["n_proxy"], "n_pw": info["n_pw"], "n_s": info["n_s"],
                       "kappa": info["kappa"], "device_bytes": info["device_bytes"]},
            "accuracy": accuracy,
            "fp64": {"value": pts64, "unit": "points/s", "ms_per_eval": 1e3 * t64 / s64,
                     "mixed_over_fp64": value / (ws * pts64)},
            "stages_ms": {k: round(v, 4) for k, v in stage_acc.items()}, "dominant_stage": dominant,
            "stage_roofline": per_stage,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": (achieved / fp32_peak) if achieved else None,
                         "traffic": STAGE_TRAFFIC.get(args.workload, {}).get(dominant),
                         "kernel": STAGE_KERNELS[d].get(dominant), "stage": dominant,
                         "peak_note": f"FP32 FMA pipes: {nsm} SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz "
                                      "(unit counts at the maximum clock; no measured FP32 peak exists)"},
            "cpu_baseline": cpu_line, "e2e": e2e, "e2e_fixed_positions": e2e_charges,
            "t_set_sources_s": t_set_sources,
            "gpu_launches": int(info["launches"]) * args.steps, "clocks": clocks,
        }
        out["config"]["launches_per_step"] = int(info["launches"])
        if not args.no_secondary:
            out["secondary"] = secondary_lines(P, torch, stream, flush, args, peaks)
    if not args.no_secondary:
        # every rank takes part in the batched line (its share of the cells)
        bl = batched_line(P, torch, stream, ncells=args.batch_cells, nmax=args.batch_nmax, ws=ws, rank=rank, pg=pg)
        if out is not None:
            out.setdefault("secondary", {})["batched"] = bl
    if out is not None:
        print(json.dumps(out))
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def secondary_lines(P, torch, stream, flush, args, peaks):
    """The 2D oblique 200k cell (mixed and FP64, accuracy on 128 oracle targets) and a bounded
    batch of 3D cells."""
    out = {}
    if args.workload != "oblique2d_200k":
        g = WORKLOADS["oblique2d_200k"]["make"]()
        n, d = g["y"].shape
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        grad = torch.empty((n, d), dtype=torch.float64, device="cuda")
        line = {"workload": WORKLOADS["oblique2d_200k"]["desc"]}
        res = {}
        for prec in ("mixed", "fp64"):
            pl = P.Plan(g["L"], EPS, precision=prec, stream=stream.cuda_stream)
            t0 = time.perf_counter()
            pl.set_sources(g["y"], g["q"])
            torch.cuda.synchronize()
            t_set = time.perf_counter() - t0
            steps = args.steps if prec == "mixed" else max(2, args.steps // 4)
            t = timed_device(pl, pot, grad, stream, flush, steps, 3)
            res[prec] = (pot.cpu().numpy().copy(), grad.cpu().numpy().copy())
            line[prec] = {"value": n * steps / t, "unit": "points/s", "ms_per_eval": 1e3 * t / steps,
                          "t_set_sources_s": t_set}
            pl.close()
        rng = np.random.default_rng(11)
        idx = np.sort(rng.choice(n, 128, replace=False))
        pref, gref, _ = oracle_sample(g, idx, nthreads=os.cpu_count())
        rel = lambda a, b: float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
        line["accuracy"] = {f"E_pot_{p}": rel(res[p][0][idx], pref) for p in res}
        line["accuracy"].update({f"E_grad_{p}": rel(res[p][1][idx], gref) for p in res})
        acc, pinfo = stage_profile(P, g, "mixed", stream, pot, grad, flush)
        fp32_peak, _, _ = fp32_peak_tflops(peaks)
        line["stages_ms"] = {k: round(v, 4) for k, v in acc.items()}
        line["stage_roofline"] = stage_roofline(acc, pinfo, d, fp32_peak)
        out["oblique2d_200k"] = line
    return out


if __name__ == "__main__":
    main()
