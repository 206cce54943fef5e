#!/usr/bin/env python
"""Benchmark: potential solves/s of the split nonlocal potential solver on a
4096 x 4096 grid (mixed precision vs FP64 on the same GPU), with the relative
error against the FP64 CPU oracle on the 512^2 stride-8 subsample, the
dominant kernel's fraction of the measured HBM bandwidth, an end-to-end
(host buffers) number, and the oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete solve (all eight kernels) of one 4096^2 density.
For N > 1 (torchrun, one rank per GPU) every rank solves its own densities
(independent problems, no data-path collective): weak scaling.
"""

from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "potential solves/s at 4096² (mixed vs FP64, same GPU) at rel err≤1e-6; %HBM peak"
WL = dict(n=4096, L=64.0, P=8.0, n_r=64, n_theta=256, count=16, seed=3)
WORKLOAD_NAME = ("rho=|u|^2, u = 16 seeded complex Gaussians, 4096^2 grid on [-64,64)^2, "
                 "P=8, 64 radial x 256 angular nodes, kappa=2, mixed precision (ES width 8)")
SUB = 8            # accuracy subsample stride (512^2 points)
N_ROT = 4          # rotating input/output pairs (4 x 268 MB > L2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle run (no accuracy / cpu_baseline keys)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-member batch measurement")
    ap.add_argument("--only-timed", action="store_true",
                    help="run only warmup + the timed mixed region (for profiler launch lists)")
    return ap.parse_args()


# --------------------------------------------------------------------------- oracle

def oracle_sample(rho: np.ndarray, node_frac: float = 1.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of one solve of
    the workload: I1 on the whole grid; the type-2 sums for a fraction of the
    polar nodes; the type-1 sums for those nodes on the 512^2 stride-8
    subsample.  Returns (estimated seconds for one full solve, phi on the
    subsample when node_frac == 1 else None, description)."""
    import oracle

    n, L = WL["n"], WL["L"]
    op = oracle.OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=WL["P"], n_r=WL["n_r"],
                             n_theta=WL["n_theta"])
    x = oracle.grid_axis(n, L)
    rows = np.arange(0, n, SUB)
    t0 = time.perf_counter()
    i1 = oracle.i1_padded_fft(rho, op)[np.ix_(rows, rows)]
    t1 = time.perf_counter()
    kx, ky, *_ = oracle.polar_nodes(op)
    D = oracle.polar_weights(op)
    m = kx.size
    take = np.arange(0, m, max(1, int(round(1.0 / node_frac))))
    frac = take.size / m
    rh = oracle.rho_hat_direct(rho, x, x, kx[take], ky[take])
    t2 = time.perf_counter()
    i2 = oracle.i2_direct_from_coeffs(D[take] * rh, kx[take], ky[take], x[rows], x[rows])
    t3 = time.perf_counter()
    sub_pts = rows.size * rows.size
    scale1 = (n * n) / sub_pts
    est = (t1 - t0) + (t2 - t1) / frac + (t3 - t2) * scale1 / frac
    desc = (f"one {n}^2 solve: I1 FFTs on the full grid; type-2 sums for {take.size} of {m} "
            f"nodes (x{1 / frac:.0f}); type-1 sums for those nodes on the {rows.size}^2 stride-{SUB} "
            f"subsample (x{scale1 / frac:.0f} to the full grid)")
    phi = (i1 + i2) if take.size == m else None
    return est, phi, desc, {"i1": t1 - t0, "type2": t2 - t1, "type1": t3 - t2}


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (read-only query) stamped with the host clock."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [f.strip() for f in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        win = [s for t, s in self.samples if t0 <= t <= t1 and len(s) >= 9]
        where = "timed region"
        if not win:
            win = [s for _, s in self.samples if len(s) >= 9]
            where = "whole run (no sample fell inside the timed region)"
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "window": "nvidia-smi unavailable"}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(s[1]) for s in win if num(s[1]) is not None]
        mx = [num(s[2]) for s in win if num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in win for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(win), "window": where}


# --------------------------------------------------------------------------- helpers

def code_only(src: str) -> str:
    """CUDA/C++ source without its comments and with whitespace runs collapsed:
    what the kernel hash covers, so that editing a comment does not mark the
    recorded counters stale (no string literal in the hashed files holds //)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return " ".join(src.split())


def kernel_hash(read=None) -> str:
    """Hash of the code of the pipeline's kernel sources; `read(name)` returns
    a file's text (default: the working tree)."""
    if read is None:
        def read(name):
            with open(os.path.join(ROOT, "paper_1409_2014_gb300", "csrc", name), encoding="utf-8") as fh:
                return fh.read()
    h = hashlib.sha256()
    for f in ("common.cuh", "kernels.cuh", "pipeline.cuh"):
        h.update(code_only(read(f)).encode())
    return h.hexdigest()[:16]


def algorithmic_bytes(stage: str, n: int, Q: int, csz: int, n_nodes: int, w: int, rsz: int,
                      n_items: int = 0, tile: int = 8) -> float:
    """Bytes one launch of a stage must move at minimum (inputs read once,
    outputs written once), for an n x n grid with band half-width Q."""
    A = csz * n * (n + 1)           # half-spectrum intermediate
    Bc = csz * n * (Q + 1)          # band columns of the row spectra
    band = csz * (Q + 1) * (2 * Q + 1)
    nodes = n_nodes * (8 + 2 * w * rsz + 8 + csz)  # q0, weights, D, c
    return float({
        "row_fwd": 8 * n * n + A + Bc,
        "col_main": 2 * A + (n + 1) * (n + 4) * 4 * (csz == 8),  # FP32: + the multiplier table rows
        "band_fwd": Bc + band,
        "interp": band + nodes,
        "spread": nodes + n_items * tile * tile * csz,     # node data in, one partial tile per item out
        "spread_reduce": n_items * tile * tile * csz + band,
        "band_inv": band + Bc,
        "row_inv": A + Bc + 8 * n * n,
    }[stage])


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_traffic(stage: str, workload: str):
    """ncu dram bytes per launch recorded for this kernel source, else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tab = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = tab.get(f"{stage}|{workload}")
    if not ent or ent.get("kernel_hash") != kernel_hash():
        return None
    return ent.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- arms

def dist_setup(use_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return world, rank, local


def replica_seed(rank: int) -> int:
    """Each rank solves its own density (independent units, no exchange)."""
    return WL["seed"] + rank


def max_over_ranks(v: float, world: int, device=None) -> float:
    """The slowest rank's time (the job's time); identity for one process."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: each rank has a fixed share)."""
    return world * units_per_rank / t_max


def run_reference(args):
    """The oracle as the reference arm: each step one bounded oracle sample."""
    world, rank, _ = dist_setup(False)
    if rank != 0:
        return
    import synth

    n, L = WL["n"], WL["L"]
    rho = synth.density_abs2(n, n, L, L, WL["seed"], WL["count"])
    # size the per-step sample so that warmup + steps fit in about three minutes
    _, _, _, comp = oracle_sample(rho, node_frac=1.0 / 64)
    budget = 180.0 / max(1, args.steps + args.warmup)
    frac = 1.0 / 64
    for f in (1.0, 1.0 / 4, 1.0 / 16):
        if comp["i1"] + (comp["type2"] + comp["type1"]) * 64 * f <= budget:
            frac = f
            break
    for _ in range(args.warmup):
        oracle_sample(rho, frac)
    ests = []
    desc = ""
    for _ in range(args.steps):
        est, _, desc, _ = oracle_sample(rho, frac)
        ests.append(est)
    est = float(np.mean(ests))
    value = 1.0 / est
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "n": n, "L": L},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_bench(dev, max_time, barrier, reps=5):
    """64 seeded densities (4-16 Gaussians) with grids drawn from {256, 512,
    1024, 2048}^2 on [-32,32)^2, P = 8, 64 x 256 nodes: mixed plans in one
    batch replayed as a CUDA graph, versus 64 separate FP64 solves."""
    import torch

    import synth
    from paper_1409_2014_gb300 import Batch, Plan

    members = synth.batch_members(seed=5, count=64)
    sizes = sorted({m[0] for m in members})
    rhos = [torch.from_numpy(synth.density_sum(n, n, 32.0, 32.0, seed=s, count=k)).to(dev)
            for n, k, s in members]
    phis = [torch.empty_like(r) for r in rhos]
    out = {"members": len(members), "sizes": {str(n): sum(1 for m in members if m[0] == n) for n in sizes},
           "domain": "[-32,32)^2, P=8, 64x256 nodes"}
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for prec in ("mixed", "fp64"):
        plans = {n: Plan(n, lx=32.0, cut_radius=8.0, n_r=64, n_theta=256, precision=prec, device=dev)
                 for n in sizes}
        if prec == "mixed":
            b = Batch([plans[m[0]] for m in members], rhos, phis)
            b.capture_graph()
            b.solve()
            barrier()
            e0.record(stream)
            for _ in range(reps):
                b.solve()
            e1.record(stream)
            barrier()
            t = max_time(e0.elapsed_time(e1) / 1000.0)
            out["mixed_graph_batch"] = {"solves_per_s": reps * len(members) / t, "ms_per_batch": 1e3 * t / reps}
            b.close()
        else:
            for (n, _, _), r, f in zip(members, rhos, phis):
                plans[n].solve(r, f)
            barrier()
            e0.record(stream)
            for _ in range(reps):
                for (n, _, _), r, f in zip(members, rhos, phis):
                    plans[n].solve(r, f)
            e1.record(stream)
            barrier()
            t = max_time(e0.elapsed_time(e1) / 1000.0)
            out["fp64_separate"] = {"solves_per_s": reps * len(members) / t, "ms_per_batch": 1e3 * t / reps}
        for p in plans.values():
            p.close()
    out["speedup"] = out["mixed_graph_batch"]["solves_per_s"] / out["fp64_separate"]["solves_per_s"]
    return out


def run_ours(args):
    import torch

    world, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1409_2014_gb300 import Plan
    from paper_1409_2014_gb300.build import build
    import synth

    build()
    n, L = WL["n"], WL["L"]
    rho_np = synth.density_abs2(n, n, L, L, replica_seed(rank), WL["count"])
    rho0 = torch.from_numpy(rho_np).to(dev)
    ins = [rho0.clone() for _ in range(N_ROT)]
    outs = [torch.empty_like(rho0) for _ in range(N_ROT)]
    del rho0

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks_dev(v: float) -> float:
        return max_over_ranks(v, world, dev)

        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    plan = Plan(n, lx=L, cut_radius=WL["P"], n_r=WL["n_r"], n_theta=WL["n_theta"],
                precision="mixed", device=dev)
    info = plan.info
    stream = torch.cuda.current_stream(dev)

    clocks = ClockSampler(local)
    for i in range(args.warmup):
        plan.solve(ins[i % N_ROT], outs[i % N_ROT])
    barrier()
    # ---- timed region: K mixed solves; per-kernel CUDA events are recorded live
    # around the first n_prof of them (events between kernels cost ~3 % per
    # solve, so not on every one)
    n_prof_req = min(args.steps, 200)
    plan.profile_begin(n_prof_req)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(stream)
    for i in range(args.steps):
        plan.solve(ins[i % N_ROT], outs[i % N_ROT])
    e1.record(stream)
    barrier()
    tw1 = time.time()
    ms_total = e0.elapsed_time(e1)
    stage_ms, n_prof = plan.profile_end()
    n_stages = len(stage_ms)
    clk = clocks.summary(tw0, tw1)
    clocks.stop()
    t_max = max_over_ranks_dev(ms_total / 1000.0)
    value = job_value(world, args.steps, t_max)
    ms_per_step = t_max * 1000.0 / args.steps
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s",
                              "ms_per_step": ms_per_step, "steps": args.steps,
                              "stages_ms_total": stage_ms, "only_timed": True}), flush=True)
        plan.close()
        return

    # ---- FP64 solver on the same GPU (same input), timed separately
    plan64 = Plan(n, lx=L, cut_radius=WL["P"], n_r=WL["n_r"], n_theta=WL["n_theta"],
                  precision="fp64", device=dev)
    k64 = max(3, min(args.steps, 50))
    for i in range(2):
        plan64.solve(ins[i % N_ROT], outs[i % N_ROT])
    barrier()
    e0.record(stream)
    for i in range(k64):
        plan64.solve(ins[i % N_ROT], outs[i % N_ROT])
    e1.record(stream)
    barrier()
    t64 = max_over_ranks_dev(e0.elapsed_time(e1) / 1000.0)
    value64 = world * k64 / t64

    # results of both paths on the first input, for the accuracy check
    phi_mixed = plan.solve(ins[0]).cpu().numpy()
    phi_64 = plan64.solve(ins[0]).cpu().numpy()
    plan64.close()

    # ---- the standard periodic FFT solver (no split, no padding) on the same input
    standard = {}
    for prec, reps in (("mixed", max(3, min(args.steps, 200))), ("fp64", max(3, min(args.steps, 20)))):
        ps = Plan(n, lx=L, partition="none", precision=prec, device=dev)
        for i in range(2):
            ps.solve(ins[i % N_ROT], outs[i % N_ROT])
        barrier()
        e0.record(stream)
        for i in range(reps):
            ps.solve(ins[i % N_ROT], outs[i % N_ROT])
        e1.record(stream)
        barrier()
        ts = max_over_ranks_dev(e0.elapsed_time(e1) / 1000.0)
        standard[prec] = {"solves_per_s": world * reps / ts, "ms_per_step": ts * 1000.0 / reps, "steps": reps}
        ps.close()

    # ---- end to end through the public API with host buffers: every step copies its
    # density from pinned host memory and its potential back (dsnu_solve_host_stream,
    # uploads and downloads overlapped with the neighbouring steps' solves)
    rho_h = torch.from_numpy(rho_np).pin_memory()
    phi_h = torch.empty_like(rho_h).pin_memory()
    ke = max(3, min(args.steps, 100))
    plan.solve_host_stream([rho_h, rho_h], [phi_h, phi_h])
    barrier()
    e0.record(stream)
    plan.solve_host_stream([rho_h] * ke, [phi_h] * ke)
    e1.record(stream)
    barrier()
    te = max_over_ranks_dev(e0.elapsed_time(e1) / 1000.0)
    e2e = {"value": world * ke / te, "unit": "solves/s", "h2d_bytes_per_step": int(rho_h.numel() * 8),
           "d2h_bytes_per_step": int(phi_h.numel() * 8), "steps": ke,
           "api": "dsnu_solve_host_stream (pinned host in/out, copies overlapped with solves)"}
    phi_e2e = phi_h.numpy().copy()
    assert np.array_equal(phi_e2e, phi_mixed), "streamed host solve differs from the device solve"

    # ---- roofline of the dominant kernel
    csz, rsz = 8, 4
    avg = {k: v / max(1, n_prof) for k, v in stage_ms.items()}
    dom = max(avg, key=avg.get)
    peak, peak_src = load_peaks()
    alg = algorithmic_bytes(dom, n, info.band_q, csz, info.n_nodes, info.kernel_width, rsz,
                            info.n_items, info.spread_tile)
    achieved = alg / (avg[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "unit": "GB/s", "frac": achieved / peak,
                "algorithmic_bytes_per_launch": alg, "avg_ms": avg[dom],
                "traffic": load_traffic(dom, "4096sq_mixed"),
                "stages_ms": {k: round(v, 5) for k, v in avg.items()},
                "stage_share": {k: round(v / sum(avg.values()), 4) for k, v in avg.items()},
                # every kernel: algorithmic bytes / live duration, as a fraction of the measured peak
                "hbm_frac_per_kernel": {
                    k: round(algorithmic_bytes(k, n, info.band_q, csz, info.n_nodes, info.kernel_width, rsz,
                                               info.n_items, info.spread_tile) / (v * 1e-3) / 1e9 / peak, 4)
                    for k, v in avg.items() if v > 0}}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "n": n, "L": L, "P": WL["P"], "n_r": WL["n_r"],
                   "n_theta": WL["n_theta"], "kernel_width": info.kernel_width, "band_q": info.band_q,
                   "spread_tile_split_chunk": [info.spread_tile, info.spread_split, info.spread_chunk],
                   "global_batch": world, "parallelism": f"independent solves x{world}",
                   "l2": f"inputs larger than L2: {N_ROT} rotating 134 MB input/output pairs"},
        "fp64": {"value": value64, "unit": "solves/s", "ms_per_step": t64 * 1000.0 / k64, "steps": k64,
                 "dtype": "f64", "mixed_speedup": value / value64},
        "roofline": roofline,
        "standard_fft": {"what": "standard periodic FFT solver (kappa = 1, p = 0), same grid and input",
                         **standard},
        "e2e": e2e,
        "gpu_launches": args.steps * n_stages,
        "clocks": clk,
    }

    if not args.no_batch:
        line["batch"] = batch_bench(dev, max_over_ranks_dev, barrier)

    if rank == 0 and not args.no_cpu_baseline:
        est, phi_ref, desc, _ = oracle_sample(rho_np, 1.0)
        sub = (slice(0, n, SUB), slice(0, n, SUB))
        acc = {}
        for name, phi in (("mixed", phi_mixed), ("fp64", phi_64)):
            d = phi[sub] - phi_ref
            acc[name] = {"rel_linf": float(np.abs(d).max() / np.abs(phi_ref).max()),
                         "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(phi_ref))}
        line["accuracy_vs_oracle"] = {"subsample": f"{n // SUB}^2 stride-{SUB}", **acc}
        line["cpu_baseline"] = {"value": 1.0 / est, "unit": "solves/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
