#!/usr/bin/env python
"""Benchmark of the two-site TDVP hot path on B300.

Workload (the configuration the metric is quoted on): the effective
Hamiltonian of a mid-chain bond of the L=60 chain, U(1)xSU(2) reduced tensors,
multiplets (Q, 2S) with Q in [-12, 12], 2S in [0, 12], Q + 2S = k (mod 2),
d(Q,S) = round(D0 exp(-Q^2/18 - S^2/4.5)) with D0 the smallest value giving a
U(1)-equivalent bond dimension >= 4096 on both outer bonds (k = 30 and 32),
entries i.i.d. complex normal from a fixed seed, each tensor normalised, exact
particle-hole-frame Fermi-Hubbard MPO with U=4, J=1.

One step = one Krylov exponential exp(-i tau H_eff) theta at that bond: k
Lanczos matvecs (H_eff theta), full re-orthogonalisation, the small
exponential, and the assembly of the result, all on the GPU.  The metric value
is the algorithmic H_eff.psi throughput (8 flops per complex multiply-add of the
reduced block products) over the whole step.

--impl reference runs the CPU oracle (U(1)xU(1) block-sparse brute force) on a
bounded sample of output blocks of the same workload expanded to U(1)xU(1).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "H_eff.psi TFLOP/s & sec/sweep, L=60 chi=4096, split vs FP64"
UNIT = "TFLOP/s"


def config2_tables():
    D0, tab = synth.gaussian_table_for_chi(4096, 30)
    left = [(Q + 30, ts, d) for (Q, ts, d) in tab]
    right = [(Q + 32, ts, d) for (Q, ts, d) in tab]
    return D0, tab, left, right


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def init_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return rank, ws


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------------------
# engine arm
# ---------------------------------------------------------------------------

def run_engine(args):
    import torch

    from paper_2606_04771_b300 import BondProblem, lib
    import ctypes as C

    rank, ws = init_dist()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    D0, tab, left, right = config2_tables()
    seed = synth.SEED_BOND + rank
    bp = BondProblem(left, right, J=1.0, U=4.0, symmetry="su2", precision=args.precision,
                     krylov_max=args.krylov, krylov_tol=0.0, stream=stream.cuda_stream, device=dev)
    keys, dims, offs, n = bp.blocks(0)
    _, ld, _, nl = bp.blocks(1)
    _, rd, _, nr = bp.blocks(2)
    g = synth.rng(seed)

    def normed(k):
        v = synth.complex_normal(g, k)
        return v / np.linalg.norm(v)

    theta_h = normed(n)
    bp.set_env(1, normed(nl))
    bp.set_env(2, normed(nr))
    flops_mv = bp.heff_flops()
    theta = torch.from_numpy(theta_h).to(f"cuda:{dev}")
    out = torch.empty_like(theta)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")  # > L2 (126 MB)

    kdim = args.krylov

    def step(x, y):
        # one Krylov exponential of tau H_eff built from kdim matvecs with full
        # re-orthogonalisation; the engine routine lives in the library
        bp.krylov_expm(x, y, tau=0.025)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step(theta, out)
        stream.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with ClockSampler(dev) as clk:
            for i in range(args.steps):
                flush.zero_()
                evs[i][0].record(stream)
                step(theta, out)
                evs[i][1].record(stream)
            stream.synchronize()
        torch.cuda.synchronize()
    barrier(ws)
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = max_over_ranks(sum(ms) / len(ms), ws)
    mv_per_step = bp.last_krylov_dim()
    flops_step = flops_mv * mv_per_step
    value = ws * flops_step / (ms_step * 1e-3) / 1e12

    # per-kernel profile of the dominant kernel (the block GEMM stages)
    pms = (C.c_double * 3)()
    pfl = (C.c_longlong * 3)()
    pby = (C.c_longlong * 3)()
    from paper_2606_04771_b300._lib import check

    check(lib().tdvp_heff_profile(bp.h, 5, pms, pfl, pby))
    stage_ms = list(pms)
    gemm_ms = stage_ms[0] + stage_ms[2]
    gemm_flops = pfl[0] + pfl[2]
    peaks, peak_kind = load_peaks()
    if args.precision == "fp64":
        peak = 1250.0 / 1000.0  # TFLOP/s, FP64 nominal (no FP64 tensor path on B300)
        bound, pnote, issued = "alu", "FP64 nominal 1.25 TFLOP/s (recipe table)", 1
    elif args.precision == "3xtf32":
        peak = peaks["bf16_tflops"] * 1.1 / 2.25
        bound, pnote, issued = "tensor", f"TF32 = {peak_kind} bf16 burst x 1.1/2.25 (nominal ratio)", 3
    else:
        peak = peaks["bf16_tflops"]
        bound, pnote, issued = "tensor", f"{peak_kind} bf16 burst (BF16X4 issues 10 digit products per MAC)", 10
    achieved = gemm_flops / (gemm_ms * 1e-3) / 1e12
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "grouped block GEMM (stages 1+3 of H_eff.psi)",
                "peak_source": pnote, "stage_ms": stage_ms,
                "tensor_pipe_frac_upper": achieved * issued / peak}

    # end to end through the C ABI with host buffers: H2D of theta, the step, D2H of the result
    host_in = theta_h.copy()
    host_out = np.empty_like(host_in)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, min(args.steps, 5))):
        bp.krylov_expm(host_in, host_out, tau=0.025)
    e2e_s = (time.perf_counter() - t0) / max(1, min(args.steps, 5))
    e2e = {"value": ws * flops_step / e2e_s / 1e12, "unit": UNIT, "h2d_bytes_per_step": int(host_in.nbytes),
           "d2h_bytes_per_step": int(host_out.nbytes)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "c128 (f64)", "3xtf32": "c128 storage, 3xTF32 products", "bf16x4": "c128 storage, BF16x4 digit products"}[args.precision],
        "data": "synthetic (seeded complex normal tensors, paper-shaped sector table)",
        "config": {"workload": "H_eff Krylov step at a mid-chain bond of L=60, U(1)xSU(2), chi=4096 (U(1)-equivalent)",
                   "chi": int(sum(d * (ts + 1) for (_, ts, d) in tab)), "chi_su2": int(sum(d for (_, _, d) in tab)),
                   "d_max": int(max(d for (_, _, d) in tab)), "multiplets": len(tab), "D0": D0,
                   "theta_elems": int(n), "matvec_gflop": flops_mv / 1e9, "krylov_dim": mv_per_step,
                   "precision": args.precision, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{ws} (independent bonds, no collective)"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": bp.launches_per_step() * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    bp.close()


# ---------------------------------------------------------------------------
# oracle arm (CPU): brute-force U(1)xU(1) blocks of the same workload
# ---------------------------------------------------------------------------

def oracle_problem(seed):
    from oracle import heff

    D0, tab, left, right = config2_tables()
    u1 = synth.to_u1u1(tab)
    lb = heff.Bond([(Q + 30, tz, d) for (Q, tz, d) in u1], su2=False)
    rb = heff.Bond([(Q + 32, tz, d) for (Q, tz, d) in u1], su2=False)
    keys = heff.theta_blocks(lb, rb)
    lk, rk = heff.left_env_blocks(lb, lb), heff.right_env_blocks(rb, rb)
    g = synth.rng(seed)
    th = [synth.complex_normal(g, (lb.sectors[k[0]][2], rb.sectors[k[4]][2])) for k in keys]
    Lb = [synth.complex_normal(g, (lb.sectors[k[0]][2], lb.sectors[k[2]][2])) for k in lk]
    Rb = [synth.complex_normal(g, (rb.sectors[k[0]][2], rb.sectors[k[2]][2])) for k in rk]
    return tab, lb, rb, keys, th, lk, Lb, rk, Rb


def cpu_baseline(budget_s=20.0, seed=synth.SEED_BOND):
    """Oracle timed on the host cores on a bounded sample of output blocks."""
    from oracle import blockwise, heff

    tab, lb, rb, keys, th, lk, Lb, rk, Rb = oracle_problem(seed)
    W = heff.shiba_mpo_tensor(1.0, 4.0)
    order = synth.rng(seed + 99).permutation(len(keys))
    t0 = time.perf_counter()
    flops, done = 0, 0
    for i in order:
        _, f = blockwise.heff2_u1_blocks(lb, rb, keys, th, lk, Lb, rk, Rb, W, [keys[i]])
        flops += f
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    total_u1 = sum(1 for _ in keys)
    rate = flops / dt / 1e12  # TFLOP/s of U(1)xU(1) algorithmic work
    return {"value": rate, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "kind": "oracle",
            "sample": f"{done} of {total_u1} U(1)xU(1) output blocks of the chi=4096 bond "
                      f"({flops / 1e9:.1f} GFLOP of U(1)xU(1) block products in {dt:.1f} s, numpy/OpenBLAS FP64)"}


def run_reference(args):
    rank, ws = init_dist()
    if rank != 0:
        return
    t = []
    vals = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(budget_s=args.cpu_seconds / max(1, args.steps))
        if i >= args.warmup:
            t.append(time.perf_counter() - t0)
            vals.append(cb["value"])
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(t), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic", "impl": "reference",
            "config": {"workload": "H_eff Krylov step at a mid-chain bond of L=60, U(1)xSU(2), chi=4096 (U(1)-equivalent)",
                       "precision": "fp64", "reference": "CPU oracle, U(1)xU(1) brute force, bounded sample"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--precision", default="bf16x4", choices=["fp64", "3xtf32", "bf16x4"])
    ap.add_argument("--krylov", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
