"""Benchmark of the STEV hot path: cell-solves/s at 1,048,576 cells.

One step = one stev_solve of every cell of the workload (32 species / 150
reactions, T0 U[800,2200] K, P U[1,5] atm, Y0 Dirichlet(0.5), dt = 1e-3 s),
i.e. one pass of the whole hot path over one batch.  The line's value is the
mixed-precision path with cp/R from the thermo network ("mixed+MLP", the
network trained on the GPU before the timed region); the same cells are
timed once with the polynomial thermo ("mixed_poly") and once on the plain
FP64 path ("plain_fp64").  Warm-up solves run the same kernel and launch
configuration on the first --warmup-cells cells.  Cells are independent,
so with N GPUs every rank solves its own batch (weak scaling, no collective on
the data path; a barrier only brackets the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

Smaller cases for profiling: --cells N and --max-iters K shrink the workload
(the line then names them in config).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-solves/s at 1M cells: mixed+MLP vs plain FP64 STEV, 1 B300; p99 latency"
UNIT = "cell-solves/s"
N_CELLS = 1 << 20

# FP64-pipe cost of CUDA's exp() and log() in DFMA-equivalents, measured on
# B300 by csrc/alu_peaks.cu (dfma 1.667/clk/SM, exp 0.104, log 0.055, div 0.222)
EXP_OPS, LOG_OPS, DIV_OPS = 16.0, 30.0, 7.5
# FP64 pipe peak: 1.667 DFMA/clk/SM x 148 SMs at the probe's 1919 MHz under load
FP64_PEAK_OPS = 4.733e11
# DRAM bytes per cell of one launch, from the ncu captures summarised in
# profiles/ (3,108- and 1,628-cell cases; reads only: the small cases' output
# writes stay in L2), scaled to the full launch by the cells it processes.
# Set to None when the kernel changes after the capture.
DRAM_BYTES_PER_CELL = {"mixed": 924160 / 3108, "fp64": 528896 / 1628, "mixed+mlp": None}


def fp64_ops_per_cell_step(S: int, R: int, Rrev: int, nnz: int) -> float:
    """Algorithmic FP64 work of one STEV iteration of one cell, in DFMA-equivalents.

    Counted from the method (not from the kernel): per species thermo (cp 4,
    H/RT 6, G/RT 7 ops), mixture and cp sums (3), gamma and concentration
    (3 + 1 division), production-rate bookkeeping (dY/dt 2, H.wdot 1),
    limiter (4 + 1 division amortised by the min), Euler (1); per reaction
    ln kf (2) + exp, reactant and product products (2), dG (3), ln kr (2) +
    exp, net rate and rOF (2); one FMA per stoichiometric entry; per
    reversible reaction the history entry (1), the N-point window sum of
    Eq. 9's D0 (N-1) and the rOF update (3); per cell-step log T, 1/T and the
    scalar updates (~12 ops + log + 2 divisions)."""
    species = S * (4 + 6 + 7 + 3 + 3 + DIV_OPS + 3 + 4 + 1)
    reactions = R * (2 + 2 + 3 + 2 + 2 + 2 * EXP_OPS)
    gather = nnz
    dft = Rrev * (1 + 12 + 3)
    scalars = 12 + LOG_OPS + 3 * DIV_OPS
    return species + reactions + gather + dft + scalars


def mixed_fp64_ops_per_cell_step(S: int) -> float:
    """FP64 work the mixed-precision plan itself requires per cell-step, in
    DFMA-equivalents: per species G/RT (7) and its split into a float pair (2)
    and the FP64 Euler update with its conversion (2); per cell log T, 1/T and
    the h / t_rem / T bookkeeping (~10).  Everything else runs on the FP32 and
    MUFU pipes, which have 64x and 16x the FP64 pipe's rate."""
    return S * (7 + 2 + 2) + LOG_OPS + DIV_OPS + 10


def workload(n_cells: int, rank: int = 0):
    from paper_1905_09395_b300 import synth
    return synth.scale_case(n_cells, seed=1 + 1000 * rank)


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" +
                                      self.FIELDS, "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.25)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 4 + k and r[4 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup(n_gpus: int):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return dist.get_rank(), dist.get_world_size(), dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def cpu_baseline(mech, T, P, Y, dt, target_s: float = 15.0, **opts):
    """The oracle as it stands on this host's cores, on a bounded sample."""
    import oracle
    cores = os.cpu_count() or 1
    n = max(cores, 8)
    t0 = time.time()
    oracle.solve(mech, T[:n], P[:n], Y[:n], dt, n_threads=cores, **opts)
    first = time.time() - t0
    # grow the sample to ~target_s of work (cells are independent and alike)
    n2 = int(min(len(T), max(n, n * target_s / max(first, 1e-3))))
    if n2 > n:
        t0 = time.time()
        oracle.solve(mech, T[:n2], P[:n2], Y[:n2], dt, n_threads=cores, **opts)
        first = time.time() - t0
        n = n2
    return {"value": n / first, "unit": UNIT, "cores": min(cores, n), "kind": "oracle",
            "sample": "first %d cells of the same workload, %.1f s" % (n, first)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle (plain C) on a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    mech, T, P, Y, dt = workload(args.cells)
    cores = os.cpu_count() or 1
    opts = {} if args.max_iters is None else {"max_iters": args.max_iters}
    per_step = max(cores, 8) * 2
    off = 0
    for _ in range(args.warmup):
        oracle.solve(mech, T[off:off + per_step], P[off:off + per_step], Y[off:off + per_step],
                     dt, n_threads=cores, **opts)
        off += per_step
    t0 = time.time()
    for _ in range(args.steps):
        oracle.solve(mech, T[off:off + per_step], P[off:off + per_step], Y[off:off + per_step],
                     dt, n_threads=cores, **opts)
        off += per_step
    el = time.time() - t0
    val = per_step * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "syn32x150, %d cells (oracle: %d-cell sample per step)"
                       % (args.cells, per_step), "precision": "fp64"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d cells per step, %d steps" % (per_step, args.steps)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def timed_solves(m, Td, Pd, Yd, dt, out, steps, warmup, warmup_cells, stream, dist=None,
                 sample_clocks=None):
    """W warm-up solves on the first warmup_cells cells (same kernel and launch
    configuration), then K timed solves of every cell, CUDA events on the
    launching stream, synchronised and barriered on both sides."""
    import torch
    nw = min(Td.shape[0], warmup_cells)
    wout = tuple(x[:nw] for x in out)
    for _ in range(warmup):
        m.solve(Td[:nw], Pd[:nw], Yd[:nw], dt, out=wout)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.time()
    for k in range(steps):
        ev[k][0].record(stream)
        m.solve(Td, Pd, Yd, dt, out=out)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.time() - t0
    barrier(dist)
    return [a.elapsed_time(b) for a, b in ev], wall, nw


def run_uneven(args):
    """Uneven independent batches (64 batches, log-uniform 1k-256k cells, the
    53/325 mechanism, dt 5e-4 s) in ONE batched launch per step, against the
    same batches as one stev_solve launch each."""
    import torch
    from paper_1905_09395_b300 import Mechanism, binding, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    mech, host_batches, dt = synth.uneven_case(args.uneven_scale)
    extra = {} if args.max_iters is None else {"max_iters": args.max_iters}
    m = Mechanism(mech, precision=binding.MIXED, **extra)
    info = None
    if args.thermo == "mlp":
        t0 = time.time()
        Ts = np.random.default_rng(2024).uniform(300.0, 3000.0, size=args.mlp_samples)
        hist = m.mlp_train(Ts, epochs=args.mlp_epochs, batch=4096, lr=2e-3, seed=7)
        m.set_options(thermo=binding.THERMO_MLP)
        info = {"final_loss": float(hist[-1]), "train_s": time.time() - t0}
    batches = [tuple(torch.from_numpy(a).to(dev) for a in b) for b in host_batches]
    total = int(sum(b[0].shape[0] for b in batches))
    # warm-up: the first batch alone, the same kernel and launch configuration
    for _ in range(args.warmup):
        m.solve_batched(batches[:1], dt)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            outs = m.solve_batched(batches, dt)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    iters = np.concatenate([o[2].cpu().numpy() for o in outs]).astype(np.int64)
    status = np.bincount(np.concatenate([o[3].cpu().numpy() for o in outs]), minlength=4)
    # the same batches as separate launches, back to back on one stream
    e0.record()
    for b in batches:
        m.solve(*b, dt)
    e1.record()
    torch.cuda.synchronize()
    ms_sep = e0.elapsed_time(e1)
    line = {"metric": "cell-solves/s, 64 uneven batches in one persistent launch", "value":
            total / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "syn53x325, 64 batches log-uniform 1k-256k cells x %g "
                                   "(%d cells), T0 U[700,2500] K, P U[1,5] atm, Y0 "
                                   "Dirichlet(0.5), dt 5e-4 s" % (args.uneven_scale, total),
                       "precision": "mixed", "thermo": args.thermo},
            "separate_launches": {"value": total / (ms_sep / 1e3), "ms": ms_sep},
            "cell_steps_per_s": float(iters.sum()) / (ms / 1e3),
            "iters": {"mean": float(iters.mean()), "p50": float(np.percentile(iters, 50)),
                      "p99": float(np.percentile(iters, 99)), "max": int(iters.max())},
            "cell_status": {"ok": int(status[0]), "maxiter": int(status[1]),
                            "nonfinite": int(status[2]), "trange": int(status[3])},
            "thermo_net": info, "gpu_launches": args.steps, "clocks": clk.summary()}
    print(json.dumps(line))
    m.close()
    return 0


def run_ours(args):
    import torch
    from paper_1905_09395_b300 import Mechanism, binding

    rank, world, dist = dist_setup(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mech, T, P, Y, dt = workload(args.cells, rank)
    S, R = mech.n_species, mech.n_reactions
    Rrev, nnz = int(mech.reversible.sum()), len(mech.rxn_species)
    extra = {} if args.max_iters is None else {"max_iters": args.max_iters}
    prec = binding.MIXED if args.precision == "mixed" else binding.FP64
    m = Mechanism(mech, precision=prec, **extra)
    mlp_info = None
    if args.precision != "mixed":
        args.thermo = "poly"
    if args.thermo == "mlp":
        t0 = time.time()
        Ts = np.random.default_rng(2024).uniform(300.0, 3000.0, size=args.mlp_samples)
        hist = m.mlp_train(Ts, epochs=args.mlp_epochs, batch=4096, lr=2e-3, seed=7)
        m.set_options(thermo=binding.THERMO_MLP)
        mlp_info = {"net": "1-64-64-%d tanh, BF16 weights, FP32 accumulate" % (3 * S),
                    "train_samples": args.mlp_samples, "epochs": args.mlp_epochs,
                    "final_loss": float(hist[-1]), "train_s": time.time() - t0,
                    "supplies": "cp/R and H/RT (energy equation), 300-3000 K"}
    n = len(T)
    Td, Pd, Yd = (torch.from_numpy(a).to(dev) for a in (T, P, Y))
    out = (torch.empty_like(Td), torch.empty_like(Yd), torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n, dtype=torch.uint8, device=dev))
    stream = torch.cuda.current_stream(dev)

    with ClockSampler(local) as clk:
        ms, wall, nw = timed_solves(m, Td, Pd, Yd, dt, out, args.steps, args.warmup,
                                    args.warmup_cells, stream, dist)
    dev_s = sum(ms) / 1e3
    it_np = out[2].cpu().numpy()
    cell_steps = int(it_np.astype(np.int64).sum())
    status = np.bincount(out[3].cpu().numpy(), minlength=4)

    t_max = dev_s
    total_cells = n * args.steps
    if dist is not None:
        t = torch.tensor([dev_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        c = torch.tensor([float(total_cells)], device=dev)
        dist.all_reduce(c)
        total_cells = int(c.item())
    value = total_cells / t_max

    # end to end through the host-pointer entry point, pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        hT, hP, hY = pin(T), pin(P), pin(Y)
        ho = (torch.empty(n, dtype=torch.float64).pin_memory().numpy(),
              torch.empty((n, S), dtype=torch.float64).pin_memory().numpy(),
              torch.empty(n, dtype=torch.int32).pin_memory().numpy(),
              torch.empty(n, dtype=torch.uint8).pin_memory().numpy())
        m.solve_host(hT[:nw], hP[:nw], hY[:nw], dt, out=tuple(x[:nw] for x in ho))
        ke = max(1, args.e2e_steps)
        barrier(dist)
        t0 = time.time()
        for _ in range(ke):
            m.solve_host(hT, hP, hY, dt, out=ho)
        el = time.time() - t0
        if dist is not None:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": n * world * ke / el, "unit": UNIT,
               "h2d_bytes_per_step": int(hT.nbytes + hP.nbytes + hY.nbytes),
               "d2h_bytes_per_step": int(sum(x.nbytes for x in ho)), "steps": ke}
    m.close()

    def one_solve(mc, ops):
        """One timed solve of the same cells by another configuration."""
        msx, _, _ = timed_solves(mc, Td, Pd, Yd, dt, out, 1, args.warmup, args.warmup_cells,
                                 stream, dist)
        itx = out[2].cpu().numpy().astype(np.int64)
        tx = msx[0] / 1e3
        if dist is not None:
            t = torch.tensor([tx], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tx = float(t.item())
        ach = ops * int(itx.sum()) / (msx[0] / 1e3)
        return {"value": n * world / tx, "unit": UNIT, "ms_per_step": tx * 1e3, "steps": 1,
                "warmup": args.warmup, "cell_steps_per_s": int(itx.sum()) / tx,
                "roofline": {"bound": "alu", "achieved": 2 * ach / 1e12,
                             "peak": 2 * FP64_PEAK_OPS / 1e12, "unit": "TFLOP/s",
                             "frac": ach / FP64_PEAK_OPS, "traffic": None,
                             "ops_per_cell_step": ops}}

    # the same cells with the polynomial thermo (what the network gains) and
    # with the plain FP64 path (what mixed precision gains)
    mixed_poly, plain = None, None
    if args.precision == "mixed" and args.thermo == "mlp" and not args.no_poly_compare:
        mp = Mechanism(mech, precision=binding.MIXED, **extra)
        mixed_poly = one_solve(mp, mixed_fp64_ops_per_cell_step(S))
        mp.close()
    if args.precision == "mixed" and not args.no_fp64_compare:
        mf = Mechanism(mech, precision=binding.FP64, **extra)
        plain = one_solve(mf, fp64_ops_per_cell_step(S, R, Rrev, nnz))
        mf.close()

    if rank != 0:
        return 0
    if args.precision == "mixed":
        ops = mixed_fp64_ops_per_cell_step(S)
        ops_note = ("FP64 work the mixed plan requires (species G/RT and split, FP64 Euler, "
                    "log T, 1/T, step bookkeeping); FP32/MUFU work not counted")
    else:
        ops = fp64_ops_per_cell_step(S, R, Rrev, nnz)
        ops_note = ("the method's FP64 work: exp = %g, log = %g, div = %g DFMA-equivalents, "
                    "measured" % (EXP_OPS, LOG_OPS, DIV_OPS))
    achieved = ops * cell_steps / (float(np.mean(ms)) / 1e3)
    bpc = DRAM_BYTES_PER_CELL.get(args.precision + ("+mlp" if args.thermo == "mlp" else ""))
    roofline = {"bound": "alu", "achieved": 2 * achieved / 1e12, "peak": 2 * FP64_PEAK_OPS / 1e12,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_OPS,
                "traffic": None if bpc is None else bpc * n,
                "traffic_note": "DRAM bytes per launch scaled from the ncu capture in profiles/",
                "pipe": "fp64 (DFMA = 2 flops); peak = measured DFMA rate of csrc/alu_peaks.cu "
                        "(1.667/clk/SM x 148 SMs x 1919 MHz)",
                "ops_per_cell_step": ops, "ops_counted": ops_note,
                "cell_steps_per_launch": cell_steps}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": "syn32x150 (32 species, 150 reversible reactions), %d cells "
                                   "per GPU, T0 U[800,2200] K, P U[1,5] atm, Y0 Dirichlet(0.5), "
                                   "dt 1e-3 s" % n,
                       "precision": args.precision,
                       "thermo": "network" if args.thermo == "mlp" else "NASA-7 polynomial",
                       "cells_per_gpu": n, "warmup_cells": nw, "max_iters": extra.get(
                           "max_iters", 200000),
                       "l2": "inputs (%d MB) larger than L2" % ((T.nbytes + P.nbytes + Y.nbytes)
                                                                >> 20),
                       "parallelism": "dp%d (independent cell batches)" % world},
            "cell_steps_per_s": cell_steps * args.steps / t_max if world == 1 else None,
            "iters": {"mean": float(it_np.mean()), "p50": float(np.percentile(it_np, 50)),
                      "p99": float(np.percentile(it_np, 99)), "max": int(it_np.max())},
            "cell_status": {"ok": int(status[0]), "maxiter": int(status[1]),
                            "nonfinite": int(status[2]), "trange": int(status[3])},
            "roofline": roofline, "gpu_launches": args.steps, "e2e": e2e,
            "mixed_poly": mixed_poly, "plain_fp64": plain, "thermo_net": mlp_info,
            "wall_s_timed": wall}
    line["clocks"] = clk.summary()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mech, T, P, Y, dt, **extra)
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["scale", "uneven"], default="scale",
                    help="uneven: 64 uneven 53/325 batches in one batched launch")
    ap.add_argument("--uneven-scale", type=float, default=1.0,
                    help="multiplies every batch size of the uneven workload")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--thermo", choices=["poly", "mlp"], default="mlp",
                    help="mlp: cp/R from the thermo network trained before timing (mixed only)")
    ap.add_argument("--no-poly-compare", action="store_true",
                    help="skip the polynomial-thermo mixed solve of the same cells")
    ap.add_argument("--mlp-samples", type=int, default=1_000_000)
    ap.add_argument("--mlp-epochs", type=int, default=30)
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 solve of the same cells (mixed runs only)")
    ap.add_argument("--cells", type=int, default=N_CELLS)
    ap.add_argument("--warmup-cells", type=int, default=16384)
    ap.add_argument("--max-iters", type=int, default=None)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
