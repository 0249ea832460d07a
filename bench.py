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

# Rates per SM and clock measured on B300 by csrc/alu_peaks.cu (lane
# operations): FP64 FMA, CUDA's exp(double), log(double) and FP64 division (all
# on the FP64 pipe); FP32 FMA; MUFU ex2.approx (the mixed path's exponentials,
# logarithms and reciprocals).  Peaks are taken at the SM clock sampled during
# the timed region.
DFMA_PER_CLK, EXP64_PER_CLK, LOG64_PER_CLK, DIV64_PER_CLK = 1.668, 0.104, 0.055, 0.222
FFMA_PER_CLK, MUFU_PER_CLK = 125.36, 31.66
N_SMS = 148
# DRAM bytes per cell of one launch, from the ncu captures summarised in
# profiles/ (reads only: the small cases' output writes stay in L2), scaled to
# the full launch by the cells it processes.  None when the kernel changed
# after its capture.
DRAM_BYTES_PER_CELL = {"mixed": 966656 / 3256, "fp64": 612608 / 1628, "mixed+mlp": 979456 / 3256}


def bf16_tflops(burst: bool = False) -> tuple:
    """The BF16 dense tensor rate of MEASURED_PEAKS.json: the sustained cuBLAS
    figure for a kernel timed inside a long step, the burst one for a kernel
    timed alone; else the profiling fallback (1.8 PFLOP/s burst, sustained
    near 1.4)."""
    key = "bf16_tflops" if burst else "bf16_tflops_sustained"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured (%s)" % ("burst" if burst else "sustained")
    except Exception:
        return (1800.0, "fallback (burst)") if burst else (1400.0, "fallback (sustained)")


def method_counts(S: int, R: int, net: bool = False) -> dict:
    """The method's work per cell-step (one STEV iteration of one cell), as
    counted from the algorithm with the sliding DFT: about 40 S + 43 R flops,
    2 R exponentials (forward and reverse rate constants, Eqs. 28-30), S
    divisions (gamma, Eqs. 6-7) and 2 logarithms (ln T); with the thermo
    network (Sec. 3) its MMA flops 2 (64 + 64 x 64 + 64 x 3S) replace about
    28 S thermo flops."""
    c = {"flops": 40 * S + 43 * R, "exp": 2 * R, "div": S, "log": 2, "mma": 0}
    if net:
        c["flops"] -= 28 * S
        c["mma"] = 2 * (64 + 64 * 64 + 64 * 3 * S)
    return c


def bound_s_per_cell_step(S: int, R: int, precision: str, net: bool, mhz: float,
                          bf16: float) -> float:
    """Composite ALU bound of one cell-step: each class of operation at the
    measured rate of the unit that executes it, t = flops / peak_fp +
    exps / peak_exp + divs / peak_div + logs / peak_log + mma / peak_bf16.
    FP64 path: flops on the FP64 pipe (FMA = 2 flops), exp / log / division
    at the rates of CUDA's double routines.  Mixed path: flops on the FP32
    pipe, exponentials, logarithms and reciprocals on MUFU, MMA flops at the
    BF16 tensor rate (bf16, TFLOP/s)."""
    clk = N_SMS * mhz * 1e6
    c = method_counts(S, R, net)
    if precision == "fp64":
        return (c["flops"] / (2 * DFMA_PER_CLK * clk) + c["exp"] / (EXP64_PER_CLK * clk) +
                c["div"] / (DIV64_PER_CLK * clk) + c["log"] / (LOG64_PER_CLK * clk))
    return (c["flops"] / (2 * FFMA_PER_CLK * clk) +
            (c["exp"] + c["div"] + c["log"]) / (MUFU_PER_CLK * clk) + c["mma"] / (bf16 * 1e12))


# The multiphase method's work per cell-step (Sec. 7.2 cells, one STEV
# iteration), counted from the algorithm with the phase temperatures held:
# phase totals, mass fractions, eps, rho_g and MW_g (33 adds, 35 divisions);
# Eqs. 44-46 (~20 flops, 1 division); 19 gamma factors (19 adds, 19
# divisions); the eleven rate laws (~71 flops, 3 divisions, 11 powers:
# Eqs. 47, 48, 50 one each, Eq. 52 three, Eq. 53 two, Eq. 55 three, rho_g^1.75
# shared); production (40 stoichiometric FMAs, 18 molar masses), phase sums
# and mass-fraction rates (72 flops, 36 divisions); Eqs. 1-5 (54 flops, 18
# divisions); Eq. 9's window sum (15); Euler (36): about 420 flops, 112
# divisions and 11 powers (each an exp and a log).
MP_COUNTS = {"flops": 420, "div": 112, "pow": 11}


def mp_bound_s_per_cell_step(mhz: float) -> float:
    """FP64 bound of one multiphase cell-step: flops on the FP64 pipe,
    divisions and pow (exp + log) at the rates of CUDA's double routines."""
    clk = N_SMS * mhz * 1e6
    c = MP_COUNTS
    return (c["flops"] / (2 * DFMA_PER_CLK * clk) + c["div"] / (DIV64_PER_CLK * clk) +
            c["pow"] * (1.0 / (EXP64_PER_CLK * clk) + 1.0 / (LOG64_PER_CLK * clk)))


def alu_roofline(precision: str, S: int, R: int, net: bool, cell_steps: float, seconds: float,
                 sm_mhz: float) -> dict:
    """Composite ALU roofline of a solve: frac = achieved cell-steps/s x the
    bound time of one cell-step.  Reported as flop rates of the bound pipe
    (FP64 FMA for the plain path, FP32 FMA for the mixed path): the peak is
    that pipe's measured rate x SMs x the sampled clock, and a cell-step's
    flop-equivalents are its bound time x that peak."""
    mhz = sm_mhz or 2032.0
    bf16, bf16_src = bf16_tflops()
    t = bound_s_per_cell_step(S, R, precision, net, mhz, bf16)
    per_clk = DFMA_PER_CLK if precision == "fp64" else FFMA_PER_CLK
    peak = 2 * per_clk * N_SMS * mhz * 1e6               # flop/s of the bound pipe
    rate = cell_steps / seconds
    return {"bound": "alu", "achieved": rate * t * peak / 1e12, "peak": peak / 1e12,
            "unit": "TFLOP/s", "frac": rate * t, "cell_steps_per_s": rate,
            "cell_steps_per_s_bound": 1.0 / t, "counts_per_cell_step": method_counts(S, R, net),
            "pipe": ("fp64 (DFMA %.3f, exp %.3f, log %.3f, div %.3f /clk/SM)"
                     % (DFMA_PER_CLK, EXP64_PER_CLK, LOG64_PER_CLK, DIV64_PER_CLK)
                     if precision == "fp64" else
                     "fp32 composite (FFMA %.2f, MUFU %.2f /clk/SM%s)"
                     % (FFMA_PER_CLK, MUFU_PER_CLK,
                        ", BF16 %.1f TFLOP/s %s" % (bf16, bf16_src) if net else "")) +
                    " (csrc/alu_peaks.cu) x %d SMs x %.0f MHz sampled" % (N_SMS, mhz)}


def spec_flag(args) -> int:
    """Mixed-precision mechanisms run the kernel compiled for them (NVRTC at
    creation, outside the timed region) unless --generic."""
    return 0 if getattr(args, "generic", False) else 1


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


def max_over_ranks(dist, x: float, device=None) -> float:
    """The slowest rank's value (time-like); x itself with one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float, device=None) -> float:
    """Every rank's x added (cells processed)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t)
    return float(t.item())


def whole_job_rate(dist, seconds: float, units: float, device=None) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: each rank its own batch, no data exchange)."""
    return sum_over_ranks(dist, units, device) / max_over_ranks(dist, seconds, device)


def cpu_baseline(mech, T, P, Y, dt, target_s: float = 15.0, keep=None, **opts):
    """The oracle as it stands on this host's cores, on a bounded sample.
    keep (a dict) receives the oracle's results on the sample cells."""
    import oracle
    cores = os.cpu_count() or 1
    n = max(cores, 8)
    t0 = time.time()
    res = oracle.solve(mech, T[:n], P[:n], Y[:n], dt, n_threads=cores, **opts)
    first = time.time() - t0
    # grow the sample to ~target_s of work (cells are independent and alike)
    n2 = int(min(len(T), max(n, n * target_s / max(first, 1e-3))))
    if n2 > n:
        t0 = time.time()
        res = oracle.solve(mech, T[:n2], P[:n2], Y[:n2], dt, n_threads=cores, **opts)
        first = time.time() - t0
        n = n2
    if keep is not None:
        keep["ref"] = res
    return {"value": n / first, "unit": UNIT, "cores": min(cores, n), "kind": "oracle",
            "sample": "first %d cells of the same workload, %.1f s" % (n, first)}


def oracle_error(gpu, ref, tol_Y, tol_T):
    """Error of GPU results against the oracle on the same cells.  STEV's final
    state is ill-conditioned on cells ringing at their limiter's amplitude (a
    rounding-size change moves them by up to ~2 Y_step^max), so the fraction
    within the target and the median say more than the maximum."""
    n = min(len(gpu[0]), len(ref[0]))
    dY = np.abs(gpu[1][:n] - ref[1][:n]).max(axis=1)
    dT = np.abs(gpu[0][:n] - ref[0][:n])
    return {"cells": int(n), "target": {"max_dY": tol_Y, "dT_K": tol_T},
            "within_target": float(np.mean((dY <= tol_Y) & (dT <= tol_T))),
            "median_dY": float(np.median(dY)), "max_dY": float(dY.max()),
            "median_dT_K": float(np.median(dT)), "max_dT_K": float(dT.max()),
            "status_equal": float(np.mean(gpu[3][:n] == ref[3][:n])),
            "note": "raw comparison on the first cells of the workload; on the 32/150 "
                    "mechanism the oracle moves nearly every cell by more than 1e-10 under a "
                    "one-ulp change of its rates, so the 1e-8 bar is checked in the tests on "
                    "step prefixes and on well-conditioned cells"}


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


L2_BYTES = 126 << 20


def inputs_fit_l2(*arrays) -> bool:
    return sum(a.nbytes for a in arrays) < L2_BYTES


def l2_note(*arrays, flushed: bool = True) -> str:
    mb = sum(a.nbytes for a in arrays) >> 20
    if not inputs_fit_l2(*arrays):
        return "inputs (%d MB) larger than L2" % mb
    if flushed:
        return "inputs (%d MB) within L2: a 256 MB buffer is written before each timed solve" % mb
    return "inputs (%d MB) within L2 (not flushed)" % mb


def timed_solves(m, Td, Pd, Yd, dt, out, steps, warmup, warmup_cells, stream, dist=None,
                 sample_clocks=None):
    """W warm-up solves on the first warmup_cells cells (same kernel and launch
    configuration), then K timed solves of every cell, CUDA events on the
    launching stream, synchronised and barriered on both sides.  When the
    inputs fit in L2, a buffer larger than L2 is written (outside the events)
    before each timed solve."""
    import torch
    nw = min(Td.shape[0], warmup_cells)
    wout = tuple(x[:nw] for x in out)
    for _ in range(warmup):
        m.solve(Td[:nw], Pd[:nw], Yd[:nw], dt, out=wout)
    flush = None
    if inputs_fit_l2(Td, Pd, Yd):
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=Td.device)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.time()
    for k in range(steps):
        if flush is not None:
            flush.zero_()
        ev[k][0].record(stream)
        m.solve(Td, Pd, Yd, dt, out=out)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.time() - t0
    barrier(dist)
    return [a.elapsed_time(b) for a, b in ev], wall, nw, (steps if flush is not None else 0)


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
    m = Mechanism(mech, precision=binding.MIXED, specialize=spec_flag(args), **extra)
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
                       "precision": "mixed", "thermo": args.thermo,
                       "l2": l2_note(*[a for b in host_batches for a in b[:3]], flushed=False)},
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


SERVE_BUDGET = 40 << 30  # device-memory admission budget of the serving workload


def _serve_mechanisms(arm, args, trained=None):
    """The 8/20 and 32/150 mechanisms for one serving arm ("mixed+mlp" or
    "fp64"); networks trained on the GPU (or taken from `trained`)."""
    from paper_1905_09395_b300 import Mechanism, binding, synth
    tabs = [synth.small_mechanism(), synth.scale_mechanism()]
    prec = binding.MIXED if arm == "mixed+mlp" else binding.FP64
    ms = [Mechanism(t, precision=prec, specialize=spec_flag(args) if arm == "mixed+mlp" else 0)
          for t in tabs]
    if arm == "mixed+mlp":
        Ts = np.random.default_rng(2024).uniform(300.0, 3000.0, size=args.mlp_samples)
        for i, m in enumerate(ms):
            if trained is not None and trained[i] is not None:
                m.mlp_set_params(*trained[i])
            else:
                m.mlp_train(Ts, epochs=args.mlp_epochs, batch=4096, lr=2e-3, seed=7)
            m.set_options(thermo=binding.THERMO_MLP)
    return tabs, ms


def serve_arm(arm, args, trained=None, rate=None, seconds=None, drain=None):
    """One serving run: the seeded Poisson request stream (rate, duration,
    sizes log-uniform 1k-512k, 8/20 and 32/150 mechanisms half and half) fed
    to a stev_server with a 40 GB admission budget, every request's inputs
    copied from pinned host memory and its results copied back.  Requests
    still unfinished `drain` seconds after the last arrival are cancelled
    (stev_server_stop) and counted as backlog; the cells they had solved
    count toward the throughput."""
    import torch
    from paper_1905_09395_b300 import Server, synth
    rate = args.serve_rate if rate is None else rate
    seconds = args.serve_seconds if seconds is None else seconds
    drain = args.serve_drain if drain is None else drain
    hi = 512 * 1024
    reqs = synth.serving_requests(seconds, rate, 1000, hi, 2, seed=4)
    tabs, ms = _serve_mechanisms(arm, args, trained)
    pools, outs = [], []
    for i, t in enumerate(tabs):
        T, P, Y = synth.make_cells(t, hi, seed=50 + i, T_range=(800.0, 2200.0),
                                   P_atm_range=(1.0, 5.0), dirichlet=0.5)
        pools.append(tuple(torch.from_numpy(a).pin_memory().numpy() for a in (T, P, Y)))
        # one output area per mechanism, shared by its requests (results are not read)
        outs.append((torch.empty(hi, dtype=torch.float64).pin_memory().numpy(),
                     torch.empty((hi, t.n_species), dtype=torch.float64).pin_memory().numpy(),
                     torch.empty(hi, dtype=torch.int32).pin_memory().numpy(),
                     torch.empty(hi, dtype=torch.uint8).pin_memory().numpy()))
    # SM shares in proportion to each mechanism's offered work: cells x cost per
    # cell, the cost timed on a warm-up solve of 16,384 pool cells on all SMs
    dev = torch.device("cuda", 0)
    cost = []
    for i, m in enumerate(ms):
        Td, Pd, Yd = (torch.from_numpy(a[:16384]).to(dev) for a in pools[i])
        for _ in range(max(1, args.warmup - 1)):
            m.solve(Td, Pd, Yd, 1e-3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.solve(Td, Pd, Yd, 1e-3)
        torch.cuda.synchronize()
        cost.append((time.perf_counter() - t0) / 16384)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    work = [cost[i] * sum(r[2] for r in reqs if r[1] == i) for i in range(2)]
    s0 = int(round(sms * work[0] / max(sum(work), 1e-30)))
    share = [min(max(s0, 4), sms - 4)]
    share.append(sms - share[0])
    srv = Server(ms, sm_share=share, mem_budget=SERVE_BUDGET, queue_len=4096)
    reports, lag, k = [], 0.0, 0
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        c0 = srv.clock()
        while True:
            now = time.perf_counter() - t0
            while k < len(reqs) and reqs[k][0] <= now:
                _, mi, n, off = reqs[k]
                T, P, Y = pools[mi]
                o = tuple(a[off:off + n] for a in outs[mi])
                srv.submit(mi, T[off:off + n], P[off:off + n], Y[off:off + n], 1e-3, out=o)
                lag = max(lag, now - reqs[k][0])
                k += 1
            if now >= seconds + drain:
                break
            if k == len(reqs) and len(reports) == len(reqs):
                break
            wait = 0.005 if k == len(reqs) else min(0.005, max(0.0, reqs[k][0] - now))
            reports += srv.poll(timeout=wait)
        t_stop = srv.clock()        # the run's end on the server clock: unfinished
        srv.stop(timeout=120.0)     # requests are censored here; cells in flight
        elapsed = time.perf_counter() - t0  # finish, nothing new starts
        while True:
            more = srv.poll()
            if not more:
                break
            reports += more
        st = srv.stats
    srv.close(timeout=120.0)
    for m in ms:
        m.close()
    done = [d for d in reports if d["status"] == 0]
    lat = np.array([d["t_done"] - d["t_submit"] for d in done]) if done else np.zeros(0)
    pct = lambda q: float(np.percentile(lat, q)) if len(lat) else None
    # every offered request's latency, an unfinished one counted as censored at
    # the run's end (a lower bound on its latency); queue wait (submit to
    # admission) and service time (admission to results) of the requests that
    # reached them
    seen = {d["id"] for d in reports}
    cens = [t_stop - d["t_submit"] for d in reports if d["status"] != 0]
    cens += [t_stop - (c0 + reqs[j][0]) for j in range(len(reqs) - len(seen))]
    lat_all = np.concatenate([lat, np.array(cens, dtype=np.float64)])
    admitted_t = [d for d in reports if d["t_admit"] > 0]
    qwait = np.array([d["t_admit"] - d["t_submit"] for d in admitted_t] +
                     [t_stop - d["t_submit"] for d in reports if d["t_admit"] <= 0])
    service = np.array([d["t_done"] - d["t_admit"] for d in done])
    q = lambda a, p: float(np.percentile(a, p)) if len(a) else None
    cells = sum(d["cells_done"] for d in reports)
    by = {}
    for i, t in enumerate(tabs):
        li = np.array([d["t_done"] - d["t_submit"] for d in done if d["mechanism"] == i])
        by[t.name] = {"sm_share": share[i], "offered_requests": sum(1 for r in reqs if r[1] == i),
                      "offered_cells": int(sum(r[2] for r in reqs if r[1] == i)),
                      "completed_requests": int(len(li)),
                      "cells_solved": int(sum(d["cells_done"] for d in reports
                                              if d["mechanism"] == i)),
                      "latency_p50_s": float(np.percentile(li, 50)) if len(li) else None,
                      "latency_p99_s": float(np.percentile(li, 99)) if len(li) else None,
                      "cost_us_per_cell_full_gpu": cost[i] * 1e6}
    # bytes copied: every admitted request's inputs, finished requests' results
    admitted = [d for d in reports if d["t_admit"] > 0]
    h2d = sum(d["n_cells"] * (8 * (2 + tabs[d["mechanism"]].n_species)) for d in admitted)
    d2h = sum(d["n_cells"] * (8 * (1 + tabs[d["mechanism"]].n_species) + 5) for d in done)
    return {"arm": arm, "value": cells / elapsed, "unit": UNIT, "elapsed_s": elapsed,
            "rate_req_per_s": rate, "arrival_window_s": seconds,
            "offered_requests": len(reqs), "offered_cells": int(sum(r[2] for r in reqs)),
            "offered_cells_per_s": sum(r[2] for r in reqs) / seconds,
            "completed_requests": len(done),
            "completed_cells": int(sum(d["n_cells"] for d in done)), "cells_solved": int(cells),
            "latency_p50_s": q(lat_all, 50), "latency_p99_s": q(lat_all, 99),
            "latency_note": "over every offered request; an unfinished one counts as censored "
                            "at the run's end (a lower bound on its latency)",
            "censored_requests": int(len(cens)),
            "finished_latency_p50_s": pct(50), "finished_latency_p99_s": pct(99),
            "latency_max_s": float(lat.max()) if len(lat) else None,
            "queue_wait_p50_s": q(qwait, 50), "queue_wait_p99_s": q(qwait, 99),
            "service_p50_s": q(service, 50), "service_p99_s": q(service, 99),
            "backlog_requests": int(len(reqs) - len(done)),
            "submit_lag_max_s": lag, "peak_resident_gb": st["peak_resident_bytes"] / 2**30,
            "kernel_launches": int(st["kernel_launches"]),
            "h2d_bytes": int(h2d), "d2h_bytes": int(d2h),
            "by_mechanism": by, "clocks": clk.summary(), "server_clock_start": c0}


def run_serve(args):
    """Serving workload: mixed+MLP and plain FP64 under the same request stream."""
    import torch
    torch.cuda.set_device(0)
    arms = [serve_arm("mixed+mlp", args)]
    if not args.no_fp64_compare:
        arms.append(serve_arm("fp64", args))
    a = arms[0]
    # the same stream at a load the mixed+MLP server sustains: half of the cell
    # rate it reached above, as requests per second of the mean request size
    light = None
    if args.serve_light_seconds > 0:
        mean_cells = a["offered_cells"] / max(a["offered_requests"], 1)
        lam = 0.5 * a["value"] / mean_cells
        light = {"rate_req_per_s": lam, "arms": [
            serve_arm(arm, args, rate=lam, seconds=args.serve_light_seconds,
                      drain=args.serve_light_seconds)
            for arm in (["mixed+mlp"] + ([] if args.no_fp64_compare else ["fp64"]))]}
    line = {"metric": "cell-solves/s under serving load (Poisson %g req/s, %g s, sizes "
                      "log-uniform 1k-512k, 8/20 and 32/150 mechanisms, 40 GB budget); "
                      "p50/p99 latency" % (args.serve_rate, args.serve_seconds),
            "value": a["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
            "ms_per_step": a["elapsed_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "serving: Poisson %g req/s for %g s (+%g s drain), sizes "
                                   "log-uniform 1k-512k cells, syn8x20 and syn32x150 half and "
                                   "half, dt 1e-3 s, 40 GB admission budget"
                                   % (args.serve_rate, args.serve_seconds, args.serve_drain),
                       "l2": "request inputs stream from host memory; pools of 512k cells "
                             "per mechanism (> L2)"},
            "latency_p50_s": a["latency_p50_s"], "latency_p99_s": a["latency_p99_s"],
            "e2e": {"value": a["value"], "unit": UNIT, "h2d_bytes_per_step": a["h2d_bytes"],
                    "d2h_bytes_per_step": a["d2h_bytes"],
                    "note": "the serving value is host to host: every request's copies are in it"},
            "gpu_launches": a["kernel_launches"], "serving": arms[0],
            "plain_fp64": arms[1] if len(arms) > 1 else None, "light_load": light,
            "clocks": a["clocks"]}
    print(json.dumps(line))
    return 0


def run_bfer(args):
    """The paper's own single-phase benchmark shape (Sec. 7.1): the BFER
    methane mechanism (6 species, 2 global reactions with real orders, Table 1
    constants) on random fixed states, t_f = 1 ms; one solve of all cells per
    step, for plain FP64, mixed precision with NASA-7 thermo and mixed with the
    thermo network (trained on the GPU before timing)."""
    import torch
    from paper_1905_09395_b300 import Mechanism, binding, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    mech = synth.bfer_mechanism()
    T, P, Y = synth.bfer_cells(mech, args.cells)
    n = len(T)
    Td, Pd, Yd = (torch.from_numpy(a).to(dev) for a in (T, P, Y))
    out = (torch.empty_like(Td), torch.empty_like(Yd), torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n, dtype=torch.uint8, device=dev))
    stream = torch.cuda.current_stream(dev)
    arms = {}
    flushes = 0
    with ClockSampler(0) as clk:
        for name, kw in (("mixed+mlp", dict(precision=binding.MIXED, specialize=spec_flag(args))),
                         ("mixed_poly", dict(precision=binding.MIXED, specialize=spec_flag(args))),
                         ("plain_fp64", dict(precision=binding.FP64))):
            m = Mechanism(mech, **kw)
            info = None
            if name == "mixed+mlp":
                t0 = time.time()
                Ts = np.random.default_rng(2024).uniform(300.0, 3000.0, size=args.mlp_samples)
                hist = m.mlp_train(Ts, epochs=args.mlp_epochs, batch=4096, lr=2e-3, seed=7)
                m.set_options(thermo=binding.THERMO_MLP)
                info = {"final_loss": float(hist[-1]), "train_s": time.time() - t0}
            ms, _, _, nflush = timed_solves(m, Td, Pd, Yd, 1e-3, out, args.steps, args.warmup,
                                            args.warmup_cells, stream)
            flushes += nflush
            it = out[2].cpu().numpy().astype(np.int64)
            st = np.bincount(out[3].cpu().numpy(), minlength=4)
            arms[name] = {"value": n / (float(np.mean(ms)) / 1e3), "unit": UNIT,
                          "ms_per_step": float(np.mean(ms)),
                          "cell_steps_per_s": float(it.sum()) / (float(np.mean(ms)) / 1e3),
                          "iters_mean": float(it.mean()), "iters_max": int(it.max()),
                          "cell_status": st.tolist(), "resident_slots": m.resident_slots,
                          "thermo_net": info}
            head = [x[:4096].cpu().numpy() for x in out]
            arms[name]["_head"] = head
            m.close()
        clocks = clk.summary()
    keep = {}
    cpu = None if args.no_cpu_baseline else cpu_baseline(mech, T, P, Y, 1e-3, keep=keep)
    for name, a in arms.items():
        head = a.pop("_head")
        if cpu is not None:
            fp64 = name == "plain_fp64"
            a["oracle_error"] = oracle_error(head, keep["ref"], 1e-8 if fp64 else 1e-4,
                                             1e-6 if fp64 else 0.5)
    # the value is the mixed-precision polynomial arm: on a 6-species
    # mechanism the polynomials cost far less than the network's MMAs
    h = arms["mixed_poly"]
    line = {"metric": "cell-solves/s, BFER methane mechanism (Sec. 7.1), random fixed states, "
                      "t_f = 1 ms", "value": h["value"], "value_arm": "mixed_poly",
            "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "bfer: 6 species (CH4 O2 CO H2O CO2 N2), MEPOX + COROX with "
                                   "Table 1 constants, %d cells, T0 U[1200,2200] K, 1 atm, "
                                   "methane-air-like Y0, dt 1e-3 s" % n,
                       "l2": l2_note(T, P, Y)},
            "arms": arms, "gpu_launches": 3 * args.steps,
            "other_launches_in_timed_region": {"l2_flush": flushes}, "clocks": clocks,
            "cpu_baseline": cpu}
    print(json.dumps(line))
    return 0


def run_accuracy(args):
    """Error of the GPU paths against the FP64 oracle on a seeded subset of
    the 1M-cell workload (16,384 cells by default): mixed + network (the
    headline), mixed with the polynomial thermo and plain FP64 solve all the
    cells on the GPU while the oracle solves the subset on the host's cores
    in a thread (the C oracle runs outside the interpreter lock)."""
    import torch
    import oracle
    from paper_1905_09395_b300 import Mechanism, binding
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    mech, T, P, Y, dt = workload(args.cells)
    n = len(T)
    idx = np.sort(np.random.default_rng(16384).choice(n, size=min(args.oracle_cells, n),
                                                      replace=False))
    cores = os.cpu_count() or 1
    ref = {}

    def run_oracle():
        t0 = time.time()
        ref["res"] = oracle.solve(mech, T[idx], P[idx], Y[idx], dt, n_threads=cores)
        ref["s"] = time.time() - t0

    th = threading.Thread(target=run_oracle)
    th.start()
    Td, Pd, Yd = (torch.from_numpy(a).to(dev) for a in (T, P, Y))
    arms = {}
    for name in ("mixed+mlp", "mixed_poly", "plain_fp64"):
        kw = (dict(precision=binding.FP64) if name == "plain_fp64" else
              dict(precision=binding.MIXED, specialize=spec_flag(args)))
        m = Mechanism(mech, **kw)
        if name == "mixed+mlp":
            Ts = np.random.default_rng(2024).uniform(300.0, 3000.0, size=args.mlp_samples)
            m.mlp_train(Ts, epochs=args.mlp_epochs, batch=4096, lr=2e-3, seed=7)
            m.set_options(thermo=binding.THERMO_MLP)
        out = [x.cpu().numpy() for x in m.solve(Td, Pd, Yd, dt)]
        m.close()
        arms[name] = [x[idx] for x in out]
    th.join()
    line = {"metric": "error against the FP64 oracle on a seeded subset of the 1M-cell workload",
            "config": {"workload": "syn32x150, %d cells; oracle on %d seeded cells (%d host "
                                   "threads, %.0f s)" % (n, len(idx), cores, ref["s"])},
            "data": "synthetic", "arms": {},
            "cpu_baseline": {"value": len(idx) / ref["s"], "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": "%d seeded cells of the workload, %.0f s" % (len(idx),
                                                                                   ref["s"])}}
    for name, g in arms.items():
        fp64 = name == "plain_fp64"
        e = oracle_error(g, ref["res"], 1e-8 if fp64 else 1e-4, 1e-6 if fp64 else 0.5)
        dY = np.abs(g[1] - ref["res"][1]).max(axis=1)
        dT = np.abs(g[0] - ref["res"][0])
        e.update({"p90_dY": float(np.percentile(dY, 90)), "p99_dY": float(np.percentile(dY, 99)),
                  "p90_dT_K": float(np.percentile(dT, 90)), "p99_dT_K": float(np.percentile(dT, 99)),
                  "within_1e-4_0.5K": float(np.mean((dY <= 1e-4) & (dT <= 0.5))),
                  "iteration_match": float(np.mean(g[2] == ref["res"][2]))})
        e["note"] = ("seeded subset (default_rng(16384)) of the workload's cells; on this "
                     "mechanism the oracle itself moves the median cell by ~3e-5 / 0.04 K under "
                     "a one-ulp change of its rates")
        line["arms"][name] = e
    print(json.dumps(line))
    return 0


def run_multiphase(args):
    """The paper's multiphase workload shape (Sec. 7.2): coal gasification
    cells (14 gas and 4 solid species, two phase temperatures, 11 reactions
    with the rate laws of Eqs. 42-56 and Table 2's constants), random
    gasifier-like states, one FP64 STEV solve of every cell per step
    (stev_mp_solve); the oracle on a bounded sample beside it."""
    import torch
    from paper_1905_09395_b300 import binding, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cells = synth.multiphase_cells(args.cells, seed=7)
    n = len(cells)
    d = torch.from_numpy(cells).to(dev)
    out = (torch.empty_like(d), torch.empty(n, dtype=torch.float64, device=dev),
           torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n, dtype=torch.uint8, device=dev))
    for _ in range(args.warmup):
        binding.mp_solve(d[:min(n, args.warmup_cells)], 1e-3,
                         out=tuple(x[:min(n, args.warmup_cells)] for x in out))
    flush = None
    if cells.nbytes < L2_BYTES:
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev[k][0].record()
            binding.mp_solve(d, 1e-3, out=out)
            ev[k][1].record()
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    it = out[2].cpu().numpy().astype(np.int64)
    st = np.bincount(out[3].cpu().numpy(), minlength=4)
    line = {"metric": "cell-solves/s, multiphase coal gasification cells (Sec. 7.2), FP64",
            "value": n / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "multiphase: 14 gas + 4 solid species, 11 reactions (Eqs. "
                                   "31-56, Table 2), %d random gasifier-like cells, T_g "
                                   "U[900,1500] K, dt 1e-3 s" % n,
                       "l2": l2_note(cells, flushed=flush is not None)},
            "cell_steps_per_s": float(it.sum()) / (ms / 1e3),
            "iters": {"mean": float(it.mean()), "p50": float(np.median(it)),
                      "max": int(it.max())},
            "cell_status": st.tolist(), "gpu_launches": args.steps,
            "other_launches_in_timed_region": {"l2_flush": args.steps if flush is not None else 0},
            "clocks": clk.summary()}
    mhz = line["clocks"]["sm_mhz"] or 2032.0
    t = mp_bound_s_per_cell_step(mhz)
    rate = line["cell_steps_per_s"]
    peak = 2 * DFMA_PER_CLK * N_SMS * mhz * 1e6
    line["roofline"] = {"bound": "alu", "achieved": rate * t * peak / 1e12, "peak": peak / 1e12,
                        "unit": "TFLOP/s", "frac": rate * t, "cell_steps_per_s_bound": 1.0 / t,
                        "counts_per_cell_step": MP_COUNTS, "traffic": None,
                        "pipe": "fp64 (DFMA %.3f, div %.3f, exp %.3f, log %.3f /clk/SM) x %d SMs "
                                "x %.0f MHz sampled" % (DFMA_PER_CLK, DIV64_PER_CLK,
                                                        EXP64_PER_CLK, LOG64_PER_CLK, N_SMS, mhz)}
    if not args.no_cpu_baseline:
        from oracle import multiphase as mp
        cores = os.cpu_count() or 1
        k = min(n, 65536)
        t0 = time.time()
        ref = mp.solve(cells[:k], 1e-3, n_threads=cores)
        el = time.time() - t0
        got = out[0][:k].cpu().numpy()
        dX = np.abs(got[:, :18] - ref[0][:, :18]).max(axis=1)
        line["cpu_baseline"] = {"value": k / el, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "first %d cells, %.1f s" % (k, el)}
        line["oracle_error"] = {"cells": k, "max_dX": float(dX.max()),
                                "within_1e-8": float(np.mean(dX <= 1e-8)),
                                "status_equal": float(np.mean(out[3][:k].cpu().numpy() == ref[3]))}
    print(json.dumps(line))
    return 0


def run_gram(args):
    """The Levenberg-Marquardt trainer's dominant contraction (Sec. 3): the
    Gauss-Newton matrix G = X X^T of the transposed Jacobian X [rows][K] of
    the 32/150 network at 512 samples (K = 49,152), TF32 tensor-core products
    with FP32 accumulation (stev_gram_tf32), timed with CUDA events."""
    import torch
    from paper_1905_09395_b300 import binding
    torch.cuda.set_device(0)
    g = torch.Generator(device="cuda").manual_seed(11)
    X = torch.randn((args.gram_rows, 49152), dtype=torch.float32, device="cuda", generator=g)
    for _ in range(args.warmup):
        binding.gram_tf32(X)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record()
        for _ in range(args.steps):
            binding.gram_tf32(X)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    n, k = X.shape
    flops = n * (n + 1) / 2 * k * 2                   # the lower triangle of G (its mirror is copied)
    bf16, src = bf16_tflops(burst=True)              # a kernel timed alone
    peak = bf16 * 1.1 / 2.25                          # TF32 at the nominal TF32:BF16 ratio
    tf = flops / (ms / 1e3) / 1e12
    line = {"metric": "TFLOP/s, Gauss-Newton matrix of the LM trainer (TF32 tensor cores)",
            "value": tf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "tf32", "data": "synthetic",
            "config": {"workload": "G = X X^T, X %d x %d FP32 (normal), lower triangle "
                                   "in 128 x 256 tiles, mirrored" % (n, k)},
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf / peak, "traffic": None,
                         "peak_note": "BF16 %s %.1f x 1.1/2.25" % (src, bf16)},
            "gpu_launches": args.steps, "clocks": clk.summary()}
    print(json.dumps(line))
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
    extra = {} if args.max_iters is None else {"max_iters": args.max_iters}
    prec = binding.MIXED if args.precision == "mixed" else binding.FP64
    m = Mechanism(mech, precision=prec, specialize=spec_flag(args) if prec == binding.MIXED else 0,
                  **extra)
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
                    "supplies": "cp/R (energy equation), 300-3000 K; H/RT and G/RT from the "
                                "NASA-7 polynomials"}
    n = len(T)
    Td, Pd, Yd = (torch.from_numpy(a).to(dev) for a in (T, P, Y))
    out = (torch.empty_like(Td), torch.empty_like(Yd), torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n, dtype=torch.uint8, device=dev))
    stream = torch.cuda.current_stream(dev)

    with ClockSampler(local) as clk:
        ms, wall, nw, nflush = timed_solves(m, Td, Pd, Yd, dt, out, args.steps, args.warmup,
                                            args.warmup_cells, stream, dist)
    dev_s = sum(ms) / 1e3
    it_np = out[2].cpu().numpy()
    cell_steps = int(it_np.astype(np.int64).sum())
    status = np.bincount(out[3].cpu().numpy(), minlength=4)
    head = [x[:4096].cpu().numpy() for x in out]   # compared with the oracle below

    t_max = max_over_ranks(dist, dev_s, dev)
    value = whole_job_rate(dist, dev_s, n * args.steps, dev)

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
        e2e = {"value": whole_job_rate(dist, el, n * ke, dev), "unit": UNIT,
               "h2d_bytes_per_step": int(hT.nbytes + hP.nbytes + hY.nbytes),
               "d2h_bytes_per_step": int(sum(x.nbytes for x in ho)), "steps": ke}
    trained_scale = m.mlp_params() if args.thermo == "mlp" else None
    m.close()

    clocks = clk.summary()

    def one_solve(mc, precision, net):
        """One timed solve of the same cells by another configuration."""
        with ClockSampler(local) as ck:
            msx, _, _, _ = timed_solves(mc, Td, Pd, Yd, dt, out, 1, args.warmup, args.warmup_cells,
                                     stream, dist)
        itx = out[2].cpu().numpy().astype(np.int64)
        tx = max_over_ranks(dist, msx[0] / 1e3, dev)
        ckx = ck.summary()
        return {"value": whole_job_rate(dist, msx[0] / 1e3, n, dev), "unit": UNIT,
                "ms_per_step": tx * 1e3, "steps": 1,
                "warmup": args.warmup, "cell_steps_per_s": int(itx.sum()) / tx,
                "roofline": dict(alu_roofline(precision, S, R, net, int(itx.sum()), msx[0] / 1e3,
                                              ckx["sm_mhz"]), traffic=None),
                "clocks": ckx}

    # the same cells with the polynomial thermo (what the network gains) and
    # with the plain FP64 path (what mixed precision gains)
    mixed_poly, plain = None, None
    if args.precision == "mixed" and args.thermo == "mlp" and not args.no_poly_compare:
        mp = Mechanism(mech, precision=binding.MIXED, specialize=spec_flag(args), **extra)
        mixed_poly = one_solve(mp, "mixed", False)
        mp.close()
    if args.precision == "mixed" and not args.no_fp64_compare:
        mf = Mechanism(mech, precision=binding.FP64, **extra)
        plain = one_solve(mf, "fp64", False)
        plain_head = [x[:4096].cpu().numpy() for x in out]
        mf.close()

    if rank != 0:
        return 0
    net = args.precision == "mixed" and args.thermo == "mlp"
    bpc = DRAM_BYTES_PER_CELL.get(args.precision + ("+mlp" if net else ""))
    roofline = alu_roofline(args.precision, S, R, net, cell_steps, float(np.mean(ms)) / 1e3,
                            clocks["sm_mhz"])
    roofline.update({"traffic": None if bpc is None else bpc * n,
                     "traffic_note": "DRAM bytes per launch scaled from the ncu capture in "
                                     "profiles/ by the cells processed",
                     "cell_steps_per_launch": cell_steps})
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
                       "kernel": ("compiled for the mechanism (NVRTC)" if args.precision == "mixed"
                                  and spec_flag(args) else "generic"),
                       "cells_per_gpu": n, "warmup_cells": nw, "max_iters": extra.get(
                           "max_iters", 200000),
                       "l2": l2_note(T, P, Y),
                       "parallelism": "dp%d (independent cell batches)" % world},
            "cell_steps_per_s": cell_steps * args.steps / t_max if world == 1 else None,
            "iters": {"mean": float(it_np.mean()), "p50": float(np.percentile(it_np, 50)),
                      "p99": float(np.percentile(it_np, 99)), "max": int(it_np.max())},
            "cell_status": {"ok": int(status[0]), "maxiter": int(status[1]),
                            "nonfinite": int(status[2]), "trange": int(status[3])},
            "roofline": roofline, "gpu_launches": args.steps,
            "other_launches_in_timed_region": {"l2_flush": nflush}, "e2e": e2e,
            "mixed_poly": mixed_poly, "plain_fp64": plain, "thermo_net": mlp_info,
            "wall_s_timed": wall}
    line["clocks"] = clocks
    if world == 1 and not args.no_serve and args.precision == "mixed" and args.thermo == "mlp":
        # p50/p99 latency under the serving load (the scale mechanism's network reused)
        keys = ("value", "unit", "rate_req_per_s", "arrival_window_s", "elapsed_s",
                "offered_cells_per_s", "completed_requests", "offered_requests", "cells_solved",
                "latency_p50_s", "latency_p99_s", "latency_note", "censored_requests",
                "finished_latency_p50_s", "finished_latency_p99_s", "latency_max_s",
                "queue_wait_p50_s", "queue_wait_p99_s", "service_p50_s", "service_p99_s",
                "by_mechanism", "clocks")
        sv = serve_arm("mixed+mlp", args, trained=[None, trained_scale])
        line["serving"] = {k: sv[k] for k in keys}
        line["serving"]["workload"] = ("Poisson %g req/s for %g s (+%g s), sizes log-uniform "
                                       "1k-512k, syn8x20 and syn32x150 half and half, 40 GB "
                                       "budget, host to host" % (args.serve_rate,
                                                                 args.serve_seconds,
                                                                 args.serve_drain))
        if args.serve_light_seconds > 0:
            # the same stream at half the cell rate the server reached above
            # (a load it sustains), as requests per second of the mean size
            lam = 0.5 * sv["value"] / (sv["offered_cells_per_s"] / args.serve_rate)
            lt = serve_arm("mixed+mlp", args, trained=[None, trained_scale], rate=lam,
                           seconds=args.serve_light_seconds, drain=args.serve_light_seconds)
            line["serving_sustainable"] = {k: lt[k] for k in keys}
            line["serving_sustainable"]["workload"] = (
                "Poisson %.3f req/s (half the measured capacity) for %g s (+%g s), same sizes "
                "and mechanisms, 40 GB budget, host to host"
                % (lam, args.serve_light_seconds, args.serve_light_seconds))
    if world == 1 and not args.no_cpu_baseline:
        keep = {}
        line["cpu_baseline"] = cpu_baseline(mech, T, P, Y, dt, keep=keep, **extra)
        fp64 = args.precision == "fp64"
        line["oracle_error"] = oracle_error(head, keep["ref"], 1e-8 if fp64 else 1e-4,
                                            1e-6 if fp64 else 0.5)
        if plain is not None:
            plain["oracle_error"] = oracle_error(plain_head, keep["ref"], 1e-8, 1e-6)
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["scale", "uneven", "serve", "bfer", "accuracy",
                                           "multiphase", "gram"],
                    default="scale",
                    help="uneven: 64 uneven 53/325 batches in one batched launch; serve: "
                         "the request loop, mixed+MLP and plain FP64; bfer: the paper's "
                         "BFER methane mechanism on random states; accuracy: the GPU paths "
                         "against the oracle on a seeded subset of the 1M cells; multiphase: "
                         "the paper's coal gasification cells (Sec. 7.2); gram: the LM "
                         "trainer's Gauss-Newton matrix on the tensor cores")
    ap.add_argument("--gram-rows", type=int, default=10624,
                    help="gram workload: rows of X (the network's parameters; 10,624 at S=32)")
    ap.add_argument("--oracle-cells", type=int, default=16384,
                    help="accuracy workload: cells the oracle solves")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="requests per second")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="arrival window")
    ap.add_argument("--serve-drain", type=float, default=5.0,
                    help="seconds after the last arrival before unfinished requests are cancelled")
    ap.add_argument("--serve-light-seconds", type=float, default=30.0,
                    help="serve workload: arrival window of the run at half the measured "
                         "mixed+MLP capacity (0 skips it)")
    ap.add_argument("--no-serve", action="store_true",
                    help="scale workload: skip the serving run beside the headline")
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
    ap.add_argument("--generic", action="store_true",
                    help="mixed precision: the generic kernel instead of the one compiled for "
                         "the mechanism")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "bfer":
        return run_bfer(args)
    if args.workload == "accuracy":
        return run_accuracy(args)
    if args.workload == "multiphase":
        return run_multiphase(args)
    if args.workload == "gram":
        return run_gram(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
