"""Writes syn32x150_conditioning.npz: the FP64 oracle's results on 96 cells
of the 32-species / 150-reaction workload (seed 11, T0 U[800,2200] K,
P U[1,5] atm, Y0 Dirichlet(0.5), dt 1e-3 s) and its own conditioning there.

The oracle at this size takes minutes (cells of up to ~30,000 steps, each
run of the 96 cells ~10 s on 8 cores, 19 full runs), so the parity tests read
these stored values instead of recomputing them.  Everything here comes from
oracle/ alone (no CUDA path):

  full_*            the full solve (T, Y, iterations, status);
  fp64_dY/dT[p]     each FP64-sized probe run's per-cell |change| (every kf by
                    one ulp, every K by 64 ulp) and fp32_dY/dT[p] each
                    FP32-sized one (kf 2^-22, K 2^-18, concentrations or net
                    rates rounded to float, reverse-term noise, the limiter's
                    and ringing thresholds by 2^-22), names in *_names;
  prefix{k}_*       the state after k = 50, 100, 200 steps (max_iters = k) and
                    the FP64 probes' per-cell spread there.

Run from the repository root:  python tests/golden/make_scale_conditioning.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1905_09395_b300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "syn32x150_conditioning.npz")
N_CELLS, SEED, DT = 96, 11, 1e-3
PREFIX_K = (50, 100, 200)


def cells():
    mech = synth.scale_mechanism()
    T, P, Y = synth.make_cells(mech, N_CELLS, seed=SEED, T_range=(800, 2200),
                               P_atm_range=(1, 5), dirichlet=0.5)
    return mech, T, P, Y


def main():
    mech, T, P, Y = cells()
    out = {"T0": T, "P0": P, "Y0": Y}
    base = oracle.solve(mech, T, P, Y, DT)
    for name, a in zip(("T", "Y", "iters", "status"), base):
        out["full_" + name] = a
    for level in ("fp64", "fp32"):
        runs = {}
        oracle.conditioning(mech, T, P, Y, DT, base=base, level=level, per_run=runs)
        names = sorted(runs)
        out[level + "_names"] = np.array(names)
        out[level + "_dY"] = np.stack([runs[k][0] for k in names])
        out[level + "_dT"] = np.stack([runs[k][1] for k in names])
        print(level, "probe runs:", names)
    for k in PREFIX_K:
        pb, sY, sT = oracle.conditioning(mech, T, P, Y, DT, max_iters=k)
        for name, a in zip(("T", "Y", "iters", "status"), pb):
            out["prefix%d_%s" % (k, name)] = a
        out["prefix%d_sY" % k] = sY
        out["prefix%d_sT" % k] = sT
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
