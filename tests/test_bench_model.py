"""The roofline model of bench.py (the composite ALU model: the method's
operations placed on the units that execute them, peaks from the measured
per-SM rates at the sampled clock): the per-cell-step counts quoted for the
32/150 workload and the fraction's arithmetic."""
import pytest

import bench


def test_operation_counts_for_32_150():
    S, R, Rrev, nnz = 32, 150, 150, 579
    assert bench.fp64_ops_per_cell_step(S, R, Rrev, nnz) == pytest.approx(10725.5)
    # FP32 pipe: 5,668 operations; MUFU: 336 (two ex2 per reaction, a
    # reciprocal per species, three scalar reciprocals, lg2 T) at the measured
    # FFMA / MUFU rate ratio
    poly = bench.mixed_ops_per_cell_step(S, R, Rrev, nnz)
    assert poly == pytest.approx(5668 + 336 * bench.FFMA_PER_CLK / bench.MUFU_PER_CLK)
    assert poly == pytest.approx(6998.4, abs=0.1)
    net = bench.mixed_ops_per_cell_step(S, R, Rrev, nnz, net=True)
    mma = 2 * (64 * 64 + 64 * S) / bench.BF16_FLOP_PER_CLK * bench.FFMA_PER_CLK
    assert net == pytest.approx(poly - 4 * S + mma)


def test_roofline_fraction():
    r = bench.alu_roofline("mixed", 7000.0, 3.5e8, 1.0, 2032.0)
    peak = bench.FFMA_PER_CLK * bench.N_SMS * 2032e6
    assert r["frac"] == pytest.approx(7000.0 * 3.5e8 / peak)
    assert r["peak"] == pytest.approx(2 * peak / 1e12)          # FMA = 2 flops
    assert r["achieved"] == pytest.approx(2 * 7000.0 * 3.5e8 / 1e12)
    f = bench.alu_roofline("fp64", 10725.5, 2.44e7, 1.0, 2032.0)
    assert f["frac"] == pytest.approx(10725.5 * 2.44e7 / (bench.DFMA_PER_CLK * 148 * 2032e6))
    assert 0.5 < f["frac"] < 0.55
