"""The roofline model of bench.py: the method's work per cell-step counted
from the algorithm (about 40 S + 43 R flops, 2 R exponentials, S divisions,
2 logarithms; the thermo network's MMA flops in place of 28 S thermo flops),
each class at the measured rate of the unit that executes it, and the
fraction's arithmetic.  The numbers below are those counts worked by hand for
the 32-species / 150-reaction workload."""
import pytest

import bench


def test_method_counts_for_32_150():
    c = bench.method_counts(32, 150)
    assert c == {"flops": 7730, "exp": 300, "div": 32, "log": 2, "mma": 0}
    n = bench.method_counts(32, 150, net=True)
    assert n["flops"] == 7730 - 28 * 32
    assert n["mma"] == 2 * (64 + 64 * 64 + 64 * 96) == 20608


def test_bound_per_cell_step_by_hand():
    clk = 148 * 2032e6
    # plain FP64: DFMA 1.668, exp 0.104, division 0.222, log 0.055 per SM and clock
    t64 = 7730 / (2 * 1.668 * clk) + 300 / (0.104 * clk) + 32 / (0.222 * clk) + 2 / (0.055 * clk)
    assert bench.bound_s_per_cell_step(32, 150, "fp64", False, 2032.0, 1400.0) == pytest.approx(t64)
    assert 1.0 / t64 == pytest.approx(5.58e7, rel=0.01)
    # mixed: FFMA 125.36, MUFU 31.66 per SM and clock; BF16 at the given TFLOP/s
    tp = 7730 / (2 * 125.36 * clk) + 334 / (31.66 * clk)
    assert bench.bound_s_per_cell_step(32, 150, "mixed", False, 2032.0, 1400.0) == pytest.approx(tp)
    tn = 6834 / (2 * 125.36 * clk) + 334 / (31.66 * clk) + 20608 / 1400e12
    assert bench.bound_s_per_cell_step(32, 150, "mixed", True, 2032.0, 1400.0) == pytest.approx(tn)
    assert 1.0 / tn == pytest.approx(7.1e9, rel=0.02)


def test_roofline_fraction_reproduces_the_measured_round_numbers():
    """Cell-step rates measured on the 1M-cell workload (FP64 2.43e7,
    polynomial mixed 4.74e8, network mixed 3.52e8 cell-steps/s at 2032 MHz)
    give fractions of about 0.43, 0.065 and 0.05 under this model."""
    f = bench.alu_roofline("fp64", 32, 150, False, 2.43e7, 1.0, 2032.0)
    assert f["frac"] == pytest.approx(0.435, abs=0.005)
    assert f["peak"] == pytest.approx(2 * 1.668 * 148 * 2032e6 / 1e12)
    assert f["achieved"] == pytest.approx(f["frac"] * f["peak"])
    p = bench.alu_roofline("mixed", 32, 150, False, 4.74e8, 1.0, 2032.0)
    assert p["frac"] == pytest.approx(0.065, abs=0.003)
    n = bench.alu_roofline("mixed", 32, 150, True, 3.52e8, 1.0, 2032.0)
    assert n["frac"] == pytest.approx(0.05, abs=0.003)
    assert n["cell_steps_per_s_bound"] * n["frac"] == pytest.approx(3.52e8)


def test_multiphase_bound_by_hand():
    """The multiphase cell-step: 420 flops on the FP64 pipe, 112 divisions and
    11 powers (exp + log) at CUDA's double rates."""
    clk = 148 * 2032e6
    t = 420 / (2 * 1.668 * clk) + 112 / (0.222 * clk) + 11 * (1 / (0.104 * clk) + 1 / (0.055 * clk))
    assert bench.mp_bound_s_per_cell_step(2032.0) == pytest.approx(t)
    assert 1.0 / t == pytest.approx(3.2e8, rel=0.03)
