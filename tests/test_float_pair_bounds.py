"""The error bound behind the mixed path's reading of "FP64 K exponent": a
species' Gibbs term of Eq. 30 in log2 units,
    g2(T) = c0 + c1 ln T + c2 / T + c3 T + c4 T^2 + c5 T^3 + c6 T^4,
evaluated the way the mixed kernels do it -- float pairs (hi + lo) for the
FP64 coefficients and for ln T, 1/T, T^2..T^4, products by FMA, sums by
TwoSum (the compensated dot product of Ogita, Rump and Oishi) -- is exact to
about 1e-11 against the same coefficients evaluated in exact decimal
arithmetic, while plain FP32 evaluation is off by ~1e-5.

This is an independent float32 emulation (numpy, round-to-nearest; an FMA is
emulated exactly through float64, where a product of two floats is exact)
written from the algorithm, not from the kernel source; the kernels' results
are checked against the oracle by the GPU tests."""
import math
from decimal import Decimal, getcontext

import numpy as np

from paper_1905_09395_b300 import synth

f32 = np.float32


def rn(x):
    return float(f32(x))


def fma(a, b, c):
    return rn(a * b + c)   # a*b of two floats is exact in float64


def two_sum(a, b):
    s = rn(a + b)
    bb = rn(s - a)
    return s, rn(rn(a - rn(s - bb)) + rn(b - bb))


def fast_two_sum(a, b):
    s = rn(a + b)
    return s, rn(b - rn(s - a))


def split(x):
    h = rn(x)
    return h, rn(x - h)


def ff_mul(x, y):
    p = rn(x[0] * y[0])
    e = fma(x[0], y[0], -p)
    e = fma(x[0], y[1], e)
    e = fma(x[1], y[0], e)
    return fast_two_sum(p, e)


def g2_float_pairs(c, T):
    Tp = split(T)
    r0 = rn(1.0 / Tp[0])
    e0 = fma(-Tp[0], r0, 1.0)
    e0 = fma(-Tp[1], r0, e0)
    inv = fast_two_sum(r0, rn(r0 * fma(e0, e0, e0)))
    lnT = split(math.log(T))
    T2 = ff_mul(Tp, Tp)
    T3 = ff_mul(T2, Tp)
    T4 = ff_mul(T2, T2)
    cp = [split(x) for x in c]
    s, e = cp[0]
    for (ch, cl), b in zip(cp[1:], (lnT, inv, Tp, T2, T3, T4)):
        p = rn(ch * b[0])
        pe = fma(ch, b[0], -p)
        pe = fma(ch, b[1], pe)
        pe = fma(cl, b[0], pe)
        s, t = two_sum(s, p)
        e = rn(e + rn(t + pe))
    return two_sum(s, e)


def test_gibbs_term_in_float_pairs_is_fp64_grade():
    getcontext().prec = 40
    mech = synth.scale_mechanism()
    a7 = np.asarray(mech.nasa7).reshape(mech.n_species, 2, 7)
    split_T = np.asarray(mech.t_range).reshape(mech.n_species, 3)[:, 1]
    L2 = 1.4426950408889634
    lp = math.log(101325.0 / 8.314462618)
    worst_pair, worst_f32 = 0.0, 0.0
    for T in np.random.default_rng(0).uniform(300.0, 3000.0, 25):
        Td = Decimal(split(T)[0]) + Decimal(split(T)[1])
        basis = [Decimal(1), Td.ln(), 1 / Td, Td, Td ** 2, Td ** 3, Td ** 4]
        for i in range(mech.n_species):
            a = a7[i, 0 if T < split_T[i] else 1]
            c = [L2 * (a[0] - a[6] - lp), L2 * (1 - a[0]), L2 * a[5], -L2 * a[1] / 2,
                 -L2 * a[2] / 6, -L2 * a[3] / 12, -L2 * a[4] / 20]
            exact = sum(Decimal(ck) * bk for ck, bk in zip(c, basis))
            h, l = g2_float_pairs(c, T)
            worst_pair = max(worst_pair, abs(float(Decimal(h) + Decimal(l) - exact)))
            # the same sum in plain FP32
            Tf = rn(T)
            b32 = [1.0, rn(math.log(Tf)), rn(1.0 / Tf), Tf, rn(Tf * Tf), rn(rn(Tf * Tf) * Tf),
                   rn(rn(Tf * Tf) * rn(Tf * Tf))]
            s = 0.0
            for ck, bk in zip(c, b32):
                s = fma(rn(ck), bk, s)
            worst_f32 = max(worst_f32, abs(float(Decimal(s) - exact)))
    assert worst_pair < 1e-11, worst_pair
    assert worst_f32 > 1e-6   # what the float pairs buy
