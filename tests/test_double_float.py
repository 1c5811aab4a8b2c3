"""Error bound of the FP32 form's double-float residual, on the CPU.

The FP32 form keeps its accurate iterate x as unevaluated pairs hi + lo of FP32 numbers and
forms the residual r = b - (pad x_i + sum_j g_ij (x_i - x_j)) with error-free
transformations: TwoSum (Knuth) for the differences and the running sum, and the FMA
TwoProduct for g times the difference, with the remaining rounding errors gathered in a
second FP32 word (Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26, 2005).

This test restates those steps with IEEE FP32 operations (numpy float32; an FMA is the
float64 product of two FP32 numbers, which is exact, plus the addend, rounded once to FP32).
It checks the claimed bound against exact rational arithmetic (fractions.Fraction) on random
stencils whose terms cancel to a residual a million times smaller than the terms:
|computed - exact| <= 2^-23 |exact| + 2^-44 * (sum of the terms' magnitudes).
A plain FP32 evaluation misses that bound by many orders of magnitude (checked below too).
The kernel itself is tested on the GPU (tests/test_gpu_df.py: convergence to tol 1e-10).
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def add(a, b):
    return f32(f32(a) + f32(b))


def sub(a, b):
    return f32(f32(a) - f32(b))


def mul(a, b):
    return f32(f32(a) * f32(b))


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def residual_df(b, gp, Xi, nbrs):
    """b - (gp Xi + sum g (Xi - Xj)) with X = (hi, lo) pairs, the kernel's order of steps."""
    S = mul(gp, Xi[0])
    C = fma(gp, Xi[1], fma(gp, Xi[0], -S))
    for g, Xj in nbrs:
        d, e = two_sum(Xi[0], -Xj[0])
        dl = add(e, sub(Xi[1], Xj[1]))
        p = mul(g, d)
        pe = fma(g, dl, fma(g, d, -p))
        S, t = two_sum(S, p)
        C = add(C, add(t, pe))
    t0, t1 = two_sum(b, -S)
    return add(t0, sub(t1, C))


def residual_fp32(b, gp, Xi, nbrs):
    q = mul(gp, Xi[0])
    for g, Xj in nbrs:
        q = add(q, mul(g, sub(Xi[0], Xj[0])))
    return sub(b, q)


def split(x):
    h = f32(x)
    return h, f32(x - np.float64(h))


def F(v):
    return Fraction(float(v))


def test_double_float_residual_bound():
    rng = np.random.default_rng(2026)
    worst_df, worst_32 = 0.0, 0.0
    for _ in range(4000):
        base = 10 ** rng.uniform(-6, 3)
        Xi = split(base * (1 + rng.normal() * 10 ** rng.uniform(-8, 0)))
        nb = [(f32(10 ** rng.uniform(-1, 2)) if rng.random() > 0.1 else f32(0),
               split(base * (1 + rng.normal() * 10 ** rng.uniform(-8, 0)))) for _ in range(6)]
        gp = f32(10 ** rng.uniform(-2, 2)) if rng.random() > 0.5 else f32(0)
        Xe = F(Xi[0]) + F(Xi[1])
        q = F(gp) * Xe + sum(F(g) * (Xe - (F(X[0]) + F(X[1]))) for g, X in nb)
        b = f32(float(q) * (1 + rng.normal() * 1e-6))  # the residual cancels to ~1e-6 of q
        exact = F(b) - q
        scale = abs(F(gp) * Xe) + sum(abs(F(g)) * (abs(Xe) + abs(F(X[0]) + F(X[1]))) for g, X in nb) + abs(F(b))
        err = abs(F(residual_df(b, gp, Xi, nb)) - exact)
        assert err <= abs(exact) * Fraction(1, 2 ** 23) + scale * Fraction(1, 2 ** 44)
        if scale > 0:
            worst_df = max(worst_df, float(err / scale))
            worst_32 = max(worst_32, float(abs(F(residual_fp32(b, gp, Xi, nb)) - exact) / scale))
    assert worst_df < 2.0 ** -44
    assert worst_32 > 1e3 * worst_df  # plain FP32 is nowhere near: the pairs are needed


def test_double_float_accumulation():
    """x += c in double-float (TwoSum, then renormalised) keeps about 48 bits."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        X = (f32(0), f32(0))
        tot = Fraction(0)
        for s in range(40):
            c = f32(rng.normal() * 10 ** rng.uniform(-8, 2) * 0.5 ** (s / 5))
            t0, t1 = two_sum(X[0], c)
            X = two_sum(t0, add(t1, X[1]))
            tot += F(c)
        assert abs(F(X[1])) <= abs(F(X[0])) * Fraction(1, 2 ** 23)
        mag = max(abs(tot), Fraction(1, 10 ** 30))
        assert abs(F(X[0]) + F(X[1]) - tot) <= mag * Fraction(1, 2 ** 40) + Fraction(1, 10 ** 40)
