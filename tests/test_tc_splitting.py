"""The arithmetic of the tensor-core face interpolation, emulated in NumPy on the CPU.

Pins the design of FR_PREC_MIXED_TC independently of the GPU: the line contraction
y_j = sum_a l_j(a) x_a (x_a double-float hi + lo, l_j the Gauss-Legendre boundary values) computed
from exponent-aligned 10-bit slices (Ozaki, Ogita, Oishi & Rump 2012) as the kernel does it:
  * every slice is an integer of at most 11 significant bits (exact in TF32);
  * every product sum an MMA forms (K <= 8 terms) is an integer below 2^24, so FP32 accumulation
    in any order is exact, and so are the level sums;
  * the double-float combination of the levels is within 2^-44 of sigma tau of the exact
    contraction: the dropped levels and slices leave 2^-51, the rest is the rounding of the
    double-float output itself (48 bits of a value up to 8 sigma tau), as in the double-float
    interpolation.  (Four slices left 2^-41, which at Ma 0.1 made the continuity residual's
    error reach 1e-6 of its largest entry on the GPU.)
And the reason for the alignment (the finding behind the choice): the same slices without a
common exponent per line (a plain hi/lo split in TF32 accumulated in FP32) leave errors near 2^-23
of the terms' size, far above the double-float path.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle.basis import Basis1D

BETA, SLICES = 10, 5
f32 = np.float32


def _df32_line(rng, N, scale):
    x = rng.standard_normal(N) * scale * rng.choice([1.0, 1e-3, 1e-7], N)
    hi = x.astype(f32)
    lo = (x - hi.astype(np.float64)).astype(f32)
    return hi, lo


def _slice_line(hi, lo):
    """The kernel's slicing, in float32 arithmetic: (slices [5][N], exponent E with max|hi| < 2^E)."""
    mx = float(np.max(np.abs(hi)))
    if mx == 0.0:
        return np.zeros((SLICES, hi.size), f32), 0
    _, E = np.frexp(mx)
    E = int(E)
    sc, sc_lo, up = f32(2.0 ** (BETA - E)), f32(2.0 ** (3 * BETA - E)), f32(2.0 ** BETA)
    X = np.zeros((SLICES, hi.size), f32)
    u = hi * sc
    X[0] = np.rint(u)
    u = (u - X[0]) * up
    X[1] = np.rint(u)
    # hi's remaining bits plus lo as an exact pair (two_sum), the pair's error carried on
    wh, wl = _two_sum(f32((u - X[1]) * up), f32(lo * sc_lo))
    X[2] = np.rint(wh)
    u = f32(f32(wh - X[2]) + wl) * up
    X[3] = np.rint(u)
    u = (u - X[3]) * up
    X[4] = np.rint(u)
    return X, E


def _slice_op(row):
    _, F = np.frexp(np.max(np.abs(row)))
    y = np.ldexp(row, -int(F))
    O = np.zeros((SLICES, row.size))
    for t in range(SLICES):
        u = np.ldexp(y, BETA)
        O[t] = np.rint(u)
        y = u - O[t]
    return O.astype(f32), int(F)


def _sig_bits(v):
    v = abs(int(v))
    return 0 if v == 0 else v.bit_length() - (len(bin(v)) - len(bin(v).rstrip("0")))


def _fp32_sum(terms, order):
    acc = f32(0.0)
    for k in order:
        acc = f32(acc + f32(terms[k]))
    return acc


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_sliced_contraction_is_exact_up_to_the_dropped_levels(p):
    rng = np.random.default_rng(100 + p)
    b = Basis1D(p)
    N = p + 1
    worst = 0.0
    for trial in range(40):
        hi, lo = _df32_line(rng, N, 10.0 ** rng.uniform(-3, 3))
        X, E = _slice_line(hi, lo)
        for s in range(SLICES):
            assert all(_sig_bits(v) <= 11 for v in X[s])
        exact_x = [Fraction(float(h)) + Fraction(float(l)) for h, l in zip(hi, lo)]
        for row in (b.l_minus, b.l_plus):
            O, F = _slice_op(row)
            D = [[int(sum(int(X[s][a]) * int(O[t][a]) for a in range(N))) for t in range(SLICES)]
                 for s in range(SLICES)]
            # Every MMA output is an integer below 2^24 and any FP32 summation order is exact.
            for s in range(SLICES):
                for t in range(SLICES):
                    assert abs(D[s][t]) < 2 ** 24
                    terms = [float(X[s][a]) * float(O[t][a]) for a in range(N)]
                    assert float(_fp32_sum(terms, rng.permutation(N))) == D[s][t]
            A = [f32(sum(D[s][L - s] for s in range(L + 1))) for L in range(SLICES)]
            assert all(abs(int(a)) < 2 ** 24 for a in A)
            # Combination into double-float, as the kernel does it.
            h0, h1 = _two_sum(A[0], f32(A[1] * f32(2.0 ** -BETA)))
            lo_ = f32(float(A[4]) * 2.0 ** (-4 * BETA)
                      + float(f32(float(A[3]) * 2.0 ** (-3 * BETA) + float(f32(A[2] * f32(2.0 ** (-2 * BETA)))))))
            r0, r1 = _two_sum(h0, f32(h1 + lo_))
            scale = Fraction(2) ** (E + F - 2 * BETA)
            got = (Fraction(float(r0)) + Fraction(float(r1))) * scale
            want = sum(Fraction(float(c)) * x for c, x in zip(row, exact_x))
            err = abs(got - want) / (Fraction(2) ** (E + F))
            worst = max(worst, float(err))
    assert worst <= 2.0 ** -44, worst


def _tf32(x):
    """Round a float32 to TF32 (10 stored mantissa bits), nearest-even."""
    b = np.asarray(x, f32).view(np.uint32).astype(np.uint64)
    r = ((b + 0xFFF + ((b >> 13) & 1)) & ~np.uint64(0x1FFF)).astype(np.uint32)
    return r.view(f32)


def test_unaligned_splits_lose_to_fp32_accumulation():
    """Without a common exponent per line the FP32 accumulator rounds: a 3-product hi/lo TF32
    split (hi hi + hi lo + lo hi) of a low-Mach energy line leaves errors near 1e-7 of the
    terms' size (measured 1.3e-7), about 2^21 times the aligned scheme's bound."""
    rng = np.random.default_rng(7)
    b = Basis1D(4)
    worst = 0.0
    for trial in range(200):
        # Energy-like line at Ma 0.1: ~178 with relative variations of 1e-3.
        x = 178.0 * (1.0 + 1e-3 * rng.standard_normal(5))
        row = b.l_plus
        xh = _tf32(x.astype(f32))
        xl = _tf32((x - xh.astype(np.float64)).astype(f32))
        ch = _tf32(row.astype(f32))
        cl = _tf32((row - ch.astype(np.float64)).astype(f32))
        terms = [float(f32(xh[a] * ch[a])) for a in range(5)] + [float(f32(xh[a] * cl[a])) for a in range(5)] + \
                [float(f32(xl[a] * ch[a])) for a in range(5)]
        got = float(_fp32_sum(terms, rng.permutation(15)))
        want = float(sum(Fraction(float(c)) * Fraction(float(v)) for c, v in zip(row, x)))
        scale = float(np.sum(np.abs(row) * np.abs(x)))
        worst = max(worst, abs(got - want) / scale)
    assert worst > 1e-8, worst
    assert worst > 2.0 ** 20 * 2.0 ** -44
