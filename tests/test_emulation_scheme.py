"""Exact-arithmetic model of the emulated FP64 trailing update (the `emulate_fp64` option of
the factorisation): checks the number-theoretic facts the CUDA kernel relies on, on the CPU.

Each row of a 32-column panel is rounded to 55 bits below its largest exponent and written
as seven balanced base-256 digits (exact in bf16); slice products are grouped by s + t <= 9
and must stay below 2^22 so that FP32 accumulators offset by 1.5 * 2^23 hold them exactly;
the groups are packed into one 64-bit integer w = 2^16 hi + round(lo / 2^16) and applied as
an FP64 value rounded once (ties away from zero), then subtracted.  The model's update error,
relative to |C| + sum |P_i||P_j|, must be that of a plain FP64 update (a few u = 2^-53 at
most).  A truncating variant (floor of the slices, w = 2^14 hi + floor(lo / 2^18)) is kept
beside it: its error, bounded relative to the row maxima, reaches several u."""
from fractions import Fraction

import numpy as np
import pytest

W = 32  # columns per block


def _bits(x):
    return int(np.float64(x).view(np.uint64))


def slice_row(row, rounded=True):
    """Biased exponent em of the row maximum and the seven digits of every value."""
    em = max(((_bits(v) >> 52) & 0x7FF) for v in row)
    digits = []
    for v in row:
        b = _bits(v)
        E = (b >> 52) & 0x7FF
        Y = 0
        if 0 < E < 0x7FF:
            sh = em - E
            M = ((b & ((1 << 52) - 1)) | (1 << 52)) << 2
            if rounded:
                Y = M if sh == 0 else (0 if sh >= 56 else ((M >> (sh - 1)) + 1) >> 1)
            else:
                Y = 0 if sh >= 55 else M >> sh
        Yb = Y + 0x808080808080
        d = [Yb >> 48] + [((Yb >> (48 - 8 * s)) & 255) - 128 for s in range(1, 7)]
        if b >> 63:
            d = [-q for q in d]
        digits.append(d)
    return em, digits


def value_of(em, d):
    """2^(em - 1021) sum_s d_s 2^(-8 (s + 1)) as an exact rational."""
    return Fraction(2) ** (em - 1021) * sum(Fraction(q, 256 ** (s + 1)) for s, q in enumerate(d))


def round_half_away(fr):
    """Fraction -> nearest FP64, ties away from zero (the kernel's integer-built conversion)."""
    if fr == 0:
        return 0.0
    sgn = -1 if fr < 0 else 1
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q = a / Fraction(2) ** (e - 52)  # in [2^52, 2^53)
    n = int(q)
    if q - n >= Fraction(1, 2):
        n += 1
    return sgn * float(Fraction(n) * Fraction(2) ** (e - 52))


def emulated_update(c, pi, pj, rounded=True):
    ei, di = slice_row(pi, rounded)
    ej, dj = slice_row(pj, rounded)
    G = {g: 0 for g in range(2, 10)}
    for s in range(7):
        for t in range(7):
            g = s + t + 2
            if g > 9:
                continue
            G[g] += sum(di[k][s] * dj[k][t] for k in range(W))
    hi = G[2] * 2**24 + G[3] * 2**16 + G[4] * 256 + G[5]
    lo = G[6] * 2**24 + G[7] * 2**16 + G[8] * 256 + G[9]
    if rounded:
        w = hi * 2**16 + ((lo + 2**15) >> 16)  # arithmetic shift: round half up
        scale = Fraction(2) ** (ei - 1021 + ej - 1021 - 56)
    else:
        w = hi * 2**14 + (lo >> 18)
        scale = Fraction(2) ** (ei - 1021 + ej - 1021 - 54)
    assert abs(w) < 2**63
    return c - round_half_away(w * scale), G


def _panel(rng, n):
    """Rows spanning several orders of magnitude, columns with their own scales, some zeros."""
    p = rng.normal(size=(n, W)) * np.exp(rng.normal(size=(n, 1)) * 3) * np.exp(rng.normal(size=(1, W)) * 1.5)
    p[rng.random(p.shape) < 0.05] = 0.0
    return p


def test_digits_reconstruct_the_55_bit_cut_exactly():
    rng = np.random.default_rng(0)
    for row in _panel(rng, 6):
        em, digits = slice_row(row)
        for v, d in zip(row, digits):
            assert 0 <= abs(d[0]) <= 128 and all(-128 <= q <= 128 for q in d)
            # exact in bf16 (the upper half of the FP32 bits): |q| <= 2^7 needs at most 8 bits
            assert all(int(np.float32(q).view(np.uint32)) & 0xFFFF == 0 for q in d)
            exact = Fraction(float(v))
            err = abs(value_of(em, d) - exact)
            assert err <= Fraction(2) ** (em - 1078)  # half a unit of the 55-bit cut, 2^(em - 1077)


def test_group_sums_fit_the_offset_fp32_accumulator():
    # worst case: every digit at +-128, 32 columns, at most 7 pairs per group
    assert 7 * W * 128 * 128 < 2**22
    rng = np.random.default_rng(1)
    p = _panel(rng, 4)
    for i in range(4):
        for j in range(4):
            _, G = emulated_update(0.0, p[i], p[j])
            assert all(abs(v) < 2**22 for v in G.values())
            # every partial sum is bounded by the sum of absolute products, so FP32 values in
            # [2^23, 2^24) hold them exactly: check that the offset keeps that range
            assert all(2**23 <= 1.5 * 2**23 + v < 2**24 for v in G.values())


@pytest.mark.parametrize("seed", [2, 3])
def test_update_error_is_that_of_plain_fp64(seed):
    rng = np.random.default_rng(seed)
    n = 6
    p = _panel(rng, n)
    C = rng.normal(size=(n, n)) * 10
    emu, trunc, plain = [], [], []
    for i in range(n):
        for j in range(n):
            exact = Fraction(float(C[i, j])) - sum(Fraction(float(p[i, k])) * Fraction(float(p[j, k])) for k in range(W))
            bound = abs(C[i, j]) + float(np.abs(p[i]) @ np.abs(p[j]))
            e, _ = emulated_update(float(C[i, j]), p[i], p[j])
            t, _ = emulated_update(float(C[i, j]), p[i], p[j], rounded=False)
            emu.append(float(abs(Fraction(e) - exact)) / bound)
            trunc.append(float(abs(Fraction(t) - exact)) / bound)
            plain.append(float(abs(Fraction(float(C[i, j] - p[i] @ p[j])) - exact)) / bound)
    u = 2.0**-53
    assert max(plain) <= 4 * u
    assert max(emu) <= 4 * u, max(emu)
    assert np.mean(emu) <= 1.5 * np.mean(plain) + 0.25 * u, (np.mean(emu), np.mean(plain))
    assert max(trunc) <= 16 * u and max(emu) < max(trunc)


def test_an_eight_7_bit_slice_cut_is_less_accurate():
    """A cut into eight 7-bit slices (56 bits) keeping the same slice pairs (s + t <= 9) drops
    larger groups: with rows and columns of mixed magnitude it is less accurate."""
    rng = np.random.default_rng(4)
    n = 5
    p = _panel(rng, n)

    def old_update(c, pi, pj):
        def cut(row):
            em = max(((_bits(v) >> 52) & 0x7FF) for v in row)
            out = []
            for v in row:
                b = _bits(v)
                E = (b >> 52) & 0x7FF
                Y = 0
                if 0 < E < 0x7FF:
                    sh = em - E
                    Y = 0 if sh >= 56 else (((b & ((1 << 52) - 1)) | (1 << 52)) << 3) >> sh
                d = [(Y >> (49 - 7 * s)) & 127 for s in range(8)]
                out.append([-q for q in d] if b >> 63 else d)
            return em, out
        ei, di = cut(pi)
        ej, dj = cut(pj)
        tot = Fraction(0)
        for s in range(8):
            for t in range(8):
                if s + t + 2 <= 9:
                    tot += Fraction(sum(di[k][s] * dj[k][t] for k in range(W)), 128 ** (s + t + 2))
        return float(Fraction(c) - Fraction(2) ** (ei - 1022 + ej - 1022) * tot)

    new, old = [], []
    for i in range(n):
        for j in range(n):
            exact = -sum(Fraction(float(p[i, k])) * Fraction(float(p[j, k])) for k in range(W))
            bound = float(np.abs(p[i]) @ np.abs(p[j]))
            new.append(float(abs(Fraction(emulated_update(0.0, p[i], p[j])[0]) - exact)) / bound)
            old.append(float(abs(Fraction(old_update(0.0, p[i], p[j])) - exact)) / bound)
    assert max(new) < max(old)
