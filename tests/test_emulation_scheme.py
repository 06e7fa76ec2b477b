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


# ---- the fixed point of the trailing matrix ---------------------------------------------
# The kernel holds the not yet factorised part of A as integers round(v 2^61) (every entry of
# K + sigma^2 I and of its Schur complements lies within the largest diagonal entry, about 1)
# and subtracts each slice-product update w 2^(e_i + e_j - 2098) shifted to that scale.

FIX = 61


def fix_shift(w, sh):
    """w 2^sh rounded to an integer, ties up (the kernel's shift of an update)."""
    if sh >= 0:
        return w << sh
    if sh < -63:
        return 0
    return ((w >> (-sh - 1)) + 1) >> 1


def fixed_update(cfix, pi, pj):
    ei, di = slice_row(pi)
    ej, dj = slice_row(pj)
    G = {g: 0 for g in range(2, 10)}
    for s in range(7):
        for t in range(7):
            g = s + t + 2
            if g <= 9:
                G[g] += sum(di[k][s] * dj[k][t] for k in range(W))
    hi = G[2] * 2**24 + G[3] * 2**16 + G[4] * 256 + G[5]
    lo = G[6] * 2**24 + G[7] * 2**16 + G[8] * 256 + G[9]
    w = hi * 2**16 + ((lo + 2**15) >> 16)
    upd = fix_shift(w, ei + ej - 2098 + FIX)
    assert abs(upd) < 2**63 and abs(cfix - upd) < 2**63  # no 64-bit overflow
    return cfix - upd


def _factor_rows(rng, n):
    """Rows of a Cholesky factor's panel: unit-bounded rows, magnitudes over several orders."""
    p = rng.normal(size=(n, W)) * np.exp(rng.normal(size=(n, 1)) * 2)
    p /= np.maximum(1.0, np.linalg.norm(p, axis=1, keepdims=True))
    p[rng.random(p.shape) < 0.05] = 0.0
    return p


@pytest.mark.parametrize("seed", [5, 6])
def test_fixed_point_update_error_is_that_of_plain_fp64(seed):
    """C in [-1, 1] held as round(C 2^61), rows of norm <= 1: the fixed-point update stays within
    a few u of the exact value relative to |C| + sum |P_i||P_j| (as the FP64 update), plus the
    fixed point's half unit 2^-62; the diagonal case (i = j, C_ii - |P_i|^2 > 0) included."""
    rng = np.random.default_rng(seed)
    n = 6
    p = _factor_rows(rng, n)
    C = rng.uniform(-1, 1, (n, n))
    u = 2.0**-53
    worst = 0.0
    for i in range(n):
        for j in range(n):
            c = float(C[i, j]) if i != j else 1.0 + 1e-4
            cfix = round(Fraction(c) * 2**FIX)
            got = Fraction(fixed_update(cfix, p[i], p[j]), 2**FIX)
            exact = Fraction(c) - sum(Fraction(float(p[i, k])) * Fraction(float(p[j, k])) for k in range(W))
            bound = abs(c) + float(np.abs(p[i]) @ np.abs(p[j]))
            err = float(abs(got - exact))
            assert err <= 4 * u * bound + 2.0 ** -61, (i, j, err / (u * bound))
            worst = max(worst, err / (u * bound))
    assert worst > 0  # the check is not vacuous


# ---- float-pair kernel values ----------------------------------------------------------
# Model of the kernel's mixed-precision entries exp(-|a - b|^2 / (2 l^2)) in float-pair
# arithmetic on FP32 world coordinates, operation for operation in numpy float32 (an FMA as
# the float64 product plus the addend, rounded once to float32: exact wherever the kernel
# relies on an FMA being error-free).

f32 = np.float32


def _fma(a, b, c):
    a, b, c = np.broadcast_arrays(np.asarray(a, f32), np.asarray(b, f32), np.asarray(c, f32))
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _two_sum(a, b):
    s = (a + b).astype(f32)
    bv = (s - a).astype(f32)
    return s, ((a - (s - bv)).astype(f32) + (b - bv)).astype(f32)


def kernel_fix_model(a, b, inv2l2):
    kL0, kL1, kL2 = f32(float.fromhex("0x1.63p-9")), f32(float.fromhex("-0x1.bd0106p-21")), f32(float.fromhex("0x1.cf79acp-48"))
    ch = f32(inv2l2)
    cl = f32(inv2l2 - float(ch))
    tab = np.array([2.0 ** (j / 256) for j in range(256)])
    Th = tab.astype(f32)
    Tl = (tab - Th.astype(np.float64)).astype(f32)
    S = np.zeros(len(a), f32)
    E = np.zeros(len(a), f32)
    for k in range(3):
        dh, dl = _two_sum(a[:, k], -b[:, k])
        p = (dh * dh).astype(f32)
        pe = _fma(dh, dh, -p)
        t, te = _two_sum(S, p)
        E = (E + (te + _fma(dl, _fma(2, dh, dl), pe)).astype(f32)).astype(f32)
        S = (t + E).astype(f32)
        E = (E - (S - t).astype(f32)).astype(f32)
    yh = (S * ch).astype(f32)
    yl = (_fma(S, ch, -yh) + _fma(S, cl, (E * ch).astype(f32))).astype(f32)
    n = np.rint((yh * f32(369.32993046757464)).astype(f32)).astype(f32)
    a0, ae = _two_sum((n * kL0).astype(f32), -yh)
    p2 = (n * kL1).astype(f32)
    b0, be = _two_sum(a0, p2)
    rh, ce = _two_sum(b0, -yl)
    rl = (((ae + be).astype(f32) + ce).astype(f32) + _fma(n, kL2, _fma(n, kL1, -p2))).astype(f32)
    q = (rh * rh).astype(f32)
    qe = _fma(rh, rh, -q)
    c34 = ((q * rh).astype(f32) * _fma(rh, f32(1 / 24), f32(1 / 6))).astype(f32)
    small = (_fma(0.5, qe, rl) + _fma(rh, rl, c34)).astype(f32)
    u, ue = _two_sum(rh, (f32(0.5) * q).astype(f32))
    eh, e4 = _two_sum(np.ones_like(u), u)
    el = (e4 + (ue + small).astype(f32)).astype(f32)
    ni = n.astype(np.int64)
    j = ni & 255
    m = (ni >> 8) + (j != 0)
    th, tl = Th[(256 - j) & 255], Tl[(256 - j) & 255]
    vh = (th * eh).astype(f32)
    vl = (_fma(th, eh, -vh) + _fma(th, el, (tl * eh).astype(f32))).astype(f32)
    # vh 2^(61 - m) is exact in binary; vl's part rounds to the integer grid
    out = np.array([round(Fraction(float(x)) * 2 ** (FIX - int(mm))) + round(Fraction(float(z)) * 2 ** (FIX - int(mm)))
                    for x, z, mm in zip(vh, vl, m)], dtype=object)
    return np.where(yh <= 43.5, out, 0)


def test_float_pair_kernel_value_model():
    """The float-pair kernel value, modelled operation for operation, against the exact value
    (FP32 world coordinates 100 m from the origin, l = 0.3): error below 2^-45 k (1 + y) + 2
    units of 2^-61 and below 2^-46 absolute; coincident points give 2^61 exactly."""
    rng = np.random.default_rng(7)
    n = 4000
    a = (np.array([103.7, -45.3, 12.9]) + rng.uniform(-1.5, 1.5, (n, 3))).astype(f32)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.concatenate([rng.uniform(0, 2.0, n // 2), rng.uniform(0, 0.3, n // 4), 10.0 ** rng.uniform(-6, -1, n // 4)])
    b = (a + d * r[:, None]).astype(f32)
    b[:10] = a[:10]
    inv2l2 = 1.0 / (2 * 0.3 * 0.3)
    got = kernel_fix_model(a, b, inv2l2)
    assert all(v == 2**FIX for v in got[:10])
    worst = 0.0
    for i in range(n):
        r2 = sum((Fraction(float(a[i, k])) - Fraction(float(b[i, k]))) ** 2 for k in range(3))
        y = float(r2 * Fraction(inv2l2))
        exact = np.exp(-np.longdouble(y)) * np.longdouble(2.0) ** FIX
        err = abs(np.longdouble(int(got[i])) - exact)
        assert err <= exact * (1 + y) * np.longdouble(2.0) ** -45 + 2, i
        assert err <= 2.0 ** (FIX - 46)
        worst = max(worst, float(err / (exact * (1 + y) + 1)))
    assert worst > 0


# ---- bordered variance (Eq. 2 as a Schur complement) ------------------------------------

def _partial_cholesky(M, n):
    """Right-looking Cholesky of the first n columns of the symmetric matrix M (lower part);
    the trailing block is left as the Schur complement."""
    M = M.copy()
    for k in range(n):
        M[k, k] = np.sqrt(M[k, k])
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k + 1:, k])
    return M


def test_bordered_factorisation_gives_the_latent_variance():
    """Appending the queries' kernel vectors to K + sigma^2 I as rows (1 on their diagonal) and
    factorising only the instance's columns leaves u = 1 - k^T (K + sigma^2 I)^-1 k on the
    appended diagonal (the latent variance, Eq. 2 read as the posterior); the rows below become
    (L^-1 k)^T; a query's value does not depend on the other appended rows; and the leading
    block is the factor of K + sigma^2 I alone."""
    rng = np.random.default_rng(17)
    N, nq, l2, s2 = 40, 9, 0.09, 1e-4
    X = rng.uniform(-0.5, 0.5, (N, 3))
    Qp = np.vstack([rng.uniform(-0.8, 0.8, (nq - 1, 3)), [[30.0, 30.0, 30.0]]])  # last: far away
    kern = lambda a, b: np.exp(-((a[:, None, :] - b[None, :, :]) ** 2).sum(-1) / (2 * l2))
    A = kern(X, X) + s2 * np.eye(N)
    Ks = kern(Qp, X)
    M = np.block([[A, Ks.T], [Ks, np.eye(nq)]])
    F = _partial_cholesky(M, N)
    u_border = np.diag(F[N:, N:])
    u_direct = 1.0 - np.einsum("ij,ij->i", Ks, np.linalg.solve(A, Ks.T).T)
    np.testing.assert_allclose(u_border, u_direct, rtol=1e-9, atol=1e-12)
    assert abs(u_border[-1] - 1.0) < 1e-12  # no support: the prior variance
    L = np.linalg.cholesky(A)
    np.testing.assert_allclose(np.tril(F[:N, :N]), L, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F[N:, :N], np.linalg.solve(L, Ks.T).T, rtol=1e-9, atol=1e-12)
    # one query alone gives the same value
    for a in (0, 4):
        Ma = np.block([[A, Ks[a:a + 1].T], [Ks[a:a + 1], np.ones((1, 1))]])
        assert abs(_partial_cholesky(Ma, N)[N, N] - u_border[a]) <= 1e-12
