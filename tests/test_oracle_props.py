"""Pins for the oracle's surface-property GP (Eq. 6), property fusion (Sec. IV-C) and the
properties carried to zero crossings and mesh vertices (Sec. IV-D)."""
import numpy as np
import pytest

VS, L = 0.1, 0.3


def _plane_points(rng, n=4000, side=1.6):
    xy = rng.uniform(-side / 2, side / 2, (n, 2))
    return np.c_[xy, 0.013 + rng.normal(0, 0.003, n)].astype(np.float32)


def test_single_point_closed_form(orc):
    """One occupied voxel with property c0: c(x) = c0 k(x, x1) / (1 + s^2) and
    w(x) = 1 - k(x, x1)^2 / (1 + s^2) at every testing voxel."""
    P = orc.params(n_props=1, sigma_prop=0.2)
    pts = np.array([[0.31, -0.22, 0.48]], np.float32)
    f = orc.frame(pts, P, props=np.array([[0.7]], np.float32))
    x1 = np.floor(pts[0].astype(np.float64) / VS + 0.5) * VS
    xs = orc.unpack_key(f.test_key) * VS
    k = np.exp(-np.sum((xs - x1) ** 2, 1) / (2 * L * L))
    s2 = 0.2 ** 2
    c0 = float(np.float32(0.7))
    np.testing.assert_allclose(f.c[:, 0], c0 * k / (1 + s2), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f.w, 1 - k * k / (1 + s2), rtol=1e-12, atol=1e-15)


def test_constant_property_equals_scaled_occupancy(orc):
    """With sigma_prop = sigma_occ and a constant property c0, Eq. 6 is c0 times the latent
    occupancy of Eq. 1 and its variance is the latent variance of Eq. 2: recovered here from
    the distance path (o = exp(-d^2 / 2 l^2), u = v / Lambda^2), which is separate code."""
    rng = np.random.default_rng(0)
    pts = _plane_points(rng)
    P = orc.params(n_props=2, sigma_prop=0.01, sigma_occ=0.01)
    props = np.tile(np.array([[0.25, -3.0]], np.float32), (len(pts), 1))
    f = orc.frame(pts, P, props=props)
    ok = (f.status == 0) & (f.d > 1e-3) & (f.d < 0.6)
    assert ok.sum() > 1000
    o = np.exp(-f.d[ok] ** 2 / (2 * L * L))
    np.testing.assert_allclose(f.c[ok, 0], 0.25 * o, rtol=1e-8)
    np.testing.assert_allclose(f.c[ok, 1], -3.0 * o, rtol=1e-8)
    lam = -L * L / (o * np.maximum(f.d[ok], 1e-3))
    u = f.v[ok] / lam ** 2
    np.testing.assert_allclose(f.w[ok], u, rtol=1e-6, atol=1e-12)


def test_linearity_and_voxel_means(orc):
    """Eq. 6 is linear in the training properties; a voxel's property is the mean of its
    points' properties, so splitting values among the points of a voxel does not matter as
    long as the mean is kept."""
    rng = np.random.default_rng(1)
    pts = _plane_points(rng, 3000)
    P = orc.params(n_props=1)
    a = rng.uniform(0, 1, (len(pts), 1)).astype(np.float32)
    b = rng.uniform(-1, 1, (len(pts), 1)).astype(np.float32)
    fa, fb = orc.frame(pts, P, props=a), orc.frame(pts, P, props=b)
    fab = orc.frame(pts, P, props=(a.astype(np.float64) + b).astype(np.float32))
    np.testing.assert_allclose(fab.c, fa.c + fb.c, atol=1e-6)  # (a + b) rounded to float32
    np.testing.assert_array_equal(fa.w, fb.w)
    # two copies of every point, with values m - e and m + e: the same frame as value m
    e = rng.uniform(0, 0.25, (len(pts), 1))
    m = np.full((len(pts), 1), 0.5)
    pts2 = np.r_[pts, pts]
    f2 = orc.frame(pts2, P, props=np.r_[m - e, m + e].astype(np.float32))
    f1 = orc.frame(pts, P, props=m.astype(np.float32))
    np.testing.assert_allclose(f2.c, f1.c, atol=1e-7)


def test_fusing_a_frame_twice(orc):
    """Eq. 8: fusing the same estimate twice keeps the property and halves its variance.
    Eq. 9: it keeps the property and doubles the weight (2 (1 - w))."""
    rng = np.random.default_rng(2)
    pts = _plane_points(rng, 2000)
    P = orc.params(n_props=1)
    f = orc.frame(pts, P, props=rng.uniform(0, 1, (len(pts), 1)).astype(np.float32))
    for mode in (0, 1):
        g = orc.Grid(fusion=mode)
        g.fuse_frame(f)
        C1, W1 = g.export_props()
        g.fuse_frame(f)
        C2, W2 = g.export_props()
        has = ~np.isnan(W1)
        assert has.sum() > 1000
        np.testing.assert_allclose(C2[has], C1[has], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(W2[has], W1[has] / 2 if mode == 0 else 2 * W1[has], rtol=1e-12)
        # keys / first-visit values: the frame's own estimates
        k = g.export()[0]
        sel = np.isin(f.test_key, k[has])
        o = np.argsort(f.test_key[sel])
        np.testing.assert_array_equal(C1[has, 0], f.c[sel][o, 0])
        np.testing.assert_array_equal(W1[has], f.w[sel][o] if mode == 0 else 1 - f.w[sel][o])


def test_property_gate_follows_the_distance(orc):
    """Properties are fused only where the distance is fused and the property estimate is
    valid; elsewhere the voxel has none (NaN)."""
    g = orc.Grid()
    key = orc.pack_key(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [3, 0, 0]]))
    d = np.array([0.1, 0.2, 0.3, np.inf])
    v = np.array([0.01, 0.01, 0.01, 0.01])
    st = np.array([0, 0, 0, 2], np.uint8)
    c = np.array([[1.0], [np.nan], [3.0], [4.0]])
    w = np.array([0.5, 0.5, 0.0, 0.5])
    g.fuse(key, d, v, st, c, w)
    k, D, V, fl = g.export()
    Cp, W = g.export_props()
    assert len(k) == 3
    assert Cp[0, 0] == 1.0 and W[0] == 0.5
    assert np.isnan(Cp[1, 0]) and np.isnan(W[1]) and np.isnan(W[2])


def test_crossing_properties_exact_for_linear_fields(orc):
    """A linear distance and a linear property field on the grid: the interpolated property
    at every zero crossing and mesh vertex is the property field at that point."""
    ijk = np.stack(np.meshgrid(*[np.arange(-8, 9)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = ijk * VS
    nrm = np.array([0.3, -0.5, 0.81])
    nrm /= np.linalg.norm(nrm)
    D = x @ nrm - 0.021
    a, b = np.array([[0.7, -0.2, 0.4], [0.1, 0.1, -0.9]]), np.array([0.3, -1.0])
    Cp = x @ a.T + b
    g = orc.Grid()
    n = len(D)
    g.fuse(orc.pack_key(ijk), D, np.ones(n), np.zeros(n, np.uint8), Cp, np.full(n, 0.5))
    xyz, _, slot, cp = g.crossings(VS, props=True)
    assert len(xyz) > 100 and cp.shape == (len(xyz), 2)
    # the FP64 crossing (before float32 rounding) is where the field is evaluated: compare to
    # the float32 point within its rounding
    np.testing.assert_allclose(cp, xyz.astype(np.float64) @ a.T + b, atol=2e-6)
    txyz, _, _, vp = g.mesh(VS, props=True)
    assert len(txyz) > 100
    np.testing.assert_allclose(vp, txyz @ a.T + b, atol=1e-12)
