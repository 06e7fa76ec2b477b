"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 path |dd| <= 1e-4 m and gradient angle <= 0.1 deg (the contract), with a
tighter typical-error check; mixed path |dd| <= 1e-3 m.  Leaf/voxel keys, training sets,
testing-voxel sets and statuses are compared bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

D_TOL = 1e-4
ANG_TOL_DEG = 0.1
D_TOL_MIXED = 1e-3


@pytest.fixture(scope="module")
def vg():
    import paper_2407_09649_gb300 as P
    P.build()
    from paper_2407_09649_gb300 import api
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return api


def _angle_deg(a, b):
    na = np.linalg.norm(a, axis=1)
    nb = np.linalg.norm(b, axis=1)
    c = np.sum(a * b, 1) / np.maximum(na * nb, 1e-300)
    return np.degrees(np.arccos(np.clip(c, -1, 1)))


def _check_mixed_var(v, rv, d, rd, floor=1e-3):
    """Mixed precision: v = (l^2 / (o d))^2 u, so a distance error dd moves v by about
    2 dd / max(d, floor) relative; the kernel values in FP32 add ~1e-3 relative to u."""
    rel = np.abs(v - rv) / np.abs(rv)
    bound = 2.0 * np.abs(d - rd) / np.maximum(rd, floor) * 1.5 + 2e-3
    assert np.all(rel <= bound), (rel.max(), np.argmax(rel - bound))


def _frame_gpu(vg, pts, **kw):
    m = vg.Map(**kw)
    f = m.build_frame(torch.from_numpy(pts).cuda())
    r = {k: v.cpu().numpy() for k, v in f.results().items()}
    inst = {k: v.cpu().numpy() for k, v in f.instances().items()}
    return m, f, r, inst


def _sort_by_key(keys, *arrs):
    o = np.argsort(keys, kind="stable")
    return (keys[o],) + tuple(a[o] for a in arrs)


def _small_scene(seed=0, n=3000):
    from paper_2407_09649_gb300 import scenes
    return scenes.sphere_plane_frame(seed, n_sphere=n, n_plane=n)


# ----------------------------------------------------------------------------------
# L-GPDF frame
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("cap", [64, 16])
def test_frame_indexing_and_training_sets_bitexact(vg, orc, cap):
    pts = _small_scene(1)
    P = orc.params(max_pts_leaf=cap)
    ref = orc.frame(pts, P)
    m, f, r, inst = _frame_gpu(vg, pts, precision="fp64", max_pts_leaf=cap)
    lk = inst["leaf_key"]
    o = np.argsort(lk)
    assert np.array_equal(lk[o], ref.leaf_key)
    assert np.array_equal(inst["n_occ"][o], ref.leaf_nocc)
    off = inst["inst_off"]
    for gi, ri in zip(o, range(len(ref.leaf_key))):
        a = inst["X"][off[gi]:off[gi + 1]]
        b = ref.X[ref.inst_off[ri]:ref.inst_off[ri + 1]]
        assert np.array_equal(a, b)
        np.testing.assert_allclose(inst["alpha"][off[gi]:off[gi + 1]], ref.alpha[ref.inst_off[ri]:ref.inst_off[ri + 1]],
                                   rtol=1e-8, atol=1e-9 * np.abs(ref.alpha).max())
    k, st = _sort_by_key(r["keys"], r["status"])
    assert np.array_equal(k, np.sort(ref.test_key))
    assert np.array_equal(st, ref.status[np.argsort(ref.test_key, kind="stable")])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_frame_values(vg, orc, precision):
    pts = _small_scene(2)
    ref = orc.frame(pts, orc.params())
    m, f, r, _ = _frame_gpu(vg, pts, precision=precision)
    k, d, v, g, s = _sort_by_key(r["keys"], r["d"], r["v"], r["grad"], r["status"])
    ro = np.argsort(ref.test_key, kind="stable")
    rd, rv, rg, rs = ref.d[ro], ref.v[ro], ref.grad[ro], ref.status[ro]
    assert np.array_equal(k, ref.test_key[ro])
    ok = rs == 0
    if precision == "fp64":
        assert np.array_equal(s, rs)
        err = np.abs(d[ok] - rd[ok])
        assert err.max() <= D_TOL and np.median(err) < 1e-9
        big = ok & (np.linalg.norm(rg, axis=1) > 0.1)
        assert _angle_deg(g[big], rg[big]).max() <= ANG_TOL_DEG
        np.testing.assert_allclose(v[ok], rv[ok], rtol=1e-5, atol=1e-12)
    else:
        mid = ok & (rd > 2e-3)
        assert np.array_equal(s[mid], rs[mid])
        assert np.abs(d[mid] - rd[mid]).max() <= D_TOL_MIXED
        big = mid & (np.linalg.norm(rg, axis=1) > 0.5)
        assert np.percentile(_angle_deg(g[big], rg[big]), 99) <= 1.0
        _check_mixed_var(v[mid], rv[mid], d[mid], rd[mid])


def test_frame_edge_cases(vg):
    m = vg.Map()
    f = m.build_frame(torch.zeros((0, 3), device="cuda"))
    assert f.n_test == 0
    bad = torch.tensor([[float("nan"), 0, 0], [1e9, 0, 0], [0, float("inf"), 1]], device="cuda")
    f = m.build_frame(bad)
    assert f.n_test == 0
    one = torch.tensor([[0.31, -0.42, 0.05]], device="cuda")
    f = m.build_frame(one)
    r = f.results()
    assert f.n_test == 27 * 512 and int((r["status"] == 0).sum()) == 27 * 512


# ----------------------------------------------------------------------------------
# fusion
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("fusion", ["invvar", "tsdf"])
def test_fusion_parity(vg, orc, fusion):
    mode = 0 if fusion == "invvar" else 1
    P = orc.params(fusion=mode)
    g_ref = orc.Grid(fusion=mode)
    m = vg.Map(precision="fp64", fusion=fusion)
    rng = np.random.default_rng(3)
    base = _small_scene(4, n=1500)
    for t in range(3):
        pts = (base + rng.normal(0, 0.02, base.shape) + np.array([0.05 * t, 0, 0])).astype(np.float32)
        ref = orc.frame(pts, P)
        g_ref.fuse_frame(ref)
        m.fuse(m.build_frame(torch.from_numpy(pts).cuda()))
    k, D, V, fl = m.export_grid()
    rk, rD, rV, rfl = g_ref.export()
    assert np.array_equal(k, rk)
    assert np.array_equal(fl, rfl)
    np.testing.assert_allclose(D, rD, rtol=1e-6, atol=D_TOL * 1e-2)
    np.testing.assert_allclose(V, rV, rtol=1e-5, atol=1e-12)
    # checkpoint / resume round trip is exact
    m2 = vg.Map(precision="fp64", fusion=fusion)
    m2.import_grid(k, D, V, fl)
    k2, D2, V2, fl2 = m2.export_grid()
    assert np.array_equal(k2, k) and np.array_equal(D2, D) and np.array_equal(V2, V) and np.array_equal(fl2, fl)


# ----------------------------------------------------------------------------------
# G-GPDF queries
# ----------------------------------------------------------------------------------
def _query_scene(seed=5):
    from paper_2407_09649_gb300 import scenes
    rng = np.random.default_rng(seed)
    surf = scenes.sphere_plane_frame(seed, n_sphere=6000, n_plane=6000)
    # a dense blob so that some neighbourhoods exceed the 1024 cap
    blob = rng.normal([1.2, -1.5, -1.0], 0.15, (2500, 3)).astype(np.float32)
    surf = np.vstack([surf, blob]).astype(np.float32)
    q = scenes.uniform_queries(seed, n=3000, lo=(-4.5, -4.5, -4.5), hi=(4.5, 4.5, 4.5))
    near = surf[rng.choice(len(surf), 1500)] + rng.normal(0, 0.1, (1500, 3)).astype(np.float32)
    q = np.vstack([q, near, [[np.nan, 0, 0]], [[40.0, 40.0, 40.0]]]).astype(np.float32)
    return surf, q


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_query_parity(vg, orc, precision):
    surf, q = _query_scene()
    S = orc.Surface(surf, orc.params())
    ref = S.query(q, want_var=True)
    assert (ref["inst_n"] == 1024).any()  # the cap selection is exercised
    m = vg.Map(precision=precision)
    m.set_surface(torch.from_numpy(surf).cuda())
    out = m.query(torch.from_numpy(q).cuda(), grad=True, var=True)
    d, g, v, s = (out[k].cpu().numpy() for k in ("d", "grad", "var", "status"))
    rd, rg, rv, rs = ref["d"], ref["grad"], ref["var"], ref["status"]
    ok = rs == 0
    assert s[-2] == 3 and s[-1] == 1
    if precision == "fp64":
        assert np.array_equal(s, rs)
        err = np.abs(d[ok] - rd[ok])
        assert err.max() <= D_TOL and np.median(err) < 1e-9
        big = ok & (np.linalg.norm(rg, axis=1) > 0.1)
        assert _angle_deg(g[big], rg[big]).max() <= ANG_TOL_DEG
        fin = ok & np.isfinite(rv)
        np.testing.assert_allclose(v[fin], rv[fin], rtol=1e-5, atol=1e-12)
    else:
        mid = ok & (rd > 2e-3) & (rd < 9.0)
        assert np.array_equal(s[mid], rs[mid])
        assert np.abs(d[mid] - rd[mid]).max() <= D_TOL_MIXED
        big = mid & (np.linalg.norm(rg, axis=1) > 0.5)
        assert np.percentile(_angle_deg(g[big], rg[big]), 99) <= 1.0
        fin = mid & np.isfinite(rv)
        _check_mixed_var(v[fin], rv[fin], d[fin], rd[fin])


def test_per_instance_launch_matches_oracle(vg, orc):
    """The plain FP64 per-instance comparison form (VGP_LAUNCH_PER_INSTANCE: one launch per GP
    instance, all FP64) meets the FP64 contract against the oracle, and gives the same bits as
    the batched FP64 form (same arithmetic, no batching)."""
    surf, q = _query_scene(11)
    q = q[::2].copy()
    S = orc.Surface(surf, orc.params())
    ref = S.query(q, want_var=True)
    res = {}
    for launch in ("per_instance", "batched"):
        m = vg.Map(precision="fp64", launch=launch)
        m.set_surface(torch.from_numpy(surf).cuda())
        res[launch] = {k: v.cpu().numpy() for k, v in m.query(torch.from_numpy(q).cuda(), grad=True, var=True).items()}
        assert m.stats()["bucket_count"][4] > 0  # instances with N > 256 (A in global memory)
    d, g, v, s = (res["per_instance"][k] for k in ("d", "grad", "var", "status"))
    rd, rg, rv, rs = ref["d"], ref["grad"], ref["var"], ref["status"]
    assert np.array_equal(s, rs)
    ok = rs == 0
    assert np.abs(d[ok] - rd[ok]).max() <= D_TOL
    big = ok & (np.linalg.norm(rg, axis=1) > 0.1)
    assert _angle_deg(g[big], rg[big]).max() <= ANG_TOL_DEG
    fin = ok & np.isfinite(rv)
    np.testing.assert_allclose(v[fin], rv[fin], rtol=1e-5, atol=1e-12)
    for k in ("d", "grad", "var", "status"):
        assert np.array_equal(res["per_instance"][k].view(np.uint8), res["batched"][k].view(np.uint8)), k


def test_query_errors(vg):
    from paper_2407_09649_gb300 import _lib
    m = vg.Map()
    with pytest.raises(_lib.VgpError) as e:
        m.query(torch.zeros((4, 3), device="cuda"))
    assert e.value.code == -6
    with pytest.raises(ValueError):
        m.set_surface(torch.zeros((4, 2), device="cuda"))
    with pytest.raises(_lib.VgpError):
        vg.Map(max_pts_group=2000)


# ----------------------------------------------------------------------------------
# independent instances: every size bucket and the bucket edges
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gp_batch_parity(vg, orc, precision):
    from paper_2407_09649_gb300 import scenes
    inst_off, X, q_off, Q = scenes.patch_sweep(n_inst=40, seed=11, q_per_inst=64)
    # force sizes on the bucket edges
    sizes = [1, 2, 31, 32, 33, 64, 65, 128, 129, 224, 225, 256, 257, 700, 1024]
    rng = np.random.default_rng(12)
    Xs, Qs = [], []
    for N in sizes:
        c = rng.uniform(-20, 20, 3)
        Xs.append(c + rng.uniform(-0.05, 0.05, (N, 3)) * np.sqrt(N))
        Qs.append(c + rng.uniform(-1, 1, (50, 3)))
    X2 = np.vstack([X.astype(np.float64)] + Xs).astype(np.float32)
    Q2 = np.vstack([Q.astype(np.float64)] + Qs).astype(np.float32)
    io2 = np.concatenate([inst_off, inst_off[-1] + np.cumsum(sizes)])
    qo2 = np.concatenate([q_off, q_off[-1] + 50 * np.arange(1, len(sizes) + 1)])
    ref = orc.gp_batch(io2, X2.astype(np.float64), qo2, Q2.astype(np.float64), orc.params())
    m = vg.Map(precision=precision)
    out = m.gp_batch(io2, X2, qo2, Q2, var=True)
    d, g, v, s = (out[k].cpu().numpy() for k in ("d", "grad", "var", "status"))
    ok = ref.status == 0
    if precision == "fp64":
        assert np.array_equal(s, ref.status)
        assert np.abs(d[ok] - ref.d[ok]).max() <= D_TOL
        big = ok & (np.linalg.norm(ref.grad, axis=1) > 0.1)
        assert _angle_deg(g[big], ref.grad[big]).max() <= ANG_TOL_DEG
        fin = ok & np.isfinite(ref.var)
        np.testing.assert_allclose(v[fin], ref.var[fin], rtol=1e-5, atol=1e-12)
    else:
        mid = ok & (ref.d > 2e-3) & (ref.d < 9.0)
        assert np.abs(d[mid] - ref.d[mid]).max() <= D_TOL_MIXED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bordered_variance_chunks(vg, orc, precision):
    """Latent variance of N > 32 instances with the emulated updates: the instance's queries are
    appended to its matrix as rows (up to 1024 per factorisation) and u is read from the Schur
    complement's diagonal (Eq. 2).  Instances of 40 to 1024 points with 1 to 700 queries, a
    non-finite query among them and queries far from the points (u near 1): the variance
    agrees with the oracle (FP64 contract) and with the per-query triangular solve of the FP64
    tensor path, and each query's bits do not depend on the other queries (the last 100
    queries of the largest instance alone, in reverse order, give the same bits)."""
    rng = np.random.default_rng(31)
    sizes = [225, 250, 600, 1000, 1024, 70, 150, 40]
    nqs = [1, 255, 256, 257, 700, 40, 600, 300]
    Xs, Qs = [], []
    for N, nq in zip(sizes, nqs):
        c = rng.uniform(-20, 20, 3)
        Xs.append(c + rng.uniform(-0.05, 0.05, (N, 3)) * np.sqrt(N))
        q = c + rng.uniform(-1, 1, (nq, 3))
        if nq > 100:
            q[7] = np.nan
            q[11] = c + 40.0  # no kernel value above underflow: u = 1
        Qs.append(q)
    X = np.vstack(Xs).astype(np.float32)
    Q = np.vstack(Qs).astype(np.float32)
    io = np.concatenate([[0], np.cumsum(sizes)])
    qo = np.concatenate([[0], np.cumsum(nqs)])
    ref = orc.gp_batch(io, X.astype(np.float64), qo, Q.astype(np.float64), orc.params())
    out = {}
    for emu in (1, 0):
        m = vg.Map(precision=precision, emulate_fp64=emu)
        out[emu] = {k: v.cpu().numpy() for k, v in m.gp_batch(io, X, qo, Q, var=True).items()}
        assert sum(m.stats()["bucket_count"][1:]) == len(sizes)  # N > 32: the emulated kernel
    d, v, s = out[1]["d"], out[1]["var"], out[1]["status"]
    assert np.array_equal(s, ref.status)
    assert s[qo[3] + 7] == 3 and s[qo[4] + 7] == 3  # bad input
    ok = ref.status == 0
    fin = ok & np.isfinite(ref.var) & (ref.var > 0)
    assert fin.sum() > 1000
    if precision == "fp64":
        np.testing.assert_allclose(v[fin], ref.var[fin], rtol=1e-5, atol=1e-12)
        # the per-query solve (FP64 tensor path) to rounding
        np.testing.assert_allclose(v[fin], out[0]["var"][fin], rtol=1e-8, atol=0)
    else:
        bound = 2.0 * np.abs(d[fin] - ref.d[fin]) / np.maximum(ref.d[fin], 1e-3) * 1.5 + 2e-3
        assert np.all(np.abs(v[fin] - ref.var[fin]) / ref.var[fin] <= bound)
    # the last instance's last 100 queries alone, reversed: the same bits per query
    sub = Q[qo[4]:qo[5]][-100:][::-1].copy()
    m = vg.Map(precision=precision, emulate_fp64=1)
    r2 = {k: v.cpu().numpy()
          for k, v in m.gp_batch(np.array([0, sizes[4]]), X[io[4]:io[5]], np.array([0, 100]), sub, var=True).items()}
    for k in ("d", "grad", "var", "status"):
        a = np.ascontiguousarray(out[1][k][qo[5] - 100:qo[5]][::-1])
        assert np.array_equal(np.ascontiguousarray(r2[k]).view(np.uint8), a.view(np.uint8)), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_chunked_queries_bit_identical(vg, orc, precision):
    """Few instances with many queries (3000 each, N from 20 to 400): the launch splits each
    instance's queries into chunks that fit the instance again, so that the queries spread over
    the GPU.  Every query's distance, gradient, variance and status are bit-identical to the
    same query answered with 40 queries per instance (not split) and to graph launches (which
    plan the chunks on the device), and agree with the oracle."""
    rng = np.random.default_rng(41)
    sizes = [20, 60, 100, 180, 400]
    nq = 3000
    Xs, Qs = [], []
    for N in sizes:
        c = rng.uniform(-20, 20, 3)
        Xs.append(c + rng.uniform(-0.05, 0.05, (N, 3)) * np.sqrt(N))
        Qs.append(c + rng.uniform(-1, 1, (nq, 3)))
    X = np.vstack(Xs).astype(np.float32)
    Q = np.vstack(Qs).astype(np.float32)
    io = np.concatenate([[0], np.cumsum(sizes)])
    qo = np.arange(len(sizes) + 1) * nq
    m = vg.Map(precision=precision, emulate_fp64=1)
    full = {k: v.cpu().numpy() for k, v in m.gp_batch(io, X, qo, Q, var=True).items()}
    pick = np.concatenate([i * nq + np.sort(rng.choice(nq, 40, replace=False)) for i in range(len(sizes))])
    sub = {k: v.cpu().numpy() for k, v in m.gp_batch(io, X, np.arange(len(sizes) + 1) * 40, Q[pick], var=True).items()}
    for k in ("d", "grad", "var", "status"):
        assert np.array_equal(np.ascontiguousarray(full[k][pick]).view(np.uint8), np.ascontiguousarray(sub[k]).view(np.uint8)), k
    # graph launches plan the chunks on the device: the same bits
    mg = vg.Map(precision=precision, emulate_fp64=1, launch="graph")
    gr = {k: v.cpu().numpy() for k, v in mg.gp_batch(io, X, qo, Q, var=True).items()}
    for k in ("d", "grad", "var", "status"):
        assert np.array_equal(np.ascontiguousarray(gr[k]).view(np.uint8), np.ascontiguousarray(full[k]).view(np.uint8)), k
    ref = orc.gp_batch(io, X.astype(np.float64), np.arange(len(sizes) + 1) * 40, Q[pick].astype(np.float64), orc.params())
    assert np.array_equal(sub["status"], ref.status)
    ok = (ref.status == 0) & (ref.d > 2e-3) & (ref.d < 9.0)
    assert ok.sum() > 100
    assert np.abs(sub["d"][ok] - ref.d[ok]).max() <= (D_TOL if precision == "fp64" else D_TOL_MIXED)
    fin = ok & np.isfinite(ref.var) & (ref.var > 0)
    if precision == "fp64":
        np.testing.assert_allclose(sub["var"][fin], ref.var[fin], rtol=1e-5, atol=1e-12)


def test_gp_batch_rejects_oversize(vg):
    from paper_2407_09649_gb300 import _lib
    m = vg.Map()
    X = np.zeros((1025, 3), np.float32)
    with pytest.raises(_lib.VgpError) as e:
        m.gp_batch([0, 1025], X, [0, 1], np.zeros((1, 3), np.float32))
    assert e.value.code == -1


# ----------------------------------------------------------------------------------
# backward
# ----------------------------------------------------------------------------------
def test_backward_parity(vg, orc):
    rng = np.random.default_rng(21)
    g = (np.arange(30) - 14.5) * 0.1
    surf = np.array([[x, y, 0.1 * np.sin(2 * x) * np.cos(y)] for x in g for y in g])
    surf = (surf + rng.normal(0, 0.01, surf.shape)).astype(np.float32)
    q = rng.uniform([-1.2, -1.2, 0.05], [1.2, 1.2, 0.9], (400, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, len(q))
    S = orc.Surface(surf, orc.params())
    rdq, rdX = S.backward(q, w)
    m = vg.Map(precision="fp64")
    m.set_surface(torch.from_numpy(surf).cuda())
    dq, dX = m.query_backward(torch.from_numpy(q).cuda(), torch.from_numpy(w).cuda())
    dq, dX = dq.cpu().numpy(), dX.cpu().numpy()
    np.testing.assert_allclose(dq, rdq, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(dX, rdX, rtol=1e-6, atol=1e-8 * np.abs(rdX).max())


def test_autograd_function(vg, orc):
    from paper_2407_09649_gb300.autograd import gpdf_distance
    rng = np.random.default_rng(22)
    g = (np.arange(20) - 9.5) * 0.1
    surf = np.array([[x, y, 0.0] for x in g for y in g]) + rng.normal(0, 0.01, (400, 3))
    surf = torch.tensor(surf, dtype=torch.float32, device="cuda", requires_grad=True)
    q = torch.tensor(rng.uniform([-0.7, -0.7, 0.1], [0.7, 0.7, 0.8], (64, 3)), dtype=torch.float32,
                     device="cuda", requires_grad=True)
    m = vg.Map(precision="fp64")
    d = gpdf_distance(q, surf, m)
    loss = torch.nn.functional.softplus(0.5 - d).sum()
    loss.backward()
    w = (-torch.sigmoid(0.5 - d)).detach().double().cpu().numpy()
    S = orc.Surface(surf.detach().cpu().numpy(), orc.params())
    rdq, rdX = S.backward(q.detach().cpu().numpy(), w)
    np.testing.assert_allclose(q.grad.cpu().numpy(), rdq, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(surf.grad.cpu().numpy(), rdX, rtol=1e-4, atol=1e-6)


def test_table_exp_matches_libm(vg):
    """The FP64 table-driven exponential used for kernel-matrix entries (mixed path) stays
    within 2 ulp of the host libm over the range the kernel uses."""
    import ctypes as C
    from paper_2407_09649_gb300 import _lib
    m = vg.Map()
    rng = np.random.default_rng(0)
    y = np.concatenate([-rng.uniform(0, 40, 200000), -rng.uniform(0, 700, 50000), [0.0, -1e-300, -699.9],
                        -np.arange(0, 50, 1 / 256.0)])
    yt = torch.from_numpy(y).cuda()
    out = torch.empty_like(yt)
    _lib.check(_lib.load().vgp_debug_exp_neg(m._h, C.c_void_p(yt.data_ptr()), C.c_void_p(out.data_ptr()), len(y),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    got = out.cpu().numpy()
    ref = np.exp(y)
    ulp = np.spacing(ref)
    assert np.max(np.abs(got - ref) / ulp) <= 2.0
    assert got[np.flatnonzero(y == 0.0)[0]] == 1.0  # e^0 exactly
    big = out.new_tensor([-800.0, -701.0])
    r = torch.empty_like(big)
    _lib.check(_lib.load().vgp_debug_exp_neg(m._h, C.c_void_p(big.data_ptr()), C.c_void_p(r.data_ptr()), 2,
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    assert r.cpu().tolist() == [0.0, 0.0]


def test_float_pair_kernel_values(vg):
    """Mixed-precision kernel values of the emulated factorisation (float-pair arithmetic on the
    FP32 pipe, fixed point round(k 2^61)) against exp(-r^2 / (2 l^2)) in extended precision, for
    FP32 world coordinates 100 m from the origin and distances from 0 to beyond the fixed
    point's range: error below 2^-45 k (1 + y) + 2 units (y = r^2 / (2 l^2)), 2^-46 at most in
    absolute terms, exact 2^61 for coincident points, 0 where k < 2^-63, symmetric bit for bit."""
    import ctypes as C
    from paper_2407_09649_gb300 import _lib
    m = vg.Map(precision="mixed", emulate_fp64=1)
    rng = np.random.default_rng(3)
    n = 400000
    xa = (np.array([103.7, -45.3, 12.9]) + rng.uniform(-1.5, 1.5, (n, 3))).astype(np.float32)
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.concatenate([rng.uniform(0, 2.0, n // 2), rng.uniform(0, 0.3, n // 4), 10.0 ** rng.uniform(-6, -1, n // 4)])
    xb = (xa + dirs * r[:, None]).astype(np.float32)
    xb[:100] = xa[:100]  # coincident
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def run(a, b):
        ta, tb = torch.from_numpy(np.ascontiguousarray(a)).cuda(), torch.from_numpy(np.ascontiguousarray(b)).cuda()
        out = torch.empty(len(a), dtype=torch.int64, device="cuda")
        _lib.check(_lib.load().vgp_debug_kernel_fix(m._h, C.c_void_p(ta.data_ptr()), C.c_void_p(tb.data_ptr()),
                                                    len(a), C.c_void_p(out.data_ptr()), st))
        return out.cpu().numpy()

    got = run(xa, xb)
    assert np.array_equal(got, run(xb, xa))  # symmetric
    assert np.all(got[:100] == 2**61)
    L = np.longdouble
    y = np.sum((xa.astype(L) - xb.astype(L)) ** 2, axis=1) / (2 * L(0.3) * L(0.3))
    exact = np.exp(-y) * L(2.0) ** 61
    err = np.abs(got.astype(L) - exact)
    assert np.all(err <= exact * (1 + y) * L(2.0) ** -45 + 2), float(np.max((err - 2) / (exact * (1 + y))))
    assert float(err.max()) <= 2.0 ** (61 - 46)
    assert np.all(got[exact < 0.125] == 0)
    big = exact > 2.0 ** 51
    print("kernel-value error relative to k (median, max over k > 2^-10):", float(np.median(err[big] / exact[big])),
          float(np.max(err[big] / exact[big])))


# ----------------------------------------------------------------------------------
# G-GPDF as blended per-leaf GPs (Eq. 10)
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_query_smooth_parity(vg, orc, precision):
    surf, q = _query_scene(9)
    P = orc.params(max_pts_leaf=128)
    S = orc.Surface(surf, P)
    for n_nodes, lam in ((8, 100.0), (3, 20.0)):
        ref = S.query_smooth(q, n_nodes=n_nodes, lam=lam, want_var=True)
        m = vg.Map(precision=precision, max_pts_leaf=128)
        m.set_surface(torch.from_numpy(surf).cuda())
        out = m.query_smooth(torch.from_numpy(q).cuda(), n_nodes=n_nodes, lam=lam, grad=True, var=True)
        d, g, v, s = (out[k].cpu().numpy() for k in ("d", "grad", "var", "status"))
        ok = ref["status"] == 0
        assert s[-2] == 3 and s[-1] == 1
        if precision == "fp64":
            assert np.array_equal(s, ref["status"])
            assert np.abs(d[ok] - ref["d"][ok]).max() <= D_TOL
            big = ok & (np.linalg.norm(ref["grad"], axis=1) > 0.1)
            assert _angle_deg(g[big], ref["grad"][big]).max() <= ANG_TOL_DEG
            fin = ok & np.isfinite(ref["var"])
            np.testing.assert_allclose(v[fin], ref["var"][fin], rtol=1e-5, atol=1e-12)
        else:
            mid = ok & (ref["d"] > 2e-3) & (ref["d"] < 9.0)
            assert np.array_equal(s[mid], ref["status"][mid])
            assert np.abs(d[mid] - ref["d"][mid]).max() <= D_TOL_MIXED


def test_autotune_keeps_results(vg):
    surf, q = _query_scene(10)
    m = vg.Map(precision="fp64")
    m.set_surface(torch.from_numpy(surf).cuda())
    qt = torch.from_numpy(q).cuda()
    a = m.query(qt, grad=True)["d"].cpu().numpy()
    cfg = m.autotune(qt)
    assert len(cfg["threads"]) == 5 and all(t % 32 == 0 for t in cfg["threads"])
    b = m.query(qt, grad=True)["d"].cpu().numpy()
    fin = np.isfinite(a)
    np.testing.assert_allclose(b[fin], a[fin], rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------------
# ray-cast testing points with signed distances (Sec. IV-B)
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_raycast_frames_and_fusion(vg, orc, precision):
    """Four frames of the room sequence, built with the sensor origin and fused in turn: the
    testing-voxel set (including the ray voxels that depend on the grid fused so far), the
    signs and statuses match the oracle bit for bit, the values within tolerance, and the
    fused grids agree after every frame."""
    from paper_2407_09649_gb300 import scenes
    room = scenes.Room(0)
    P = orc.params(max_pts_leaf=512)
    g_ref = orc.Grid()
    m = vg.Map(precision=precision, max_pts_leaf=512)
    tol = D_TOL if precision == "fp64" else D_TOL_MIXED
    for k in range(4):
        pts = room.frame(3 * k, seed=0)[::4]
        origin, *_ = room.camera_pose(3 * k)
        known = g_ref.export()[0]
        ref = orc.frame(pts, P, origin=origin, normal_steps=3, known=known)
        f = m.build_frame(torch.from_numpy(pts).cuda(), origin=origin)
        r = {kk: v.cpu().numpy() for kk, v in f.results().items()}
        o = np.argsort(r["keys"], kind="stable")
        ro = np.argsort(ref.test_key, kind="stable")
        assert np.array_equal(r["keys"][o], ref.test_key[ro])
        assert np.array_equal(r["status"][o], ref.status[ro])
        ok = ref.status[ro] == 0
        rd, d = ref.d[ro], r["d"][o]
        if precision == "fp64":
            assert np.abs(d[ok] - rd[ok]).max() <= tol
        else:
            mid = ok & (np.abs(rd) > 2e-3)
            assert np.abs(d[mid] - rd[mid]).max() <= tol
        sg = ref.sign[ro]
        nz = ok & (np.abs(rd) > 1e-6)
        assert np.array_equal(np.sign(d[nz]), sg[nz].astype(np.float64))
        g_ref.fuse_frame(ref)
        m.fuse(f)
        k1, D1, V1, fl1 = m.export_grid()
        k2, D2, V2, fl2 = g_ref.export()
        assert np.array_equal(k1, k2) and np.array_equal(fl1, fl2)
        err = np.abs(D1 - D2)
        if precision == "fp64":
            assert err.max() <= tol
        else:
            # Fused values are averages weighted by the inferred variances (Eq. 8); in mixed
            # precision those carry ~1e-3 relative error, which moves an average by that fraction
            # of the spread between the fused frames' distances.
            assert np.mean(err <= tol) >= 0.999 and err.max() <= 5 * tol


def test_launch_shapes_give_identical_results(vg):
    """Large neighbourhoods (N up to 1024, A in global memory): every launch shape of the
    solve, with the panel staged in shared memory or read through L1/L2 with two CTAs per SM,
    gives bit-identical distances, gradients and variances."""
    rng = np.random.default_rng(8)
    u = rng.normal(size=(150000, 3))
    surf = (1.3 * u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    q = (surf[rng.integers(0, len(surf), 20000)] * rng.uniform(0.6, 1.4, (20000, 1))).astype(np.float32)
    m = vg.Map(precision="mixed")
    m.set_surface(torch.from_numpy(surf).cuda())
    qt = torch.from_numpy(q).cuda()
    ref = {k: v.cpu().numpy() for k, v in m.query(qt, grad=True, var=True).items()}
    assert m.stats()["bucket_count"][4] > 50  # instances with N > 256
    for threads, per_sm, stage in [((384, 512, 256, 128, 64), (2, 0, 0, 0, 0), 0),
                                   ((256, 256, 128, 64, 32), (2, 0, 0, 0, 0), 0),
                                   ((256, 512, 256, 128, 64), (3, 0, 0, 0, 0), 0),
                                   ((512, 512, 256, 128, 64), (1, 0, 0, 0, 0), 1)]:
        m.set_launch(threads, per_sm, stage)
        out = {k: v.cpu().numpy() for k, v in m.query(qt, grad=True, var=True).items()}
        for k in ("d", "grad", "var", "status"):
            assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k


@pytest.mark.parametrize("emulate", [0, 1])
def test_graph_launch_mode_matches_direct(vg, emulate):
    """VGP_LAUNCH_GRAPH (device-planned buckets, the solve replayed as a CUDA graph) gives
    bit-identical frames (with surface properties), fused grids and G-GPDF queries to the
    direct batched launches, and updates its executable graph in place between calls; with
    emulate_fp64 = 1 the N > 224 buckets (leaves of 225..256 points, neighbourhoods up to 1024)
    run the emulated factorisation in both modes."""
    from paper_2407_09649_gb300 import scenes
    room = scenes.Room(0)
    frames = [torch.from_numpy(room.frame(k, seed=0)[::2]).cuda() for k in range(4)]
    props = [torch.rand((f.shape[0], 2), device="cuda", generator=torch.Generator("cuda").manual_seed(k))
             for k, f in enumerate(frames)]
    for precision in ("mixed", "fp64"):
        maps = {mode: vg.Map(precision=precision, max_pts_leaf=256, n_props=2, launch=mode, emulate_fp64=emulate)
                for mode in ("batched", "graph")}
        res = {}
        for mode, m in maps.items():
            out = []
            for k, (f, p) in enumerate(zip(frames, props)):
                fr = m.build_frame(f, origin=room.camera_pose(k)[0], props=p)
                r = {kk: v.cpu().numpy() for kk, v in fr.results().items()}
                c, w = (t.cpu().numpy() for t in fr.props())
                o = np.argsort(r["keys"])  # result order is unspecified; keys are unique
                out.append(({kk: v[o] for kk, v in r.items()}, c[o], w[o]))
                m.fuse(fr)
            m.update_surface()
            ss = room.surface_samples(seed=3)
            rng = np.random.default_rng(3)
            q = torch.from_numpy((ss[rng.integers(0, len(ss), 20000)]
                                  + rng.normal(0, 0.2, (20000, 3))).astype(np.float32)).cuda()
            qo = {kk: v.cpu().numpy() for kk, v in m.query(q, grad=True, var=True).items()}
            big = m.stats()["bucket_count"][4]
            so = {kk: v.cpu().numpy() for kk, v in m.query_smooth(q, n_nodes=8, var=True).items()}
            res[mode] = (out, m.export_grid(), qo, so, m.stats(), big)
        a, b = res["batched"], res["graph"]
        for (ra, ca, wa), (rb, cb, wb) in zip(a[0], b[0]):
            for k in ("keys", "d", "v", "grad", "status"):
                assert np.array_equal(ra[k].view(np.uint8), rb[k].view(np.uint8)), k
            assert np.array_equal(ca.view(np.uint8), cb.view(np.uint8))
            assert np.array_equal(wa.view(np.uint8), wb.view(np.uint8))
        for x, y in zip(a[1], b[1]):
            assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))
        for k in ("d", "grad", "var", "status"):
            assert np.array_equal(a[2][k].view(np.uint8), b[2][k].view(np.uint8)), k
            assert np.array_equal(a[3][k].view(np.uint8), b[3][k].view(np.uint8)), k
        st = b[4]
        assert st["graph_replays"] >= 10 and st["graph_instantiations"] <= 4
        assert b[5] > 0  # the G-GPDF query solved instances with N > 256


def test_results_repeatable_across_calls_maps_and_launch_modes(vg, orc):
    """Results depend on nothing but the inputs: on the sphere surface with 20k queries, whose
    densest leaves hold more than 4096 points (their point lists are sorted in global memory
    by the surface binning, so every instance lists its points in index order), two calls of
    one map, a call on a subset of the queries, a second map with its own surface binning and
    a graph-mode map give bit-identical distances, gradients, variances and statuses, with the
    emulated FP64-accurate updates and without."""
    rng = np.random.default_rng(8)
    u = rng.normal(size=(150000, 3))
    surf = (1.3 * u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    q = (surf[rng.integers(0, len(surf), 20000)] * rng.uniform(0.6, 1.4, (20000, 1))).astype(np.float32)
    assert np.unique(orc.leaf_key_of_points(surf, 0.1), return_counts=True)[1].max() > 4096
    qt = torch.from_numpy(q).cuda()
    st = torch.from_numpy(surf).cuda()
    keys = ("d", "grad", "var", "status")
    for precision in ("mixed", "fp64"):
        for emu in (1, 0):
            def run(m, qq=qt):
                return {k: v.cpu().numpy() for k, v in m.query(qq, grad=True, var=True).items()}
            m = vg.Map(precision=precision, emulate_fp64=emu)
            m.set_surface(st)
            ref = run(m)
            assert m.stats()["bucket_count"][4] > 50
            other = {"second call": run(m)}
            sub = run(m, qt[7000:12000])
            m2 = vg.Map(precision=precision, emulate_fp64=emu)
            m2.set_surface(st)
            other["second map"] = run(m2)
            mg = vg.Map(precision=precision, emulate_fp64=emu, launch="graph")
            mg.set_surface(st)
            other["graph mode"] = run(mg)
            for name, r in other.items():
                for k in keys:
                    assert np.array_equal(r[k].view(np.uint8), ref[k].view(np.uint8)), (precision, emu, name, k)
            for k in keys:
                assert np.array_equal(sub[k].view(np.uint8), ref[k][7000:12000].view(np.uint8)), (precision, emu, k)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_emulated_trailing_updates(vg, orc, precision):
    """emulate_fp64 = 1 (trailing updates of N > 224 instances on the bf16 tensor cores with
    exact slice products) agrees with the FP64 tensor path to rounding on large
    neighbourhoods and on full L-GPDF leaves, and the FP64 map stays within the FP64 contract
    against the oracle.  In mixed precision the gradient is an FP32 sum whose own error
    (well inside the mixed tolerance) follows last-bit changes of alpha, so it is compared at
    that scale."""
    rng = np.random.default_rng(8)
    u = rng.normal(size=(150000, 3))
    surf = (1.3 * u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    q = (surf[rng.integers(0, len(surf), 20000)] * rng.uniform(0.6, 1.4, (20000, 1))).astype(np.float32)
    qt = torch.from_numpy(q).cuda()
    out = {}
    for emu in (0, 1):
        m = vg.Map(precision=precision, emulate_fp64=emu)
        m.set_surface(torch.from_numpy(surf).cuda())
        out[emu] = {k: v.cpu().numpy() for k, v in m.query(qt, grad=True, var=True).items()}
        assert m.stats()["bucket_count"][4] > 50
    a, b = out[0], out[1]
    assert np.array_equal(a["status"], b["status"])
    ok = a["status"] == 0
    g_tol = 1e-5 if precision == "fp64" else 5e-3
    assert np.abs(a["d"][ok] - b["d"][ok]).max() <= (1e-7 if precision == "fp64" else 1e-5)
    assert np.abs(a["grad"][ok] - b["grad"][ok]).max() <= g_tol
    fin = ok & np.isfinite(a["var"]) & (a["var"] > 1e-12)
    assert np.median(np.abs(a["var"][fin] - b["var"][fin]) / a["var"][fin]) <= 1e-6
    if precision == "fp64":
        sel = rng.choice(np.flatnonzero(ok), 300, replace=False)
        ref = orc.Surface(surf, orc.params()).query(q[sel], want_var=False)
        assert np.array_equal(ref["status"], b["status"][sel])
        assert np.abs(b["d"][sel] - ref["d"]).max() <= D_TOL
    # full L-GPDF leaves: a volume, every leaf holds 512 occupied voxels
    pts = torch.from_numpy(rng.uniform(0.0, 2.4, (200000, 3)).astype(np.float32)).cuda()
    fr = {}
    for emu in (0, 1):
        m = vg.Map(precision=precision, max_pts_leaf=512, emulate_fp64=emu)
        f = m.build_frame(pts)
        assert m.stats()["bucket_count"][4] >= 27
        r = {k: v.cpu().numpy() for k, v in f.results().items()}
        o = np.argsort(r["keys"])
        fr[emu] = {k: v[o] for k, v in r.items()}
    assert np.array_equal(fr[0]["keys"], fr[1]["keys"]) and np.array_equal(fr[0]["status"], fr[1]["status"])
    ok = fr[0]["status"] == 0
    assert np.abs(fr[0]["d"][ok] - fr[1]["d"][ok]).max() <= (1e-7 if precision == "fp64" else 1e-5)
    # the testing voxels' variance: per-voxel solve (plain) against the bordered factorisation
    # of the lattice instances (emulated)
    fin = ok & np.isfinite(fr[0]["v"]) & (fr[0]["v"] > 0)
    rel = np.abs(fr[1]["v"][fin] - fr[0]["v"][fin]) / fr[0]["v"][fin]
    assert fin.sum() > 1000 and np.median(rel) <= 1e-6
    assert rel.max() <= (1e-5 if precision == "fp64" else 1e-2)
