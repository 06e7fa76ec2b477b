"""Pins for the oracle's zero crossings and marching cubes over the fused grid (Sec. IV-D).

The grid values are set directly (a first fusion with v = 1 stores D = d, Eq. 8), so each
pin controls D exactly: a linear field (crossings on the plane), a sphere's signed distance
(a closed genus-0 mesh), and every one of the 256 sign patterns of a cell (closed, outward
oriented surfaces)."""
from collections import Counter

import numpy as np
import pytest

VS = 0.1


def _grid(orc, ijk, D):
    g = orc.Grid()
    n = len(D)
    g.fuse(orc.pack_key(ijk), np.asarray(D, np.float64), np.ones(n), np.zeros(n, np.uint8))
    return g


def _box(lo, hi):
    r = [np.arange(lo[a], hi[a]) for a in range(3)]
    return np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)


def _edge_id(key, axis):
    return (int(key), int(axis))


def _directed_edges(ek, ea):
    E = Counter()
    for t in range(len(ek)):
        v = [_edge_id(ek[t, j], ea[t, j]) for j in range(3)]
        for j in range(3):
            E[(v[j], v[(j + 1) % 3])] += 1
    return E


def _closed_and_consistent(ek, ea):
    """Every directed mesh edge appears once and its reverse once: a closed, consistently
    oriented surface."""
    E = _directed_edges(ek, ea)
    return all(m == 1 and E.get((b, a), 0) == 1 for (a, b), m in E.items())


def _volume(xyz):
    """Signed volume enclosed by a closed triangle mesh (divergence theorem)."""
    return float(np.einsum("ij,ij->i", xyz[:, 0], np.cross(xyz[:, 1], xyz[:, 2])).sum() / 6.0)


def test_plane_crossings_closed_form_and_brute_force_count(orc):
    """Linear D = n.x - c: every crossing lies on the plane (linear interpolation is exact
    for a linear field), and there is exactly one crossing per sign-changing axis edge,
    counted by brute force over the dense box."""
    rng = np.random.default_rng(3)
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    lo, hi = np.array([-13, -9, -11]), np.array([11, 14, 12])
    ijk = _box(lo, hi)
    c = 0.0371
    D = (ijk * VS) @ nrm - c
    g = _grid(orc, ijk, D)
    xyz, owner, slot = g.crossings(VS)
    assert len(xyz) > 100
    # on the plane up to float32 rounding of the coordinates
    res = np.abs(xyz.astype(np.float64) @ nrm - c)
    assert np.all(res <= (np.abs(xyz.astype(np.float64)) @ np.abs(nrm)) * 2.0 ** -24 + 1e-15)
    # brute-force edge count over the dense array
    Dd = D.reshape(*(hi - lo))
    ins = Dd < 0
    cnt = (ins[1:] != ins[:-1]).sum() + (ins[:, 1:] != ins[:, :-1]).sum() + (ins[:, :, 1:] != ins[:, :, :-1]).sum()
    assert len(xyz) == cnt
    # each crossing is owned by the edge end whose voxel holds its float32 point
    o = orc.unpack_key(owner)
    axis = slot // 2
    p = xyz.astype(np.float64)
    assert np.array_equal(np.floor(p / VS + 0.5).astype(np.int64), o)
    for a in range(3):
        off = np.abs(p[:, a] - o[:, a] * VS)
        assert np.all(xyz[axis != a, a] == (o[axis != a, a] * VS).astype(np.float32))
        assert np.all(off[axis == a] <= 0.5 * VS * (1 + 1e-6))
    # one crossing per edge
    lower = o.copy()
    minus = (slot % 2) == 0
    lower[minus, axis[minus]] -= 1
    ids = set(zip(orc.pack_key(lower).tolist(), axis.tolist()))
    assert len(ids) == len(xyz)


def test_sphere_mesh_closed_genus0_outward(orc):
    """Signed distance of a sphere inside the box: a closed mesh with Euler characteristic
    2, normals pointing to increasing D, vertices within the interpolation error of the
    sphere, and every zero crossing used as a mesh vertex."""
    R, c = 0.63, np.array([0.013, 0.021, -0.017])
    ijk = _box([-10, -10, -10], [11, 11, 11])
    D = np.linalg.norm(ijk * VS - c, axis=1) - R
    g = _grid(orc, ijk, D)
    xyz, ek, ea = g.mesh(VS)
    assert _closed_and_consistent(ek, ea)
    V = {_edge_id(ek[t, j], ea[t, j]) for t in range(len(ek)) for j in range(3)}
    E = len(_directed_edges(ek, ea)) // 2
    assert len(V) - E + len(ek) == 2
    nrm = np.cross(xyz[:, 1] - xyz[:, 0], xyz[:, 2] - xyz[:, 0])
    assert np.all(np.einsum("ij,ij->i", nrm, xyz.mean(1) - c) > 0)
    r = np.linalg.norm(xyz.reshape(-1, 3) - c, axis=1)
    assert np.abs(r - R).max() <= VS * VS / R
    assert 0.9 * (4 / 3) * np.pi * R ** 3 < _volume(xyz) < (4 / 3) * np.pi * R ** 3
    cx, owner, slot = g.crossings(VS)
    o = orc.unpack_key(owner)
    axis = slot // 2
    minus = (slot % 2) == 0
    o[minus, axis[minus]] -= 1
    assert set(zip(orc.pack_key(o).tolist(), axis.tolist())) == V


@pytest.mark.parametrize("case", range(256))
def test_every_cell_case_closed_and_outward(orc, case):
    """One cell with corner signs from `case` inside an all-outside shell: the mesh is
    closed and consistently oriented, encloses a positive volume, and that volume lies
    within the voxels of the inside corners (crossings at edge midpoints)."""
    ijk = _box([0, 0, 0], [4, 4, 4])
    D = np.full(len(ijk), 0.5)
    inside = 0
    for k in range(8):
        if (case >> k) & 1:
            w = np.array([1 + (k & 1), 1 + ((k >> 1) & 1), 1 + ((k >> 2) & 1)])
            D[np.all(ijk == w, axis=1)] = -0.5
            inside += 1
    g = _grid(orc, ijk, D)
    xyz, ek, ea = g.mesh(VS)
    if inside == 0:
        assert len(xyz) == 0
        return
    assert _closed_and_consistent(ek, ea)
    vol = _volume(xyz)
    assert 0 < vol <= inside * VS ** 3 * (1 + 1e-9)


def test_ambiguous_face_keeps_diagonal_inside_corners_apart(orc):
    """Two inside corners that share only a face diagonal get two separate triangles; the
    complementary pattern (two outside corners on a diagonal) gets one joined surface."""
    def cell(mask, sign):
        ijk = _box([0, 0, 0], [2, 2, 2])
        D = np.array([sign * (-0.5 if (mask >> (x + 2 * y + 4 * z)) & 1 else 0.5) for x, y, z in ijk])
        return _grid(orc, ijk, D).mesh(VS)

    xyz, ek, ea = cell(0b00001001, 1.0)  # corners 0 and 3 inside
    assert len(xyz) == 2
    a = {_edge_id(ek[0, j], ea[0, j]) for j in range(3)}
    b = {_edge_id(ek[1, j], ea[1, j]) for j in range(3)}
    assert not (a & b)
    xyz, ek, ea = cell(0b00001001, -1.0)  # corners 0 and 3 outside
    assert len(xyz) == 4
    verts = [{_edge_id(ek[t, j], ea[t, j]) for j in range(3)} for t in range(4)]
    # one connected polygon fan: every triangle shares an edge-vertex with another
    assert all(any(verts[t] & verts[u] for u in range(4) if u != t) for t in range(4))


def test_random_interior_signs_give_closed_surfaces(orc):
    """Random inside/outside voxels in a 7^3 block inside an outside shell: every ambiguous
    face is resolved the same way from both cells, so the mesh is closed."""
    rng = np.random.default_rng(11)
    ijk = _box([-4, -4, -4], [5, 5, 5])
    D = rng.uniform(0.05, 1.0, len(ijk))
    interior = np.all(np.abs(ijk) <= 3, axis=1)
    flip = interior & (rng.random(len(ijk)) < 0.45)
    D[flip] *= -1
    xyz, ek, ea = _grid(orc, ijk, D).mesh(VS)
    assert len(xyz) > 200
    assert _closed_and_consistent(ek, ea)
    assert _volume(xyz) > 0


def test_active_only_selects_latest_fusion_leaves(orc):
    """Crossings of the leaves touched by the latest fusion are exactly the all-leaf
    crossings whose owner voxel lies in one of those leaves."""
    R, c = 0.63, np.array([0.013, 0.021, -0.017])
    ijk = _box([-10, -10, -10], [11, 11, 11])
    D = np.linalg.norm(ijk * VS - c, axis=1) - R
    g = _grid(orc, ijk, D)
    sel = ijk[:, 0] >= 3  # a second fusion touching only leaves with x >= 0
    n = int(sel.sum())
    g.fuse(orc.pack_key(ijk[sel]), D[sel], np.ones(n), np.zeros(n, np.uint8))
    allx, allo, alls = g.crossings(VS)
    actx, acto, acts = g.crossings(VS, active_only=True)
    k, _, _, fl = g.export()
    act_leaves = set(orc.pack_key(np.floor_divide(orc.unpack_key(k[(fl & 1) == 1]), 8)).tolist())
    own_leaf = orc.pack_key(np.floor_divide(orc.unpack_key(allo), 8))
    keep = np.array([int(x) in act_leaves for x in own_leaf])
    assert 0 < keep.sum() < len(allx)
    assert np.array_equal(acto, allo[keep]) and np.array_equal(acts, alls[keep])
    assert np.array_equal(actx, allx[keep])
    _, ek, _ = g.mesh(VS, active_only=True)
    _, ek_all, _ = g.mesh(VS)
    assert 0 < len(ek) < len(ek_all)


def test_surface_store_replaces_active_leaves_only(orc):
    """The G-GPDF training set after an update: the touched leaves carry the new crossings,
    every other leaf keeps what it had."""
    R, c = 0.63, np.array([0.013, 0.021, -0.017])
    ijk = _box([-10, -10, -10], [11, 11, 11])
    D = np.linalg.norm(ijk * VS - c, axis=1) - R
    g = _grid(orc, ijk, D)
    st = orc.SurfaceStore(VS)
    st.update(g)
    full, _, _ = g.crossings(VS)
    a = st.points()
    assert len(a) == len(full)
    assert {tuple(p) for p in a.tolist()} == {tuple(p) for p in full.tolist()}
    old = dict(st.leaf)
    # move the sphere: refuse only leaves with x >= 0 (voxels x >= 0 are in those leaves)
    sel = ijk[:, 0] >= 0
    D2 = np.linalg.norm(ijk * VS - (c + [0.05, 0, 0]), axis=1) - R
    n = int(sel.sum())
    g.fuse(orc.pack_key(ijk[sel]), D2[sel], np.full(n, 1e-12), np.zeros(n, np.uint8))
    st.update(g)
    newx, _, _ = g.crossings(VS, active_only=True)
    lk = orc.leaf_key_of_points(newx, VS)
    k, _, _, fl = g.export()
    act = set(orc.pack_key(np.floor_divide(orc.unpack_key(k[(fl & 1) == 1]), 8)).tolist())
    for leaf, pts in old.items():
        if leaf not in act:
            assert np.array_equal(st.leaf[leaf], pts)
    for leaf in act:
        exp = newx[lk == leaf]
        if len(exp):
            assert np.array_equal(st.leaf[leaf], exp)
        else:
            assert leaf not in st.leaf
