"""Edge cases of the mapping paths on the GPU: empty maps and frames through marching cubes
and training-set updates, a sensor origin that is not finite, properties fused with the
TSDF-style weights of Eq. 9, and the graph launch mode on empty batches."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vg():
    import paper_2407_09649_gb300 as P
    P.build()
    return P


def test_empty_map_mesh_and_surface(vg):
    m = vg.Map(precision="fp64")
    r = m.extract_mesh()
    assert r["crossings"][0].shape == (0, 3) and r["triangles"][0].shape == (0, 3, 3)
    assert m.update_surface() == 0
    q = torch.zeros((5, 3), device="cuda")
    out = m.query(q)
    assert np.all(out["status"].cpu().numpy() == 1)  # no support
    assert np.all(np.isinf(out["d"].cpu().numpy()))


def test_empty_frame_touches_nothing(vg, orc):
    """A frame without points fuses nothing: afterwards no leaf is active, the active-leaf
    extraction is empty and the training set keeps what it had."""
    from paper_2407_09649_gb300 import scenes
    room = scenes.Room(0)
    m = vg.Map(precision="fp64", max_pts_leaf=256)
    pts = torch.from_numpy(room.frame(0, seed=0)[::4]).cuda()
    o = room.camera_pose(0)[0]
    m.fuse(m.build_frame(pts, origin=o))
    n0 = m.update_surface()
    kept = m.surface_points().cpu().numpy()
    assert n0 > 100
    f = m.build_frame(torch.zeros((0, 3), device="cuda"), origin=o)
    assert f.n_test == 0
    m.fuse(f)
    r = m.extract_mesh(active_only=True)
    assert r["crossings"][0].shape[0] == 0 and r["triangles"][0].shape[0] == 0
    assert m.update_surface() == n0
    assert np.array_equal(m.surface_points().cpu().numpy(), kept)


def test_nonfinite_origin_tests_only_occupied_voxels(vg, orc):
    """With an origin that is not finite there are no rays and no oriented normals: the
    testing voxels are the occupied voxels, all with sign +, on both sides."""
    from paper_2407_09649_gb300 import scenes
    room = scenes.Room(0)
    pts = room.frame(2, seed=0)[::4]
    P = orc.params(max_pts_leaf=256)
    o = np.array([np.nan, 1.0, 1.0])
    ref = orc.frame(pts, P, origin=o)
    m = vg.Map(precision="fp64", max_pts_leaf=256)
    f = m.build_frame(torch.from_numpy(pts).cuda(), origin=o)
    r = {k: v.cpu().numpy() for k, v in f.results().items()}
    assert np.array_equal(np.sort(r["keys"]), np.sort(ref.test_key))
    assert np.all(ref.sign == 1)
    ok = r["status"] == 0
    assert np.all(r["d"][ok] >= 0)


def test_tsdf_property_fusion_matches_oracle(vg, orc):
    """Eq. 9 weights for the distance and the properties, three frames, FP64 map."""
    from paper_2407_09649_gb300 import scenes
    room = scenes.Room(0)
    P = orc.params(max_pts_leaf=256, n_props=1, fusion=1)
    g = orc.Grid(fusion=1)
    m = vg.Map(precision="fp64", max_pts_leaf=256, n_props=1, fusion="tsdf")
    rng = np.random.default_rng(4)
    for k in range(3):
        pts = room.frame(4 * k, seed=0)[::3]
        props = rng.uniform(0, 1, (len(pts), 1)).astype(np.float32)
        origin = room.camera_pose(4 * k)[0]
        f = orc.frame(pts, P, origin=origin, known=g.export()[0], props=props)
        g.fuse_frame(f)
        m.fuse(m.build_frame(torch.from_numpy(pts).cuda(), origin=origin, props=torch.from_numpy(props).cuda()))
    k1, D1, V1, _ = m.export_grid()
    k2, D2, V2, _ = g.export()
    assert np.array_equal(k1, k2)
    assert np.abs(D1 - D2).max() <= 1e-4 and np.abs(V1 - V2).max() <= 1e-6
    _, C1, W1 = m.export_props()
    C2, W2 = g.export_props()
    has = ~np.isnan(W2)
    assert np.array_equal(~np.isnan(W1), has) and has.mean() > 0.5
    assert np.abs(C1[has] - C2[has]).max() <= 1e-6 and np.abs(W1[has] - W2[has]).max() <= 1e-6


def test_graph_mode_on_empty_and_tiny_batches(vg):
    m = vg.Map(precision="mixed", launch="graph")
    f = m.build_frame(torch.zeros((0, 3), device="cuda"))
    assert f.n_test == 0
    one = torch.tensor([[0.31, 0.22, -0.14]], device="cuda")
    f = m.build_frame(one)
    r = f.results()
    assert m.stats()["graph_replays"] > 0  # the solve ran as a graph, not skipped
    assert r["keys"].shape[0] == 27 * 512
    mb = vg.Map(precision="mixed")
    rb = mb.build_frame(one).results()
    a = np.argsort(r["keys"].cpu().numpy())
    b = np.argsort(rb["keys"].cpu().numpy())
    assert np.array_equal(r["d"].cpu().numpy()[a].view(np.uint64), rb["d"].cpu().numpy()[b].view(np.uint64))
