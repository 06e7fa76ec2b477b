"""Pins of the oracle's ray-cast testing points (Sec. IV-B): Bresenham lines have the length,
connectivity and closeness of a voxel line; normals of planar surfaces are the plane normal;
normal voxels and ray voxels carry the sign given by the sensor side; signed distances of a
wall scene match the signed distance to the wall."""
import numpy as np


def _wall(x0=2.0, half=1.2, step=0.02, seed=0):
    rng = np.random.default_rng(seed)
    y, z = np.meshgrid(np.arange(-half, half, step), np.arange(-half, half, step))
    pts = np.c_[np.full(y.size, x0), y.ravel(), z.ravel()] + rng.normal(0, 0.002, (y.size, 3))
    return pts.astype(np.float32)


def test_wall_normals_and_signs(orc):
    P = orc.params(max_pts_leaf=512)
    pts = _wall()
    origin = np.array([0.03, 0.02, 0.01])
    F = orc.frame(pts, P, origin=origin, normal_steps=3, known=None)
    ijk = orc.unpack_key(F.test_key)
    # the wall is the voxel plane i = 20; normal voxels at i = 20 -+ k carry sign +- (sensor at i = 0)
    inner = (np.abs(ijk[:, 1]) <= 9) & (np.abs(ijk[:, 2]) <= 9)
    for k in (1, 2, 3):
        front = inner & (ijk[:, 0] == 20 - k)
        back = inner & (ijk[:, 0] == 20 + k)
        assert front.sum() > 100 and back.sum() > 100
        assert np.all(F.sign[front] == 1) and np.all(F.sign[back] == -1)
    assert set(np.unique(ijk[inner, 0])) <= set(range(17, 24))
    ok = inner & (F.status == 0)
    x = ijk[:, 0] * 0.1
    wall_x = pts[:, 0].mean()
    sd = wall_x - x  # signed distance to the wall, positive on the sensor side
    far = ok & (np.abs(sd) > 0.05)
    assert np.max(np.abs(F.d[far] - sd[far])) < 0.02
    assert np.all(np.sign(F.d[far]) == np.sign(sd[far]))


def test_rays_are_voxel_lines(orc):
    """With every voxel of a box known, the ray voxels of each surface voxel are its whole
    Bresenham line: max|delta| voxels from the origin voxel, 26-connected, within one voxel of
    the segment."""
    P = orc.params(max_pts_leaf=512)
    rng = np.random.default_rng(1)
    pts = (np.array([1.5, -0.7, 0.9]) + rng.normal(0, 0.02, (40, 3))).astype(np.float32)
    origin = np.array([-0.3, 0.4, -0.2])
    g = np.stack(np.meshgrid(*[np.arange(-8, 22)] * 3, indexing="ij"), -1).reshape(-1, 3)
    known = orc.pack_key(g)
    F = orc.frame(pts, P, origin=origin, normal_steps=0, known=known)
    ijk_o = np.floor(origin / 0.1 + 0.5).astype(np.int64)
    occ = np.unique(np.floor(pts.astype(np.float64) / 0.1 + 0.5).astype(np.int64), axis=0)
    keys = set(int(k) for k in F.test_key)
    for s in occ:
        d = s - ijk_o
        m = np.argmax(np.abs(d))
        n = abs(d[m])
        # reconstruct the line voxels from the testing set: one voxel per step of the dominant axis
        line = []
        for i in range(n):
            t = i / n
            ideal = ijk_o + t * d
            cands = [ideal.round().astype(np.int64) + np.array(o) for o in np.ndindex(3, 3, 3)]
            cands = [c - 1 for c in cands]
            cands = [c for c in cands if c[m] == ijk_o[m] + np.sign(d[m]) * i and int(orc.pack_key(c)) in keys]
            assert cands, (s, i)
            best = min(cands, key=lambda c: np.sum((c - ideal) ** 2))
            assert np.max(np.abs(best - ideal)) <= 1.0
            line.append(best)
        for a, b in zip(line[:-1], line[1:]):
            assert np.max(np.abs(a - b)) == 1


def test_jacobi_normal_matches_eigh(orc):
    """A tilted planar patch: the normal voxels lie along the plane normal computed by LAPACK
    (numpy.linalg.eigh) from the same integer scatter."""
    P = orc.params(max_pts_leaf=512)
    u = np.array([1.0, 0.0, 0.3]) / np.linalg.norm([1.0, 0.0, 0.3])
    v = np.array([0.0, 1.0, 0.0])
    a, b = np.meshgrid(np.arange(-0.6, 0.6, 0.01), np.arange(-0.6, 0.6, 0.01))
    pts = (np.array([0.0, 0.0, 1.5]) + a.reshape(-1, 1) * u + b.reshape(-1, 1) * v).astype(np.float32)
    origin = np.array([0.0, 0.0, 0.0])
    F = orc.frame(pts, P, origin=origin, normal_steps=2, known=None)
    occ = np.unique(np.floor(pts.astype(np.float64) / 0.1 + 0.5).astype(np.int64), axis=0)
    occ_set = {tuple(x) for x in occ}
    keys = {int(k): s for k, s in zip(F.test_key, F.sign)}
    checked = 0
    for s in occ[::7]:
        offs = [np.array(o) - 1 for o in np.ndindex(3, 3, 3) if tuple(s + np.array(o) - 1) in occ_set]
        if len(offs) < 3:
            continue
        O = np.array(offs, dtype=np.float64)
        n_ = len(O)
        M = n_ * O.T @ O - np.outer(O.sum(0), O.sum(0))
        w, V = np.linalg.eigh(M)
        if w[1] - w[0] < 1e-6 * max(1.0, w[2]):
            continue  # degenerate smallest eigenvalue: eigenvector not unique
        nrm = V[:, 0]
        if nrm @ (origin - s * 0.1) < 0:
            nrm = -nrm
        for k in (1, 2, -1, -2):
            vv = s + np.floor(k * nrm + 0.5).astype(np.int64)
            assert keys.get(int(orc.pack_key(vv))) is not None, (s, k)
        checked += 1
    assert checked > 20
