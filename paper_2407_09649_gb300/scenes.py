"""Seeded synthetic scenes shared by the CUDA path's tests/benchmarks and the oracle's.

This module only draws inputs: point clouds, query points and patch instances.  It holds
none of the method's arithmetic (no voxel keys, no kernel, no GP algebra), so both the
oracle and the CUDA path can take their inputs from here without sharing any of the
computation they are compared on.

The paper evaluates on RGB-D and LiDAR scans of rooms and campuses (Sec. V); those
datasets are not available, so each generator below builds a scene of the same structure:
surfaces sampled by a depth sensor or area-uniformly, 0.1 m voxels, 8^3 leaves.

All randomness is numpy ``PCG64`` with an explicit seed.  Every function returns float32
arrays (the dtype the sensor path delivers) unless stated otherwise.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    bg = np.random.PCG64(seed)
    if stream:
        bg = bg.jumped(stream)
    return np.random.Generator(bg)


# --------------------------------------------------------------------------------------
# Sphere + plane single frame: 20k surface points, 10k queries in [-4, 4]^3.
# --------------------------------------------------------------------------------------
def sphere_plane_frame(seed: int = 0, n_sphere: int = 10_000, n_plane: int = 10_000,
                       radius: float = 2.0, plane_z: float = -1.0, half: float = 4.0,
                       noise: float = 0.01) -> np.ndarray:
    """Half the points uniform on a sphere of radius 2 m at the origin, half uniform on
    the plane z=-1 over [-4,4]^2, plus isotropic Gaussian noise (sigma 0.01 m)."""
    rng = _rng(seed)
    s = rng.standard_normal((n_sphere, 3))
    s *= radius / np.linalg.norm(s, axis=1, keepdims=True)
    p = np.empty((n_plane, 3))
    p[:, :2] = rng.uniform(-half, half, (n_plane, 2))
    p[:, 2] = plane_z
    pts = np.vstack([s, p])
    pts += rng.normal(0.0, noise, pts.shape)
    return pts.astype(np.float32)


def uniform_queries(seed: int = 0, n: int = 10_000, lo=(-4.0, -4.0, -4.0),
                    hi=(4.0, 4.0, 4.0)) -> np.ndarray:
    """Uniform query points in an axis-aligned box (second PCG64 stream of ``seed``)."""
    rng = _rng(seed, stream=1)
    return rng.uniform(np.asarray(lo), np.asarray(hi), (n, 3)).astype(np.float32)


# --------------------------------------------------------------------------------------
# Room + circling depth camera: a sequence of ray-cast frames.
# --------------------------------------------------------------------------------------
class Room:
    """A 20x10x3 m box with 30 axis-aligned boxes on the floor and 10 spheres."""

    def __init__(self, seed: int = 0, size=(20.0, 10.0, 3.0), n_boxes: int = 30,
                 n_spheres: int = 10, cam_centre=(10.0, 5.0, 1.5), cam_radius: float = 3.0):
        rng = _rng(seed)
        self.size = np.asarray(size, dtype=np.float64)
        self.cam_centre = np.asarray(cam_centre, dtype=np.float64)
        self.cam_radius = float(cam_radius)
        boxes = []
        while len(boxes) < n_boxes:
            s = rng.uniform(0.2, 2.0, 3)
            c = rng.uniform(s[:2] / 2, self.size[:2] - s[:2] / 2)
            lo = np.array([c[0] - s[0] / 2, c[1] - s[1] / 2, 0.0])
            hi = np.array([c[0] + s[0] / 2, c[1] + s[1] / 2, s[2]])
            if self._blocks_camera(lo, hi):
                continue
            boxes.append((lo, hi))
        self.box_lo = np.array([b[0] for b in boxes])
        self.box_hi = np.array([b[1] for b in boxes])
        sph = []
        while len(sph) < n_spheres:
            r = rng.uniform(0.2, 1.0)
            c = rng.uniform([r, r, r], self.size - r)
            if self._sphere_blocks_camera(c, r):
                continue
            sph.append((c, r))
        self.sph_c = np.array([s[0] for s in sph])
        self.sph_r = np.array([s[1] for s in sph])

    def _blocks_camera(self, lo, hi, clearance=0.4):
        th = np.linspace(0, 2 * np.pi, 256, endpoint=False)
        cam = self.cam_centre + self.cam_radius * np.c_[np.cos(th), np.sin(th), np.zeros_like(th)]
        inside = np.all((cam > lo - clearance) & (cam < hi + clearance), axis=1)
        return bool(inside.any())

    def _sphere_blocks_camera(self, c, r, clearance=0.4):
        th = np.linspace(0, 2 * np.pi, 256, endpoint=False)
        cam = self.cam_centre + self.cam_radius * np.c_[np.cos(th), np.sin(th), np.zeros_like(th)]
        return bool((np.linalg.norm(cam - c, axis=1) < r + clearance).any())

    def camera_pose(self, k: int, n_poses: int = 50):
        th = 2 * np.pi * k / n_poses
        origin = self.cam_centre + self.cam_radius * np.array([np.cos(th), np.sin(th), 0.0])
        fwd = np.array([np.cos(th), np.sin(th), 0.0])
        up = np.array([0.0, 0.0, 1.0])
        right = np.cross(fwd, up)
        return origin, fwd, right, up

    def raycast(self, origin, dirs):
        """Range along each unit ray to the nearest surface (room walls, boxes, spheres)."""
        o = np.asarray(origin, dtype=np.float64)
        d = dirs
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            # room interior: exit distance
            t_hi = np.where(d > 0, (self.size - o) * inv, np.where(d < 0, (0.0 - o) * inv, np.inf))
            t = t_hi.min(axis=1)
            # boxes: slab entry distance
            for lo, hi in zip(self.box_lo, self.box_hi):
                t0 = (lo - o) * inv
                t1 = (hi - o) * inv
                tmin = np.minimum(t0, t1).max(axis=1)
                tmax = np.maximum(t0, t1).min(axis=1)
                hit = (tmax >= tmin) & (tmin > 0)
                t = np.where(hit & (tmin < t), tmin, t)
            for c, r in zip(self.sph_c, self.sph_r):
                oc = o - c
                b = d @ oc
                cc = oc @ oc - r * r
                disc = b * b - cc
                th = -b - np.sqrt(np.maximum(disc, 0.0))
                hit = (disc >= 0) & (th > 0)
                t = np.where(hit & (th < t), th, t)
        return t

    def frame(self, k: int, seed: int = 0, width: int = 400, height: int = 250,
              fov_x_deg: float = 90.0, fov_y_deg: float = 60.0, noise: float = 0.02,
              n_poses: int = 50) -> np.ndarray:
        """World-frame points of one pinhole depth frame (width*height rays)."""
        origin, fwd, right, up = self.camera_pose(k, n_poses)
        u = (np.arange(width) + 0.5) / width * 2 - 1
        v = (np.arange(height) + 0.5) / height * 2 - 1
        uu, vv = np.meshgrid(u * np.tan(np.radians(fov_x_deg) / 2),
                             v * np.tan(np.radians(fov_y_deg) / 2))
        dirs = fwd[None] + uu.reshape(-1, 1) * right[None] + vv.reshape(-1, 1) * up[None]
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        t = self.raycast(origin, dirs)
        rng = _rng(seed + 1000 * (k + 1))
        t = t + rng.normal(0.0, noise, t.shape)
        return (origin[None] + t[:, None] * dirs).astype(np.float32)

    def surface_samples(self, seed: int = 0, density: float = 100.0) -> np.ndarray:
        """Area-uniform noise-free samples (``density`` per m^2) of every exposed surface of
        the room: walls, floor, ceiling, box faces and spheres."""
        rng = _rng(seed, stream=2)
        faces = []  # (origin, e1, e2) parallelograms
        X, Y, Z = self.size
        faces += [(np.array([0, 0, 0.]), np.array([X, 0, 0.]), np.array([0, Y, 0.])),
                  (np.array([0, 0, Z]), np.array([X, 0, 0.]), np.array([0, Y, 0.])),
                  (np.array([0, 0, 0.]), np.array([X, 0, 0.]), np.array([0, 0, Z])),
                  (np.array([0, Y, 0.]), np.array([X, 0, 0.]), np.array([0, 0, Z])),
                  (np.array([0, 0, 0.]), np.array([0, Y, 0.]), np.array([0, 0, Z])),
                  (np.array([X, 0, 0.]), np.array([0, Y, 0.]), np.array([0, 0, Z]))]
        for lo, hi in zip(self.box_lo, self.box_hi):
            s = hi - lo
            ex, ey, ez = np.diag(s)
            faces += [(lo + np.array([0, 0, s[2]]), ex, ey),
                      (lo, ex, ez), (lo + np.array([0, s[1], 0]), ex, ez),
                      (lo, ey, ez), (lo + np.array([s[0], 0, 0]), ey, ez)]
        out = []
        for o, e1, e2 in faces:
            area = np.linalg.norm(np.cross(e1, e2))
            n = rng.poisson(area * density)
            ab = rng.uniform(0, 1, (n, 2))
            out.append(o + ab[:, :1] * e1 + ab[:, 1:] * e2)
        for c, r in zip(self.sph_c, self.sph_r):
            n = rng.poisson(4 * np.pi * r * r * density)
            s = rng.standard_normal((n, 3))
            s /= np.linalg.norm(s, axis=1, keepdims=True)
            out.append(c + r * s)
        P = np.vstack(out)
        keep = ~self.inside_obstacle(P, margin=1e-6)
        return P[keep].astype(np.float32)

    def inside_obstacle(self, P, margin=0.0):
        P = np.asarray(P, dtype=np.float64)
        inside = np.zeros(len(P), dtype=bool)
        for lo, hi in zip(self.box_lo, self.box_hi):
            inside |= np.all((P > lo + margin) & (P < hi - margin), axis=1)
        for c, r in zip(self.sph_c, self.sph_r):
            inside |= np.linalg.norm(P - c, axis=1) < r - margin
        return inside

    def trajectories(self, seed: int = 2, n_traj: int = 256, n_way: int = 64,
                     shrink: float = 0.5) -> np.ndarray:
        """Catmull-Rom splines through 4 control points uniform in the room shrunk by
        ``shrink`` metres; returns float32 [n_traj, n_way, 3]."""
        rng = _rng(seed)
        cp = rng.uniform(shrink, self.size - shrink, (n_traj, 4, 3))
        # centripetal-free (uniform) Catmull-Rom through P0..P3 with clamped end tangents
        P = np.concatenate([cp[:, :1], cp, cp[:, -1:]], axis=1)  # [T, 6, 3]
        segs = 3
        s = np.linspace(0, segs, n_way, endpoint=True)
        seg = np.minimum(s.astype(int), segs - 1)
        t = (s - seg)[None, :, None]
        p0 = P[:, seg]
        p1 = P[:, seg + 1]
        p2 = P[:, seg + 2]
        p3 = P[:, seg + 3]
        t2, t3 = t * t, t * t * t
        out = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)
        return out.astype(np.float32)


# --------------------------------------------------------------------------------------
# City: ground plane + random boxes, area-uniform surface samples, 10M queries.
# --------------------------------------------------------------------------------------
class City:
    """A 100x100x10 m city: a ground plane and ``n_boxes`` random boxes (footprint sides
    U(2,15) m, height U(2,10) m)."""

    def __init__(self, seed: int = 0, extent=(100.0, 100.0, 10.0), n_boxes: int = 200):
        rng = _rng(seed)
        self.extent = np.asarray(extent, dtype=np.float64)
        fp = rng.uniform(2.0, 15.0, (n_boxes, 2))
        h = rng.uniform(2.0, 10.0, n_boxes)
        c = rng.uniform(fp / 2, self.extent[:2] - fp / 2)
        self.box_lo = np.c_[c - fp / 2, np.zeros(n_boxes)]
        self.box_hi = np.c_[c + fp / 2, h]
        # faces: ground + per box roof and 4 walls, as (origin, e1, e2, outward normal)
        faces = [(np.zeros(3), np.array([self.extent[0], 0, 0]), np.array([0, self.extent[1], 0]),
                  np.array([0, 0, 1.0]))]
        for lo, hi in zip(self.box_lo, self.box_hi):
            s = hi - lo
            ex, ey, ez = np.diag(s)
            faces += [(lo + np.array([0, 0, s[2]]), ex, ey, np.array([0, 0, 1.0])),
                      (lo, ex, ez, np.array([0, -1.0, 0])),
                      (lo + np.array([0, s[1], 0]), ex, ez, np.array([0, 1.0, 0])),
                      (lo, ey, ez, np.array([-1.0, 0, 0])),
                      (lo + np.array([s[0], 0, 0]), ey, ez, np.array([1.0, 0, 0]))]
        self.f_o = np.array([f[0] for f in faces])
        self.f_e1 = np.array([f[1] for f in faces])
        self.f_e2 = np.array([f[2] for f in faces])
        self.f_n = np.array([f[3] for f in faces])
        self.f_area = np.linalg.norm(np.cross(self.f_e1, self.f_e2), axis=1)

    def _cell_table(self):
        # boxes overlapping each 1 m ground cell, padded with -1
        if getattr(self, "_cells", None) is None:
            nx, ny = int(np.ceil(self.extent[0])), int(np.ceil(self.extent[1]))
            lists = [[] for _ in range(nx * ny)]
            for b, (lo, hi) in enumerate(zip(self.box_lo, self.box_hi)):
                for ix in range(max(int(np.floor(lo[0])) - 1, 0), min(int(np.floor(hi[0])) + 2, nx)):
                    for iy in range(max(int(np.floor(lo[1])) - 1, 0), min(int(np.floor(hi[1])) + 2, ny)):
                        lists[ix * ny + iy].append(b)
            k = max(1, max(len(x) for x in lists))
            tab = np.full((nx * ny, k), -1, dtype=np.int64)
            for c, x in enumerate(lists):
                tab[c, :len(x)] = x
            self._cells = (nx, ny, tab)
        return self._cells

    def inside_box(self, P, margin=0.0):
        P = np.asarray(P, dtype=np.float64)
        nx, ny, tab = self._cell_table()
        ix = np.clip(np.floor(P[:, 0]).astype(np.int64), 0, nx - 1)
        iy = np.clip(np.floor(P[:, 1]).astype(np.int64), 0, ny - 1)
        cand = tab[ix * ny + iy]
        inside = np.zeros(len(P), dtype=bool)
        for j in range(cand.shape[1]):
            b = cand[:, j]
            has = b >= 0
            bb = np.where(has, b, 0)
            lo = self.box_lo[bb] + margin
            hi = self.box_hi[bb] - margin
            inside |= has & np.all((P > lo) & (P < hi), axis=1)
        return inside

    def _sample_faces(self, rng, n):
        f = rng.choice(len(self.f_area), size=n, p=self.f_area / self.f_area.sum())
        ab = rng.uniform(0, 1, (n, 2))
        P = self.f_o[f] + ab[:, :1] * self.f_e1[f] + ab[:, 1:] * self.f_e2[f]
        return P, self.f_n[f]

    def surface(self, n: int = 2_000_000, seed: int = 0, chunk: int = 1 << 20) -> np.ndarray:
        """``n`` area-uniform samples on exposed faces (samples hidden inside another box
        are rejected and redrawn), no noise."""
        rng = _rng(seed, stream=1)
        got, total = [], 0
        while total < n:
            P, _ = self._sample_faces(rng, chunk)
            P = P[~self.inside_box(P, margin=1e-6)]
            got.append(P)
            total += len(P)
        return np.vstack(got)[:n].astype(np.float32)

    def queries(self, n: int = 10_000_000, seed: int = 1, frac_free: float = 0.7,
                max_offset: float = 0.5, chunk: int = 1 << 21) -> np.ndarray:
        """``frac_free`` uniform in free space (rejecting points inside boxes), the rest a
        surface sample pushed out along its normal by U(0, max_offset) m."""
        rng = _rng(seed)
        n_free = int(round(n * frac_free))
        n_near = n - n_free
        free, total = [], 0
        while total < n_free:
            P = rng.uniform(0, self.extent, (chunk, 3))
            P = P[~self.inside_box(P)]
            free.append(P)
            total += len(P)
        near, total = [], 0
        while total < n_near:
            P, N = self._sample_faces(rng, chunk)
            P = P + N * rng.uniform(0, max_offset, (chunk, 1))
            P = P[~self.inside_box(P, margin=-1e-6)]
            near.append(P)
            total += len(P)
        Q = np.vstack([np.vstack(free)[:n_free], np.vstack(near)[:n_near]])
        Q = Q[rng.permutation(len(Q))]
        return Q.astype(np.float32)


# --------------------------------------------------------------------------------------
# Independent patch instances (the batched sweep): N log-uniform in [4, 1024].
# --------------------------------------------------------------------------------------
def patch_sweep(n_inst: int = 200_000, seed: int = 4, n_min: int = 4, n_max: int = 1024,
                q_per_inst: int = 512, noise: float = 0.01, spacing: float = 0.1,
                box: float = 50.0):
    """Noisy planar / spherical-cap patches (alternating), N = floor(exp(U(ln n_min,
    ln(n_max+1)))) points each at about ``spacing`` metres, queried at ``q_per_inst``
    points uniform in the patch's bounding box grown by 0.5 m.

    Returns ``(inst_off int64[I+1], X float32[sum N,3], q_off int64[I+1], Q float32[.,3])``.
    """
    rng = _rng(seed)
    N = np.floor(np.exp(rng.uniform(np.log(n_min), np.log(n_max + 1), n_inst))).astype(np.int64)
    N = np.clip(N, n_min, n_max)
    inst_off = np.zeros(n_inst + 1, dtype=np.int64)
    np.cumsum(N, out=inst_off[1:])
    T = int(inst_off[-1])
    inst = np.repeat(np.arange(n_inst), N)
    kind = inst % 2  # 0 planar, 1 spherical cap
    # random orthonormal frame per instance
    a = rng.standard_normal((n_inst, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    tmp = np.where(np.abs(a[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    b = np.cross(a, tmp)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    c = np.cross(a, b)
    centre = rng.uniform(-box, box, (n_inst, 3))
    radius = rng.uniform(0.2, 1.0, n_inst)
    u = rng.uniform(0, 1, (T, 2))
    side = spacing * np.sqrt(N.astype(np.float64))
    # planar: square of side 0.1 sqrt(N) in the (b, c) plane
    s_i = side[inst]
    plane = (u[:, :1] - 0.5) * s_i[:, None] * b[inst] + (u[:, 1:] - 0.5) * s_i[:, None] * c[inst]
    # spherical cap of area N * spacing^2 about axis a, centre offset so the cap apex sits at
    # the instance centre
    R = radius[inst]
    area = N[inst] * spacing * spacing
    cos_t = np.maximum(1.0 - area / (2 * np.pi * R * R), -1.0)
    z = cos_t + (1.0 - cos_t) * u[:, 0]
    phi = 2 * np.pi * u[:, 1]
    rxy = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    cap = R[:, None] * (z[:, None] * a[inst] + (rxy * np.cos(phi))[:, None] * b[inst]
                        + (rxy * np.sin(phi))[:, None] * c[inst]) - R[:, None] * a[inst]
    X = np.where(kind[:, None] == 0, plane, cap) + centre[inst]
    X += rng.normal(0.0, noise, X.shape)
    # queries: uniform in each instance's AABB grown by 0.5 m
    lo = np.full((n_inst, 3), np.inf)
    hi = np.full((n_inst, 3), -np.inf)
    np.minimum.at(lo, inst, X)
    np.maximum.at(hi, inst, X)
    lo -= 0.5
    hi += 0.5
    q_off = np.arange(n_inst + 1, dtype=np.int64) * q_per_inst
    qi = np.repeat(np.arange(n_inst), q_per_inst)
    Q = lo[qi] + rng.uniform(0, 1, (n_inst * q_per_inst, 3)) * (hi - lo)[qi]
    return inst_off, X.astype(np.float32), q_off, Q.astype(np.float32)
