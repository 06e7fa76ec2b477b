"""Python access to the plain FP64 CPU oracle (``vgpdf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the package's smoke check and the benchmark's
CPU-baseline leg use this module; the product path never does.  It shares no code with the
CUDA path; the two meet only on the seeded inputs of ``paper_2407_09649_gb300.scenes``.

Every function here is argument marshalling around the C oracle, which cites the paper
passage it follows (Eqs. 1-5 for the GP algebra and reverting, Eqs. 7-9 for fusion,
Sec. IV-A/B/D for voxelisation, closest-node choice and the G-GPDF neighbourhood).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vgpdf_oracle.c")
_LIB = os.path.join(_HERE, "_vgpdf_oracle.so")

ST_OK, ST_NO_SUPPORT, ST_CLAMPED, ST_BAD_INPUT, ST_FACTOR_FAIL = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over instances)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("voxel_size", C.c_double), ("lengthscale", C.c_double),
                ("sigma_occ", C.c_double), ("d_max", C.c_double), ("d_var_floor", C.c_double),
                ("max_pts_leaf", C.c_int32), ("max_pts_group", C.c_int32),
                ("max_leaf_search", C.c_int32), ("fusion", C.c_int32),
                ("sigma_prop", C.c_double), ("n_props", C.c_int32), ("pad_", C.c_int32)]


def params(voxel_size=0.1, lengthscale=0.3, sigma_occ=0.01, d_max=10.0, d_var_floor=1e-3,
           max_pts_leaf=64, max_pts_group=1024, max_leaf_search=8, fusion=0, sigma_prop=0.1,
           n_props=0) -> Params:
    return Params(voxel_size, lengthscale, sigma_occ, d_max, d_var_floor, max_pts_leaf,
                  max_pts_group, max_leaf_search, fusion, sigma_prop, n_props, 0)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp = C.c_void_p
        i64 = C.c_int64
        L.or_index_points.argtypes = [C.POINTER(Params), vp, i64, vp, vp, vp, vp, vp]
        L.or_gp_fit.argtypes = [vp, C.c_int, C.POINTER(Params), vp, vp]
        L.or_gp_fit.restype = C.c_int
        L.or_gp_batch.argtypes = [C.POINTER(Params), i64, vp, vp, vp, vp, C.c_int] + [vp] * 8
        L.or_gp_batch.restype = C.c_int
        L.or_frame_build.argtypes = [C.POINTER(Params), vp, i64]
        L.or_frame_build.restype = vp
        L.or_frame_build2.argtypes = [C.POINTER(Params), vp, i64, vp, C.c_int, vp, i64]
        L.or_frame_build2.restype = vp
        L.or_frame_build3.argtypes = [C.POINTER(Params), vp, vp, i64, vp, C.c_int, vp, i64]
        L.or_frame_build3.restype = vp
        L.or_frame_props.argtypes = [vp, vp, vp]
        L.or_frame_props.restype = C.c_int
        L.or_frame_signs.argtypes = [vp, vp]
        L.or_frame_free.argtypes = [vp]
        L.or_frame_count.argtypes = [vp, C.c_int]
        L.or_frame_count.restype = i64
        L.or_frame_leaves.argtypes = [vp] * 6
        L.or_frame_tests.argtypes = [vp] * 7
        L.or_grid_new.restype = vp
        L.or_grid_free.argtypes = [vp]
        L.or_grid_fuse.argtypes = [vp, C.c_int, vp, vp, vp, vp, i64]
        L.or_grid_fuse2.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, C.c_int, i64]
        L.or_grid_fuse2.restype = C.c_int
        L.or_grid_export_props.argtypes = [vp, vp, vp]
        L.or_grid_export_props.restype = C.c_int
        L.or_grid_size.argtypes = [vp]
        L.or_grid_size.restype = i64
        L.or_grid_export.argtypes = [vp] * 5
        L.or_grid_crossings.argtypes = [vp, C.c_double, C.c_int, vp, vp, vp, vp]
        L.or_grid_crossings.restype = i64
        L.or_grid_mesh.argtypes = [vp, C.c_double, C.c_int, vp, vp, vp, vp]
        L.or_grid_mesh.restype = i64
        L.or_surface_new.argtypes = [C.POINTER(Params), vp, i64]
        L.or_surface_new.restype = vp
        L.or_surface_free.argtypes = [vp]
        L.or_surface_leaves.argtypes = [vp, vp, vp, vp]
        L.or_surface_leaves.restype = i64
        L.or_surface_instance.argtypes = [vp, C.c_uint64, vp]
        L.or_surface_instance.restype = i64
        L.or_query_smooth_nodes.argtypes = [vp, vp, i64, C.c_int, vp]
        L.or_query_smooth_nodes.restype = C.c_int
        L.or_surface_leaf_capped.argtypes = [vp, C.c_uint64, C.c_int, vp]
        L.or_surface_leaf_capped.restype = i64
        L.or_query.argtypes = [vp, vp, i64, C.c_int, vp, vp, vp, vp, vp, vp]
        L.or_query_backward.argtypes = [vp, vp, i64, vp, vp, vp]
        L.or_query_smooth.argtypes = [vp, vp, i64, C.c_int, C.c_double, C.c_int, vp, vp, vp, vp, vp]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


# ------------------------------------------------------------------------------------
def index_points(pts, P: Params | None = None):
    """Voxel index, voxel key, leaf key, in-leaf bit and validity of each point."""
    P = P or params()
    pts = _f32(pts)
    n = len(pts)
    ijk = np.zeros((n, 3), np.int64)
    vk = np.zeros(n, np.uint64)
    lk = np.zeros(n, np.uint64)
    bit = np.zeros(n, np.int32)
    ok = np.zeros(n, np.uint8)
    lib().or_index_points(C.byref(P), _p(pts), n, _p(ijk), _p(vk), _p(lk), _p(bit), _p(ok))
    return ijk, vk, lk, bit, ok.astype(bool)


def gp_fit(X, P: Params | None = None):
    """Packed lower Cholesky factor of K + sigma^2 I and alpha = (K + sigma^2 I)^-1 1."""
    P = P or params()
    X = _f64(X).reshape(-1, 3)
    N = len(X)
    Lp = np.zeros(N * (N + 1) // 2 + 1)
    al = np.zeros(max(N, 1))
    ok = lib().or_gp_fit(_p(X), N, C.byref(P), _p(Lp), _p(al))
    return bool(ok), Lp[: N * (N + 1) // 2], al[:N]


@dataclass
class BatchResult:
    d: np.ndarray
    grad: np.ndarray
    var: np.ndarray
    status: np.ndarray
    occ: np.ndarray
    grad_occ: np.ndarray
    u: np.ndarray
    alpha: np.ndarray


def gp_batch(inst_off, X, q_off, Q, P: Params | None = None, want_var: bool = True) -> BatchResult:
    """Independent instances: inst ``I`` trains on ``X[inst_off[I]:inst_off[I+1]]`` and
    answers ``Q[q_off[I]:q_off[I+1]]``."""
    P = P or params()
    inst_off = np.ascontiguousarray(inst_off, np.int64)
    q_off = np.ascontiguousarray(q_off, np.int64)
    X = _f64(X).reshape(-1, 3)
    Q = _f64(Q).reshape(-1, 3)
    nq = len(Q)
    r = BatchResult(np.zeros(nq), np.zeros((nq, 3)), np.zeros(nq), np.zeros(nq, np.uint8),
                    np.zeros(nq), np.zeros((nq, 3)), np.zeros(nq), np.zeros(len(X)))
    rc = lib().or_gp_batch(C.byref(P), len(inst_off) - 1, _p(inst_off), _p(X), _p(q_off), _p(Q),
                           int(want_var), _p(r.d), _p(r.grad), _p(r.var), _p(r.status), _p(r.occ),
                           _p(r.grad_occ), _p(r.u), _p(r.alpha))
    if rc != 0:
        raise MemoryError("oracle gp_batch failed")
    return r


def gp_single(X, Q, P: Params | None = None, want_var: bool = True) -> BatchResult:
    X = _f64(X).reshape(-1, 3)
    Q = _f64(Q).reshape(-1, 3)
    return gp_batch([0, len(X)], X, [0, len(Q)], Q, P, want_var)


# ------------------------------------------------------------------------------------
@dataclass
class Frame:
    leaf_key: np.ndarray
    leaf_nocc: np.ndarray
    inst_off: np.ndarray
    X: np.ndarray
    alpha: np.ndarray
    test_key: np.ndarray
    test_inst_key: np.ndarray
    d: np.ndarray
    v: np.ndarray
    grad: np.ndarray
    status: np.ndarray
    sign: np.ndarray = None
    c: np.ndarray = None  # surface-property means (n_test, n_props), Eq. 6
    w: np.ndarray = None  # surface-property variances (n_test,)


def frame(pts, P: Params | None = None, origin=None, normal_steps: int = 3, known=None, props=None) -> Frame:
    """One L-GPDF frame: voxelise, fit one GP per leaf, infer at all testing voxels.  Without
    ``origin`` the testing voxels are the dilated GP leaves; with the sensor ``origin`` they are
    the ray-cast set of Sec. IV-B (``known``: sorted voxel keys with earlier measurements) and
    the distances are signed.  ``props`` (n, P.n_props) float32 gives each point's surface
    properties; the frame then also infers their means and variances (Eq. 6)."""
    P = P or params()
    pts = _f32(pts)
    L = lib()
    pr = None
    if props is not None and P.n_props > 0:
        pr = np.ascontiguousarray(np.asarray(props, np.float32).reshape(len(pts), P.n_props))
    if origin is None:
        h = L.or_frame_build3(C.byref(P), _p(pts), _p(pr) if pr is not None else None, len(pts), None, 0, None, 0)
    else:
        o = np.ascontiguousarray(origin, np.float64)
        kn = np.ascontiguousarray(np.sort(np.asarray(known if known is not None else [], np.uint64)), np.uint64)
        h = L.or_frame_build3(C.byref(P), _p(pts), _p(pr) if pr is not None else None, len(pts), _p(o),
                              int(normal_steps), _p(kn) if len(kn) else None, len(kn))
    if not h:
        raise MemoryError("oracle frame build failed")
    try:
        nl, T, nt = (L.or_frame_count(h, w) for w in (0, 1, 2))
        f = Frame(np.zeros(nl, np.uint64), np.zeros(nl, np.int32), np.zeros(nl + 1, np.int64),
                  np.zeros((T, 3)), np.zeros(T), np.zeros(nt, np.uint64), np.zeros(nt, np.uint64),
                  np.zeros(nt), np.zeros(nt), np.zeros((nt, 3)), np.zeros(nt, np.uint8))
        L.or_frame_leaves(h, _p(f.leaf_key), _p(f.leaf_nocc), _p(f.inst_off), _p(f.X), _p(f.alpha))
        L.or_frame_tests(h, _p(f.test_key), _p(f.test_inst_key), _p(f.d), _p(f.v), _p(f.grad),
                         _p(f.status))
        f.sign = np.zeros(nt, np.int8)
        L.or_frame_signs(h, _p(f.sign))
        if pr is not None:
            f.c = np.zeros((nt, P.n_props))
            f.w = np.zeros(nt)
            L.or_frame_props(h, _p(f.c), _p(f.w))
    finally:
        L.or_frame_free(h)
    return f


class Grid:
    """Global fused grid (sorted voxel records) with probabilistic fusion."""

    def __init__(self, fusion: int = 0):
        self.h = lib().or_grid_new()
        self.fusion = fusion

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_grid_free(self.h)
            self.h = None

    def fuse(self, key, d, v, status, c=None, w=None):
        key = np.ascontiguousarray(key, np.uint64)
        d = _f64(d)
        v = _f64(v)
        status = np.ascontiguousarray(status, np.uint8)
        if c is None:
            lib().or_grid_fuse(self.h, self.fusion, _p(key), _p(d), _p(v), _p(status), len(key))
            return
        c = np.ascontiguousarray(np.asarray(c, np.float64).reshape(len(key), -1))
        w = _f64(w)
        rc = lib().or_grid_fuse2(self.h, self.fusion, _p(key), _p(d), _p(v), _p(status), _p(c), _p(w), c.shape[1],
                                 len(key))
        if rc != 0:
            raise ValueError("at most 4 property channels")

    def fuse_frame(self, f: Frame):
        self.fuse(f.test_key, f.d, f.v, f.status, f.c, f.w)

    def export_props(self):
        """Fused surface properties (n, n_props) and their variances (weights for Eq. 9) in key
        order; NaN where no property was fused."""
        L = lib()
        n = L.or_grid_size(self.h)
        npr = L.or_grid_export_props(self.h, None, None)
        Cp = np.zeros((n, npr))
        W = np.zeros(n)
        L.or_grid_export_props(self.h, _p(Cp), _p(W))
        return Cp, W

    def export(self):
        n = lib().or_grid_size(self.h)
        k = np.zeros(n, np.uint64)
        D = np.zeros(n)
        V = np.zeros(n)
        fl = np.zeros(n, np.uint8)
        lib().or_grid_export(self.h, _p(k), _p(D), _p(V), _p(fl))
        return k, D, V, fl

    def crossings(self, voxel_size: float, active_only: bool = False, props: bool = False):
        """Zero crossings owned by the voxels of all leaves (or of the leaves touched by the
        latest fusion): float32 points (n, 3), owner voxel keys, slots 2 axis + (+ side); with
        ``props`` also the interpolated fused properties (n, n_props)."""
        L = lib()
        n = L.or_grid_crossings(self.h, float(voxel_size), int(active_only), None, None, None, None)
        npr = L.or_grid_export_props(self.h, None, None)
        xyz = np.zeros((n, 3), np.float32)
        owner = np.zeros(n, np.uint64)
        slot = np.zeros(n, np.uint8)
        cp = np.zeros((n, npr))
        L.or_grid_crossings(self.h, float(voxel_size), int(active_only), _p(xyz), _p(owner), _p(slot), _p(cp))
        return (xyz, owner, slot, cp) if props else (xyz, owner, slot)

    def mesh(self, voxel_size: float, active_only: bool = False, props: bool = False):
        """Marching-cubes triangle soup: xyz (T, 3, 3) FP64, edge keys (T, 3), edge axes (T, 3);
        with ``props`` also the interpolated fused properties per vertex (T, 3, n_props)."""
        L = lib()
        n = L.or_grid_mesh(self.h, float(voxel_size), int(active_only), None, None, None, None)
        npr = L.or_grid_export_props(self.h, None, None)
        xyz = np.zeros((n, 3, 3))
        ek = np.zeros((n, 3), np.uint64)
        ea = np.zeros((n, 3), np.uint8)
        vp_ = np.zeros((n, 3, npr))
        L.or_grid_mesh(self.h, float(voxel_size), int(active_only), _p(xyz), _p(ek), _p(ea), _p(vp_))
        return (xyz, ek, ea, vp_) if props else (xyz, ek, ea)


def leaf_key_of_points(xyz, voxel_size: float) -> np.ndarray:
    """Leaf key of each float32 point (voxel floor(p / vs + 1/2), leaf floor(voxel / 8))."""
    p = np.asarray(xyz, np.float32).astype(np.float64)
    ijk = np.floor(p / voxel_size + 0.5).astype(np.int64)
    lf = np.floor_divide(ijk, 8)
    return pack_key(lf) if len(p) else np.zeros(0, np.uint64)


class SurfaceStore:
    """Zero-crossing training set of the G-GPDF, kept per leaf (Sec. IV-D): after each
    fusion the leaves it touched get their crossings recomputed and replace their old ones;
    the other leaves keep theirs."""

    def __init__(self, voxel_size: float):
        self.vs = float(voxel_size)
        self.leaf = {}

    def update(self, grid: Grid):
        k, _, _, fl = grid.export()
        keys = k[(fl & 1) == 1]
        for a in np.unique(pack_key(np.floor_divide(unpack_key(keys), 8))).tolist() if len(keys) else []:
            self.leaf.pop(int(a), None)
        xyz, _, _ = grid.crossings(self.vs, active_only=True)
        lk = leaf_key_of_points(xyz, self.vs)
        for a in np.unique(lk).tolist():
            self.leaf[int(a)] = xyz[lk == a]

    def points(self) -> np.ndarray:
        """All stored crossings, leaves in ascending key order (in-leaf order kept)."""
        if not self.leaf:
            return np.zeros((0, 3), np.float32)
        return np.concatenate([self.leaf[k] for k in sorted(self.leaf)], 0)


class Surface:
    """G-GPDF training set: surface points binned by leaf."""

    def __init__(self, pts, P: Params | None = None):
        self.P = P or params()
        self.pts = _f32(pts)
        self.h = lib().or_surface_new(C.byref(self.P), _p(self.pts), len(self.pts))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_surface_free(self.h)
            self.h = None

    def leaves(self):
        L = lib()
        nl = L.or_surface_leaves(self.h, None, None, None)
        key = np.zeros(nl, np.uint64)
        off = np.zeros(nl + 1, np.int64)
        L.or_surface_leaves(self.h, _p(key), _p(off), None)
        idx = np.zeros(int(off[-1]), np.int64)
        L.or_surface_leaves(self.h, None, None, _p(idx))
        return key, off, idx

    def instance(self, centre_key: int) -> np.ndarray:
        L = lib()
        n = L.or_surface_instance(self.h, C.c_uint64(int(centre_key)), None)
        out = np.zeros(max(n, 1), np.int64)
        L.or_surface_instance(self.h, C.c_uint64(int(centre_key)), _p(out))
        return out[:n]

    def query(self, q, want_var: bool = True):
        q = _f32(q)
        n = len(q)
        d = np.zeros(n)
        g = np.zeros((n, 3))
        v = np.zeros(n)
        st = np.zeros(n, np.uint8)
        ik = np.zeros(n, np.uint64)
        iN = np.zeros(n, np.int32)
        lib().or_query(self.h, _p(q), n, int(want_var), _p(d), _p(g), _p(v), _p(st), _p(ik), _p(iN))
        return dict(d=d, grad=g, var=v if want_var else None, status=st, inst_key=ik, inst_n=iN)

    def smooth_nodes(self, q, n_nodes: int = 8) -> np.ndarray:
        """Leaf keys of the nodes each query blends in query_smooth, nearest first, 0 past the
        last node: (n, n_nodes) uint64."""
        q = _f32(q)
        keys = np.zeros((len(q), int(n_nodes)), np.uint64)
        lib().or_query_smooth_nodes(self.h, _p(q), len(q), int(n_nodes), _p(keys))
        return keys

    def leaf_capped(self, key: int, cap: int) -> np.ndarray:
        """Sorted point indices of the node GP of leaf ``key`` (at most ``cap`` points, those
        nearest the leaf centre)."""
        L = lib()
        n = L.or_surface_leaf_capped(self.h, C.c_uint64(int(key)), int(cap), None)
        out = np.zeros(max(n, 1), np.int64)
        L.or_surface_leaf_capped(self.h, C.c_uint64(int(key)), int(cap), _p(out))
        return out[:n]

    def query_smooth(self, q, n_nodes: int = 8, lam: float = 100.0, want_var: bool = True):
        """G-GPDF as per-leaf GPs blended by the smooth minimum of Eq. 10."""
        q = _f32(q)
        n = len(q)
        d = np.zeros(n)
        g = np.zeros((n, 3))
        v = np.zeros(n)
        st = np.zeros(n, np.uint8)
        nn = np.zeros(n, np.int32)
        lib().or_query_smooth(self.h, _p(q), n, int(n_nodes), float(lam), int(want_var), _p(d), _p(g), _p(v),
                              _p(st), _p(nn))
        return dict(d=d, grad=g, var=v if want_var else None, status=st, n_nodes=nn)

    def backward(self, q, dL_dd):
        q = _f32(q)
        n = len(q)
        dL_dd = _f64(dL_dd)
        dq = np.zeros((n, 3))
        dX = np.zeros((len(self.pts), 3))
        lib().or_query_backward(self.h, _p(q), n, _p(dL_dd), _p(dq), _p(dX))
        return dq, dX


# ------------------------------------------------------------------------------------
def unpack_key(k):
    """Integer (x, y, z) of a packed 3x21-bit key (bias 2^20)."""
    k = np.asarray(k, dtype=np.uint64)
    m = np.uint64(0x1FFFFF)
    x = ((k >> np.uint64(42)) & m).astype(np.int64) - (1 << 20)
    y = ((k >> np.uint64(21)) & m).astype(np.int64) - (1 << 20)
    z = (k & m).astype(np.int64) - (1 << 20)
    return np.stack([x, y, z], axis=-1)


def pack_key(ijk):
    ijk = np.asarray(ijk, dtype=np.int64) + (1 << 20)
    return ((ijk[..., 0].astype(np.uint64) << np.uint64(42))
            | (ijk[..., 1].astype(np.uint64) << np.uint64(21)) | ijk[..., 2].astype(np.uint64))
