"""Thin Python binding of the C ABI (``include/vgpdf.h``) over torch CUDA tensors.

Argument marshalling only: every step of the path runs in the CUDA library.  PyTorch
provides device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


class _CudaView:
    """Zero-copy view of library-owned device memory for ``torch.as_tensor``."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _view(ptr, shape, typestr, dtype):
    n = int(np.prod(shape)) if len(shape) else 1
    if n == 0 or not ptr:
        return torch.empty(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaView(ptr, shape, typestr), device="cuda").clone()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f32(x, name: str) -> torch.Tensor:
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor or numpy array")
    x = x.to(device="cuda", dtype=torch.float32).contiguous()
    if x.dim() != 2 or x.shape[1] != 3:
        raise ValueError(f"{name}: expected shape [n, 3], got {tuple(x.shape)}")
    return x


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def make_params(**kw) -> L.VgpParams:
    lib = L.load()
    p = L.VgpParams()
    lib.vgp_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": L.VGP_FP64, "mixed": L.VGP_MIXED}[v]
        if k == "launch" and isinstance(v, str):
            v = {"batched": L.VGP_LAUNCH_BATCHED, "per_instance": L.VGP_LAUNCH_PER_INSTANCE,
                 "graph": L.VGP_LAUNCH_GRAPH}[v]
        if k == "fusion" and isinstance(v, str):
            v = {"invvar": L.VGP_FUSE_INVVAR, "tsdf": L.VGP_FUSE_TSDF}[v]
        if not hasattr(p, k):
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class Frame:
    """An L-GPDF frame: leaf GPs and testing-voxel results (library-owned)."""

    def __init__(self, gmap: "Map", handle):
        self._map = gmap
        self._h = handle

    def results(self) -> dict:
        lib = L.load()
        n = C.c_int64()
        k, d, v, g, s = (C.c_void_p() for _ in range(5))
        L.check(lib.vgp_frame_results(self._h, C.byref(n), C.byref(k), C.byref(d), C.byref(v), C.byref(g),
                                      C.byref(s)))
        torch.cuda.current_stream().synchronize()
        n = n.value
        return dict(keys=_view(k.value, (n,), "<u8", torch.uint64), d=_view(d.value, (n,), "<f8", torch.float64),
                    v=_view(v.value, (n,), "<f8", torch.float64),
                    grad=_view(g.value, (n, 3), "<f8", torch.float64),
                    status=_view(s.value, (n,), "|u1", torch.uint8))

    def props(self):
        """Surface-property means (n_test, n_props) and variances (n_test,) of the testing
        voxels, in the order of results(); None for a frame without properties."""
        lib = L.load()
        npr = C.c_int32()
        c, w = C.c_void_p(), C.c_void_p()
        L.check(lib.vgp_frame_props(self._h, C.byref(npr), C.byref(c), C.byref(w)))
        if npr.value == 0:
            return None
        n = C.c_int64()
        L.check(lib.vgp_frame_results(self._h, C.byref(n), None, None, None, None, None))
        torch.cuda.current_stream().synchronize()
        return (_view(c.value, (n.value, npr.value), "<f8", torch.float64),
                _view(w.value, (n.value,), "<f8", torch.float64))

    def instances(self) -> dict:
        lib = L.load()
        nl, T = C.c_int64(), C.c_int64()
        lk, no, off, X, al = (C.c_void_p() for _ in range(5))
        L.check(lib.vgp_frame_instances(self._h, C.byref(nl), C.byref(T), C.byref(lk), C.byref(no), C.byref(off),
                                        C.byref(X), C.byref(al)))
        torch.cuda.current_stream().synchronize()
        nl, T = nl.value, T.value
        return dict(leaf_key=_view(lk.value, (nl,), "<u8", torch.uint64),
                    n_occ=_view(no.value, (nl,), "<i4", torch.int32),
                    inst_off=_view(off.value, (nl + 1,), "<i8", torch.int64),
                    X=_view(X.value, (T, 3), "<f8", torch.float64), alpha=_view(al.value, (T,), "<f8", torch.float64))

    @property
    def n_test(self) -> int:
        n = C.c_int64()
        L.check(L.load().vgp_frame_results(self._h, C.byref(n), None, None, None, None, None))
        return n.value

    def close(self):
        if self._h:
            L.load().vgp_frame_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Map:
    """A GP distance-field map on the current CUDA device (see ``include/vgpdf.h``)."""

    def __init__(self, **params):
        lib = L.load()
        self.params = make_params(**params)
        h = C.c_void_p()
        L.check(lib.vgp_create(C.byref(self.params), C.byref(h)))
        self._h = h
        self._surface = None
        self._surface_key = None

    # -- L-GPDF ----------------------------------------------------------------------
    def build_frame(self, pts, origin=None, props=None) -> Frame:
        """L-GPDF of one frame; with the sensor ``origin`` (3 floats) the testing voxels are
        the ray-cast set and distances are signed; ``props`` (n, n_props) float32 adds the
        surface-property GP (Eq. 6)."""
        pts = _dev_f32(pts, "pts")
        h = C.c_void_p()
        o = None
        if origin is not None:
            o = (C.c_double * 3)(*[float(x) for x in origin])
        if props is None:
            L.check(L.load().vgp_build_frame(self._h, _ptr(pts), pts.shape[0], o, _stream(), C.byref(h)))
        else:
            if isinstance(props, np.ndarray):
                props = torch.from_numpy(np.ascontiguousarray(props, np.float32))
            pr = props.to(device="cuda", dtype=torch.float32).reshape(pts.shape[0], -1).contiguous()
            L.check(L.load().vgp_build_frame_props(self._h, _ptr(pts), _ptr(pr), pts.shape[0], o, _stream(),
                                                   C.byref(h)))
        return Frame(self, h)

    def export_props(self):
        """Fused surface properties (n, n_props) and variances in the order of export_grid."""
        lib = L.load()
        n = C.c_int64(0)
        L.check(lib.vgp_export_props(self._h, C.byref(n), None, None, None, _stream()))
        npr = self.params.n_props
        k = np.zeros(n.value, np.uint64)
        Cp = np.zeros((n.value, npr))
        W = np.zeros(n.value)
        if n.value:
            L.check(lib.vgp_export_props(self._h, C.byref(n), k.ctypes.data_as(C.c_void_p),
                                         Cp.ctypes.data_as(C.c_void_p), W.ctypes.data_as(C.c_void_p), _stream()))
        return k, Cp, W

    def import_props(self, keys, Cp, W) -> None:
        keys = np.ascontiguousarray(keys, np.uint64)
        Cp = np.ascontiguousarray(Cp, np.float64)
        W = np.ascontiguousarray(W, np.float64)
        L.check(L.load().vgp_import_props(self._h, len(keys), keys.ctypes.data_as(C.c_void_p),
                                          Cp.ctypes.data_as(C.c_void_p), W.ctypes.data_as(C.c_void_p), _stream()))

    def fuse(self, frame: Frame) -> None:
        L.check(L.load().vgp_fuse(self._h, frame._h, _stream()))

    def export_grid(self):
        lib = L.load()
        n = C.c_int64(0)
        L.check(lib.vgp_export_grid(self._h, C.byref(n), None, None, None, None, _stream()))
        k = np.zeros(n.value, np.uint64)
        D = np.zeros(n.value)
        V = np.zeros(n.value)
        fl = np.zeros(n.value, np.uint8)
        if n.value:
            L.check(lib.vgp_export_grid(self._h, C.byref(n), k.ctypes.data_as(C.c_void_p),
                                        D.ctypes.data_as(C.c_void_p), V.ctypes.data_as(C.c_void_p),
                                        fl.ctypes.data_as(C.c_void_p), _stream()))
        return k[:n.value], D[:n.value], V[:n.value], fl[:n.value]

    def import_grid(self, keys, D, V, flags) -> None:
        keys = np.ascontiguousarray(keys, np.uint64)
        D = np.ascontiguousarray(D, np.float64)
        V = np.ascontiguousarray(V, np.float64)
        flags = np.ascontiguousarray(flags, np.uint8)
        L.check(L.load().vgp_import_grid(self._h, len(keys), keys.ctypes.data_as(C.c_void_p),
                                         D.ctypes.data_as(C.c_void_p), V.ctypes.data_as(C.c_void_p),
                                         flags.ctypes.data_as(C.c_void_p), _stream()))

    # -- G-GPDF ----------------------------------------------------------------------
    def set_surface(self, pts) -> None:
        pts = _dev_f32(pts, "pts")
        L.check(L.load().vgp_set_surface(self._h, _ptr(pts), pts.shape[0], _stream()))
        self._surface = pts
        self._surface_key = (pts.data_ptr(), tuple(pts.shape), pts._version)

    def extract_mesh(self, active_only: bool = False, triangles: bool = True) -> dict:
        """Zero crossings and marching-cubes triangles of the fused grid (vgp_extract_mesh):
        ``crossings`` = (xyz float32 (n, 3), owner voxel keys, slots), ``triangles`` =
        (xyz float64 (T, 3, 3), edge keys (T, 3), edge axes (T, 3))."""
        lib = L.load()
        h = C.c_void_p()
        L.check(lib.vgp_extract_mesh(self._h, int(active_only), int(triangles), _stream(), C.byref(h)))
        try:
            n = C.c_int64()
            x, o, sl = C.c_void_p(), C.c_void_p(), C.c_void_p()
            L.check(lib.vgp_mesh_crossings(h, C.byref(n), C.byref(x), C.byref(o), C.byref(sl)))
            n = n.value
            cross = (_view(x.value, (n, 3), "<f4", torch.float32), _view(o.value, (n,), "<u8", torch.uint64),
                     _view(sl.value, (n,), "|u1", torch.uint8))
            nt = C.c_int64()
            L.check(lib.vgp_mesh_triangles(h, C.byref(nt), C.byref(x), C.byref(o), C.byref(sl)))
            nt = nt.value
            tri = (_view(x.value, (nt, 3, 3), "<f8", torch.float64), _view(o.value, (nt, 3), "<u8", torch.uint64),
                   _view(sl.value, (nt, 3), "|u1", torch.uint8))
            npr = C.c_int32()
            L.check(lib.vgp_mesh_props(h, C.byref(npr), C.byref(x), C.byref(o)))
            npr = npr.value
            props = None
            if npr:
                props = (_view(x.value, (n, npr), "<f8", torch.float64),
                         _view(o.value, (nt, 3, npr), "<f8", torch.float64))
        finally:
            lib.vgp_mesh_destroy(h)
        return dict(crossings=cross, triangles=tri, props=props)

    def update_surface(self) -> int:
        """Refresh the G-GPDF training set from the zero crossings of the leaves the latest
        fusion touched and train the G-GPDF on it (vgp_update_surface).  Returns its size."""
        L.check(L.load().vgp_update_surface(self._h, _stream()))
        pts = self.surface_points()
        self._surface = pts
        self._surface_key = (pts.data_ptr(), tuple(pts.shape), pts._version)
        return pts.shape[0]

    def surface_points(self) -> torch.Tensor:
        """Copy of the map's kept G-GPDF training set (float32 (n, 3))."""
        n, x = C.c_int64(), C.c_void_p()
        L.check(L.load().vgp_surface_points(self._h, C.byref(n), C.byref(x)))
        return _view(x.value, (n.value, 3), "<f4", torch.float32)

    def surface_is(self, pts: torch.Tensor) -> bool:
        return self._surface_key == (pts.data_ptr(), tuple(pts.shape), pts._version)

    def query(self, q, grad: bool = True, var: bool = False, out: dict | None = None) -> dict:
        q = _dev_f32(q, "q")
        n = q.shape[0]
        out = out or {}
        d = out.get("d") if out.get("d") is not None else torch.empty(n, dtype=torch.float64, device="cuda")
        g = (out.get("grad") if out.get("grad") is not None else torch.empty((n, 3), dtype=torch.float64, device="cuda")) if grad else None
        v = (out.get("var") if out.get("var") is not None else torch.empty(n, dtype=torch.float64, device="cuda")) if var else None
        s = out.get("status") if out.get("status") is not None else torch.empty(n, dtype=torch.uint8, device="cuda")
        L.check(L.load().vgp_query_distance_gradient(self._h, _ptr(q), n, _ptr(d), _ptr(g), _ptr(v), _ptr(s),
                                                     _stream()))
        return dict(d=d, grad=g, var=v, status=s)

    def query_smooth(self, q, n_nodes: int = 8, lam: float = 100.0, grad: bool = True, var: bool = False) -> dict:
        """G-GPDF as per-leaf GPs blended by the smooth minimum of Eq. 10 (vgp_query_smooth)."""
        q = _dev_f32(q, "q")
        n = q.shape[0]
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        g = torch.empty((n, 3), dtype=torch.float64, device="cuda") if grad else None
        v = torch.empty(n, dtype=torch.float64, device="cuda") if var else None
        s = torch.empty(n, dtype=torch.uint8, device="cuda")
        L.check(L.load().vgp_query_smooth(self._h, _ptr(q), n, int(n_nodes), float(lam), _ptr(d), _ptr(g), _ptr(v),
                                          _ptr(s), _stream()))
        return dict(d=d, grad=g, var=v, status=s)

    def debug_query_plan(self, q) -> dict:
        """Selection of vgp_query_distance_gradient for these queries (vgp_debug_query_plan):
        ``inst_key`` (centre leaf per instance), ``inst_off`` / ``point_idx`` (surface point
        indices per instance) and ``q_inst`` (instance per query, negative if none)."""
        q = _dev_f32(q, "q")
        lib = L.load()
        ni, T = C.c_int64(), C.c_int64()
        L.check(lib.vgp_debug_query_plan(self._h, _ptr(q), q.shape[0], _stream(), C.byref(ni), C.byref(T),
                                         None, None, None, None))
        key = np.zeros(ni.value, np.uint64)
        off = np.zeros(ni.value + 1, np.int64)
        idx = np.zeros(T.value, np.int64)
        qi = np.zeros(q.shape[0], np.int32)
        h = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
        L.check(lib.vgp_debug_query_plan(self._h, _ptr(q), q.shape[0], _stream(), C.byref(ni), C.byref(T), h(key),
                                         h(off), h(idx), h(qi)))
        return dict(inst_key=key, inst_off=off, point_idx=idx, q_inst=qi)

    def debug_smooth_plan(self, q, n_nodes: int = 8) -> dict:
        """Node selection of vgp_query_smooth (vgp_debug_smooth_plan): ``node_key``,
        ``inst_off`` / ``point_idx`` per node GP, and ``pair_inst`` (n, n_nodes) nodes of each
        query nearest first, -1 past the last."""
        q = _dev_f32(q, "q")
        lib = L.load()
        ni, T = C.c_int64(), C.c_int64()
        L.check(lib.vgp_debug_smooth_plan(self._h, _ptr(q), q.shape[0], int(n_nodes), _stream(), C.byref(ni),
                                          C.byref(T), None, None, None, None))
        key = np.zeros(ni.value, np.uint64)
        off = np.zeros(ni.value + 1, np.int64)
        idx = np.zeros(T.value, np.int64)
        pi = np.zeros((q.shape[0], int(n_nodes)), np.int32)
        h = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
        L.check(lib.vgp_debug_smooth_plan(self._h, _ptr(q), q.shape[0], int(n_nodes), _stream(), C.byref(ni),
                                          C.byref(T), h(key), h(off), h(idx), h(pi)))
        return dict(node_key=key, inst_off=off, point_idx=idx, pair_inst=pi)

    def autotune(self, q) -> dict:
        """Pick the fastest launch shape per size bucket on these queries (vgp_autotune)."""
        q = _dev_f32(q, "q")
        L.check(L.load().vgp_autotune(self._h, _ptr(q), q.shape[0], _stream()))
        st = self.stats()
        return {"threads": list(st["cfg_threads"]), "per_sm": list(st["cfg_per_sm"]),
                "stage_panel": int(st["cfg_stage_panel"]), "bucket_ms": list(st["t_bucket_ms"])}

    def set_launch(self, threads, per_sm, stage_panel: int = 1) -> None:
        """Pin the GP solve launch shapes per size bucket (vgp_set_launch)."""
        t = (C.c_int32 * 5)(*[int(x) for x in threads])
        p = (C.c_int32 * 5)(*[int(x) for x in per_sm])
        L.check(L.load().vgp_set_launch(self._h, t, p, int(stage_panel)))

    def query_backward(self, q, dL_dd, want_dq: bool = True, want_dX: bool = True):
        q = _dev_f32(q, "q")
        n = q.shape[0]
        dL_dd = dL_dd.to(device="cuda", dtype=torch.float64).contiguous()
        dq = torch.empty((n, 3), dtype=torch.float64, device="cuda") if want_dq else None
        m = self._surface.shape[0] if self._surface is not None else 0
        dX = torch.empty((m, 3), dtype=torch.float64, device="cuda") if want_dX else None
        L.check(L.load().vgp_query_backward(self._h, _ptr(q), n, _ptr(dL_dd), _ptr(dq), _ptr(dX), _stream()))
        return dq, dX

    # -- independent instances ---------------------------------------------------------
    def gp_batch(self, inst_off, X, q_off, Q, var: bool = True) -> dict:
        inst_off = torch.as_tensor(inst_off, dtype=torch.int64).to("cuda").contiguous()
        q_off = torch.as_tensor(q_off, dtype=torch.int64).to("cuda").contiguous()
        X = _dev_f32(X, "X")
        Q = _dev_f32(Q, "Q")
        n = Q.shape[0]
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        v = torch.empty(n, dtype=torch.float64, device="cuda") if var else None
        s = torch.empty(n, dtype=torch.uint8, device="cuda")
        L.check(L.load().vgp_gp_batch(self._h, inst_off.shape[0] - 1, _ptr(inst_off), _ptr(X), _ptr(q_off), _ptr(Q),
                                      _ptr(d), _ptr(g), _ptr(v), _ptr(s), _stream()))
        return dict(d=d, grad=g, var=v, status=s)

    def stats(self) -> dict:
        st = L.VgpStats()
        L.check(L.load().vgp_get_stats(self._h, C.byref(st)))
        out = {k: getattr(st, k) for k, _ in L.VgpStats._fields_}
        for k in ("bucket_count", "t_bucket_ms", "cfg_threads", "cfg_per_sm"):
            out[k] = list(getattr(st, k))
        return out

    def sync(self):
        L.check(L.load().vgp_sync(self._h))

    def close(self):
        if getattr(self, "_h", None):
            L.load().vgp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
