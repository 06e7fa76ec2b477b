"""The C ABI library builds, loads and exports every function that include/vgpdf.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vgpdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vgp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2407_09649_gb300 as P
    P.build()
    from paper_2407_09649_gb300 import _lib
    return _lib.load()


def test_header_declares_the_entry_points():
    names = _declared()
    for required in ("vgp_build_frame", "vgp_fuse", "vgp_query_distance_gradient", "vgp_query_backward",
                     "vgp_gp_batch", "vgp_set_surface", "vgp_export_grid", "vgp_import_grid"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2407_09649_gb300 import _lib
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(_declared()) <= bound


def test_param_struct_layout_matches_header(lib):
    import ctypes as C
    from paper_2407_09649_gb300 import _lib
    p = _lib.VgpParams()
    lib.vgp_default_params(C.byref(p))
    assert abs(p.voxel_size - 0.1) < 1e-15 and abs(p.lengthscale - 0.3) < 1e-15
    assert p.max_pts_leaf == 64 and p.max_pts_group == 1024 and p.max_leaf_search == 8
    assert p.precision == _lib.VGP_MIXED and p.fusion == _lib.VGP_FUSE_INVVAR
    assert C.sizeof(_lib.VgpParams) == 5 * 8 + 8 * 4 + 8 + 2 * 4 and p.profile == 0 and p.normal_steps == 3
    assert abs(p.sigma_prop - 0.1) < 1e-15 and p.n_props == 0


def test_create_rejects_bad_params_without_touching_the_gpu(lib):
    import ctypes as C
    from paper_2407_09649_gb300 import _lib
    p = _lib.VgpParams()
    lib.vgp_default_params(C.byref(p))
    p.max_pts_group = 5000
    h = C.c_void_p()
    assert lib.vgp_create(C.byref(p), C.byref(h)) == -1
    assert b"max_pts_group" in lib.vgp_last_error()
    lib.vgp_default_params(C.byref(p))
    p.launch = 3
    assert lib.vgp_create(C.byref(p), C.byref(h)) == -1
    assert b"launch" in lib.vgp_last_error()
    assert lib.vgp_destroy(None) == 0


def _canon(tri):
    """Rotate a triangle so its smallest vertex comes first (orientation kept)."""
    i = tri.index(min(tri))
    return tri[i:] + tri[:i]


def test_marching_cubes_table_matches_the_oracle_face_walk(lib, orc):
    """The library's host-built per-mask triangle table (used by the kernels) gives, for all
    256 inside masks, the same oriented triangles as the oracle's face walk on a single cell."""
    import ctypes as C
    import numpy as np
    tab = (C.c_uint8 * (256 * 16))()
    ntri = (C.c_uint8 * 256)()
    lib.vgp_debug_mc_table(tab, ntri)
    tab = np.frombuffer(tab, np.uint8).reshape(256, 16)
    ntri = np.frombuffer(ntri, np.uint8)
    ijk = np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for mask in range(256):
        lib_tris = []
        for t in range(int(ntri[mask])):
            tri = []
            for j in range(3):
                e = int(tab[mask, 3 * t + j])
                axis = e >> 2
                u, w = (axis + 1) % 3, (axis + 2) % 3
                lc = ((e & 1) << u) | (((e >> 1) & 1) << w)
                tri.append((lc, axis))
            lib_tris.append(_canon(tri))
        D = np.array([-0.5 if (mask >> (x + 2 * y + 4 * z)) & 1 else 0.5 for x, y, z in ijk])
        g = orc.Grid()
        g.fuse(orc.pack_key(ijk), D, np.ones(8), np.zeros(8, np.uint8))
        _, ek, ea = g.mesh(0.1)
        c = orc.unpack_key(ek)
        ref = [_canon([(int(c[t, j, 0] + 2 * c[t, j, 1] + 4 * c[t, j, 2]), int(ea[t, j])) for j in range(3)])
               for t in range(len(ek))]
        assert sorted(lib_tris) == sorted(ref), mask
