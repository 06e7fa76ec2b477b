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
    assert C.sizeof(_lib.VgpParams) == 5 * 8 + 8 * 4 and p.profile == 0 and p.normal_steps == 3


def test_create_rejects_bad_params_without_touching_the_gpu(lib):
    import ctypes as C
    from paper_2407_09649_gb300 import _lib
    p = _lib.VgpParams()
    lib.vgp_default_params(C.byref(p))
    p.max_pts_group = 5000
    h = C.c_void_p()
    assert lib.vgp_create(C.byref(p), C.byref(h)) == -1
    assert b"max_pts_group" in lib.vgp_last_error()
    assert lib.vgp_destroy(None) == 0
