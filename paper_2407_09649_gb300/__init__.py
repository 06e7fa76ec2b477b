"""GB300-native batched local Gaussian-process distance fields (the data-parallel hot path of
VDB-GPDF, arXiv 2407.09649): a C-ABI CUDA library (``include/vgpdf.h``, ``libvgpdf.so``) and
a thin Python binding.

    from paper_2407_09649_gb300 import Map
    m = Map(precision="mixed")
    f = m.build_frame(points)        # L-GPDF of one frame
    m.fuse(f)                        # probabilistic fusion into the global grid
    m.set_surface(surface_points)    # G-GPDF training set
    out = m.query(q, grad=True, var=True)
"""
from .build import build  # noqa: F401


def __getattr__(name):
    # torch-dependent parts load lazily so that ``build`` works without a GPU
    if name in ("Map", "Frame", "make_params"):
        from . import api
        return getattr(api, name)
    if name in ("gpdf_distance", "GPDFDistance"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
