"""vgp_gp_batch_static: the batched GP solve for callers that cannot allocate device memory
(a fixed memory budget, a real-time loop that must not enter the allocator).  It keeps all
its scratch in one static device array inside the library.

Checks, through the C ABI, that two calls in a row give the same results as the allocating
entry point vgp_gp_batch (within the parity tolerances used elsewhere), and that sizes beyond
the documented maximum are refused with a clear error.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _call_static(lib, L, params, inst_off, X, q_off, Q, want_var=True):
    io = torch.as_tensor(inst_off, dtype=torch.int64).cuda()
    qo = torch.as_tensor(q_off, dtype=torch.int64).cuda()
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Qd = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).cuda()
    n = Qd.shape[0]
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    v = torch.empty(n, dtype=torch.float64, device="cuda") if want_var else None
    s = torch.empty(n, dtype=torch.uint8, device="cuda")
    p = lambda t: None if t is None else C.c_void_p(t.data_ptr())  # noqa: E731
    rc = lib.vgp_gp_batch_static(C.byref(params), io.shape[0] - 1, p(io), p(Xd), p(qo), p(Qd), p(d), p(g), p(v), p(s),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        return rc, None
    torch.cuda.synchronize()
    return rc, dict(d=d.cpu().numpy(), grad=g.cpu().numpy(), var=None if v is None else v.cpu().numpy(),
                    status=s.cpu().numpy())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_static_batch_matches_allocating_batch_twice(precision):
    import paper_2407_09649_gb300 as P
    P.build()
    from paper_2407_09649_gb300 import _lib as L, scenes
    from paper_2407_09649_gb300.api import Map, make_params
    lib = L.load()
    params = make_params(precision=precision)
    m = Map(precision=precision)
    for seed in (31, 32):  # two calls in a row share the static scratch
        inst_off, X, q_off, Q = scenes.patch_sweep(n_inst=3000, seed=seed, n_min=1, n_max=64, q_per_inst=40)
        Q[5] = np.nan
        rc, got = _call_static(lib, L, params, inst_off, X, q_off, Q)
        assert rc == 0, L.load().vgp_last_error()
        ref = m.gp_batch(inst_off, X, q_off, Q, var=True)
        ref = {k: t.cpu().numpy() for k, t in ref.items()}
        assert np.array_equal(got["status"], ref["status"])
        ok = ref["status"] == 0
        assert np.abs(got["d"][ok] - ref["d"][ok]).max() <= 1e-9
        np.testing.assert_allclose(got["grad"][ok], ref["grad"][ok], rtol=1e-9, atol=1e-12)
        fin = ok & np.isfinite(ref["var"])
        np.testing.assert_allclose(got["var"][fin], ref["var"][fin], rtol=1e-9, atol=1e-15)
        assert got["status"][5] == L.ST_BAD_INPUT


def test_static_batch_refuses_oversize():
    import paper_2407_09649_gb300 as P
    P.build()
    from paper_2407_09649_gb300 import _lib as L
    from paper_2407_09649_gb300.api import make_params
    lib = L.load()
    params = make_params()
    X = np.zeros((65, 3), np.float32)
    rc, _ = _call_static(lib, L, params, [0, 65], X, [0, 1], np.zeros((1, 3), np.float32))
    assert rc == -1 and b"more than 64 points" in lib.vgp_last_error()
    rc, _ = _call_static(lib, L, params, np.zeros(70000, np.int64), np.zeros((1, 3), np.float32),
                         np.zeros(70000, np.int64), np.zeros((1, 3), np.float32))
    assert rc == -1 and b"instances exceed" in lib.vgp_last_error()
    # a negative first offset is refused before any point is read
    rc, _ = _call_static(lib, L, params, [-5, 3], np.zeros((3, 3), np.float32), [0, 1], np.zeros((1, 3), np.float32))
    assert rc == -1 and b"negative, decreasing" in lib.vgp_last_error()
