"""Differentiation through G-GPDF at the room-map size: a torch.autograd.Function over
vgp_query_distance_gradient / vgp_query_backward on 256 trajectories x 64 waypoints,
loss = sum softplus(0.5 m - d).  Checked against the FP64 oracle's backward pass (exact
derivative of the same discrete structure) and against central finite differences of the
GPU forward (FP64 path, steps h = 1e-4 m and h/2 combined by Richardson extrapolation) on
waypoint and surface coordinates away from voxel boundaries."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _far_from_voxel_boundary(x, vs=0.1, margin=2e-3):
    f = x / vs + 0.5
    return np.abs(f - np.round(f)) * vs > margin


@pytest.fixture(scope="module")
def room_case():
    import paper_2407_09649_gb300 as P
    P.build()
    from paper_2407_09649_gb300 import scenes
    room = scenes.Room(0)
    X = room.surface_samples(seed=0, density=100.0)
    W = room.trajectories(seed=2).reshape(-1, 3)
    return X, W


def test_backward_matches_oracle_at_room_size(room_case, orc):
    from paper_2407_09649_gb300.api import Map
    from paper_2407_09649_gb300.autograd import gpdf_distance
    X, W = room_case
    m = Map(precision="fp64")
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    d = gpdf_distance(Wt, Xt, m)
    loss = torch.nn.functional.softplus(0.5 - d).sum()
    loss.backward()
    S = orc.Surface(X, orc.params())
    ref = S.query(W, want_var=False)
    ok = ref["status"] == 0
    assert ok.mean() > 0.99
    np.testing.assert_allclose(d.detach().cpu().numpy()[ok], ref["d"][ok], rtol=0, atol=1e-4)
    w = -1.0 / (1.0 + np.exp(-(0.5 - ref["d"])))
    rdq, rdX = S.backward(W, w)
    gq = Wt.grad.cpu().numpy()
    gX = Xt.grad.cpu().numpy()
    np.testing.assert_allclose(gq, rdq, rtol=1e-5, atol=1e-7)
    # 10,000 surface points among those the waypoints' neighbourhoods touch
    touched = np.flatnonzero(np.abs(rdX).sum(1) > 0)
    rng = np.random.default_rng(3)
    sel = rng.choice(touched, min(10_000, len(touched)), replace=False)
    np.testing.assert_allclose(gX[sel], rdX[sel], rtol=1e-5, atol=1e-7 * np.abs(rdX).max())


def _central(f, A, i, a, h):
    Ap, Am = A.copy(), A.copy()
    Ap[i, a] += h
    Am[i, a] -= h
    step = float(Ap[i, a]) - float(Am[i, a])
    return (f(Ap) - f(Am)) / step, step / 2


def _richardson(f, A, i, a, h):
    """Central differences at h and h/2 (float32 coordinates, so the actual steps are used)
    combined to cancel the h^2 truncation term.  None when the two disagree grossly, which
    means a step crossed a discrete change (leaf membership or the nearest-first cap)."""
    d1, s1 = _central(f, A, i, a, h)
    d2, s2 = _central(f, A, i, a, h / 2)
    if abs(d1 - d2) > 1e-2 * max(1.0, abs(d1)):
        return None
    return (s1 * s1 * d2 - s2 * s2 * d1) / (s1 * s1 - s2 * s2)


def test_gradients_match_central_differences(room_case):
    from paper_2407_09649_gb300.api import Map
    X, W = room_case
    m = Map(precision="fp64")
    Xt = torch.from_numpy(X).cuda()
    Wt = torch.from_numpy(W).cuda()

    def loss_of(Wq, Xs):
        m.set_surface(Xs)
        d = m.query(Wq, grad=False, var=False)["d"]
        return float(torch.nn.functional.softplus(0.5 - d).sum().item()), d

    L0, d0 = loss_of(Wt, Xt)
    w = (-torch.sigmoid(0.5 - d0)).double()
    m.set_surface(Xt)
    dq, dX = m.query_backward(Wt, w)
    dq, dX = dq.cpu().numpy(), dX.cpu().numpy()
    rng = np.random.default_rng(4)
    h = 1e-4
    checked = 0
    for i in rng.choice(len(W), 64, replace=False):
        a = int(rng.integers(3))
        if not _far_from_voxel_boundary(W[i, a]):
            continue
        fd = _richardson(lambda Wq: loss_of(torch.from_numpy(Wq).cuda(), Xt)[0], W, i, a, h)
        if fd is None:
            continue
        assert abs(fd - dq[i, a]) <= 2e-4 * max(1.0, abs(fd)), (i, a, fd, dq[i, a])
        checked += 1
    touched = np.flatnonzero(np.abs(dX).sum(1) > 1e-6)
    for j in rng.choice(touched, 48, replace=False):
        a = int(rng.integers(3))
        if not _far_from_voxel_boundary(X[j, a]):
            continue
        fd = _richardson(lambda Xs: loss_of(Wt, torch.from_numpy(Xs).cuda())[0], X, j, a, h)
        if fd is None:
            continue
        assert abs(fd - dX[j, a]) <= 2e-4 * max(1.0, abs(fd)) + 1e-5, (j, a, fd, dX[j, a])
        checked += 1
    assert checked >= 50
