"""The sharded N > 1 path on CPU: two gloo ranks.

* G-GPDF over x slabs of leaves (each rank keeps its slab plus a halo of max_leaf_search + 1
  leaves, queries routed to the owner of their leaf and answered there, results routed back):
  every output equals the single-rank oracle's bit for bit, with the surface given whole to
  every rank and with each rank holding only its own part of it.  The scene puts surface near
  the slab boundary, queries on both sides of it, queries whose 27-leaf neighbourhood is empty
  (fallback centre leaf within max_leaf_search) and queries without support.
* Independent instances split by N^3 cost: the all-gathered results equal the single-rank
  oracle's bit for bit.

The per-rank solver is the FP64 oracle; on GPUs the same routing drives the CUDA library.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene():
    from paper_2407_09649_gb300 import scenes
    rng = np.random.default_rng(21)
    sph = scenes.sphere_plane_frame(0, n_sphere=1500, n_plane=0)
    # a 24 m strip of the plane z = -1, longer than two slabs and their halos
    strip = np.c_[rng.uniform(-12, 12, 3000), rng.uniform(-2, 2, 3000), -1 + rng.normal(0, 0.01, 3000)]
    # a sparse cluster of points far above the plane: queries next to it use a fallback
    # centre leaf, queries far from everything have no support
    isl = rng.normal([0.3, 0.2, 3.2], 0.05, (30, 3))
    surf = np.vstack([sph, strip, isl]).astype(np.float32)
    q = np.c_[rng.uniform(-12.5, 12.5, 1200), rng.uniform(-3, 3, 1200), rng.uniform(-3, 4.5, 1200)].astype(np.float32)
    near = isl[rng.integers(0, len(isl), 80)] + rng.normal(0, 0.6, (80, 3)).astype(np.float32)
    q = np.vstack([q, near, [[np.nan, 0.0, 0.0]], [[30.0, 30.0, 30.0]]]).astype(np.float32)
    return surf, q


def _equal_bits(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _run(rank, world, out)
    except Exception:  # report instead of leaving the parent waiting
        import traceback
        out.put({"rank": rank, "error": traceback.format_exc()})
    finally:
        dist.destroy_process_group()


def _run(rank, world, out):
    import torch
    import torch.distributed as dist
    if True:
        import oracle
        from paper_2407_09649_gb300 import scenes, shard
        oracle.set_threads(2)
        P = oracle.params()
        surf, qall = _scene()
        # this rank's queries: an interleaved share of the workload
        myq = qall[rank::world]
        ref = oracle.Surface(surf, P).query(myq, want_var=True)

        def make_solver(local):
            S = oracle.Surface(local.numpy(), P)

            def solve(qq):
                r = S.query(qq.numpy(), want_var=True)
                return {"d": r["d"], "grad": r["grad"], "var": r["var"], "status": r["status"]}
            return solve

        res = {"rank": rank}
        for replicated in (True, False):
            sh = shard.ShardedGGPDF(make_solver, voxel_size=P.voxel_size, max_leaf_search=P.max_leaf_search)
            given = surf if replicated else np.array_split(surf, world)[rank]
            n_local = sh.set_surface(torch.from_numpy(np.ascontiguousarray(given)), replicated=replicated)
            got = sh.query(torch.from_numpy(myq))
            own = shard.owner_of(shard.leaf_x(torch.from_numpy(myq), P.voxel_size), sh.bounds).numpy()
            tag = "repl" if replicated else "dist"
            res[tag] = {"n_local": n_local, "n_surface": len(surf), "routed_away": int((own != rank).sum()),
                        "equal": all(_equal_bits(got[k].numpy(), ref[k]) for k in ("d", "grad", "var"))
                        and np.array_equal(got["status"].numpy(), ref["status"]),
                        "bounds": sh.bounds}
        res["statuses"] = sorted(set(int(s) for s in ref["status"]))
        # independent instances, split by cost
        io, X, qo, Q = scenes.patch_sweep(n_inst=60, seed=9, n_min=4, n_max=300, q_per_inst=8)
        single = oracle.gp_batch(io, X.astype(np.float64), qo, Q.astype(np.float64), P)

        def solve_batch(a, b, c, d):
            r = oracle.gp_batch(a, b.astype(np.float64), c, d.astype(np.float64), P)
            return {"d": r.d, "grad": r.grad, "var": r.var, "status": r.status}

        sb = shard.sharded_gp_batch(solve_batch, io, X, qo, Q)
        cuts = shard.split_by_cost(io, world)
        res["batch_equal"] = (_equal_bits(sb["d"], single.d) and _equal_bits(sb["grad"], single.grad)
                              and _equal_bits(sb["var"], single.var) and np.array_equal(sb["status"], single.status))
        res["batch_cuts"] = cuts.tolist()
        out.put(res)
        dist.barrier()


def test_two_gloo_ranks_sharded_results_equal_single_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([out.get(timeout=600) for _ in procs], key=lambda r: r["rank"])
    for p in procs:
        p.join(timeout=60)
    for r in res:
        assert "error" not in r, r.get("error")
    for p in procs:
        assert p.exitcode == 0
    for r in res:
        for tag in ("repl", "dist"):
            assert r[tag]["equal"], (r["rank"], tag)
            assert r[tag]["n_local"] < r[tag]["n_surface"]  # each rank holds a part of the surface
            assert r[tag]["routed_away"] > 0  # some of its queries were answered by the other rank
        assert r["repl"]["bounds"] == r["dist"]["bounds"]
        assert r["batch_equal"]
    assert res[0]["repl"]["bounds"] == res[1]["repl"]["bounds"]
    assert {0, 1, 3} <= set(res[0]["statuses"]) | set(res[1]["statuses"])  # ok, no support, bad input
    cuts = res[0]["batch_cuts"]
    assert 0 < cuts[1] < cuts[2]  # both ranks got instances


def test_split_by_cost_balances_n_cubed():
    from paper_2407_09649_gb300 import shard
    rng = np.random.default_rng(0)
    N = np.floor(np.exp(rng.uniform(np.log(4), np.log(1025), 5000))).astype(np.int64)
    io = np.concatenate([[0], np.cumsum(N)])
    for world in (2, 4, 8):
        cuts = shard.split_by_cost(io, world)
        assert cuts[0] == 0 and cuts[-1] == len(N) and np.all(np.diff(cuts) >= 0)
        cost = np.array([np.sum(N[a:b].astype(np.float64) ** 3) for a, b in zip(cuts[:-1], cuts[1:])])
        assert cost.max() <= cost.sum() / world + 1025.0 ** 3  # within one instance of even


def test_slab_bounds_split_evenly_and_route_every_leaf():
    import torch
    from paper_2407_09649_gb300 import shard
    rng = np.random.default_rng(1)
    pts = torch.from_numpy(rng.uniform(-20, 20, (20000, 3)).astype(np.float32))
    lx = shard.leaf_x(pts, 0.1)
    b = shard.slab_bounds(lx, 4, collective=False)
    own = shard.owner_of(lx, b)
    share = np.bincount(own.numpy(), minlength=4) / len(pts)
    assert np.all(np.abs(share - 0.25) < 0.02)
    assert b == sorted(b)
    # the leaf index matches the oracle's voxel and leaf convention
    import oracle
    k = oracle.unpack_key(oracle.leaf_key_of_points(pts.numpy(), 0.1))[:, 0]
    assert np.array_equal(k, lx.numpy())
    bad = torch.tensor([[np.nan, 0, 0], [np.inf, 0, 0], [3e38, 0, 0]], dtype=torch.float32)
    assert torch.all((shard.owner_of(shard.leaf_x(bad, 0.1), b) >= 0) & (shard.owner_of(shard.leaf_x(bad, 0.1), b) < 4))
