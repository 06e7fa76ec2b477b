"""Sharding of the G-GPDF and of independent GP instances over ranks (one process per GPU).

GP instances are independent (Sec. IV-A, IV-D), so the path partitions without changing any
result:

* Maps and G-GPDF queries: spatial slabs of leaves along x.  Rank r owns the leaves whose x
  leaf index lies in [b_r, b_r+1) and keeps the surface points of its slab plus a halo of
  H = max_leaf_search + 1 leaves on each side.  That halo is everything a query of the slab can
  reach: its centre leaf lies within max_leaf_search leaves of the query leaf (Chebyshev), and
  its instance holds the centre leaf's 27-leaf neighbourhood.  Local points keep the global
  order, so the cap's tie-break (lower point index) is unchanged, and every result equals the
  single-rank result bit for bit.  Queries travel to the owner of their leaf in one all-to-all
  and the results come back in a second; the slab bounds split the surface points evenly and
  come from an all-reduced histogram, so every rank derives the same bounds.
* Independent instances (gp_batch): contiguous ranges of instances with equal sums of N^3,
  the factorisation cost; each rank solves its range and the results are all-gathered.

The exchanges use torch.distributed on the tensors' device (CPU tensors with gloo, CUDA
tensors with NCCL).  The per-rank solver is a callable, so the same routing drives the GPU
library or, in tests, the CPU oracle.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import torch
import torch.distributed as dist

# |leaf index| bound used when routing: finite points beyond the voxel range are answered as
# bad input by any rank, so they only need a valid owner
_LEAF_CLAMP = 1 << 40


def leaf_x(points: torch.Tensor, voxel_size: float) -> torch.Tensor:
    """x leaf index floor(floor(x / vs + 1/2) / 8) of float32 points [n, 3], in FP64 with the
    library's rounding (IEEE division, then addition, no contraction); int64, 0 for
    non-finite points."""
    x = points[:, 0].to(torch.float64)
    ijk = torch.floor(x / voxel_size + 0.5)
    ijk = torch.where(torch.isfinite(ijk), ijk, torch.zeros_like(ijk))
    ijk = ijk.clamp(-8.0 * _LEAF_CLAMP, 8.0 * _LEAF_CLAMP).to(torch.int64)
    return torch.div(ijk, 8, rounding_mode="floor")


def slab_bounds(lx: torch.Tensor, world: int, group=None, collective: bool = True) -> list[int]:
    """Bounds b_0 < ... < b_world of the x leaf slabs (b_0 and b_world open), splitting the
    surface points evenly by their x leaf indices lx.  collective=True: lx are this rank's
    points and the histogram is all-reduced over the ranks; False: lx already holds every
    point (each rank derives the same bounds alone)."""
    dev = lx.device
    big = torch.iinfo(torch.int64).max
    lo = torch.tensor([lx.min().item() if lx.numel() else big], dtype=torch.int64, device=dev)
    hi = torch.tensor([lx.max().item() if lx.numel() else -big], dtype=torch.int64, device=dev)
    reduce = collective and world > 1
    if reduce:
        dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
        dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    lo, hi = int(lo.item()), int(hi.item())
    if lo > hi:  # no surface anywhere: everything goes to rank 0
        return [-_LEAF_CLAMP] + [_LEAF_CLAMP] * world
    hist = torch.bincount(lx - lo, minlength=hi - lo + 1).to(torch.int64)
    if reduce:
        dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    cum = torch.cumsum(hist, 0).cpu().numpy()
    total = int(cum[-1])
    bounds = [-_LEAF_CLAMP]
    for r in range(1, world):
        # the slab of rank r - 1 ends after the first leaf column at which the cumulative
        # count reaches r / world of the points
        k = int(np.searchsorted(cum, (total * r + world - 1) // world, side="left"))
        bounds.append(max(lo + k + 1, bounds[-1]))
    bounds.append(_LEAF_CLAMP)
    return bounds


def owner_of(lx: torch.Tensor, bounds: list[int]) -> torch.Tensor:
    """Rank owning each x leaf index: the r with bounds[r] <= lx < bounds[r + 1]."""
    b = torch.tensor(bounds[1:-1], dtype=torch.int64, device=lx.device)
    return torch.bucketize(lx, b, right=True)


def _exchange(x: torch.Tensor, send_counts: list[int], group=None) -> tuple[torch.Tensor, list[int]]:
    """all-to-all of the rows of x (grouped by destination rank in rank order); returns the
    received rows (grouped by source rank in rank order) and the receive counts."""
    world = len(send_counts)
    sc = torch.tensor(send_counts, dtype=torch.int64, device=x.device)
    rc = torch.empty_like(sc)
    dist.all_to_all_single(rc, sc, group=group)
    recv_counts = [int(v) for v in rc.tolist()]
    out = x.new_empty((sum(recv_counts),) + tuple(x.shape[1:]))
    dist.all_to_all_single(out, x.contiguous(), output_split_sizes=recv_counts, input_split_sizes=send_counts,
                           group=group)
    assert world == dist.get_world_size(group)
    return out, recv_counts


class ShardedGGPDF:
    """G-GPDF distance queries over a surface partitioned in x slabs of leaves.

    ``make_solver(points)`` builds the rank's local solver from its slab + halo of surface
    points (float32 [m, 3], global order); the solver maps query points (float32 [n, 3]) to a
    dict of d [n], grad [n, 3], var [n] (or None) and status [n], as
    ``vgp_query_distance_gradient`` does.
    """

    def __init__(self, make_solver: Callable, voxel_size: float = 0.1, max_leaf_search: int = 8, group=None):
        self.make_solver = make_solver
        self.vs = float(voxel_size)
        self.halo = int(max_leaf_search) + 1
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.bounds = None
        self.solver = None
        self.n_local = 0

    def set_surface(self, points: torch.Tensor, replicated: bool = True) -> int:
        """Partition the surface.  replicated=True: every rank passes the whole surface and
        keeps its slab + halo.  replicated=False: every rank passes its own points (the global
        surface is the rank-major concatenation) and the points travel to every rank whose
        slab + halo holds them.  Returns the number of local points.  Collective."""
        lx = leaf_x(points, self.vs)
        if replicated:
            self.bounds = slab_bounds(lx, self.world, collective=False)
            lo, hi = self.bounds[self.rank] - self.halo, self.bounds[self.rank + 1] + self.halo
            keep = (lx >= lo) & (lx < hi)
            local = points[keep]
        else:
            self.bounds = slab_bounds(lx, self.world, self.group)
            order, counts = [], []
            for r in range(self.world):
                lo, hi = self.bounds[r] - self.halo, self.bounds[r + 1] + self.halo
                sel = torch.nonzero((lx >= lo) & (lx < hi)).flatten()
                order.append(sel)
                counts.append(int(sel.numel()))
            local = points if self.world == 1 else _exchange(points[torch.cat(order)], counts, self.group)[0]
        self.n_local = int(local.shape[0])
        self.solver = self.make_solver(local)
        return self.n_local

    def query(self, q: torch.Tensor) -> dict:
        """Answer the rank's queries q (float32 [n, 3]); every rank calls this (collective)."""
        if self.world == 1:
            res = self.solver(q)
            return {"d": torch.as_tensor(res["d"]), "grad": torch.as_tensor(res["grad"]),
                    "var": None if res.get("var") is None else torch.as_tensor(res["var"]),
                    "status": torch.as_tensor(res["status"]).to(torch.uint8)}
        own = owner_of(leaf_x(q, self.vs), self.bounds)
        perm = torch.argsort(own, stable=True)
        counts = torch.bincount(own, minlength=self.world).tolist()
        recv, rcounts = _exchange(q[perm], counts, self.group)
        res = self.solver(recv)
        n = recv.shape[0]
        packed = torch.empty((n, 6), dtype=torch.float64, device=q.device)
        packed[:, 0] = torch.as_tensor(res["d"], device=q.device)
        packed[:, 1:4] = torch.as_tensor(res["grad"], device=q.device).reshape(n, 3)
        var = res.get("var")
        packed[:, 4] = torch.as_tensor(var, device=q.device) if var is not None else float("nan")
        packed[:, 5] = torch.as_tensor(res["status"], device=q.device).to(torch.float64)
        back, _ = _exchange(packed, rcounts, self.group)
        out = torch.empty_like(back)
        out[perm] = back
        return {"d": out[:, 0].contiguous(), "grad": out[:, 1:4].contiguous(),
                "var": out[:, 4].contiguous() if var is not None else None, "status": out[:, 5].to(torch.uint8)}


def split_by_cost(inst_off: np.ndarray, world: int) -> np.ndarray:
    """Instance bounds c_0 = 0 <= ... <= c_world = n_inst of contiguous ranges with about equal
    sums of N^3 (the Cholesky cost), from the instance offsets (int64 [n_inst + 1])."""
    N = np.diff(np.asarray(inst_off, dtype=np.int64)).astype(np.float64)
    cost = np.cumsum(N ** 3)
    total = cost[-1] if len(cost) else 0.0
    cuts = [0]
    for r in range(1, world):
        cuts.append(max(int(np.searchsorted(cost, total * r / world, side="left")) + 1, cuts[-1]))
    cuts.append(len(N))
    return np.minimum(np.array(cuts, dtype=np.int64), len(N))


def sharded_gp_batch(solve: Callable, inst_off: np.ndarray, X: np.ndarray, q_off: np.ndarray, Q: np.ndarray,
                     group=None) -> dict:
    """Independent instances split by cost over the ranks: rank r solves instances
    [c_r, c_r+1) with ``solve(inst_off, X, q_off, Q) -> dict(d, grad, var, status)`` (arrays
    of its queries) and the per-query results of all ranks are all-gathered in instance order.
    Every rank passes the same full batch.  Collective."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    cuts = split_by_cost(inst_off, world)
    a, b = int(cuts[rank]), int(cuts[rank + 1])
    io = np.asarray(inst_off[a:b + 1], dtype=np.int64)
    qo = np.asarray(q_off[a:b + 1], dtype=np.int64)
    res = solve(io - io[0], X[io[0]:io[-1]], qo - qo[0], Q[qo[0]:qo[-1]])
    n = int(qo[-1] - qo[0])
    packed = torch.empty((n, 6), dtype=torch.float64)
    packed[:, 0] = torch.as_tensor(np.asarray(res["d"], dtype=np.float64))
    packed[:, 1:4] = torch.as_tensor(np.asarray(res["grad"], dtype=np.float64).reshape(n, 3))
    var = res.get("var")
    packed[:, 4] = torch.as_tensor(np.asarray(var, dtype=np.float64)) if var is not None else float("nan")
    packed[:, 5] = torch.as_tensor(np.asarray(res["status"]).astype(np.float64))
    sizes = [int(q_off[cuts[r + 1]] - q_off[cuts[r]]) for r in range(world)]
    if world > 1:  # all-gather padded to the largest share, then trimmed
        m = max(sizes)
        pad = torch.zeros((m, 6), dtype=torch.float64)
        pad[:n] = packed
        gathered = [torch.empty((m, 6), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, pad, group=group)
        allp = torch.cat([g[:sz] for g, sz in zip(gathered, sizes)])
    else:
        allp = packed
    return {"d": np.ascontiguousarray(allp[:, 0].numpy()), "grad": np.ascontiguousarray(allp[:, 1:4].numpy()),
            "var": np.ascontiguousarray(allp[:, 4].numpy()) if var is not None else None,
            "status": allp[:, 5].numpy().astype(np.uint8)}
