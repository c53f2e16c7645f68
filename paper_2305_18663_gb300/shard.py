"""Sharded nodal pass over several ranks (EDiSt, Section III-B, Alg. 5).

Every rank holds a replica of the graph, the assignment b and the blockmodel
M.  Each rank decides a disjoint set of vertices against the frozen (b, M),
the ranks exchange the new labels (one allgather, 4 bytes per vertex in
total), and every rank applies the full set of decisions to its replica.
Because a decision depends only on the frozen state and on the Philox
counter (sweep_id, v), the result is the single-rank sweep bit for bit, for
any number of ranks.

The degree-balanced dealing of Section III-B (vertices sorted by degree, cut
into chunks of 2 x world, rank r taking the r-th highest and the r-th lowest
of each chunk) gives each rank a scattered vertex set.  `dealt_order` turns it
into contiguous ranges by relabelling the vertices once, so that each rank's
pass is one `sbp_nodal_decide` over [lo, hi) and its slice of the exchange is
contiguous.

The merge phase is not sharded: a rank computes every block's merge
proposals itself (their draws are keyed by round and block, so all ranks
agree without an exchange).

The exchange runs on `torch.distributed` with whatever backend the process
group has (NCCL with device tensors, gloo with host tensors).
"""

from __future__ import annotations

import numpy as np

__all__ = ["deal_vertices", "dealt_order", "relabel_edges", "allgather_slices", "sharded_sweep"]


def deal_vertices(degrees: np.ndarray, world: int, rank: int) -> np.ndarray:
    """Vertex ids a rank handles in a sharded nodal pass (Section III-B):
    vertices sorted by degree are cut into chunks of 2*world; rank r takes
    the r-th highest and the r-th lowest of each chunk."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = np.argsort(-np.asarray(degrees), kind="stable")
    n = order.size
    pos = np.arange(n)
    chunk_pos = pos % (2 * world)
    mine = (chunk_pos == rank) | (chunk_pos == 2 * world - 1 - rank)
    return np.sort(order[mine])


def dealt_order(degrees: np.ndarray, world: int) -> tuple[np.ndarray, list[tuple[int, int]]]:
    """Relabelling that makes each rank's dealt set one contiguous range.

    Returns (new_to_old, ranges): vertex new_to_old[i] of the input graph
    becomes vertex i; rank r owns the new ids [ranges[r][0], ranges[r][1]).
    Within a rank the vertices keep their ascending original order."""
    parts = [deal_vertices(degrees, world, r) for r in range(world)]
    new_to_old = np.concatenate(parts).astype(np.int64) if parts else np.zeros(0, np.int64)
    ranges, lo = [], 0
    for p in parts:
        ranges.append((lo, lo + p.size))
        lo += p.size
    return new_to_old, ranges


def relabel_edges(src: np.ndarray, dst: np.ndarray, new_to_old: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Edge list of the relabelled graph (same edge order)."""
    old_to_new = np.empty_like(new_to_old)
    old_to_new[new_to_old] = np.arange(new_to_old.size)
    return old_to_new[np.asarray(src)].astype(np.int32), old_to_new[np.asarray(dst)].astype(np.int32)


def allgather_slices(local, ranges: list[tuple[int, int]], group=None):
    """All ranks' slices concatenated in rank order (the exchange of Alg. 5).

    local: this rank's slice (a 1-D torch tensor of length hi - lo of its
    range).  Slices may have different lengths, including zero: each is
    padded to the longest before the collective."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if len(ranges) != world:
        raise ValueError("one range per rank")
    lo, hi = ranges[rank]
    if local.ndim != 1 or local.numel() != hi - lo:
        raise ValueError("local slice does not match this rank's range")
    width = max(h - l for l, h in ranges)
    buf = torch.zeros(max(width, 1), dtype=local.dtype, device=local.device)
    buf[: local.numel()] = local
    out = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    return torch.cat([out[r][: h - l] for r, (l, h) in enumerate(ranges)])


def sharded_sweep(model, sweep_id: int, ranges: list[tuple[int, int]], group=None, stats: bool = False):
    """One nodal pass with this rank deciding its range, the new labels
    exchanged, and the full set applied to this rank's replica."""
    import torch
    import torch.distributed as dist

    from . import sbp_commit, sbp_get_pending, sbp_nodal_decide, sbp_set_pending

    rank = dist.get_rank(group)
    lo, hi = ranges[rank]
    n = ranges[-1][1]
    if n != model.g.n:
        raise ValueError("ranges must cover the graph")
    dev = torch.device("cuda", torch.cuda.current_device())
    sbp_nodal_decide(model.h, sweep_id, lo, hi)
    # gloo gathers host tensors, NCCL device tensors
    host = dist.get_backend(group) == "gloo"
    mine = torch.empty(hi - lo, dtype=torch.int32, device="cpu" if host else dev)
    sbp_get_pending(model.h, lo, hi, mine)  # synchronous: the labels are in place on return
    full = allgather_slices(mine, ranges, group)
    if not host:
        torch.cuda.current_stream(dev).synchronize()  # the model may run on another stream
    sbp_set_pending(model.h, 0, n, full)
    return sbp_commit(model.h, stats=stats)
