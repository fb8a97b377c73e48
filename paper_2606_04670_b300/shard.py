"""Evaluation over several GPUs, one process per GPU (torch.distributed: NCCL between GPUs,
gloo for the multi-process CPU tests).

The paper's reductions shard naturally (Sec. 5: O(N) independent work per query, N^2 for the
Lipschitz constant, nothing stored per pair):

* Query-sharded evaluation (data replicated): each rank evaluates its slice of the queries
  with lip_eval; there is no exchange beyond collecting the outputs (``gather_outputs``).
* Data-sharded evaluation (each rank holds a slice of the data, e.g. when N is too large
  for one GPU): ``eval_data_sharded`` runs the library's per-rank steps around two
  exchanges: one all-reduce MIN of packed 64-bit keys (FP32 bound value, then global data
  index), then the owner of each winner re-evaluates it in FP64 and one all-reduce MIN /
  MAX spreads the exact bounds.  The result equals single-GPU lip_eval bit for bit.
* Lipschitz-constant estimate with the data replicated: the tile pairs of the N^2/2 pair
  triangle are shared out block-cyclically (lip_estimate_M_part), and one all_gather of
  each rank's 4-number result lets every rank pick the winner with lip_estimate_M's rule.

The per-rank steps are methods of a "shard" object, so the same exchange code drives the
CUDA library (``DeviceShard``) and the tests' host-side stand-ins.  No kernel of one rank
ever waits on another rank: all waiting happens inside the collectives.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

NO_KEY = (1 << 63) - 1          # key of "no candidate" (INT64_MAX)


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[begin, end) of rank's contiguous share of n items (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    return n * rank // world, n * (rank + 1) // world


class DeviceShard:
    """This rank's slice of the data in a LipFit handle, whose first point has global index
    ``index_base``: the per-rank steps of the data-sharded evaluation and of the shared
    estimate, on this process's GPU."""

    def __init__(self, model, index_base: int):
        self.model = model
        self.index_base = int(index_base)

    def scan(self, Q):
        return self.model.shard_scan(Q, self.index_base)

    def reeval(self, Q, key_up, key_lo):
        return self.model.shard_reeval(Q, self.index_base, key_up, key_lo)

    def finish(self, key_up, key_lo, hi64, lo64) -> Dict:
        return self.model.shard_finish(key_up, key_lo, hi64, lo64)

    def estimate_part(self, part: int, nparts: int) -> List[float]:
        return self.model.estimate_M_part(part, nparts)


def _dist():
    import torch.distributed as dist
    return dist


def eval_data_sharded(shard, Q, group=None) -> Dict:
    """g, lo, hi, idx_up, idx_lo (global indices) of every query Q (the same Q on every
    rank) over the union of the ranks' data.  Every rank returns the full outputs."""
    import torch
    dist = _dist()
    key_up, key_lo = shard.scan(Q)
    keys = torch.stack([key_up, key_lo])
    dist.all_reduce(keys, op=dist.ReduceOp.MIN, group=group)
    hi64, lo64 = shard.reeval(Q, keys[0], keys[1])
    dist.all_reduce(hi64, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(lo64, op=dist.ReduceOp.MAX, group=group)
    return shard.finish(keys[0], keys[1], hi64, lo64)


def gather_outputs(out: Dict, counts: Sequence[int], dst: int = 0, group=None):
    """Query-sharded evaluation's collection step: rank r's outputs (counts[r] queries each)
    concatenated in rank order on rank ``dst`` (None on the others).  Uses all_gather of
    equal-sized (padded) buffers, which every backend provides."""
    import torch
    dist = _dist()
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if len(counts) != world:
        raise ValueError("one count per rank")
    width = max(max(counts), 1)
    result = {}
    for k in sorted(out):
        t = out[k]
        pad = torch.zeros((width,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[: t.shape[0]] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        if rank == dst:
            result[k] = torch.cat([parts[r][: counts[r]] for r in range(world)])
    return result if rank == dst else None


def _better(a: Sequence[float], b: Sequence[float]) -> bool:
    """lip_estimate_M's order of candidates [M, i, j, key]: a part without a pair (i < 0)
    loses; then the larger key (the part's exact FP64 maximum); then the lower i, then the
    lower j."""
    if b[1] < 0:
        return a[1] >= 0
    if a[1] < 0:
        return False
    if a[3] != b[3]:
        return a[3] > b[3]
    if a[1] != b[1]:
        return a[1] < b[1]
    return a[2] < b[2]


def estimate_M_sharded(shard, group=None, device=None) -> Tuple[float, int, int]:
    """(M_est, i, j) over all pairs, each rank computing its block-cyclic share (the data
    replicated on every rank); equal to lip_estimate_M on one GPU bit for bit."""
    import torch
    dist = _dist()
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    mine = torch.tensor(shard.estimate_part(rank, world), dtype=torch.float64, device=device)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    best = [0.0, -1.0, -1.0, -1.0]
    for p in parts:
        c = p.tolist()
        if _better(c, best):
            best = c
    return best[0], int(best[1]), int(best[2])
