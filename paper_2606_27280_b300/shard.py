"""Entry-range sharding of the exact search across ranks (one process per GPU).

The database is cut into contiguous entry ranges, one per rank.  Each rank holds
an index over its range and answers every query exactly over it; one exchange
step -- an all-gather of the per-rank answers (nq * k * 16 bytes a rank) -- and
the lexicographic merge of hn_merge_topk (similarity descending, global index
ascending: the tie rule of Theorem 2) give the answer over the whole database,
because the exact maximum of Theorem 1 is associative.  Thresholds are not
shared between ranks: each rank's search is exact on its own.

``gather_and_merge`` is the exchange step on its own: device tensors merge with
the library's kernel, host tensors (a gloo group, or results gathered through
host memory) with its host function.  ``ShardedIndex`` puts a local index in
front of it.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import hn


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Entries [lo, hi) of rank `rank` when n entries are cut into `world` contiguous
    ranges of sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    return n * rank // world, n * (rank + 1) // world


def gather_and_merge(local_idx: torch.Tensor, local_sim: torch.Tensor, id_offset: int, group=None,
                     stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """All-gather every rank's (nq, k) answers over its own entries (shard-local int64
    indices, -1 for none; float64 similarities) and its global index offset, then merge.
    Returns the (nq, k) global answers on every rank."""
    if local_idx.dim() != 2 or local_sim.shape != local_idx.shape:
        raise ValueError("local_idx, local_sim: (nq, k)")
    world = dist.get_world_size(group)
    dev = local_idx.device
    idx_parts = [torch.empty_like(local_idx) for _ in range(world)]
    sim_parts = [torch.empty_like(local_sim) for _ in range(world)]
    dist.all_gather(idx_parts, local_idx.contiguous(), group=group)
    dist.all_gather(sim_parts, local_sim.contiguous(), group=group)
    off = torch.tensor([id_offset], dtype=torch.int64, device=dev)
    off_parts = [torch.empty_like(off) for _ in range(world)]
    dist.all_gather(off_parts, off, group=group)
    idx = torch.stack(idx_parts)
    sim = torch.stack(sim_parts)
    offs = torch.cat(off_parts)
    if dev.type == "cuda":
        return hn.merge_topk(idx, sim, offs, stream=stream)
    i, s = hn.merge_topk_host(idx.numpy(), sim.numpy(), offs.numpy())
    return torch.from_numpy(i), torch.from_numpy(s)


class ShardedIndex:
    """This rank's part of an entry-range sharded index.  `x_local` holds the rank's
    HN-normalised entries (rows [id_offset, id_offset + len) of the whole database)."""

    def __init__(self, x_local: torch.Tensor, k: int, alpha: float, id_offset: int, prefix: int = hn.PREFIX_BF16,
                 group=None, stream=None):
        self.index = hn.Index(x_local, k, alpha, prefix=prefix, stream=stream)
        self.n_local = x_local.shape[0]
        self.id_offset = int(id_offset)
        self.group = group

    def search(self, q: torch.Tensor, topk: int = 1, stream=None, **search_kw):
        """Exact top-`topk` of every row of q over the whole sharded database (every rank
        passes the same queries): (idx, sim) of shape (nq, topk), global indices."""
        nq = q.shape[0]
        kk = min(topk, self.n_local)
        if topk == 1:
            r = self.index.search(q, stream=stream, **search_kw)
            li, ls = r.idx.view(nq, 1), r.sim.view(nq, 1)
        else:
            r = self.index.search_topk(q, kk, stream=stream, **search_kw)
            li, ls = r.idx, r.sim
            if kk < topk:   # a shard smaller than k: pad with empty slots
                pad = topk - kk
                li = torch.cat([li, torch.full((nq, pad), -1, dtype=torch.int64, device=q.device)], 1)
                ls = torch.cat([ls, torch.full((nq, pad), float("-inf"), dtype=torch.float64, device=q.device)], 1)
        return gather_and_merge(li, ls, self.id_offset, group=self.group, stream=stream)

    def close(self) -> None:
        self.index.close()
