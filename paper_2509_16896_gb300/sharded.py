"""One filter on several devices: target rows split across the ranks of a process group,
the source set replicated (include/yy.h, the section on one filter across several devices).

Per step every rank predicts its rows against all nodes, updates them (yy_update_shard),
exchanges its rows' log-weights and its record with every other rank (two all-gathers:
n_pad values and G x (2r + 4) doubles), merges (yy_merge_shards; every rank computes the same
result from the same gathered buffers) and restarts redundantly.  The arithmetic is in the
library; this module only moves buffers.
"""
from __future__ import annotations

from . import binding


def exchange(rows, record, dist):
    """All-gathers every rank's rows (equal chunks, rank order) and records; returns
    (rows of all ranks concatenated, records stacked [G][2r + 4])."""
    import torch
    G = dist.get_world_size()
    rows_list = [torch.empty_like(rows) for _ in range(G)]
    rec_list = [torch.empty_like(record) for _ in range(G)]
    dist.all_gather(rows_list, rows)
    dist.all_gather(rec_list, record)
    return torch.cat(rows_list), torch.stack(rec_list)


class ShardedFilter:
    """A filter handle on this rank's device, owning chunk `rank` of `world size` of the
    target rows."""

    def __init__(self, cfg, dist, device: str, stream=None):
        import torch
        self.torch = torch
        self.dist = dist
        self.G = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0
        self.f = binding.Filter(cfg, device=device, stream=stream)
        self.f.set_shard(self.rank, self.G)
        _, chunk = self.f.shard_rows()
        dt = torch.float64 if self.f.fp64 else torch.float32
        self.rows = torch.empty(chunk, dtype=dt, device=device)
        self.record = torch.empty(2 * cfg.r + 4, dtype=torch.float64, device=device)

    def init_nodes(self, poly, scramble, center, halfwidth=None) -> None:
        self.f.init_nodes(poly, scramble, center, halfwidth)
        self.f.set_shard(self.rank, self.G)   # work list of this shard's tiles

    def step(self, dy_dev, restart: bool = True) -> None:
        """One filter step: prediction, shard update, exchange, merge, automatic restart."""
        self.f.predict()
        self.f.update_shard(dy_dev, self.rows, self.record)
        with self.torch.cuda.stream(self.f.stream):
            if self.dist is not None and self.G > 1:
                rows_all, recs = exchange(self.rows, self.record, self.dist)
            else:
                rows_all, recs = self.rows, self.record.view(1, -1)
        self.f.merge_shards(rows_all, recs, self.G)
        if restart:
            self.f.restart(binding.RESTART_AUTO)

    def estimate(self):
        return self.f.estimate()
