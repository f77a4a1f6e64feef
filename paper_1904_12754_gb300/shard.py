"""Sharded solves over torch.distributed: the exchange of mlmc_plan_set_shard.

Every rank holds the whole plan and walks its part of each level's new walk
indices (mlmc_shard_range); before each controller decision the library
calls the exchange, which sums the ranks' per-level row sums and totals in
place.  Here that sum is one torch.distributed all-reduce: NCCL on a device
buffer, or gloo on a host buffer.  This module only marshals the buffer and
the callback; the walks, the sums and the decisions run in the library.
"""
from __future__ import annotations

from . import mlmc as M


class DistExchange:
    """The exchange buffer and callback for one plan (or a fixed size).

    group: a torch.distributed process group (None: the default group).
    device: where the buffer lives; None picks "cuda" for the NCCL backend and
    "cpu" otherwise.  count: buffer size in doubles (default: the plan's
    mlmc_shard_buffer_doubles)."""

    def __init__(self, plan=None, group=None, device=None, count: int = None):
        import torch
        import torch.distributed as dist
        self._dist = dist
        self._group = group
        if device is None:
            device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        if count is None:
            count = plan.shard_buffer_doubles()
        self.buf = torch.zeros(int(count), dtype=torch.float64, device=device)
        self.failures = 0

        def _exchange(n, _ctx):
            try:
                view = self.buf[:n]
                self._dist.all_reduce(view, op=self._dist.ReduceOp.SUM, group=self._group)
                if view.is_cuda:
                    torch.cuda.current_stream().synchronize()
                return 0
            except Exception:  # reported to the library as a failed exchange
                self.failures += 1
                return 1

        self.callback = M.EXCHANGE_FN(_exchange)
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        if plan is not None:
            self.attach(plan)

    def attach(self, plan):
        """Make `plan` this rank's shard of the solve."""
        plan.set_shard(self.rank, self.world, self.callback, self.buf)
