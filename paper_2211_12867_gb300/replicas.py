"""Independent replicas on several GPUs of one node.

The Icarus update does not shard across GPUs here: every rank runs its own
replica of the workload (its own seed), and the ranks only meet to line up
their timed regions and to take the slowest rank's time.  A run's throughput
is the units all ranks processed divided by that time (weak scaling).
"""
from __future__ import annotations

import os


class ReplicaGroup:
    """Rank bookkeeping from the torchrun environment (RANK, WORLD_SIZE,
    LOCAL_RANK); a process group only when WORLD_SIZE > 1."""

    def __init__(self, backend="nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                import torch
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.dist = dist

    @property
    def seed(self):
        """Seed of this rank's replica (its inputs differ from the others')."""
        return self.rank

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x):
        """The largest of the ranks' values of x (every rank gets it)."""
        if self.dist is None:
            return float(x)
        import torch
        dev = f"cuda:{self.local}" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank, seconds_max):
        """Whole-job throughput: units of all ranks over the slowest rank's
        time."""
        return units_per_rank * self.world / seconds_max

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None
