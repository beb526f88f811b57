"""Independent replicas of the workload, one process per GPU.

The solve does not shard on one box: every rank builds and solves its own
system (weak scaling), so the ranks exchange no field data.  They meet only
on the host, to start the timed region together (barrier) and to report the
slowest rank's time (max over ranks).  The backend is NCCL for GPU runs and
gloo for the CPU tests of this logic.
"""
from __future__ import annotations

import os


class Replicas:
    """Rank/world from the torchrun environment; a process group only when
    WORLD_SIZE > 1."""

    def __init__(self, backend: str = "nccl", device=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v: float) -> float:
        """Maximum of v over all ranks (every rank gets it)."""
        if self.dist is None:
            return float(v)
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64,
                         device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        """Sum of v over all ranks (units processed by the whole job)."""
        if self.dist is None:
            return float(v)
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64,
                         device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None
