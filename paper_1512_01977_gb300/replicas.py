"""Replica runs over several GPUs of one node.

The update has no cross-solve arithmetic, so N GPUs run N independent solves
(replicas): there is no data-path collective.  The only communication is the
measurement's barrier and the max over ranks of the timed region, over
torch.distributed (NCCL on GPUs, gloo on CPU).  Rank, world size and the
rendezvous come from the environment torchrun sets (RANK, WORLD_SIZE,
LOCAL_RANK, MASTER_ADDR, MASTER_PORT).
"""
import os


def world():
    """(world_size, rank, local_rank) from the environment (1, 0, 0 when unset)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Replicas:
    """Process-group wrapper: init, barrier, max over ranks, teardown."""

    def __init__(self, backend=None, device=None):
        import torch
        import torch.distributed as dist

        self.dist = dist
        self.ws, self.rank, self.local = world()
        self.device = device
        self.backend = backend or ("nccl" if device is not None and device.type == "cuda" else "gloo")
        self.active = self.ws > 1
        if self.active and not dist.is_initialized():
            kw = {"device_id": device} if self.backend == "nccl" and device is not None else {}
            dist.init_process_group(self.backend, **kw)
        self._torch = torch

    def barrier(self):
        if self.active:
            self.dist.barrier()
        if self.device is not None and self.device.type == "cuda":
            self._torch.cuda.synchronize(self.device)

    def max(self, x):
        """Maximum of a float over all ranks (x itself for one rank)."""
        if not self.active:
            return float(x)
        dev = self.device if self.backend == "nccl" else "cpu"
        t = self._torch.tensor([float(x)], dtype=self._torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.active and self.dist.is_initialized():
            self.dist.destroy_process_group()


def aggregate_rate(units_per_rank, world_size, max_seconds):
    """Whole-job rate: all units every rank processed / the slowest rank's time."""
    return world_size * units_per_rank / max_seconds
