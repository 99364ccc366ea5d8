"""Host-side helpers for running the march on several GPUs of one node.

Solves are independent (every batch row -- photon energy, incidence angle,
request -- marches alone, and z is sequential within a row), so several
GPUs either run independent replicas or split the rows of a batch; no step
of the march exchanges data between GPUs.  What crosses ranks is host-side
bookkeeping only: a barrier around timed regions, the maximum of the ranks'
times, and, when a batch is split, gathering the rows' results to rank 0.

One process per GPU, launched by torchrun (RANK / WORLD_SIZE / MASTER_*
from the environment); NCCL when the tensors live on a GPU, gloo on the
host (the CPU tests run two gloo ranks).
"""

from __future__ import annotations

import os

import numpy as np


def shard(n_rows: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced share [begin, end) of ``n_rows`` rows for
    ``rank`` of ``world``: the first n_rows % world ranks take one extra."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_rows, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


class Ranks:
    """World view of one process: rank, size, barrier, reductions, gather."""

    def __init__(self, backend: str | None = None, device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend or ("nccl" if device is not None else "gloo"))
            self.dist = dist

    def _tensor(self, values, dtype):
        import torch
        t = torch.as_tensor(np.asarray(values), dtype=dtype)
        return t.to(self.device) if self.device is not None else t

    def barrier(self, sync=None):
        """Barrier across ranks; ``sync`` (e.g. torch.cuda.synchronize) runs
        on both sides so that no device work straddles it."""
        if sync is not None:
            sync()
        if self.dist is not None:
            self.dist.barrier()
        if sync is not None:
            sync()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = self._tensor([x], torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = self._tensor([x], torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def gather_rows(self, local: np.ndarray, n_rows: int) -> np.ndarray | None:
        """Reassemble a batch split by ``shard``: every rank passes its rows
        (leading axis), rank 0 receives all ``n_rows`` in row order, the
        other ranks None."""
        local = np.ascontiguousarray(local)
        if self.dist is None:
            return local
        import torch
        b, e = shard(n_rows, self.rank, self.world)
        if local.shape[0] != e - b:
            raise ValueError("local rows do not match this rank's shard")
        width = -(-n_rows // self.world)                  # rows of the largest shard
        tail = local.shape[1:]
        view = local.view(np.float64) if np.iscomplexobj(local) else local.astype(np.float64)
        pad = np.zeros((width,) + view.shape[1:], np.float64)
        pad[: view.shape[0]] = view
        t = self._tensor(pad, torch.float64)
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t)
        if self.rank != 0:
            return None
        rows = []
        for r, p in enumerate(parts):
            rb, re_ = shard(n_rows, r, self.world)
            rows.append(p.cpu().numpy()[: re_ - rb])
        full = np.concatenate(rows, axis=0)
        if np.iscomplexobj(local):
            return full.view(local.dtype).reshape((n_rows,) + tail)
        return full.astype(local.dtype).reshape((n_rows,) + tail)

    def close(self):
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()
        self.dist = None
