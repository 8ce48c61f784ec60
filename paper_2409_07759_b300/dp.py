"""Data parallelism for the window step of Alg. 1, one process per GPU.

Each rank keeps a full replica of the Gaussian buffer and renders its own
share of the window's views (forward with the fused L1 term, backward). The
per-Gaussian gradients are then summed over ranks by one all-reduce of the
gradient rows of the eligible slots (active at a frame of the step and not
frozen: the only ones whose gradient can be nonzero, the same on every
replica), packed by the library, each rank's contribution weighted by its
share of the views so that the sum is the gradient of the loss over the whole
window (the L1 term is a mean over views). The optimiser / SGLD noise / relocation step
that follows runs on every replica from the same reduced gradients, the same
seed and the same step counter, so the counter-based random streams (Philox,
keyed by seed and step) give identical updates and the replicas stay equal
without exchanging parameters.

The view partition and the reduction are plain host logic over
torch.distributed; they work with any backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Optional


def shard_views(n_views: int, rank: int, world: int) -> list:
    """Indices of the views rank `rank` renders out of a window of `n_views`:
    a strided partition, so each rank sees every frame of the window when
    there are at least `world` views per frame."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return list(range(rank, n_views, world))


def view_weight(local_views: int, total_views: int) -> float:
    """Factor on a rank's gradients (and loss) before the sum: its share of
    the window's views. The per-rank L1 term is a mean over its own views, so
    sum_r (V_r / V) * mean_r = the mean over all V views."""
    if local_views < 0 or total_views <= 0 or local_views > total_views:
        raise ValueError(f"{local_views} local views of {total_views}")
    return local_views / total_views


class GradientReducer:
    """Callable (flat_grads, loss, rows=None) -> None: scales the gradients and
    the loss by the rank's view share and sums them over the process group in
    place.

    With rows (an object with pack(scale) -> (packed, n) and unpack(packed, n),
    such as RowExchange) only the n packed rows, already scaled, are summed --
    the eligible slots, the only ones whose gradient can be nonzero and which
    every replica finds alike -- and written back; the rest of flat is left as
    it is (zero). Otherwise the whole flat buffer is scaled and summed."""

    def __init__(self, local_views: int, total_views: int, group=None):
        self.weight = view_weight(local_views, total_views)
        self.group = group
        self.last_exchanged = 0  # floats summed by the last call

    def __call__(self, flat, loss=None, rows=None):
        import torch.distributed as dist
        if rows is None:
            if self.weight != 1.0:
                flat.mul_(self.weight)
            dist.all_reduce(flat, group=self.group)
            self.last_exchanged = flat.numel()
        else:
            packed, n = rows.pack(self.weight)
            part = packed[:n]
            dist.all_reduce(part, group=self.group)
            rows.unpack(packed, n)
            self.last_exchanged = part.numel()
        if loss is not None:
            if self.weight != 1.0:
                loss.mul_(self.weight)
            dist.all_reduce(loss, group=self.group)


class RowExchange:
    """The library's packing of the eligible slots' gradient rows (one
    swgs_grad_pack per step, one count read, one swgs_grad_unpack after the
    sum). Buffers are allocated once, for the state's capacity."""

    def __init__(self, renderer, state, grads, frames):
        import torch
        self.r, self.state, self.grads = renderer, state, grads
        self.frames = list(frames)
        K = (state.sh_degree + 1) ** 2
        self.row = 11 + 3 * K
        n = max(1, state.n)
        self.ids = torch.empty(n, dtype=torch.int32, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.packed = torch.empty((n, self.row), dtype=torch.float32, device="cuda")

    def pack(self, scale=1.0):
        self.r.grad_pack(self.state, self.grads, self.frames, self.ids, self.count, self.packed,
                         scale=scale)
        return self.packed, int(self.count.item())

    def unpack(self, packed, n):
        self.r.grad_unpack(self.grads, self.ids, self.count, packed)


def total_views(local_views: int, group=None, device: Optional[str] = None) -> int:
    """Sum of the ranks' view counts (one small all-reduce at set-up)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_views], dtype=torch.int64, device=device)
    dist.all_reduce(t, group=group)
    return int(t.item())
