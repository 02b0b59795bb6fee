"""Frame sharding across ranks (one process per GPU).

Frames are independent in the decoder, so a job of `total` frames splits into
contiguous frame ranges, one per rank, with no exchange on the data path.
Channel noise is drawn by the counter-based generator from each frame's
global index, so a frame's LLRs do not depend on how the frames are split.
Only integer counters (frames, bit and frame errors, iterations) and timings
are reduced at the end.
"""
from __future__ import annotations

from dataclasses import dataclass, field


def frame_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """(first global frame, count) of `rank`'s share of `total` frames;
    the first total % world ranks take one extra frame."""
    if world <= 0 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


@dataclass
class Counts:
    """Decode statistics that add across shards."""

    frames: int = 0
    bit_errors: int = 0
    frame_errors: int = 0
    iterations: int = 0
    unsatisfied: int = 0  # frames whose final syndrome is nonzero
    extra: dict = field(default_factory=dict)

    def add_decode(self, bits, iters, ok, sent) -> None:
        """Accumulate one decoded batch (numpy arrays) against the sent words."""
        import numpy as np

        err = np.asarray(bits) != np.asarray(sent)
        self.frames += int(err.shape[0])
        self.bit_errors += int(err.sum())
        self.frame_errors += int(err.any(axis=1).sum())
        self.iterations += int(np.asarray(iters).sum())
        self.unsatisfied += int((np.asarray(ok) == 0).sum())

    def as_list(self) -> list[int]:
        return [self.frames, self.bit_errors, self.frame_errors, self.iterations, self.unsatisfied]

    @classmethod
    def from_list(cls, v) -> "Counts":
        return cls(*[int(x) for x in v])


def allreduce_counts(counts: Counts, group=None) -> Counts:
    """Sum counters over the ranks of a torch.distributed group (any backend)."""
    import torch
    import torch.distributed as dist

    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor(counts.as_list(), dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return Counts.from_list(t.cpu().tolist())
