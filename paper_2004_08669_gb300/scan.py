"""Temperature scans across several GPUs: one process per GPU, each running a
contiguous block of the betas, then a host-side gather of the observables.

The betas of a scan are independent runs of Algorithm 3 of arXiv:2004.08669
(Sec. III sweeps the temperature one run at a time), so the scan shards with
no exchange in the data path: the only communication is one gather of small
host objects (the per-beta observables) after the work is done.  On one GPU
the library's own scan (ctm_scan_*) overlaps the betas of a block; this module
only splits the betas between ranks and collects the results.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Half-open range [lo, hi) of the n betas that `rank` of `world` takes:
    contiguous blocks whose sizes differ by at most one, lower ranks first."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world size {world}")
    if n < 0:
        raise ValueError("n must be >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def gather_results(local: list, rank: int, world: int, group=None) -> Optional[list]:
    """Concatenate every rank's list of results in rank order on rank 0
    (other ranks get None).  Uses torch.distributed's object gather on
    `group` (a gloo group, so no device memory is involved)."""
    if world == 1:
        return list(local)
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object(local, parts, dst=0, group=group)
    if rank != 0:
        return None
    out = []
    for p in parts:
        out.extend(p)
    return out


def run_sharded(betas: Sequence[float], run_block: Callable[[List[float]], list], rank: int = 0, world: int = 1,
                group=None) -> Optional[list]:
    """Run `run_block` on this rank's block of betas (it returns one result
    per beta, in order) and gather all results on rank 0 in beta order."""
    lo, hi = shard_range(len(betas), rank, world)
    local = run_block(list(betas[lo:hi]))
    if len(local) != hi - lo:
        raise RuntimeError(f"run_block returned {len(local)} results for {hi - lo} betas")
    return gather_results(local, rank, world, group)
