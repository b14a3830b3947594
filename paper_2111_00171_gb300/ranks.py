"""Work split and timing across ranks: one process per GPU.

Each pattern of a scan is matched on its own (section "Correlation Pattern
Matching": the correlation, its maximum and the refinement use the plan and
that pattern alone), so ranks exchange nothing on the data path.  A rank
matches either its own scan (weak scaling) or a contiguous slice of one CSR
scan (strong scaling).  The only collectives are the barriers around a timed
region and the maximum of the elapsed times over ranks.

The helpers take numpy arrays or torch tensors and work under any
``torch.distributed`` backend: NCCL on GPUs, gloo on the host.
"""

import os


def rank_env():
    """(world_size, rank, local_rank) from the launcher's environment; (1, 0, 0)
    for a plain single-process run."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank environment: rank {rank} of {world}")
    return world, rank, local


def pattern_range(n_patterns, world, rank):
    """Contiguous patterns [lo, hi) of ``rank``: the first n % world ranks take
    one pattern more, so counts differ by at most one and the ranges tile
    [0, n_patterns) in rank order."""
    if world < 1 or not 0 <= rank < world or n_patterns < 0:
        raise ValueError("pattern_range: need world >= 1, 0 <= rank < world, n >= 0")
    base, extra = divmod(n_patterns, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def csr_slice(row_ptr, qx, qy, intensity, world, rank):
    """This rank's patterns of a CSR scan as a CSR scan of its own.

    Returns (row_ptr', qx', qy', I', lo, hi): row_ptr' = row_ptr[lo:hi+1] -
    row_ptr[lo] starts at 0 as the match entry point requires, and the peak
    arrays are views of the peaks [row_ptr[lo], row_ptr[hi])."""
    n = len(row_ptr) - 1
    lo, hi = pattern_range(n, world, rank)
    p0, p1 = int(row_ptr[lo]), int(row_ptr[hi])
    rp = row_ptr[lo:hi + 1] - row_ptr[lo]
    return rp, qx[p0:p1], qy[p0:p1], intensity[p0:p1], lo, hi


def _reduce(value, op):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value):
    """Maximum of ``value`` over all ranks (the value itself on one rank)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX if dist.is_available() else None)


def sum_over_ranks(value):
    """Sum of ``value`` over all ranks (the value itself on one rank)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM if dist.is_available() else None)


def barrier():
    """Barrier over all ranks; nothing on one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
