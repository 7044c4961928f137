"""Host logic of the multi-GPU mode: replicas only.

Code blocks and cells are independent and a TB needs only its own CBs, so N
GPUs run N independent replicas: rank r serves its own block of cells (its
HARQ soft buffers stay on its GPU) and there is no collective on the data
path.  The only cross-rank traffic is the timing reduction of a benchmark:
the slowest rank's time and the sum of the bits all ranks decoded.
"""


def cell_block(n_cells_total, world, rank):
    """Contiguous block of cell ids served by `rank` (sizes differ by <= 1)."""
    base, extra = divmod(n_cells_total, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def rank_seed(seed, rank):
    """Seed of a rank's synthetic traffic (distinct per rank)."""
    return seed + 7919 * rank


def reduce_time_bits(seconds, bits, device=None):
    """Max of `seconds` and sum of `bits` over all ranks of the default
    process group (gloo on CPU, NCCL on GPU).  Returns (max_s, total_bits)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    b = torch.tensor([float(bits)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())
