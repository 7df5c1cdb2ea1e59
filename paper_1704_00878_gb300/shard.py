"""One center-star MSA split across processes (one GPU each).

Every alignment to the center is independent (the map step of the paper's
Figure 3), so the sequences shard into contiguous blocks with the center
replicated.  The one exchange is the reduce of Figure 3: each process's
per-slot insertion maxima G are combined by an elementwise maximum, after
which every process writes its own rows of the common alignment.  The exact
center adds a gather of the candidates' distance row sums.

The collectives go through torch.distributed (NCCL between GPUs; gloo in the
CPU tests).  The per-process work is the C ABI of libmsa.
"""
import numpy as np


def shard_bounds(n, world, rank):
    """Contiguous block [lo, hi) of n items for `rank` of `world`."""
    per, extra = divmod(n, world)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def _tensor(x, device):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).to(device)


def global_insert_maxima(local_G, device="cpu", group=None):
    """Elementwise maximum of every process's slot maxima (Figure 3's reduce)."""
    import torch.distributed as dist
    t = _tensor(np.asarray(local_G, dtype=np.int64), device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.cpu().numpy().astype(np.int32)


def gather_rowsums(local_rowsum, n, device="cpu", group=None):
    """Row sums of every candidate from per-process blocks (shard_bounds
    order) -> the full int64[n] vector on every process."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    full = torch.zeros(n, dtype=torch.int64, device=device)
    rank = dist.get_rank(group)
    lo, hi = shard_bounds(n, world, rank)
    full[lo:hi] = _tensor(np.asarray(local_rowsum, dtype=np.int64), device)
    dist.all_reduce(full, group=group)  # blocks are disjoint: the sum assembles them
    return full.cpu().numpy()


def max_over_ranks(x, device="cpu", group=None):
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_msa(letters, offsets, center, matrix, alphabet, gap_open, gap_extend, device,
                group=None):
    """This process's rows of the MSA of the whole set, aligned to `center`
    (an input index), with one allreduce-max of G between processes.
    Returns (lo, hi, rows uint8[hi-lo, W], W)."""
    import torch.distributed as dist
    from . import binding as b
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    n = offsets.size - 1
    lo, hi = shard_bounds(n, world, rank)
    # the shard plus the center (its own alignment is dropped unless it is ours)
    idx = list(range(lo, hi)) + [center]
    seqs = [letters[offsets[i]:offsets[i + 1]] for i in idx]
    off = np.zeros(len(seqs) + 1, np.int64)
    off[1:] = np.cumsum([s.size for s in seqs])
    flat = np.concatenate(seqs).astype(np.uint8)
    with b.Context(matrix, alphabet, gap_open, gap_extend) as h:
        b.msa_load(h, flat, off)
        b.msa_align_to_center(h, len(seqs) - 1)
        G = global_insert_maxima(b.msa_insert_maxima(h), device, group)
        rows, W = b.msa_merge_gaps_with(h, G)
    return lo, hi, rows[:hi - lo], W
