"""One center-star MSA split across processes (one GPU each).

Every alignment to the center is independent (the map step of the paper's
Figure 3), so the sequences shard into contiguous blocks with the center
replicated.  The exchanges are the two reduces of the method:

- the exact center: every process computes its share of the pairs
  (msa_center_partial: a range of the all-pairs triangle, or a chunk of the
  reference sample) as per-sequence similarity sums; one allreduce-sum gives
  every process the whole set's sums, from which msa_center_combine takes the
  row sums and the center;
- Figure 3's reduce of the inserted-space matrix: each process's per-slot
  insertion maxima G are combined by an elementwise maximum, after which every
  process writes its own rows of the common alignment.

The collectives go through torch.distributed (NCCL between GPUs; gloo in the
CPU tests).  The per-process work is a backend: GpuBackend drives libmsa's C
ABI on this process's GPU; any object with the same five methods can stand in
(the CPU tests use the oracle).
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


def global_sums(local_sums, device="cpu", group=None):
    """Elementwise sum of every process's partial similarity sums (uint64
    values below 2^63, carried as int64 for the collective)."""
    import torch.distributed as dist
    t = _tensor(np.asarray(local_sums, dtype=np.uint64).astype(np.int64), device)
    dist.all_reduce(t, group=group)
    return t.cpu().numpy().astype(np.uint64)


def max_over_ranks(x, device="cpu", group=None):
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


class GpuBackend:
    """This process's share of the work through libmsa on its current GPU.

    center_partial / center_combine run on a context holding the whole set
    (every process needs every sequence to meet its share of the pairs);
    align_block loads this process's block plus the center into a second
    context, whose insert_maxima / merge_with follow."""

    def __init__(self, letters, offsets, matrix, alphabet, gap_open, gap_extend):
        from . import binding as b
        self.b = b
        self.letters = np.ascontiguousarray(letters, dtype=np.uint8)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.args = (matrix, alphabet, gap_open, gap_extend)
        self.whole = b.Context(*self.args)
        b.msa_load(self.whole.h, self.letters, self.offsets)
        self.block = None

    def center_partial(self, shard, nshards, refs=None):
        return self.b.msa_center_partial(self.whole.h, shard, nshards, refs)

    def center_combine(self, sums, nref=0):
        c, _ = self.b.msa_center_combine(self.whole.h, sums, nref)
        return c, self.b.msa_center_rowsums(self.whole.h)

    def align_block(self, lo, hi, center):
        idx = list(range(lo, hi)) + [int(center)]
        seqs = [self.letters[self.offsets[i]:self.offsets[i + 1]] for i in idx]
        off = np.zeros(len(seqs) + 1, np.int64)
        off[1:] = np.cumsum([s.size for s in seqs])
        if self.block is None:
            self.block = self.b.Context(*self.args)
        self.b.msa_load(self.block.h, np.concatenate(seqs), off)
        self.b.msa_align_to_center(self.block.h, len(seqs) - 1)

    def insert_maxima(self):
        return self.b.msa_insert_maxima(self.block.h)

    def merge_with(self, G):
        rows, W = self.b.msa_merge_gaps_with(self.block.h, G)
        return rows, W

    def close(self):
        for c in (self.whole, self.block):
            if c is not None:
                c.close()


def sharded_center(backend, refs=None, device="cpu", group=None):
    """The exact center of the whole set (EXACT, or EXACT_SAMPLED over refs):
    this process's share of the pairs, one allreduce-sum, then the row sums
    and their argmin.  Returns (center, rowsum int64[n])."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    local = backend.center_partial(rank, world, refs)
    total = global_sums(local, device, group)
    return backend.center_combine(total, 0 if refs is None else len(refs))


def sharded_msa(backend, n, center, device="cpu", group=None):
    """This process's rows of the MSA of the whole set, aligned to `center`
    (an input index), with one allreduce-max of G between processes.
    Returns (lo, hi, rows uint8[hi-lo, W], W)."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    lo, hi = shard_bounds(n, world, rank)
    # the block plus the center (its own alignment is dropped unless it is ours)
    backend.align_block(lo, hi, center)
    G = global_insert_maxima(backend.insert_maxima(), device, group)
    rows, W = backend.merge_with(G)
    return lo, hi, rows[:hi - lo], W
