"""The host logic of a center-star MSA split across processes, with two and
three gloo ranks on the CPU: shard.sharded_center (each rank's share of the
exact center's pairs, one allreduce-sum, the row sums and their argmin) and
shard.sharded_msa (each rank's block of alignments, the allreduce-max of the
slot maxima G of Figure 3's reduce, its rows of the common alignment) give
the single-process oracle's center, row sums and MSA.  A stand-in backend
does each rank's GPU work with the oracle (this machine has no GPU); the GPU
backend's calls are tested on a GPU in tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ONE = 1 << 16


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    import oracle
    from seqgen import generate, scoring
    letters, offsets, w, _ = generate("plain_protein_200", n=37, seed=12)
    alph, M, _, _ = scoring(w.kind)
    return oracle.Problem(letters, offsets, alph, M, w.gap_open, w.gap_extend), letters, offsets


class OracleShard:
    """Stand-in for shard.GpuBackend: the same five calls, computed with the
    oracle.  Its share of the pairs is its own (round robin over the first
    index), which the collective must not depend on."""

    def __init__(self, prob, letters, offsets):
        import oracle
        self.oracle, self.prob, self.letters, self.offsets = oracle, prob, letters, offsets
        n = prob.n
        self.self = oracle.pair_scores(prob, np.stack([np.arange(n)] * 2, 1)).astype(np.int64)

    def _sim(self, pairs):
        S = self.oracle.pair_scores(self.prob, pairs).astype(np.int64)
        m = np.maximum(self.self[pairs[:, 0]], self.self[pairs[:, 1]])
        return np.where(m > 0, (S * ONE) // np.maximum(m, 1), ONE).astype(np.uint64)

    def center_partial(self, shard, nshards, refs=None):
        n = self.prob.n
        out = np.zeros(n, np.uint64)
        if refs is None:
            pairs = np.array([(i, j) for i in range(shard, n, nshards) for j in range(i + 1, n)],
                             np.int64).reshape(-1, 2)
            if pairs.size:
                sim = self._sim(pairs)
                np.add.at(out, pairs[:, 0], sim)
                np.add.at(out, pairs[:, 1], sim)
        else:
            mine = [int(r) for k, r in enumerate(refs) if k % nshards == shard]
            pairs = np.array([(i, r) for r in mine for i in range(n)], np.int64).reshape(-1, 2)
            if pairs.size:
                np.add.at(out, pairs[:, 0], self._sim(pairs))
        return out

    def center_combine(self, sums, nref=0):
        n = self.prob.n
        cnt = nref if nref else n - 1
        rowsum = cnt * ONE - np.asarray(sums, np.int64)
        return int(np.argmin(rowsum)), rowsum

    def align_block(self, lo, hi, center):
        self.lo, self.hi, self.center = lo, hi, center
        _, ins, occ = self.oracle.align_all(self.prob, center)
        self.ins, self.occ = ins[lo:hi], occ[lo:hi]

    def insert_maxima(self):
        lc = self.prob.length(self.center)
        return self.ins.max(axis=0) if self.ins.size else np.zeros(lc + 1, np.int64)

    def merge_with(self, G):
        o, prob, lo, hi = self.oracle, self.prob, self.lo, self.hi
        sub_off = self.offsets[lo:hi + 1] - self.offsets[lo]
        sub = o.Problem(self.letters[self.offsets[lo]:self.offsets[hi]], sub_off, prob.alphabet,
                        prob.M, prob.o, prob.e)
        lc = prob.length(self.center)
        W = lc + int(np.asarray(G).sum())
        rows = np.zeros((hi - lo, W), np.uint8)
        G32 = np.ascontiguousarray(G, np.int32)
        rc = o.lib().orc_write_rows(o._p(sub.res), o._p(sub.off), hi - lo, lc,
                                    o._p(np.ascontiguousarray(self.ins)),
                                    o._p(np.ascontiguousarray(self.occ)), o._p(G32), W,
                                    prob.alphabet.encode(), o._p(rows))
        assert rc == 0
        return rows, W


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1704_00878_gb300 import shard
        prob, letters, offsets = _problem()
        backend = OracleShard(prob, letters, offsets)
        center, rowsum = shard.sharded_center(backend)
        refs = np.array([1, 4, 6, 9, 20, 33, 36])
        s_center, s_rowsum = shard.sharded_center(backend, refs=refs)
        lo, hi, rows, W = shard.sharded_msa(backend, prob.n, center)
        np.save(os.path.join(out_dir, "r%d.npy" % rank),
                {"rowsum": rowsum, "center": center, "s_rowsum": s_rowsum, "s_center": s_center,
                 "lo": lo, "hi": hi, "rows": rows, "W": W,
                 "tmax": shard.max_over_ranks(float(rank + 1))}, allow_pickle=True)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_reproduce_single_process(world, tmp_path):
    import oracle
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    prob, letters, offsets = _problem()
    oc, orow = oracle.exact_center(prob)
    refs = np.array([1, 4, 6, 9, 20, 33, 36])
    osc, osrow = oracle.exact_center(prob, refs=refs)
    *_, oW, orows = oracle.msa(prob, oc)
    res = [np.load(os.path.join(str(tmp_path), "r%d.npy" % r), allow_pickle=True).item()
           for r in range(world)]
    covered = 0
    for r in res:
        assert (r["rowsum"] == orow).all() and r["center"] == oc
        assert (r["s_rowsum"] == osrow).all() and r["s_center"] == osc
        assert r["tmax"] == float(world)
        # every rank's rows, written with the global G, are the single-process rows
        assert r["W"] == oW and (r["rows"] == orows[r["lo"]:r["hi"]]).all()
        covered += r["hi"] - r["lo"]
    assert covered == prob.n


def test_shard_bounds_cover_everything():
    from paper_1704_00878_gb300 import shard
    for n in (1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
