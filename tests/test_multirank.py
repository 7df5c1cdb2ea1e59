"""The host logic of a center-star MSA split across processes, with two gloo
ranks on the CPU: the allreduce-max of the slot maxima G (Figure 3's reduce)
and the gather of the exact center's row sums reproduce the single-process
results.  The oracle stands in for each rank's GPU work."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


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


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1704_00878_gb300 import shard
        prob, letters, offsets = _problem()
        n = prob.n
        lo, hi = shard.shard_bounds(n, world, rank)
        # exact center: this rank's candidates against every sequence
        local = oracle.center_rowsums(prob, np.arange(lo, hi))
        rowsum = shard.gather_rowsums(local, n)
        center = int(np.argmin(rowsum))
        # alignment of this rank's rows, then the global slot maxima
        seg, ins, occ = oracle.align_all(prob, center)
        G = shard.global_insert_maxima(ins[lo:hi].max(axis=0))
        np.save(os.path.join(out_dir, "r%d.npy" % rank),
                {"rowsum": rowsum, "center": center, "G": G, "lo": lo, "hi": hi,
                 "tmax": shard.max_over_ranks(float(rank + 1))}, allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_two_ranks_reproduce_single_process(tmp_path):
    import oracle
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    prob, letters, offsets = _problem()
    oc, orow = oracle.exact_center(prob)
    _, ins, occ = oracle.align_all(prob, oc)
    oG, oW, orows = oracle.merge(prob, oc, ins, occ)
    res = [np.load(os.path.join(str(tmp_path), "r%d.npy" % r), allow_pickle=True).item()
           for r in range(world)]
    for r in res:
        assert (r["rowsum"] == orow).all() and r["center"] == oc
        assert (r["G"] == oG).all()
        assert r["tmax"] == float(world)
    # every rank's rows, written with the global G, are the single-process rows
    lib = oracle.lib()
    for r in res:
        lo, hi = r["lo"], r["hi"]
        sub_off = offsets[lo:hi + 1] - offsets[lo]
        sub = oracle.Problem(letters[offsets[lo]:offsets[hi]], sub_off, prob.alphabet, prob.M,
                             prob.o, prob.e)
        W = prob.length(oc) + int(r["G"].sum())
        rows = np.zeros((hi - lo, W), np.uint8)
        ins_b = np.ascontiguousarray(ins[lo:hi])
        occ_b = np.ascontiguousarray(occ[lo:hi])
        G32 = np.ascontiguousarray(r["G"], np.int32)
        rc = lib.orc_write_rows(oracle._p(sub.res), oracle._p(sub.off), hi - lo, prob.length(oc),
                                oracle._p(ins_b), oracle._p(occ_b), oracle._p(G32), W,
                                prob.alphabet.encode(), oracle._p(rows))
        assert rc == 0 and W == oW
        assert (rows == orows[lo:hi]).all()


def test_shard_bounds_cover_everything():
    from paper_1704_00878_gb300 import shard
    for n in (1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
