"""The exact center split into shards through the C ABI on one GPU: the sum of
every shard's partial similarity sums (msa_center_partial) gives, through
msa_center_combine, the center and row sums of the single selection and of
the oracle, for any number of shards, all pairs or a reference sample; and
shard.GpuBackend runs sharded_center / sharded_msa in a one-rank group."""
import os
import socket

import numpy as np
import pytest

import oracle
from tests._gpu import binding, workload, make_ctx, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nshards", [1, 2, 3, 5])
def test_partial_sums_combine_to_the_exact_center(nshards):
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=90, seed=17)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    oc, orow = oracle.exact_center(prob)
    refs = np.array([3, 8, 13, 21, 34, 55, 89])
    osc, osrow = oracle.exact_center(prob, refs=refs)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c1, s1 = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        total = sum(b.msa_center_partial(h, k, nshards) for k in range(nshards))
        c, s = b.msa_center_combine(h, total)
        rows = b.msa_center_rowsums(h)
        stotal = sum(b.msa_center_partial(h, k, nshards, refs=refs) for k in range(nshards))
        sc, ss = b.msa_center_combine(h, stotal, nref=len(refs))
        srows = b.msa_center_rowsums(h)
        with pytest.raises(b.MSAError):
            b.msa_center_partial(h, nshards, nshards)
    assert (rows == orow).all() and c == oc == c1 and s == s1 == orow[oc]
    assert (srows == osrow).all() and sc == osc and ss == osrow[osc]


def test_gpu_backend_in_a_one_rank_group(tmp_path):
    import torch.distributed as dist
    from paper_1704_00878_gb300 import shard
    letters, offsets, w, alph, M = workload("plain_protein_200", n=40, seed=5)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        backend = shard.GpuBackend(letters, offsets, M, alph, w.gap_open, w.gap_extend)
        center, rowsum = shard.sharded_center(backend)
        lo, hi, rows, W = shard.sharded_msa(backend, prob.n, center)
        backend.close()
    finally:
        dist.destroy_process_group()
    oc, orow = oracle.exact_center(prob)
    *_, oW, orows = oracle.msa(prob, oc)
    assert center == oc and (rowsum == orow).all()
    assert (lo, hi) == (0, prob.n) and W == oW and (rows == orows).all()
