"""Failure detection without a GPU fault: an allocation cap on the host side
(forced allocation failure) and the bounded waits of the tensor-core
convolution made to run out on purpose (no load is ever issued), each
followed by a normal call on the same context."""
import numpy as np
import pytest

import oracle
from oracle import net
from tests._gpu import binding, workload, make_ctx, oracle_problem

pytestmark = pytest.mark.gpu


def test_memory_cap_fails_cleanly_and_context_recovers():
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=40, seed=3)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        held0, _ = b.msa_memory(h)
        b.msa_set_memory_limit(h, held0 + 4096)
        with pytest.raises(b.MSAError) as ei:
            b.msa_load(h, letters, offsets)
            b.msa_select_center(h, b.MSA_CENTER_EXACT)
        assert ei.value.code == b.MSA_ENOMEM
        assert "device memory limit" in str(ei.value)
        b.msa_set_memory_limit(h, 0)
        b.msa_load(h, letters, offsets)
        c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        held, peak = b.msa_memory(h)
        with pytest.raises(b.MSAError) as ei:
            b.msa_set_memory_limit(h, -1)
        assert ei.value.code == b.MSA_EINVAL
    oc, orow = oracle.exact_center(prob)
    assert c == oc and s == orow[oc]
    assert 0 < held <= peak


def test_tensor_core_wait_timeout_is_reported_and_context_recovers():
    b = binding()
    letters, offsets, w, alph, M = workload("learned_center_50k", n=12, seed=2)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        assert b.msa_debug_wait_timeout(h)
        b.msa_load(h, letters, offsets)
        b.msa_selector_init(h, seed=5)
        params = net.unflatten(b.msa_selector_params(h).astype(np.float64))
        emb = b.msa_selector_embed(h)
    oemb = net.embed_all(params, [prob.seq(i) for i in range(prob.n)])
    assert np.linalg.norm(emb - oemb) / np.linalg.norm(oemb) < 3e-2
