"""The path at its documented size limits, bit for bit against the oracle:
sequences of the maximum length (MSA_MAX_LEN residues: the center kernels'
longest queries, int32 cells, the most passes of the alignment kernels), the
anchored path's longest sequences (one residue short of MSA_MAX_LEN) and the
tree of such an MSA."""
import numpy as np
import pytest

import oracle
from oracle import nj as T
from seqgen import blosum62, dna_matrix, pack_sequences, STANDARD_AA
from tests._gpu import binding, make_ctx, oracle_problem
from tests.test_gpu_anchored import _check as anchored_check
from tests.test_gpu_parity import run_pipeline, check_against_oracle

pytestmark = pytest.mark.gpu


def mutants(rng, ancestor, pool, lengths, rate):
    """Copies of the ancestor with substitutions at `rate`, cut to `lengths`
    (each from a random start)."""
    out = []
    for L in lengths:
        s = ancestor.copy()
        hit = rng.random(s.size) < rate
        s[hit] = pool[rng.integers(0, pool.size, int(hit.sum()))]
        start = int(rng.integers(0, ancestor.size - L + 1))
        out.append(s[start:start + L])
    return out


def test_maximum_length_proteins():
    b = binding()
    alph, M = blosum62()
    rng = np.random.default_rng(17)
    pool = np.frombuffer(STANDARD_AA.encode(), np.uint8)
    Lmax = b.MSA_MAX_LEN
    ancestor = pool[rng.integers(0, pool.size, Lmax)]
    seqs = mutants(rng, ancestor, pool, [Lmax, Lmax, 5000, 1, 777], 0.3)
    letters, offsets = pack_sequences(seqs)
    prob = oracle_problem(letters, offsets, alph, M, 11, 1)
    oc, orow = oracle.exact_center(prob)
    with make_ctx(alph, M, 11, 1) as h:
        b.msa_load(h, letters, offsets)
        c, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        assert c == oc and (b.msa_center_rowsums(h) == orow).all()
        for center in sorted({c, 0}):  # the exact center and a maximum-length one
            out = run_pipeline(b, h, letters, offsets, center)
            check_against_oracle(prob, center, *out)
        joins, lengths = b.msa_nj_tree(h)  # of the last MSA
    _, _, _, _, _, orows = oracle.msa(prob, center)
    oj, ol = T.nj(T.msa_distances(orows))
    assert (joins == oj).all() and (lengths == ol).all()


def test_anchored_path_at_its_longest_sequences():
    b = binding()
    alph, M = dna_matrix(2, -3)
    rng = np.random.default_rng(23)
    pool = np.frombuffer(b"ACGT", np.uint8)
    L = b.MSA_MAX_LEN - 1
    ancestor = pool[rng.integers(0, 4, L)]
    seqs = [ancestor.copy()] + mutants(rng, ancestor, pool, [L, L - 3, 4000, 9], 0.02)
    letters, offsets = pack_sequences(seqs)
    prob = oracle_problem(letters, offsets, alph, M, 5, 2)
    with make_ctx(alph, M, 5, 2) as h:
        b.msa_load(h, letters, offsets)
        anchored_check(b, h, prob, 0, 8, letters, offsets)
        # one residue longer is beyond the anchored path's positions
        seqs2 = seqs + [np.concatenate([ancestor, pool[:1]])]
        l2, o2 = pack_sequences(seqs2)
        b.msa_load(h, l2, o2)
        with pytest.raises(b.MSAError) as ei:
            b.msa_align_anchored(h, 0, 8)
        assert ei.value.code == b.MSA_ERANGE
