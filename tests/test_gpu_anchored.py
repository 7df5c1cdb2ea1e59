"""The anchored alignment (the paper's trie path for similar nucleotides) on
the GPU against the oracle's: inserted-space rows, segments and the merged
MSA bit for bit, on the similar-DNA workload for several segment lengths,
with sequences sent to the local path (no match, a long unmatched stretch)
and on proteins."""
import numpy as np
import pytest

import oracle
from seqgen import dna_matrix, pack_sequences
from tests._gpu import binding, workload, make_ctx, oracle_problem

pytestmark = pytest.mark.gpu


def _check(b, h, prob, center, k, letters, offsets):
    scores = np.zeros(prob.n, np.int32)
    nf = b.msa_align_anchored(h, center, k, scores)
    seg, ins, occ = b.msa_alignment_info(h)
    rows, W = b.msa_merge_gaps(h)
    oseg, oins, oocc = oracle.anchored_all(prob, center, k)
    assert (ins == oins).all() and (occ == oocc).all()
    assert (seg == oseg).all() and (scores == oseg[:, 0]).all()
    oG, oW, orows = oracle.merge(prob, center, oins, oocc)
    assert W == oW and (rows == orows).all()
    return nf


@pytest.mark.parametrize("k", [8, 12, 16])
def test_similar_dna_matches_the_oracle(k):
    b = binding()
    letters, offsets, w, alph, M = workload("similar_dna_100k", n=300, seed=7)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        nf = _check(b, h, prob, 0, k, letters, offsets)
    print("k", k, "sequences on the local path", nf)


def test_local_path_for_unanchored_and_long_stretches():
    """A random sequence (no match), one with a 120-residue foreign stretch
    between anchors (longer than the 80 a lane aligns), and similar ones."""
    b = binding()
    alph, M = dna_matrix(2, -3)
    rng = np.random.default_rng(3)
    bases = np.frombuffer(b"ACGT", np.uint8)
    center = bases[rng.integers(0, 4, 600)]
    seqs = [center.copy()]
    seqs.append(bases[rng.integers(0, 4, 300)])                          # unrelated
    seqs.append(np.concatenate([center[:200], bases[rng.integers(0, 4, 120)], center[320:]]))
    for _ in range(20):                                                   # similar
        s = center.copy()
        hit = rng.random(s.size) < 0.03
        s[hit] = bases[rng.integers(0, 4, int(hit.sum()))]
        seqs.append(s[int(rng.integers(0, 40)):s.size - int(rng.integers(0, 40))])
    letters, offsets = pack_sequences(seqs)
    prob = oracle_problem(letters, offsets, alph, M, 5, 2)
    with make_ctx(alph, M, 5, 2) as h:
        b.msa_load(h, letters, offsets)
        nf = _check(b, h, prob, 0, 12, letters, offsets)
    assert nf >= 2


def test_proteins_with_short_segments():
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=60, seed=4)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        _check(b, h, prob, 5, 4, letters, offsets)
        with pytest.raises(b.MSAError):
            b.msa_align_anchored(h, 5, 13)          # 13 x 5 bits > 64
