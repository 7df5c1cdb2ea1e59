"""Pins for the oracle's anchored alignment (the paper's trie path for similar
nucleotides: matched center segments are skipped, unmatched stretches
aligned): hand-worked fixtures, brute-force optimal global alignment of the
stretches between anchors, the local path when nothing anchors, and the merge
invariants of the rows it produces.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from seqgen import dna_matrix, generate
from tests import _pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    out = []
    for ln in open(os.path.join(GOLDEN, "anchored_cases.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        f = [x.strip() for x in ln.split("|")]
        ints = lambda x: [int(v) for v in x.split()]
        out.append(dict(name=f[0], k=int(f[1]), c=f[2], x=f[3], seg=tuple(ints(f[4])),
                        ins=ints(f[5]), occ=ints(f[6])))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked_anchored(case):
    alph, M = dna_matrix(2, -3)
    c = oracle.encode(case["c"].encode(), alph)
    x = oracle.encode(case["x"].encode(), alph)
    ins, occ, seg = oracle.anchored(c, x, M, 5, 2, case["k"])
    assert seg == case["seg"]
    assert list(ins) == case["ins"] and list(occ) == case["occ"]


def _global_brute(a, b, M, o, e):
    """Best affine score of a global alignment of a and b (every path)."""
    return max(_pins.score_path(list(a), list(b), p, M, o, e)
               for p in _pins._paths(len(a), len(b)))


@pytest.mark.parametrize("seed", range(30))
def test_stretch_is_an_optimal_global_alignment(seed):
    """Two anchors made of letters the stretches never use, one unmatched
    center segment between them: the alignment's score is the anchors' plus
    the best global alignment of the stretches (every path enumerated), and
    its columns re-score to it."""
    rng = np.random.default_rng(300 + seed)
    K = 6                                   # 0-3: stretch letters; 4, 5: anchors
    M = np.full((K, K), -3, np.int8)
    np.fill_diagonal(M, 2)
    M[:4, :4] = rng.integers(-4, 3, size=(4, 4))
    M[:4, :4] = np.triu(M[:4, :4]) + np.triu(M[:4, :4], 1).T
    np.fill_diagonal(M, 2)
    o = int(rng.integers(2, 6)); e = int(rng.integers(1, o + 1))
    k = 3
    a1, a2 = [4, 5, 4], [5, 4, 5]
    while True:
        sc = list(rng.integers(0, 4, k))
        sx = list(rng.integers(0, 4, int(rng.integers(0, 5))))
        if not any(sx[i:i + k] == sc for i in range(len(sx) - k + 1)):
            break
    c = np.array(a1 + sc + a2, np.uint8)
    x = np.array(a1 + sx + a2, np.uint8)
    ins, occ, seg = oracle.anchored(c, x, M, o, e, k)
    anchors = sum(int(M[v, v]) for v in a1 + a2)
    assert seg[0] == anchors + _global_brute(sc, sx, M, o, e)
    assert seg[1:] == (0, 0, len(c), len(x))
    cols = _pins.pairwise_columns(ins, occ, len(c), len(x))
    total, prev = 0, None
    for ci, si in cols:
        if ci is not None and si is not None:
            total += int(M[c[ci - 1]][x[si - 1]]); prev = "M"
        elif ci is None:
            total -= e if prev == "I" else o; prev = "I"
        else:
            total -= e if prev == "D" else o; prev = "D"
    assert total == seg[0]


def test_identical_sequences_align_residue_for_residue():
    alph, M = dna_matrix(2, -3)
    rng = np.random.default_rng(5)
    c = rng.integers(0, 4, 200).astype(np.uint8)
    for k in (4, 8, 16):
        ins, occ, seg = oracle.anchored(c, c, M, 5, 2, k)
        assert (occ[1:] == 1).all() and (ins == 0).all()
        assert seg[0] == 2 * (200 // k * k) and seg[1:3] == (0, 0)


def test_no_anchor_is_the_local_path():
    alph, M = dna_matrix(2, -3)
    rng = np.random.default_rng(6)
    c = rng.integers(0, 4, 60).astype(np.uint8)
    x = rng.integers(0, 4, 50).astype(np.uint8)
    k = 40                                   # one 40-residue segment: never found
    ins, occ, seg = oracle.anchored(c, x, M, 5, 2, k)
    v, codes, end = oracle.sw(c, x, M, 5, 2, codes=True)
    oins, oocc, oseg = oracle.traceback(codes, v, end)
    assert (ins == oins).all() and (occ == oocc).all() and seg == (v,) + oseg


def test_similar_dna_rows_merge_into_an_msa():
    """On a sample of the similar-DNA workload, the anchored rows account for
    every residue, and the merged MSA keeps every sequence and the center."""
    letters, offsets, w, _ = generate("similar_dna_100k", n=40, seed=3)
    alph, M = dna_matrix(2, -3)
    prob = oracle.Problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    center = 0
    seg, ins, occ = oracle.anchored_all(prob, center, 16)
    lc = prob.length(center)
    for t in range(prob.n):
        assert int(ins[t].sum()) + int(occ[t].sum()) == prob.length(t)
    G, W, rows = oracle.merge(prob, center, ins, occ)
    assert W == lc + int(G.sum())
    for t in range(prob.n):
        assert bytes(rows[t]).replace(b"-", b"") == bytes(letters[offsets[t]:offsets[t + 1]])
    # on 2 % divergence nearly every residue pair of the anchored region is a match
    assert (occ[:, 1:].mean() > 0.9)
