"""Recomputing the local-alignment DP inside any box that contains the
traced path (H = 0 and no open gap on the box's top row and left column)
reproduces that path: same segment, same inserted residues and aligned
center residues inside it.  This is the property a traceback-light
alignment (codes only inside the segment's box) rests on; checked with the
oracle on random pairs with small alphabets and gap costs that make ties
common."""
import numpy as np
import pytest

import oracle
from seqgen import dna_matrix


def random_case(rng):
    K = int(rng.integers(2, 5))
    M = dna_matrix()[1][:K, :K].astype(np.int8) if rng.random() < 0.5 else \
        np.where(np.eye(K, dtype=bool), int(rng.integers(1, 4)), -int(rng.integers(1, 4))).astype(np.int8)
    e = int(rng.integers(1, 3))
    o = e + int(rng.integers(0, 4))
    c = rng.integers(0, K, size=int(rng.integers(3, 40))).astype(np.uint8)
    s = rng.integers(0, K, size=int(rng.integers(3, 40))).astype(np.uint8)
    return c, s, M, o, e


def inner(ins, occ, i1, i2):
    """Inserted residues between aligned center residues, and which center
    residues are aligned, strictly inside the segment (slots i1+1 .. i2-1,
    residues i1+1 .. i2)."""
    return ins[i1 + 1:i2].tolist(), occ[i1 + 1:i2 + 1].tolist()


@pytest.mark.parametrize("seed", range(6))
def test_box_recompute_reproduces_the_traced_path(seed):
    rng = np.random.default_rng(1000 + seed)
    checked = 0
    for _ in range(150):
        c, s, M, o, e = random_case(rng)
        best, codes, end = oracle.sw(c, s, M, o, e, codes=True)
        if best <= 0:
            continue
        ins, occ, (i1, j1, i2, j2) = oracle.traceback(codes, best, end)
        assert (i2, j2) == end
        # the minimal box and a few larger ones (corner above and left of
        # the path's start, far edges at the best cell)
        corners = [(i1, j1)] + [(int(rng.integers(0, i1 + 1)), int(rng.integers(0, j1 + 1)))
                                for _ in range(3)]
        for bi, bj in corners:
            bb, bcodes, bend = oracle.sw(c[bi:i2], s[bj:j2], M, o, e, codes=True)
            assert bb == best
            assert bend == (i2 - bi, j2 - bj)
            bins, bocc, (ki1, kj1, ki2, kj2) = oracle.traceback(bcodes, bb, bend)
            assert (ki1 + bi, kj1 + bj, ki2 + bi, kj2 + bj) == (i1, j1, i2, j2)
            assert inner(bins, bocc, ki1, ki2) == inner(ins, occ, i1, i2)
            checked += 1
    assert checked > 200


def reversed_local_h(c, s, M, o, e):
    """H of the local alignment (Eq. 1-2, a gap of k costing o + (k-1) e) of
    the two sequences as given, written out cell by cell: (len(c)+1) x
    (len(s)+1), row and column 0 zero."""
    NEG = -(1 << 40)
    H = np.zeros((len(c) + 1, len(s) + 1), np.int64)
    F = np.full(len(s) + 1, NEG, np.int64)
    for i in range(1, len(c) + 1):
        E = NEG
        for j in range(1, len(s) + 1):
            E = max(H[i, j - 1] - o, E - e)
            F[j] = max(H[i - 1, j] - o, F[j] - e)
            H[i, j] = max(0, H[i - 1, j - 1] + int(M[c[i - 1], s[j - 1]]), E, F[j])
    return H


@pytest.mark.parametrize("seed", range(3))
def test_reverse_pass_corner_holds_the_traced_start(seed):
    """The reverse pass of the traceback-light alignment: on the two prefixes
    ending at the best cell, both read backwards, no cell scores above the
    best score S, and the largest reversed row P and column Q of cells scoring
    S give a corner (i2 - P, j2 - Q) above and left of the traced segment's
    start (i1, j1) -- so the box from that corner holds the traced path."""
    rng = np.random.default_rng(2000 + seed)
    checked = 0
    for _ in range(150):
        c, s, M, o, e = random_case(rng)
        best, codes, end = oracle.sw(c, s, M, o, e, codes=True)
        if best <= 0:
            continue
        ins, occ, (i1, j1, i2, j2) = oracle.traceback(codes, best, end)
        H = reversed_local_h(c[:i2][::-1], s[:j2][::-1], M, o, e)
        assert H.max() == best
        ps, qs = np.nonzero(H == best)
        assert i2 - ps.max() <= i1 and j2 - qs.max() <= j1
        # and the box from that corner, its row rounded down to 16, gives back
        # the traced path (the box-recompute property above)
        bi, bj = (i2 - ps.max()) & ~15, j2 - qs.max()
        bb, bcodes, bend = oracle.sw(c[bi:i2], s[bj:j2], M, o, e, codes=True)
        assert bb == best and bend == (i2 - bi, j2 - bj)
        _, _, seg = oracle.traceback(bcodes, bb, bend)
        assert (seg[0] + bi, seg[1] + bj) == (i1, j1)
        checked += 1
    assert checked > 100
