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
