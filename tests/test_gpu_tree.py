"""The neighbour-joining tree on the GPU against the tree oracle, through the
C ABI: distances of the merged rows and every join (children and branch
lengths) bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import nj as T
from tests._gpu import binding, workload, make_ctx, oracle_problem
from tests.test_oracle_nj import random_tree

pytestmark = pytest.mark.gpu


def any_ctx():
    from seqgen import dna_matrix
    alph, M = dna_matrix()
    return make_ctx(alph, M, 5, 2)


@pytest.mark.parametrize("n,seed", [(3, 1), (4, 2), (40, 3), (300, 4), (700, 5)])
def test_nj_of_additive_distances(n, seed):
    """Distances read off a random tree: the GPU joins equal the oracle's
    (which recovers the tree); 700 rows cross the packing of the matrix."""
    b = binding()
    tj, tl, D = random_tree(np.random.default_rng(seed), n)
    oj, ol = T.nj(D)
    with any_ctx() as h:
        joins, lengths = b.msa_nj(h, D)
    assert (joins == oj).all() and (lengths == ol).all()
    assert T.splits(joins, lengths, n) == T.splits(tj, tl, n)


def test_nj_ties_small_and_unbalanced():
    b = binding()
    cases = [np.zeros((1, 1), np.int64), np.array([[0, 7], [7, 0]], np.int64)]
    eq = np.full((9, 9), 2, np.int64)
    np.fill_diagonal(eq, 0)
    cases.append(eq)  # every Q ties at every join
    rng = np.random.default_rng(7)
    R = rng.integers(0, 1 << 20, size=(600, 600)).astype(np.int64)
    R = np.triu(R, 1)
    cases.append(R + R.T)  # no tree behind it: odd and negative updates floor
    with any_ctx() as h:
        for D in cases:
            oj, ol = T.nj(D)
            joins, lengths = b.msa_nj(h, D)
            assert (joins == oj).all() and (lengths == ol).all(), D.shape


def test_nj_from_device_memory_and_range_check():
    import torch
    b = binding()
    _, _, D = random_tree(np.random.default_rng(9), 50)
    oj, ol = T.nj(D)
    with any_ctx() as h:
        joins, lengths = b.msa_nj(h, torch.from_numpy(D).cuda())
        assert (joins == oj).all() and (lengths == ol).all()
        big = np.array([[0, 1 << 42, 1 << 42], [1 << 42, 0, 1 << 42], [1 << 42, 1 << 42, 0]],
                       np.int64)
        with pytest.raises(b.MSAError) as ei:
            b.msa_nj(h, big)
        assert ei.value.code == b.MSA_ERANGE
        joins, lengths = b.msa_nj(h, D)  # the context stays usable
        assert (joins == oj).all()


@pytest.mark.parametrize("name,n", [("plain_protein_200", 200), ("batched_uneven_10k", 700),
                                    ("similar_dna_100k", 120)])
def test_tree_of_the_msa(name, n):
    """The whole path to the tree: MSA rows, their distances and the joins
    equal the oracle's, computed from the oracle's own MSA."""
    b = binding()
    letters, offsets, w, alph, M = workload(name, n=n, seed=21)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    center = int(np.argsort(np.diff(offsets), kind="stable")[n // 2])
    _, _, _, _, _, orows = oracle.msa(prob, center)
    od = T.msa_distances(orows)
    oj, ol = T.nj(od)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        with pytest.raises(b.MSAError):
            b.msa_tree_distances(h)  # before an alignment and merge
        b.msa_align_to_center(h, center)
        b.msa_merge_gaps(h, want_rows=False)
        d = b.msa_tree_distances(h)
        joins, lengths = b.msa_nj_tree(h)
    assert (d == od).all()
    assert (joins == oj).all() and (lengths == ol).all()
