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


@pytest.mark.parametrize("name,n,frac,cap", [("batched_uneven_10k", 600, 0.1, 6),
                                             ("similar_dna_100k", 400, 0.1, 8),
                                             ("plain_protein_200", 200, 0.2, 5),
                                             ("plain_protein_200", 120, 0.1, 1)])
def test_clustered_tree_of_the_msa(name, n, frac, cap):
    """The clustered tree (sample tree cut into clusters, rows labelled, one
    outgroup-rooted tree per cluster, grafted back): joins, branch lengths and
    labels equal the oracle's on its own MSA."""
    b = binding()
    letters, offsets, w, alph, M = workload(name, n=n, seed=33)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    center = int(np.argsort(np.diff(offsets), kind="stable")[n // 2])
    _, _, _, _, _, orows = oracle.msa(prob, center)
    sample = np.sort(np.random.default_rng(4).choice(n, max(2, int(frac * n)), replace=False))
    oj, ol, oc = T.cluster_tree(T.msa_distances(orows), sample, cap)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        with pytest.raises(b.MSAError):
            b.msa_nj_cluster_tree(h, sample, cap)  # before a merge
        b.msa_align_to_center(h, center)
        b.msa_merge_gaps(h, want_rows=False)
        joins, lengths, cluster = b.msa_nj_cluster_tree(h, sample, cap)
        with pytest.raises(b.MSAError):
            b.msa_nj_cluster_tree(h, [0, n], cap)  # a row out of range
    assert (cluster == oc).all()
    assert (joins == oj).all() and (lengths == ol).all()
    print(name, "clusters", int(cluster.max()) + 1)


def test_clustered_tree_degenerate_cuts():
    """One sample row (a single cluster: the NJ tree of all rows) and every
    row sampled with a cap above them (no cut): both equal the oracle's and,
    as unrooted trees, the plain NJ tree."""
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=90, seed=8)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    _, _, _, _, _, orows = oracle.msa(prob, 5)
    D = T.msa_distances(orows)
    nj_splits = T.splits(*T.nj(D), 90)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        b.msa_align_to_center(h, 5)
        b.msa_merge_gaps(h, want_rows=False)
        for sample, cap in (([17], 1), (np.arange(90), 90)):
            oj, ol, oc = T.cluster_tree(D, sample, cap)
            joins, lengths, cluster = b.msa_nj_cluster_tree(h, sample, cap)
            assert (joins == oj).all() and (lengths == ol).all() and (cluster == oc).all()
            assert T.splits(joins, lengths, 90) == nj_splits
