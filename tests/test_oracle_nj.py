"""Pins of the tree oracle (oracle/nj.py) against what fixes it from outside:
p-distances counted by hand, and neighbour joining's exactness on additive
distances (distances read off a tree are recovered as that tree, topology and
branch lengths; Saitou and Nei, as cited by the paper's tree section)."""
import os

import numpy as np
import pytest

from oracle import nj as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nj_cases.txt")


def load_fixture():
    rows, pairs, mode = [], [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("rows", "pairs"):
            mode = line
            continue
        if mode == "rows":
            rows.append(np.frombuffer(line.encode(), np.uint8))
        else:
            pairs.append([int(x) for x in line.split()])
    return np.stack(rows), pairs


def test_pdistances_match_hand_counts():
    rows, pairs = load_fixture()
    mism, comp = T.msa_counts(rows)
    d = T.msa_distances(rows)
    for a, b, mm, cc, dd in pairs:
        assert (mism[a, b], comp[a, b], d[a, b]) == (mm, cc, dd), (a, b)
        assert (mism[b, a], comp[b, a], d[b, a]) == (mm, cc, dd), (b, a)


def random_tree(rng, n, lo=2, hi=40):
    """A random rooted binary tree on n leaves with even integer branch lengths:
    (joins, lengths) in the oracle's format (children by node id) and the
    leaf-to-leaf path lengths (an additive metric)."""
    nodes = list(range(n))
    joins, lengths = [], []
    nxt = n
    while len(nodes) > 1:
        a, b = rng.choice(len(nodes), size=2, replace=False)
        x, y = nodes[a], nodes[b]
        la, lb = (2 * int(v) for v in rng.integers(lo // 2, hi // 2 + 1, size=2))
        joins.append((x, y))
        lengths.append((float(la), float(lb)))
        nodes = [v for k, v in enumerate(nodes) if k not in (a, b)] + [nxt]
        nxt += 1
    # path lengths: depth of every leaf below each node
    below = {i: {i: 0} for i in range(n)}
    D = np.zeros((n, n), np.int64)
    for t, ((x, y), (lx, ly)) in enumerate(zip(joins, lengths)):
        dx = {k: v + int(lx) for k, v in below[x].items()}
        dy = {k: v + int(ly) for k, v in below[y].items()}
        for i, di in dx.items():
            for j, dj in dy.items():
                D[i, j] = D[j, i] = di + dj
        below[n + t] = {**dx, **dy}
    return joins, lengths, D


@pytest.mark.parametrize("n", [3, 4, 5, 8, 13, 40])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_additive_distances_give_back_their_tree(n, seed):
    rng = np.random.default_rng(1000 * n + seed)
    tj, tl, D = random_tree(rng, n)
    joins, lengths = T.nj(D)
    assert joins.shape == (n - 1, 2)
    want = T.splits(tj, tl, n)
    got = T.splits(joins, lengths, n)
    assert got == want


def test_three_leaves_join_by_the_classic_formulas():
    D = np.array([[0, 10, 14], [10, 0, 18], [14, 18, 0]])
    joins, lengths = T.nj(D)
    # every Q equals -(d01 + d02 + d12): the tie goes to the smallest pair
    assert joins.tolist() == [[0, 1], [3, 2]]
    assert lengths[0].tolist() == [(10 + 14 - 18) / 2, (10 + 18 - 14) / 2]
    assert lengths[1].tolist() == [(14 + 18 - 10) / 4, (14 + 18 - 10) / 4]


def test_ties_go_to_the_smallest_slots():
    # all distances 2: first (0, 1); the new node (5) keeps slot 0 at distance
    # 1 from every other leaf, and Q ties between (slot 0, 2) and the pairs of
    # leaves (-6 each), so slot 0 joins leaf 2 next
    D = np.full((5, 5), 2, np.int64)
    np.fill_diagonal(D, 0)
    joins, lengths = T.nj(D)
    assert joins[0].tolist() == [0, 1] and joins[1].tolist() == [5, 2]
    assert lengths[0].tolist() == [1.0, 1.0]


def test_fixed_point_update_floors():
    # non-additive: (d(i,k) + d(j,k) - d(i,j)) is odd for k = 2 and negative
    # for k = 3; the update floors both
    D = np.array([[0, 5, 4, 0], [5, 0, 2, 1], [4, 2, 0, 9], [0, 1, 9, 0]], np.int64)
    joins, lengths = T.nj(D)
    assert len(joins) == 3
    mism = T.splits(joins, lengths, 4)
    assert len(mism) == 5  # 4 leaf edges + 1 inner edge


def test_one_and_two_rows():
    j, l = T.nj(np.zeros((1, 1), np.int64))
    assert j.shape == (0, 2)
    j, l = T.nj(np.array([[0, 7], [7, 0]]))
    assert j.tolist() == [[0, 1]] and l.tolist() == [[3.5, 3.5]]


def test_newick_of_a_small_tree():
    D = np.array([[0, 10, 14], [10, 0, 18], [14, 18, 0]])
    joins, lengths = T.nj(D)
    assert T.newick(joins, lengths, ["a", "b", "c"]) == "((a:3.0,b:7.0):5.5,c:5.5);"


# ------------------------------------------------------------- clustered tree

def clade_forest(rng, sizes, short=(2, 10), long=(200, 400)):
    """A tree of clades with even integer branches: each clade a random
    rooted binary tree of short branches, the clade roots joined by a random
    backbone of long branches; with 2 sampled leaves on each side of every
    clade root (None when a side has fewer than 2 leaves).  Returns (joins,
    lengths, D, sample)."""
    n = sum(sizes)
    joins, lengths, roots, sample = [], [], [], []
    nxt, base = n, 0
    for m in sizes:
        nodes = list(range(base, base + m))
        while len(nodes) > 1:
            a, b = rng.choice(len(nodes), size=2, replace=False)
            joins.append((nodes[a], nodes[b]))
            lengths.append(tuple(float(2 * int(v)) for v in rng.integers(short[0] // 2, short[1] // 2 + 1, 2)))
            nodes = [v for k, v in enumerate(nodes) if k not in (a, b)] + [nxt]
            nxt += 1
        roots.append(nodes[0])
        base += m
    lv = {i: [i] for i in range(n)}
    for t, (x, y) in enumerate(joins):
        lv[n + t] = lv[x] + lv[y]
    for r in roots:
        x, y = joins[r - n]
        if len(lv[x]) < 2 or len(lv[y]) < 2:
            return None
        sample += list(rng.choice(lv[x], 2, replace=False)) + list(rng.choice(lv[y], 2, replace=False))
    nodes = list(roots)
    while len(nodes) > 1:
        a, b = rng.choice(len(nodes), size=2, replace=False)
        joins.append((nodes[a], nodes[b]))
        lengths.append(tuple(float(2 * int(v)) for v in rng.integers(long[0] // 2, long[1] // 2 + 1, 2)))
        nodes = [v for k, v in enumerate(nodes) if k not in (a, b)] + [nxt]
        nxt += 1
    depth = {i: {i: 0} for i in range(n)}
    D = np.zeros((n, n), np.int64)
    for t, ((x, y), (lx, ly)) in enumerate(zip(joins, lengths)):
        dx = {k: v + int(lx) for k, v in depth[x].items()}
        dy = {k: v + int(ly) for k, v in depth[y].items()}
        for i, di in dx.items():
            for j, dj in dy.items():
                D[i, j] = D[j, i] = di + dj
        depth[n + t] = {**dx, **dy}
    return joins, lengths, D, sorted(int(s) for s in sample)


@pytest.mark.parametrize("seed", [1, 3, 5, 12, 21, 30])
def test_cluster_tree_recovers_a_forest_of_clades(seed):
    """Clades far apart, each sampled on both sides of its root, a cap of the
    4 sampled rows per clade: the clusters are the clades, every row's nearest
    sample row lies in its clade, and the merged tree is the generating tree
    (topology and branch lengths)."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        sizes = [int(v) for v in rng.integers(6, 14, size=int(rng.integers(3, 7)))]
        forest = clade_forest(rng, sizes)
        if forest is not None:
            break
    tj, tl, D, S = forest
    n = D.shape[0]
    joins, lengths, cluster = T.cluster_tree(D, S, 4)
    assert joins.shape == (n - 1, 2)
    assert T.splits(joins, lengths, n) == T.splits(tj, tl, n)
    starts = np.cumsum([0] + sizes)
    for c in range(len(sizes)):  # one cluster per clade
        assert len(set(cluster[starts[c]:starts[c + 1]])) == 1
    assert len(set(cluster)) == len(sizes)


def test_cluster_tree_without_a_cut_is_the_nj_tree():
    _, _, D = random_tree(np.random.default_rng(77), 25)
    joins, lengths, cluster = T.cluster_tree(D, list(range(25)), 25)
    oj, ol = T.nj(D)
    assert T.splits(joins, lengths, 25) == T.splits(oj, ol, 25)
    assert (cluster == 0).all()


def test_cluster_labels_and_post_order():
    """Labels by the definition, written out by brute force: a sample row in
    its own cluster, any other row with its nearest sample row (ties to the
    smaller row); the output lists children before their parents."""
    rng = np.random.default_rng(5)
    n = 60
    R = rng.integers(0, 50, size=(n, n)).astype(np.int64)
    D = np.triu(R, 1) + np.triu(R, 1).T
    S = sorted(int(v) for v in rng.choice(n, 12, replace=False))
    joins, lengths, cluster = T.cluster_tree(D, S, 3)
    Sset = set(S)
    for i in range(n):
        if i in Sset:
            continue
        best = min(S, key=lambda s: (int(D[i, s]), s))
        assert cluster[i] == cluster[best]
    # clusters are numbered by their smallest sample row
    firsts = [min(s for s in S if cluster[s] == c) for c in range(cluster.max() + 1)]
    assert firsts == sorted(firsts)
    for t, (a, b) in enumerate(joins):
        assert a < n + t and b < n + t
    assert sorted(set(joins.ravel().tolist())) == list(range(2 * n - 2))


def test_midpoint_root_of_a_hand_tree():
    """Leaves 0..3 on the tree ((0:1,1:2):3,(2:4,3:10)): the longest path is
    1 -> 3 (2 + 3 + 10 = 15), its middle 7.5 from leaf 3, on the edge to 3:
    the root splits it into 7.5 (toward 3) and 2.5 (toward the rest)."""
    joins = [(0, 1), (2, 3), (4, 5)]
    lengths = [(1.0, 2.0), (4.0, 10.0), (3.0, 0.0)]
    kids, root = T._midpoint_rooted(joins, lengths, 4)
    assert sorted((w, l) for w, l in kids[root]) == sorted([(3, 7.5), (5, 2.5)])
