"""Oracle of the phylogenetic tree over the MSA (test infrastructure only:
the tests, the smoke check and the bench's CPU baseline use it; the product
path never imports it).

The paper builds the tree of the aligned sequences by neighbour joining (the
section on NJ trees with Spark, Figure 4, citing Saitou and Nei), but states
neither the distance nor the arithmetic.  Readings, shared with the GPU tree:

- distance of two MSA rows: the p-distance over the columns where both rows
  hold a residue (gap '-' in either row: the column is not compared), in
  fixed point: d = floor(2^20 * mismatches / compared); d = 2^20 when no
  column is compared;
- neighbour joining on those integers, m nodes active: r_i = sum_k d(i, k)
  over the active k; Q(i, j) = (m - 2) d(i, j) - r_i - r_j for active i < j
  (slots numbered as the input rows, a new node taking the slot of the first
  of its two children); the smallest Q joins, ties to the smallest i, then
  the smallest j; branch lengths ((m - 2) d(i, j) + r_i - r_j) / (2 (m - 2))
  to i and ((m - 2) d(i, j) - r_i + r_j) / (2 (m - 2)) to j, each one double
  division of two integers; the new node's distances
  d(u, k) = floor((d(i, k) + d(j, k) - d(i, j)) / 2); when two nodes remain
  they join at the middle of the edge between them (d / 2 each), which roots
  the tree.  Node ids: the rows are 0 .. n-1, the t-th join creates n + t.

Exact integer arithmetic except the branch lengths, which are one correctly
rounded division each, so the GPU tree equals this one bit for bit.
"""
import numpy as np

DSCALE = 1 << 20
GAP = ord("-")


def msa_counts(rows):
    """(mismatches, compared) int64[n, n] of the MSA rows (uint8 letters, '-'
    for gaps): compared = columns where both rows hold a residue, mismatches =
    those of them whose residues differ."""
    rows = np.ascontiguousarray(rows, dtype=np.uint8)
    n = rows.shape[0]
    res = rows != GAP
    mism = np.zeros((n, n), np.int64)
    comp = np.zeros((n, n), np.int64)
    for a in range(n):
        both = res & res[a]
        comp[a] = both.sum(axis=1)
        mism[a] = (both & (rows != rows[a])).sum(axis=1)
    return mism, comp


def msa_distances(rows):
    """Fixed-point p-distances int64[n, n] of the MSA rows."""
    mism, comp = msa_counts(rows)
    return np.where(comp > 0, (DSCALE * mism) // np.maximum(comp, 1), DSCALE).astype(np.int64)


def nj(d):
    """Neighbour joining of the integer distance matrix d (n x n, symmetric,
    zero diagonal).  Returns (joins int64[n-1, 2] node ids, lengths
    float64[n-1, 2]); joins[t] creates node n + t, the last one is the root
    (empty for n = 1)."""
    D = np.array(d, dtype=np.int64)
    n = D.shape[0]
    if n < 2:
        return np.zeros((0, 2), np.int64), np.zeros((0, 2), np.float64)
    node = list(range(n))
    active = list(range(n))
    joins, lengths = [], []
    big = np.iinfo(np.int64).max
    while len(active) > 2:
        m = len(active)
        A = np.array(active)
        sub = D[np.ix_(A, A)]
        r = sub.sum(axis=1)
        Q = (m - 2) * sub - r[:, None] - r[None, :]
        Q[np.tril_indices(m)] = big  # pairs i < j only
        x, y = divmod(int(np.argmin(Q)), m)  # first minimum: smallest i, then j
        i, j = int(A[x]), int(A[y])
        dij = int(D[i, j])
        den = float(2 * (m - 2))
        bl_i = float((m - 2) * dij + int(r[x]) - int(r[y])) / den
        bl_j = float((m - 2) * dij - int(r[x]) + int(r[y])) / den
        joins.append((node[i], node[j]))
        lengths.append((bl_i, bl_j))
        for k in active:
            if k != i and k != j:
                D[i, k] = D[k, i] = (int(D[i, k]) + int(D[j, k]) - dij) >> 1
        D[i, i] = 0
        node[i] = n + len(joins) - 1
        active.remove(j)
    a, b = active
    joins.append((node[a], node[b]))
    half = float(D[a, b]) / 2.0
    lengths.append((half, half))
    return np.array(joins, np.int64), np.array(lengths, np.float64)


def newick(joins, lengths, names=None):
    """The rooted tree in Newick form (leaves named by `names` or their row)."""
    n = len(joins) + 1
    names = names or [str(i) for i in range(n)]
    text = {i: names[i] for i in range(n)}
    for t, ((a, b), (la, lb)) in enumerate(zip(joins, lengths)):
        text[n + t] = "(%s:%r,%s:%r)" % (text[int(a)], float(la), text[int(b)], float(lb))
    return text[n + len(joins) - 1] + ";" if len(joins) else names[0] + ";"


def splits(joins, lengths, n):
    """The tree as {frozenset of leaves below an edge: edge length}, with the
    two root edges merged into one edge (the unrooted tree NJ estimates)."""
    below = {i: frozenset([i]) for i in range(n)}
    edges = {}
    for t, ((a, b), (la, lb)) in enumerate(zip(joins, lengths)):
        u = n + t
        below[u] = below[int(a)] | below[int(b)]
        for c, l in ((int(a), la), (int(b), lb)):
            s = below[c]
            key = min(s, frozenset(range(n)) - s, key=lambda z: (len(z), sorted(z)))
            edges[key] = edges.get(key, 0.0) + l
    return edges
