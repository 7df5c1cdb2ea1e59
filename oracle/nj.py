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


# ----------------------------------------------------------------------------
# The tree of a large set by clusters (the paper's tree section, Figure 4: a
# ~10 % sample is clustered, every sequence is labelled with a cluster, one
# tree is built per cluster, and the cluster trees are merged).  Reading,
# shared with the GPU:
#   1. the NJ tree of the sample rows (the sample sorted ascending), rooted at
#      the middle of its longest leaf-to-leaf path (the path found from the
#      smallest sample leaf: its farthest leaf, then that leaf's farthest;
#      ties to the smaller leaf; lengths summed from that second end; a
#      middle that falls on a node roots on that node's edge toward the second
#      end);
#   2. clusters: starting from its root, the subtree holding the most sample
#      rows (ties: the smaller node id) is replaced by its two children until
#      no subtree holds more than `cap` sample rows; clusters are numbered in
#      the order of their smallest sample row;
#   3. a sample row belongs to its own cluster; any other row to the cluster of
#      its nearest sample row (smallest distance, ties: the smaller row);
#   4. per cluster, the NJ tree of its rows plus an outgroup -- the sample row
#      outside the cluster nearest to the cluster's sample rows (ties: the
#      smaller outgroup row, then the smaller cluster row) -- rooted where the
#      outgroup joins it, the outgroup then removed (one cluster: the NJ tree
#      of all rows as it is rooted; one row: that leaf);
#   5. every cluster's subtree of the sample tree is replaced by the cluster's
#      tree, the edge above it keeping its length;
#   6. output in post-order, each node's children ordered by their smallest
#      row, internal nodes numbered n, n + 1, ... in that order.


def _reroot(joins, lengths, nleaf, out_leaf):
    """The tree of (joins, lengths) over leaves 0..nleaf-1 as an unrooted tree
    (the root's two edges one edge), rooted where leaf `out_leaf` joins it and
    without that leaf: {node: [(child, length), ...]}, root."""
    adj = {}

    def link(a, b, l):
        adj.setdefault(a, []).append((b, l))
        adj.setdefault(b, []).append((a, l))
    T = len(joins)
    for t in range(T - 1):
        (a, b), (la, lb) = joins[t], lengths[t]
        link(nleaf + t, int(a), float(la))
        link(nleaf + t, int(b), float(lb))
    (a, b), (la, lb) = joins[T - 1], lengths[T - 1]
    link(int(a), int(b), float(la) + float(lb))
    root = adj[out_leaf][0][0]
    children, stack, seen = {}, [root], {root, out_leaf}
    while stack:
        v = stack.pop()
        children[v] = []
        for w, l in adj[v]:
            if w not in seen:
                seen.add(w)
                children[v].append((w, l))
                stack.append(w)
    return children, root


def _unrooted(joins, lengths, nleaf):
    """Adjacency {node: [(neighbour, length)]} of the tree of (joins, lengths)
    with the root's two edges joined into one."""
    adj = {}

    def link(a, b, l):
        adj.setdefault(a, []).append((b, l))
        adj.setdefault(b, []).append((a, l))
    T = len(joins)
    for t in range(T - 1):
        (a, b), (la, lb) = joins[t], lengths[t]
        link(nleaf + t, int(a), float(la))
        link(nleaf + t, int(b), float(lb))
    (a, b), (la, lb) = joins[T - 1], lengths[T - 1]
    link(int(a), int(b), float(la) + float(lb))
    for v in adj:
        adj[v].sort()
    return adj


def _farthest(adj, src, nleaf):
    """(leaf farthest from src, its distance, parent links of the search):
    distances summed along the path from src, ties to the smaller leaf."""
    dist, par, stack = {src: 0.0}, {src: None}, [src]
    while stack:
        v = stack.pop()
        for w, l in adj[v]:
            if w not in dist:
                dist[w] = dist[v] + l
                par[w] = (v, l)
                stack.append(w)
    best = min((v for v in dist if v < nleaf), key=lambda v: (-dist[v], v))
    return best, dist[best], par


def _midpoint_rooted(joins, lengths, nleaf):
    """The tree rooted at the middle of its longest leaf-to-leaf path:
    {node: [(child, length), ...]}, root (a new node "r" on that edge)."""
    adj = _unrooted(joins, lengths, nleaf)
    a, _, _ = _farthest(adj, 0, nleaf)
    b, total, par = _farthest(adj, a, nleaf)
    half = total / 2.0
    # walk from b toward a: the edge (v, u) where the path passes the middle
    v, walked = b, 0.0
    while True:  # the last edge of the path at the latest (negative lengths)
        u, l = par[v]
        if walked + l >= half or u == a:
            break
        walked += l
        v = u
    x = half - walked  # distance from v along the edge toward u
    adj[v] = [(w, ll) for w, ll in adj[v] if w != u]
    adj[u] = [(w, ll) for w, ll in adj[u] if w != v]
    adj["r"] = [(v, x), (u, l - x)]
    adj[v].append(("r", x))
    adj[u].append(("r", l - x))
    children, stack, seen = {}, ["r"], {"r"}
    while stack:
        w = stack.pop()
        children[w] = []
        for y, ll in adj[w]:
            if y not in seen:
                seen.add(y)
                children[w].append((y, ll))
                stack.append(y)
    return children, "r"


def cluster_tree(D, sample, cap):
    """The clustered tree of the rows of the n x n distance matrix D.
    Returns (joins int64[n-1, 2], lengths float64[n-1, 2], cluster int32[n])."""
    import sys
    D = np.asarray(D, dtype=np.int64)
    n = D.shape[0]
    sys.setrecursionlimit(max(sys.getrecursionlimit(), 4 * n + 1000))  # trees as deep as n
    S = sorted(set(int(s) for s in sample))
    m = len(S)
    sj, sl = nj(D[np.ix_(S, S)])
    # sample tree, midpoint-rooted: node -> [(child, length)], sample-local
    # leaf ids 0..m-1
    if m > 1:
        kids, root_s = _midpoint_rooted(sj, sl, m)
    else:
        kids, root_s = {0: []}, 0
    leaves = {}

    def gather(v):
        if v not in leaves:
            leaves[v] = [v] if not kids.get(v) else sum((gather(w) for w, _ in kids[v]), [])
        return leaves[v]
    gather(root_s)
    order = {v: k for k, v in enumerate(sorted((v for v in leaves if not isinstance(v, str)),
                                               key=lambda v: v))}
    order["r"] = -1
    cuts = [root_s]
    while True:
        big = max(cuts, key=lambda v: (len(leaves[v]), -order[v]))
        if len(leaves[big]) <= cap:
            break
        cuts.remove(big)
        cuts += [kids[big][0][0], kids[big][1][0]]
    cuts.sort(key=lambda v: min(S[l] for l in leaves[v]))
    q = len(cuts)
    of_leaf = {}
    for c, v in enumerate(cuts):
        for l in leaves[v]:
            of_leaf[l] = c
    cluster = np.zeros(n, np.int32)
    for i in range(n):
        if i in S:
            cluster[i] = of_leaf[S.index(i)]
        else:
            k = min(range(m), key=lambda x: (int(D[i, S[x]]), S[x]))
            cluster[i] = of_leaf[k]
    # the final tree as {node: [(child, length)]}; rows keep ids 0..n-1,
    # other nodes get private keys
    tree, key = {}, [n]

    def fresh():
        key[0] += 1
        return ("x", key[0])

    def graft(children, root, name):
        """Copy a rooted tree whose leaves are named by `name` into `tree`."""
        def walk(v):
            if v not in children or not children[v]:
                return name(v)
            u = fresh()
            tree[u] = [(walk(w), l) for w, l in children[v]]
            return u
        return walk(root)

    cl_root = {}
    for c, v in enumerate(cuts):
        R = [int(i) for i in np.flatnonzero(cluster == c)]
        if len(R) == 1:
            cl_root[v] = R[0]
            continue
        if q == 1:
            jj, ll = nj(D[np.ix_(R, R)])
            ch = {len(R) + t: [(int(a), float(la)), (int(b), float(lb))]
                  for t, ((a, b), (la, lb)) in enumerate(zip(jj, ll))}
            cl_root[v] = graft(ch, 2 * len(R) - 2, lambda x: R[x])
            continue
        inside = [S[l] for l in leaves[v]]
        outside = [s for s in S if cluster[s] != c]
        o = min(outside, key=lambda s: (min(int(D[t, s]) for t in inside), s))
        U = sorted(R + [o])
        jj, ll = nj(D[np.ix_(U, U)])
        ch, r = _reroot(jj, ll, len(U), U.index(o))
        cl_root[v] = graft(ch, r, lambda x: U[x])
    if q == 1:
        root = cl_root[cuts[0]]
    else:
        def walk_s(v):
            if v in cl_root:
                return cl_root[v]
            u = fresh()
            tree[u] = [(walk_s(w), l) for w, l in kids[v]]
            return u
        root = walk_s(root_s)
    # post-order, children by smallest row
    low = {}

    def lowest(v):
        if v not in low:
            low[v] = v if not isinstance(v, tuple) else min(lowest(w) for w, _ in tree[v])
        return low[v]
    joins, lengths, ids = [], [], {}

    def emit(v):
        if not isinstance(v, tuple):
            return v
        (a, la), (b, lb) = sorted(tree[v], key=lambda e: lowest(e[0]))
        ia, ib = emit(a), emit(b)
        joins.append((ia, ib))
        lengths.append((la, lb))
        ids[v] = n + len(joins) - 1
        return ids[v]
    if n > 1:
        emit(root)
    return (np.array(joins, np.int64).reshape(-1, 2), np.array(lengths, np.float64).reshape(-1, 2),
            cluster)
