"""Pins for the CPU oracle: it is checked against things other than itself
(brute-force enumeration, the literal cubic Eq. 2, textbook special cases,
invariants and hand-worked fixtures).  CPU only."""
import os

import numpy as np
import pytest

import oracle
from seqgen import blosum62, dna_matrix, generate, STANDARD_AA, PROTEIN_LETTERS
from tests import _pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_matrix(rng, K, symmetric=True):
    M = rng.integers(-6, 7, size=(K, K)).astype(np.int8)
    if symmetric:
        M = np.triu(M) + np.triu(M, 1).T
    return M.astype(np.int8)


def rand_gaps(rng):
    e = int(rng.integers(1, 4))
    o = e + int(rng.integers(0, 6))
    return o, e


# ----------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(40))
def test_score_and_best_cell_equal_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    K = int(rng.integers(2, 5))
    M = rand_matrix(rng, K, symmetric=bool(seed % 2))
    o, e = rand_gaps(rng)
    la = int(rng.integers(1, 6))
    lb = int(rng.integers(1, 6))
    A = rng.integers(0, K, la)
    B = rng.integers(0, K, lb)
    best, ending = _pins.brute_local(list(A), list(B), M, o, e)
    v, codes, end = oracle.sw(A, B, M, o, e, codes=True)
    assert v == best
    # best cell: smallest i, then smallest j, among cells whose best ending
    # alignment reaches the maximum
    if best == 0:
        assert end == (0, 0)
    else:
        cells = sorted(c for c, s in ending.items() if s == best)
        assert end == cells[0]


@pytest.mark.parametrize("seed", range(4))
def test_length_six_brute_force(seed):
    rng = np.random.default_rng(77 + seed)
    M = rand_matrix(rng, 3)
    o, e = rand_gaps(rng)
    A = rng.integers(0, 3, 6)
    B = rng.integers(0, 3, 6)
    best, _ = _pins.brute_local(list(A), list(B), M, o, e)
    assert oracle.sw(A, B, M, o, e) == best


# ----------------------------------------------------------- literal Eq. (2)

@pytest.mark.parametrize("seed", range(12))
def test_gotoh_equals_literal_eq2(seed):
    rng = np.random.default_rng(2000 + seed)
    K = int(rng.integers(3, 8))
    M = rand_matrix(rng, K, symmetric=bool(seed % 3))
    o, e = rand_gaps(rng)
    A = rng.integers(0, K, int(rng.integers(1, 41)))
    B = rng.integers(0, K, int(rng.integers(1, 41)))
    H = _pins.eq2_literal(A, B, M, o, e)
    v, _, end = oracle.sw(A, B, M, o, e, codes=True)
    assert v == int(H.max())
    assert end == _pins.first_argmax(H)


@pytest.mark.parametrize("seed", range(8))
def test_equal_open_extend_is_linear_gap_sw(seed):
    rng = np.random.default_rng(3000 + seed)
    _, M = blosum62()
    g = int(rng.integers(1, 12))
    A = rng.integers(0, 20, int(rng.integers(1, 60)))
    B = rng.integers(0, 20, int(rng.integers(1, 60)))
    assert oracle.sw(A, B, M, g, g) == _pins.linear_sw(A, B, M, g)


# ----------------------------------------------------------- invariants

def test_self_score_is_diagonal_sum_for_blosum62():
    _, M = blosum62()
    rng = np.random.default_rng(5)
    for _ in range(20):
        A = rng.integers(0, 20, int(rng.integers(1, 300)))
        assert oracle.sw(A, A, M, 11, 1) == int(sum(int(M[a][a]) for a in A))


def test_symmetry_and_nonnegativity():
    _, M = blosum62()
    rng = np.random.default_rng(6)
    for _ in range(20):
        A = rng.integers(0, 24, int(rng.integers(1, 200)))
        B = rng.integers(0, 24, int(rng.integers(1, 200)))
        s1 = oracle.sw(A, B, M, 11, 1)
        assert s1 == oracle.sw(B, A, M, 11, 1) and s1 >= 0


def test_blosum62_table_properties():
    letters, M = blosum62()
    assert letters == PROTEIN_LETTERS
    assert (M == M.T).all()
    d = np.diag(M).astype(int)
    # dominance: s(a,b) <= (s(a,a) + s(b,b)) / 2, which makes d(A,B) >= 0
    assert (2 * M.astype(int) <= d[:, None] + d[None, :]).all()
    assert M[letters.index("W"), letters.index("W")] == 11
    assert M[letters.index("A"), letters.index("A")] == 4


# ----------------------------------------------------------- golden fixtures

def _golden_matrix(spec):
    if spec == "dna":
        return dna_matrix(2, -3)
    if spec == "abc":
        M = np.full((3, 3), -20, np.int8)
        np.fill_diagonal(M, 10)
        return "ABC", M
    if spec == "abcdxy":
        M = np.full((6, 6), -20, np.int8)
        np.fill_diagonal(M, 10)
        M[2, 4] = M[4, 2] = 14
        return "ABCDXY", M
    raise KeyError(spec)


def _golden_cases():
    out = []
    for ln in open(os.path.join(GOLDEN, "traceback_cases.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        f = [x.strip() for x in ln.split("|")]
        out.append(dict(name=f[0], matrix=f[1], o=int(f[2]), e=int(f[3]), c=f[4], s=f[5],
                        score=int(f[6]), end=tuple(map(int, f[7].split())),
                        seg=tuple(map(int, f[8].split())),
                        ins=list(map(int, f[9].split())), occ=list(map(int, f[10].split()))))
    return out


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hand_worked_traceback(case):
    alphabet, M = _golden_matrix(case["matrix"])
    c = oracle.encode(case["c"].encode(), alphabet)
    s = oracle.encode(case["s"].encode(), alphabet)
    v, codes, end = oracle.sw(c, s, M, case["o"], case["e"], codes=True)
    assert v == case["score"]
    assert end == case["end"]
    ins, occ, seg = oracle.traceback(codes, v, end)
    assert seg == case["seg"]
    assert list(ins) == case["ins"]
    assert list(occ) == case["occ"]


def _sp_cases():
    out = []
    for ln in open(os.path.join(GOLDEN, "sp_cases.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        f = [x.strip() for x in ln.split("|")]
        out.append((f[0], f[1].split(), int(f[2])))
    return out


@pytest.mark.parametrize("case", _sp_cases(), ids=lambda c: c[0])
def test_hand_counted_sp(case):
    _, rows, sp = case
    msa = np.array([list(r.encode()) for r in rows], dtype=np.uint8)
    assert oracle.sp_pairwise(msa) == sp
    assert oracle.sp_columns(msa) == sp


# ----------------------------------------------------------- traceback validity

@pytest.mark.parametrize("seed", range(10))
def test_traceback_is_an_optimal_path(seed):
    rng = np.random.default_rng(4000 + seed)
    K = int(rng.integers(3, 6))
    M = rand_matrix(rng, K)
    o, e = rand_gaps(rng)
    A = rng.integers(0, K, int(rng.integers(1, 30)))
    B = rng.integers(0, K, int(rng.integers(1, 30)))
    v, codes, end = oracle.sw(A, B, M, o, e, codes=True)
    ins, occ, seg = oracle.traceback(codes, v, end)
    assert int(ins.sum()) + int(occ.sum()) == len(B)
    cols = _pins.pairwise_columns(ins, occ, len(A), len(B))
    assert _pins.rescore_segment(cols, A, B, seg, M, o, e) == v
    # flank pairs outside the segment are gap-free except the surplus residues
    i1, j1, i2, j2 = seg
    for ci, si in cols:
        if ci is not None and si is not None and not (i1 < ci <= i2):
            assert ci - si == (i1 - j1 if ci <= i1 else i2 - j2)


# ----------------------------------------------------------- merge + SP

def _small_problem(name="plain_protein_200", n=24, seed=None):
    letters, offsets, w, _ = generate(name, n=n, seed=seed)
    alph, M = (blosum62() if w.kind == "protein" else dna_matrix(2, -3))
    return oracle.Problem(letters, offsets, alph, M, w.gap_open, w.gap_extend), letters, offsets


def test_merge_invariants():
    prob, letters, offsets = _small_problem(n=30)
    center = 7
    seg, ins, occ, G, W, msa = oracle.msa(prob, center)
    lc = prob.length(center)
    assert W == lc + int(G.sum())
    assert (G == ins.max(axis=0)).all()
    for t in range(prob.n):
        row = bytes(msa[t])
        assert row.replace(b"-", b"") == bytes(letters[offsets[t]:offsets[t + 1]])
    # the center's own row is the center with G[j] gaps in slot j
    crow = bytes(msa[center])
    exp = b"".join(b"-" * int(G[j]) + (bytes([letters[offsets[center] + j]]) if j < lc else b"")
                   for j in range(lc + 1))
    assert crow == exp
    # projecting (center, row t) and dropping gap-gap columns gives the row's
    # pairwise alignment (ins/occ), and its segment re-scores to the score
    for t in range(prob.n):
        pairs = [(a, b) for a, b in zip(msa[center], msa[t]) if not (a == 45 and b == 45)]
        cols = _pins.pairwise_columns(ins[t], occ[t], lc, prob.length(t))
        assert len(pairs) == len(cols)
        for (a, b), (ci, si) in zip(pairs, cols):
            assert (a == 45) == (ci is None) and (b == 45) == (si is None)
        assert _pins.rescore_segment(cols, prob.seq(center), prob.seq(t), tuple(seg[t, 1:]),
                                     prob.M, prob.o, prob.e) == seg[t, 0]


def _msa_golden():
    out = []
    for ln in open(os.path.join(GOLDEN, "msa_cases.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        f = [x.strip() for x in ln.split("|")]
        rows = []
        for ent in f[2].split(";"):
            seq, ins, occ = [x.strip() for x in ent.split("/")]
            rows.append((seq, [int(v) for v in ins.split()], [int(v) for v in occ.split()]))
        out.append(dict(name=f[0], center=f[1], rows=rows, G=[int(v) for v in f[3].split()],
                        W=int(f[4]), msa=f[5].split()))
    return out


@pytest.mark.parametrize("case", _msa_golden(), ids=lambda c: c["name"])
def test_hand_written_merge(case):
    """Inserted residues are left-justified in their slot (gaps after them)."""
    alphabet, M = dna_matrix(2, -3)
    seqs = [r[0].encode() for r in case["rows"]]
    assert seqs[0] == case["center"].encode()
    offsets = np.concatenate([[0], np.cumsum([len(x) for x in seqs])])
    prob = oracle.Problem(np.frombuffer(b"".join(seqs), np.uint8), offsets, alphabet, M, 5, 2)
    ins = np.array([r[1] for r in case["rows"]], dtype=np.uint16)
    occ = np.array([r[2] for r in case["rows"]], dtype=np.uint8)
    G, W, msa = oracle.merge(prob, 0, ins, occ)
    assert list(G) == case["G"] and W == case["W"]
    assert [bytes(r).decode() for r in msa] == case["msa"]


def test_sp_columns_equal_pairwise():
    prob, _, _ = _small_problem(n=20)
    *_, msa = oracle.msa(prob, 3)
    assert oracle.sp_columns(msa) == oracle.sp_pairwise(msa)
    rng = np.random.default_rng(9)
    rnd = rng.choice(np.frombuffer(b"ACG-", np.uint8), size=(13, 31))
    assert oracle.sp_columns(rnd) == oracle.sp_pairwise(rnd)


# ----------------------------------------------------------- exact center

ONE = 1 << 16


def _distance_matrix(S):
    """d(A,B) = 2^16 - floor(2^16 S(A,B) / max(S(A,A), S(B,B))), 0 when that max is 0."""
    S = np.asarray(S, dtype=np.int64)
    m = np.maximum(np.diag(S)[:, None], np.diag(S)[None, :])
    d = np.zeros_like(S)
    pos = m > 0
    d[pos] = ONE - (S[pos] * ONE) // m[pos]
    return d


@pytest.mark.parametrize("seed", range(3))
def test_exact_center_equals_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    K = 3
    M = rand_matrix(rng, K)
    np.fill_diagonal(M, rng.integers(2, 6, K))
    o, e = rand_gaps(rng)
    seqs = [rng.integers(0, K, int(rng.integers(1, 5))) for _ in range(9)]
    S = np.array([[_pins.brute_local(list(a), list(b), M, o, e)[0] for b in seqs] for a in seqs])
    d = _distance_matrix(S)
    rowsum = d.sum(axis=1)
    letters = "".join("ABC"[x] for s in seqs for x in s).encode()
    offsets = np.concatenate([[0], np.cumsum([len(s) for s in seqs])])
    prob = oracle.Problem(np.frombuffer(letters, np.uint8), offsets, "ABC", M, o, e)
    c, rs = oracle.exact_center(prob)
    assert (rs == rowsum).all()
    assert c == int(np.argmin(rowsum))
    # a reference subset sums over that subset only
    refs = np.array([1, 4, 6])
    c2, rs2 = oracle.exact_center(prob, refs=refs)
    exp2 = d[:, refs].sum(axis=1)
    assert (rs2 == exp2).all() and c2 == int(np.argmin(exp2))


def _center_golden():
    out = []
    for ln in open(os.path.join(GOLDEN, "center_cases.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        f = [x.strip() for x in ln.split("|")]
        ints = lambda x: [int(v) for v in x.split()]
        out.append(dict(name=f[0], matrix=f[1], o=int(f[2]), e=int(f[3]), seqs=f[4].split(),
                        self=ints(f[5]), S=ints(f[6]), d=ints(f[7]), rowsum=ints(f[8]),
                        center=int(f[9])))
    return out


def _center_matrix(spec):
    M = np.full((2, 2), -1, np.int8)
    M[0, 0] = 2
    M[1, 1] = 2 if spec == "ab" else 0
    return "AB", M


@pytest.mark.parametrize("case", _center_golden(), ids=lambda c: c["name"])
def test_hand_worked_center(case):
    alphabet, M = _center_matrix(case["matrix"])
    seqs = [s.encode() for s in case["seqs"]]
    offsets = np.concatenate([[0], np.cumsum([len(s) for s in seqs])])
    prob = oracle.Problem(np.frombuffer(b"".join(seqs), np.uint8), offsets, alphabet, M,
                          case["o"], case["e"])
    n = prob.n
    iu = [(i, j) for i in range(n) for j in range(i + 1, n)]
    assert list(oracle.pair_scores(prob, [(i, i) for i in range(n)])) == case["self"]
    assert list(oracle.pair_scores(prob, iu)) == case["S"]
    # d of each pair: the row sum over a single reference
    for (i, j), dv in zip(iu, case["d"]):
        _, rs = oracle.exact_center(prob, refs=np.array([j]))
        assert rs[i] == dv
        _, rs = oracle.exact_center(prob, refs=np.array([i]))
        assert rs[j] == dv
    c, rs = oracle.exact_center(prob)
    assert list(rs) == case["rowsum"]
    assert c == case["center"]


def test_distance_properties_on_protein_set():
    prob, _, _ = _small_problem(n=12)
    pairs = np.array([(i, j) for i in range(prob.n) for j in range(prob.n)])
    S = oracle.pair_scores(prob, pairs).reshape(prob.n, prob.n)
    assert (S == S.T).all()
    d = _distance_matrix(S)
    # zero on the diagonal, symmetric, and in [0, 2^16] under BLOSUM62's
    # dominance s(a,b) <= (s(a,a) + s(b,b)) / 2 (a local score never exceeds
    # the larger self score)
    assert (np.diag(d) == 0).all() and (d == d.T).all()
    assert (d >= 0).all() and (d <= ONE).all()
    _, rs = oracle.exact_center(prob)
    assert (rs == d.sum(axis=1)).all()


def _workload_subset(name, m, seed, keep_first=False):
    letters, offsets, w, _ = generate(name, n=min(w_n(name), 4000))
    rng = np.random.default_rng(seed)
    n = offsets.size - 1
    idx = np.sort(rng.choice(n, size=m, replace=False))
    if keep_first:
        idx = np.unique(np.concatenate([[0], idx[1:]]))
    seqs = [letters[offsets[i]:offsets[i + 1]] for i in idx]
    alph, M = (blosum62() if w.kind == "protein" else dna_matrix(2, -3))
    offs = np.concatenate([[0], np.cumsum([len(s) for s in seqs])])
    return oracle.Problem(np.concatenate(seqs), offs, alph, M, w.gap_open, w.gap_extend)


def w_n(name):
    from seqgen import WORKLOADS
    return WORKLOADS[name].n


@pytest.mark.parametrize("name", ["batched_uneven_10k", "learned_center_50k"])
def test_exact_center_is_not_a_length_proxy(name):
    """On 200-sequence samples of the uneven multi-family protein sets the
    center is neither the shortest nor the longest sequence (the row sums of
    S(A,A) + S(B,B) - 2 S(A,B) rank sequences by length: correlation 1.00
    and the shortest sequence as center on these samples)."""
    prob = _workload_subset(name, 200, 3)
    lens = np.diff(prob.off)
    c, rs = oracle.exact_center(prob)
    corr = float(np.corrcoef(rs, lens)[0, 1])
    print(f"{name}: center length {lens[c]}, length range {lens.min()}-{lens.max()}, "
          f"corr(row sum, length) {corr:+.3f}")
    lo, hi = np.percentile(lens, [10, 90])
    assert lo <= lens[c] <= hi
    assert abs(corr) < 0.99


def test_exact_center_ranks_the_common_ancestor_first():
    """Short peptides cut (and mutated) from one 500-residue ancestor, with the
    ancestor itself in the set: the ancestor's local alignments reach a large
    fraction of every peptide's self score, so its row sum is among the
    smallest 2 % (the shortest peptide's is not)."""
    prob = _workload_subset("short_peptides_1m", 200, 1, keep_first=True)
    c, rs = oracle.exact_center(prob)
    lens = np.diff(prob.off)
    assert lens[0] == 500
    assert int((rs < rs[0]).sum()) <= 0.02 * prob.n
    assert int((rs < rs[int(np.argmin(lens))]).sum()) > 0.5 * prob.n
