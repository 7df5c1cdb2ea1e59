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


def test_sp_columns_equal_pairwise():
    prob, _, _ = _small_problem(n=20)
    *_, msa = oracle.msa(prob, 3)
    assert oracle.sp_columns(msa) == oracle.sp_pairwise(msa)
    rng = np.random.default_rng(9)
    rnd = rng.choice(np.frombuffer(b"ACG-", np.uint8), size=(13, 31))
    assert oracle.sp_columns(rnd) == oracle.sp_pairwise(rnd)


# ----------------------------------------------------------- exact center

@pytest.mark.parametrize("seed", range(3))
def test_exact_center_equals_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    K = 3
    M = rand_matrix(rng, K)
    np.fill_diagonal(M, rng.integers(2, 6, K))
    o, e = rand_gaps(rng)
    seqs = [rng.integers(0, K, int(rng.integers(1, 5))) for _ in range(9)]
    S = np.array([[_pins.brute_local(list(a), list(b), M, o, e)[0] for b in seqs] for a in seqs])
    d = np.diag(S)[:, None] + np.diag(S)[None, :] - 2 * S
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


def test_distance_properties_on_protein_set():
    prob, _, _ = _small_problem(n=12)
    pairs = np.array([(i, j) for i in range(prob.n) for j in range(prob.n)])
    S = oracle.pair_scores(prob, pairs).reshape(prob.n, prob.n)
    assert (S == S.T).all()
    d = np.diag(S)[:, None] + np.diag(S)[None, :] - 2 * S.astype(np.int64)
    assert (np.diag(d) == 0).all() and (d >= 0).all()
