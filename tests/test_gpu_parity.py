"""GPU path vs the CPU oracle through the C ABI: bit-exact scores, best cells,
traceback codes, inserted-space rows, merged MSAs, SP costs and centers."""
import numpy as np
import pytest

import oracle
from seqgen import reference_sample, blosum62, dna_matrix, STANDARD_AA, pack_sequences
from tests._gpu import binding, workload, make_ctx, oracle_problem, random_set

pytestmark = pytest.mark.gpu


def run_pipeline(b, h, letters, offsets, center):
    b.msa_load(h, letters, offsets)
    scores = np.zeros(offsets.size - 1, np.int32)
    b.msa_align_to_center(h, center, scores)
    seg, ins, occ = b.msa_alignment_info(h)
    rows, W = b.msa_merge_gaps(h)
    sp = b.msa_sp_score(h)
    return scores, seg, ins, occ, rows, W, sp


def check_against_oracle(prob, center, scores, seg, ins, occ, rows, W, sp):
    oseg, oins, oocc, oG, oW, orows = oracle.msa(prob, center)
    assert (scores == oseg[:, 0]).all()
    assert (seg == oseg).all()
    assert (ins == oins).all()
    assert (occ == oocc).all()
    assert W == oW
    assert (rows == orows).all()
    assert sp == oracle.sp_columns(orows)


# ------------------------------------------------------------- pair scores

@pytest.mark.parametrize("precision", [0, 2])
def test_pair_scores_random_lengths(precision):
    b = binding()
    rng = np.random.default_rng(11)
    alph, M = blosum62()
    letters, offsets = random_set(rng, 60, 1, 1300, alph, STANDARD_AA)
    prob = oracle_problem(letters, offsets, alph, M, 11, 1)
    pairs = rng.integers(0, 60, size=(300, 2))
    pairs[:60] = np.stack([np.arange(60), np.arange(60)], 1)  # self pairs
    with make_ctx(alph, M, 11, 1, precision=precision) as h:
        b.msa_load(h, letters, offsets)
        got = b.msa_pair_scores(h, pairs)
    assert (got == oracle.pair_scores(prob, pairs)).all()


# ------------------------------------------------------------- center

def test_exact_center_plain_protein_200():
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200")
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    oc, orow = oracle.exact_center(prob)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        rows = b.msa_center_rowsums(h)
    assert (rows == orow).all()
    assert c == oc and s == orow[oc]


def test_exact_center_graph_on_any_stream():
    """The length-bucketed center kernels run as one captured CUDA graph
    launched on the context's stream: on the legacy default stream and on a
    side stream, twice in a row on one context, the row sums are the
    oracle's."""
    import torch
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=150, seed=9)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    oc, orow = oracle.exact_center(prob)
    for stream in (None, torch.cuda.Stream()):
        with make_ctx(alph, M, w.gap_open, w.gap_extend, stream=stream) as h:
            b.msa_load(h, letters, offsets)
            for _ in range(2):
                c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT)
                assert c == oc and s == orow[oc]
                assert (b.msa_center_rowsums(h) == orow).all()


@pytest.mark.parametrize("precision,sat", [(2, 0), (1, 0), (1, 300)])
def test_exact_center_precisions_and_overflow_recheck(precision, sat):
    """int32 cells, packed int16 cells, and packed cells with a low overflow
    guard (most pairs re-run in int32) all give the oracle's row sums."""
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=120, seed=5)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    oc, orow = oracle.exact_center(prob)
    with make_ctx(alph, M, w.gap_open, w.gap_extend, precision=precision, sat_limit=sat) as h:
        b.msa_load(h, letters, offsets)
        c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        rows = b.msa_center_rowsums(h)
    assert (rows == orow).all() and c == oc


def test_sampled_center():
    b = binding()
    letters, offsets, w, alph, M = workload("learned_center_50k", n=400, seed=3)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    refs = reference_sample(400, 37, seed=9)
    oc, orow = oracle.exact_center(prob, refs=refs)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT_SAMPLED, refs=refs)
        rows = b.msa_center_rowsums(h)
    assert (rows == orow).all() and c == oc and s == orow[oc]


# ------------------------------------------------------------- alignment + merge

@pytest.mark.parametrize("lanes", [0, 1, 2, 4])
@pytest.mark.parametrize("precision", [0, 2])
def test_codes_and_best_cells_bitexact(precision, lanes):
    """Codes of every cell: int16 lanes carrying two subjects (automatic
    precision; odd sorted positions are recomputed in the high lane) and
    int32 cells, with the modelled group width and with 1 (every lane its
    own subjects, the center in 16-row passes), 2 and 4 lanes per group.
    Both extension bits match everywhere; the source bits match wherever
    H > 0 (the oracle's source is nonzero): where H = 0 the traceback stops
    on the score it carries, so the packed kernel stores no zero source
    there (1, 2 or 3 instead)."""
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=13, seed=2)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    center = 4
    with make_ctx(alph, M, w.gap_open, w.gap_extend, precision=precision) as h:
        b.msa_set_align_group(h, lanes)
        b.msa_load(h, letters, offsets)
        b.msa_align_to_center(h, center)
        seg, _, _ = b.msa_alignment_info(h)
        for t in range(prob.n):
            codes = b.msa_debug_codes(h, t, prob.length(t))
            v, ocodes, end = oracle.sw(prob.seq(center), prob.seq(t), M, w.gap_open, w.gap_extend,
                                       codes=True)
            pos = (ocodes & 3) != 0
            assert ((codes & 12) == (ocodes & 12)).all(), t
            assert (codes[pos] == ocodes[pos]).all(), t
            assert ((codes[~pos] & 3) != 0).all() or precision == 2, t
            if precision == 2:
                assert (codes == ocodes).all(), t
            assert seg[t, 0] == v and (seg[t, 3], seg[t, 4]) == end


def test_msa_bitexact_plain_protein_200():
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200")
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        out = run_pipeline(b, h, letters, offsets, c)
    check_against_oracle(prob, c, *out)


def test_msa_long_center_multipass():
    """Center longer than one 512-row pass, ragged lengths up to 2000."""
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=150, seed=8)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    lens = np.diff(offsets)
    center = int(np.argmax(lens))
    assert lens[center] > 1024
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        out = run_pipeline(b, h, letters, offsets, center)
    check_against_oracle(prob, center, *out)


@pytest.mark.parametrize("budget,lanes,cta", [(1, 8, 256), (300_000, 32, 256), (300_000, 16, 256),
                                              (1, 1, 256), (300_000, 1, 256), (300_000, 2, 256),
                                              (300_000, 4, 256), (1, 8, 384), (300_000, 16, 384),
                                              (300_000, 32, 384)])
def test_msa_in_code_batches(budget, lanes, cta):
    """Codes budgets that split the alignment into one subject per batch and
    into a few batches, with each group width and CTA size of the alignment
    kernels, give the same MSA as the oracle."""
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=60, seed=12)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_set_codes_budget(h, budget)
        b.msa_set_align_group(h, lanes)
        b.msa_set_align_threads(h, cta)
        with pytest.raises(b.MSAError):
            b.msa_set_align_threads(h, 512)
        with pytest.raises(b.MSAError):
            b.msa_set_codes_budget(h, 0)
        for bad in (12, 3, 64, -1):
            with pytest.raises(b.MSAError):
                b.msa_set_align_group(h, bad)
        out = run_pipeline(b, h, letters, offsets, 7)
    check_against_oracle(prob, 7, *out)


def test_msa_dna_workload():
    b = binding()
    letters, offsets, w, alph, M = workload("similar_dna_100k", n=40, seed=4)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        oc, _ = oracle.exact_center(prob)
        assert c == oc
        out = run_pipeline(b, h, letters, offsets, c)
    check_against_oracle(prob, c, *out)


# ------------------------------------------------------------- edge cases

def test_edge_cases_tiny_and_degenerate():
    b = binding()
    alph, M = dna_matrix(2, -3)
    cases = [
        [b"A"],                                   # one sequence of length one
        [b"A", b"C", b"G"],                       # no positive cell anywhere
        [b"AAAA", b"CCCC", b"AAAA"],              # zero-score pairs and duplicates
        [b"ACGT" * 40, b"ACGT" * 40, b"ACGT" * 40],  # identical rows
        [b"A", b"ACGTACGTTTGACCA" * 50, b"GG"],    # very uneven
    ]
    for seqs in cases:
        letters, offsets = pack_sequences(seqs)
        prob = oracle_problem(letters, offsets, alph, M, 5, 2)
        with make_ctx(alph, M, 5, 2) as h:
            b.msa_load(h, letters, offsets)
            c, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
            assert c == oracle.exact_center(prob)[0]
            out = run_pipeline(b, h, letters, offsets, c)
        check_against_oracle(prob, c, *out)


def test_errors_are_reported():
    b = binding()
    alph, M = dna_matrix(2, -3)
    with make_ctx(alph, M, 5, 2) as h:
        with pytest.raises(b.MSAError) as ei:
            b.msa_load(h, np.frombuffer(b"ACGTX", np.uint8), np.array([0, 5]))
        assert ei.value.code == b.MSA_EINVAL
        with pytest.raises(b.MSAError) as ei:
            b.msa_load(h, np.frombuffer(b"ACGT", np.uint8), np.array([0, 2, 2, 4]))
        assert ei.value.code == b.MSA_EINVAL
        long = np.frombuffer(b"A" * (b.MSA_MAX_LEN + 1), np.uint8)
        with pytest.raises(b.MSAError) as ei:
            b.msa_load(h, long, np.array([0, long.size]))
        assert ei.value.code == b.MSA_ERANGE
        b.msa_load(h, np.frombuffer(b"ACGTAC", np.uint8), np.array([0, 3, 6]))
        with pytest.raises(b.MSAError) as ei:
            b.msa_merge_gaps(h)
        assert ei.value.code == b.MSA_ESTATE
        with pytest.raises(b.MSAError) as ei:
            b.msa_select_center(h, b.MSA_CENTER_LEARNED)
        assert ei.value.code == b.MSA_ESTATE
    with pytest.raises(b.MSAError):
        b.msa_create(M, alph, 1, 2)               # open < extend
    asym = M.copy()
    asym[0, 1] = 5
    with pytest.raises(b.MSAError):
        b.msa_create(asym, alph, 5, 2)


def test_device_buffers_in_and_out():
    import torch
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=30, seed=6)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    dlet = torch.from_numpy(letters).cuda()
    with make_ctx(alph, M, w.gap_open, w.gap_extend,
                  stream=torch.cuda.current_stream()) as h:
        b.msa_load(h, dlet, offsets)
        dsc = torch.zeros(prob.n, dtype=torch.int32, device="cuda")
        b.msa_align_to_center(h, 3, dsc)
        _, W = b.msa_merge_gaps(h, want_rows=False)
        drows = torch.zeros((prob.n, W), dtype=torch.uint8, device="cuda")
        b.msa_merge_gaps(h, out=drows)
    oseg, _, _, _, oW, orows = oracle.msa(prob, 3)
    assert (dsc.cpu().numpy() == oseg[:, 0]).all()
    assert W == oW and (drows.cpu().numpy() == orows).all()


# ------------------------------------------------------------- full-size workload

def test_batched_uneven_10k_full_size_sampled():
    """The 10,000-sequence workload in the benchmark's launch configuration:
    row sums of sampled candidates and sampled MSA rows checked one by one
    against the oracle, invariants on every row."""
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k")
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    n = prob.n
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        rowsum = b.msa_center_rowsums(h)
        scores = np.zeros(n, np.int32)
        b.msa_align_to_center(h, c, scores)
        seg, ins, occ = b.msa_alignment_info(h)
        rows, W = b.msa_merge_gaps(h)
        sp = b.msa_sp_score(h)
    assert c == int(np.argmin(rowsum)) and s == rowsum[c]
    rng = np.random.default_rng(1)
    # the shortest sequences are the queries stacked several to a pass
    order = np.argsort(np.diff(offsets), kind="stable")
    sample = [c] + list(rng.choice(n, 2, replace=False)) + [int(order[0]), int(order[5])]
    orow = oracle.center_rowsums(prob, sample)
    assert (rowsum[sample] == orow).all(), (sample, rowsum[sample], orow)
    # sampled rows of the alignment, one by one
    lc = prob.length(c)
    for t in rng.choice(n, 25, replace=False):
        v, codes, end = oracle.sw(prob.seq(c), prob.seq(t), prob.M, prob.o, prob.e, codes=True)
        oins, oocc, oseg = oracle.traceback(codes, v, end)
        assert scores[t] == v and tuple(seg[t, 1:]) == oseg
        assert (ins[t] == oins).all() and (occ[t] == oocc).all()
    G = ins.max(axis=0)
    assert W == lc + int(G.sum())
    for t in range(0, n, 97):
        assert bytes(rows[t]).replace(b"-", b"") == bytes(letters[offsets[t]:offsets[t + 1]])
    assert sp == oracle.sp_columns(rows)


def test_autotuned_selection_is_unchanged():
    """The autotuner only changes which kernel variant runs, never a result."""
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=300, seed=12)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    oc, orow = oracle.exact_center(prob)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        rates = b.msa_autotune(h)
        c, s = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        rows = b.msa_center_rowsums(h)
    assert rates.shape[1] >= 9 and (rates > 0).sum() >= 9
    assert (rows == orow).all() and c == oc


def test_autotuned_alignment_is_unchanged():
    """The alignment tuner times every group width in packed and int32 cells
    and keeps the fastest; the MSA is the oracle's whatever it keeps."""
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=120, seed=14)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    center = 11
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        rates, (lanes, packed, cta) = b.msa_align_autotune(h, center)
        out = run_pipeline(b, h, letters, offsets, center)
    assert rates.shape == (3, 6) and (rates > 0).sum() == 15 and lanes in b.ALIGN_LANES
    assert cta in (256, 384) and (cta == 256 or (packed and lanes >= 8))
    check_against_oracle(prob, center, *out)


def test_short_peptides_against_their_center():
    """Peptides cut from a 500-residue ancestor (which is sequence 0):
    sampled exact center (240 references: enough work that the short
    reference queries are stacked several to a pass) and the whole MSA,
    bit-exact."""
    b = binding()
    letters, offsets, w, alph, M = workload("short_peptides_1m", n=1500, seed=5)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    refs = reference_sample(prob.n, 240, seed=3)
    oc, orow = oracle.exact_center(prob, refs=refs)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        c, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT_SAMPLED, refs=refs)
        assert (b.msa_center_rowsums(h) == orow).all() and c == oc
        out = run_pipeline(b, h, letters, offsets, 0)
    check_against_oracle(prob, 0, *out)


def test_split_set_merges_to_the_same_msa():
    """Two halves aligned in separate contexts (each with the center), merged
    with the elementwise maximum of their slot maxima, give the rows of the
    single-context MSA (the sharded path's exchange, on one GPU)."""
    b = binding()
    from seqgen import split_sequences
    letters, offsets, w, alph, M = workload("plain_protein_200", n=60, seed=13)
    center = 17
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        b.msa_align_to_center(h, center)
        full, W = b.msa_merge_gaps(h)
    seqs = split_sequences(letters, offsets)
    parts, Gs = [], []
    for lo, hi in ((0, 31), (31, 60)):
        sub = seqs[lo:hi] + [seqs[center]]
        sl, so = pack_sequences(sub)
        parts.append((lo, hi, sl, so))
        with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
            b.msa_load(h, sl, so)
            b.msa_align_to_center(h, len(sub) - 1)
            Gs.append(b.msa_insert_maxima(h))
    G = np.maximum(Gs[0], Gs[1])
    for lo, hi, sl, so in parts:
        with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
            b.msa_load(h, sl, so)
            b.msa_align_to_center(h, hi - lo)
            rows, W2 = b.msa_merge_gaps_with(h, G)
            with pytest.raises(b.MSAError):
                b.msa_merge_gaps_with(h, np.zeros_like(G) if G.any() else G - 1)
        assert W2 == W and (rows[:hi - lo] == full[lo:hi]).all()
