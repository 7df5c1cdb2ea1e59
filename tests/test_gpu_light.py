"""The traceback-light alignment (MSA_ALIGN_BOX) against the oracle: a score
pass to each subject's best cell, a reverse pass to a corner above and left of
its traced segment, codes only inside the box between.  Every result must equal
the oracle's full alignment bit for bit (scores, segments, inserted spaces,
merged MSA, SP), and every box must hold the oracle's traced segment."""
import numpy as np
import pytest

import oracle
from seqgen import dna_matrix, pack_sequences
from tests._gpu import binding, workload, make_ctx, oracle_problem, random_set
from tests.test_gpu_parity import run_pipeline, check_against_oracle

pytestmark = pytest.mark.gpu


def light_pipeline(b, h, letters, offsets, center):
    b.msa_set_align_mode(h, b.MSA_ALIGN_BOX)
    out = run_pipeline(b, h, letters, offsets, center)
    boxes = b.msa_align_boxes(h, offsets.size - 1)
    return out, boxes


def check_boxes(prob, center, boxes):
    """Each box ends at the oracle's best cell, starts on a 16-row boundary
    above and left of the segment's start, and lies inside the matrix."""
    oseg = oracle.msa(prob, center)[0]
    Lc = prob.length(center)
    for r in range(prob.n):
        sc, i1, j1, i2, j2 = (int(v) for v in oseg[r])
        i0, j0, bi2, bj2 = (int(v) for v in boxes[r])
        if sc <= 0:
            assert (i0, j0, bi2, bj2) == (0, 0, 0, 0)
            continue
        assert (bi2, bj2) == (i2, j2), r
        assert i0 % 16 == 0 and 0 <= i0 <= i1 and 0 <= j0 <= j1, (r, boxes[r], oseg[r])
        assert i2 <= Lc and j2 <= prob.length(r)


def box_fraction(prob, center, boxes):
    Lc = prob.length(center)
    lens = np.diff(prob.off)
    area = ((boxes[:, 2] - boxes[:, 0]).astype(np.int64) * (boxes[:, 3] - boxes[:, 1])).sum()
    return area / float(Lc * lens.sum())


def test_light_peptides_against_their_center():
    """Peptides cut from their 500-residue ancestor: each box spans about the
    peptide's own length, a fraction of the matrix."""
    b = binding()
    letters, offsets, w, alph, M = workload("short_peptides_1m", n=1500, seed=5)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        out, boxes = light_pipeline(b, h, letters, offsets, 0)
        ms, _ = b.msa_stage_times(h)
    check_against_oracle(prob, 0, *out)
    check_boxes(prob, 0, boxes)
    assert box_fraction(prob, 0, boxes) < 0.4
    assert ms["light_score"] > 0 and ms["light_corner"] > 0 and ms["light_box"] > 0


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8, 16, 32])
def test_light_protein_every_group_width(lanes):
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=80, seed=21)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    center = 5
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_set_align_group(h, lanes)
        b.msa_load(h, letters, offsets)
        out, boxes = light_pipeline(b, h, letters, offsets, center)
    check_against_oracle(prob, center, *out)
    check_boxes(prob, center, boxes)


@pytest.mark.parametrize("budget", [1, 200_000])
def test_light_long_center_multipass_and_batches(budget):
    """A center longer than two 512-row passes (the reverse windows and the
    boxes then span several passes) with ragged subjects up to 2000 long, in
    one subject per code batch and in a few batches."""
    b = binding()
    letters, offsets, w, alph, M = workload("batched_uneven_10k", n=120, seed=8)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    lens = np.diff(offsets)
    center = int(np.argmax(lens))
    assert lens[center] > 1024
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_set_codes_budget(h, budget)
        b.msa_load(h, letters, offsets)
        out, boxes = light_pipeline(b, h, letters, offsets, center)
    check_against_oracle(prob, center, *out)
    check_boxes(prob, center, boxes)


def test_light_dna_and_a_short_center():
    """Similar DNA (segments span the matrix), then the same set against its
    shortest member (many subjects longer than the center)."""
    b = binding()
    letters, offsets, w, alph, M = workload("similar_dna_100k", n=40, seed=4)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    shortest = int(np.argmin(np.diff(offsets)))
    for center in (3, shortest):
        with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
            b.msa_load(h, letters, offsets)
            out, boxes = light_pipeline(b, h, letters, offsets, center)
        check_against_oracle(prob, center, *out)
        check_boxes(prob, center, boxes)


@pytest.mark.parametrize("seed", range(4))
def test_light_ties_in_small_alphabets(seed):
    """Two- and three-letter sequences under small gap costs: equal scores
    everywhere, so the best cell, the corner and the box's own best cell all
    meet ties (first cell by row then column; the corner the largest row and
    column reaching the best score)."""
    b = binding()
    rng = np.random.default_rng(100 + seed)
    alph, M = dna_matrix(2, -3)
    emit = "AC" if seed % 2 == 0 else "ACG"
    letters, offsets = random_set(rng, 70, 1, 90, alph, emit)
    for o, e in ((3, 1), (5, 2), (4, 4)):
        prob = oracle_problem(letters, offsets, alph, M, o, e)
        center = int(rng.integers(0, 70))
        with make_ctx(alph, M, o, e) as h:
            b.msa_load(h, letters, offsets)
            out, boxes = light_pipeline(b, h, letters, offsets, center)
        check_against_oracle(prob, center, *out)
        check_boxes(prob, center, boxes)


def test_light_edge_cases():
    b = binding()
    alph, M = dna_matrix(2, -3)
    cases = [
        [b"A"],
        [b"A", b"C", b"G"],                       # no positive cell anywhere
        [b"AAAA", b"CCCC", b"AAAA"],
        [b"ACGT" * 40, b"ACGT" * 40, b"ACGT" * 40],
        [b"A", b"ACGTACGTTTGACCA" * 50, b"GG"],
        [b"ACGT" * 200, b"TTTTACGTACGTTTTT", b"GGGG" + b"ACGT" * 3],  # segments deep in a long center
    ]
    for seqs in cases:
        letters, offsets = pack_sequences(seqs)
        prob = oracle_problem(letters, offsets, alph, M, 5, 2)
        for center in range(len(seqs)):
            with make_ctx(alph, M, 5, 2) as h:
                b.msa_load(h, letters, offsets)
                out, boxes = light_pipeline(b, h, letters, offsets, center)
            check_against_oracle(prob, center, *out)
            check_boxes(prob, center, boxes)


def test_light_mode_switches_and_errors():
    b = binding()
    letters, offsets, w, alph, M = workload("plain_protein_200", n=30, seed=3)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        for bad in (-1, 2, 7):
            with pytest.raises(b.MSAError):
                b.msa_set_align_mode(h, bad)
        b.msa_load(h, letters, offsets)
        with pytest.raises(b.MSAError):          # no alignment yet
            b.msa_align_boxes(h, 30)
        out = run_pipeline(b, h, letters, offsets, 2)   # the full mode
        check_against_oracle(prob, 2, *out)
        with pytest.raises(b.MSAError):          # the last alignment was full
            b.msa_align_boxes(h, 30)
        out, boxes = light_pipeline(b, h, letters, offsets, 2)
        check_against_oracle(prob, 2, *out)
        check_boxes(prob, 2, boxes)
        b.msa_set_align_mode(h, b.MSA_ALIGN_FULL)
        out = run_pipeline(b, h, letters, offsets, 2)
        check_against_oracle(prob, 2, *out)
    # int32 cells (no packed path): the box mode runs the full alignment
    with make_ctx(alph, M, w.gap_open, w.gap_extend, precision=b.MSA_INT32) as h:
        b.msa_load(h, letters, offsets)
        b.msa_set_align_mode(h, b.MSA_ALIGN_BOX)
        out = run_pipeline(b, h, letters, offsets, 2)
        check_against_oracle(prob, 2, *out)
        with pytest.raises(b.MSAError):
            b.msa_align_boxes(h, 30)


@pytest.mark.parametrize("kind", ["dna", "protein"])
def test_light_at_the_longest_packed_centers(kind):
    """The longest centers the packed cells take: MSA_MAX_LEN residues of DNA
    (reverse windows of up to 16 passes of 512 rows) and 2,900 residues of
    protein under BLOSUM62 (the int16 bound), with subjects from full length
    down to short reads cut from anywhere in the center."""
    from tests.test_gpu_limits import mutants
    from seqgen import blosum62, STANDARD_AA
    b = binding()
    rng = np.random.default_rng(31 if kind == "dna" else 37)
    if kind == "dna":
        alph, M = dna_matrix(2, -3)
        pool = np.frombuffer(b"ACGT", np.uint8)
        L, o, e, rate = b.MSA_MAX_LEN, 5, 2, 0.02
        lengths = [L, L - 100, 3000, 200, 40, 17]
    else:
        alph, M = blosum62()
        pool = np.frombuffer(STANDARD_AA.encode(), np.uint8)
        L, o, e, rate = 2900, 11, 1, 0.3
        lengths = [L, 2000, 300, 60, 25]
    ancestor = pool[rng.integers(0, pool.size, L)]
    seqs = [ancestor.copy()] + mutants(rng, ancestor, pool, lengths, rate)
    letters, offsets = pack_sequences(seqs)
    prob = oracle_problem(letters, offsets, alph, M, o, e)
    with make_ctx(alph, M, o, e) as h:
        b.msa_load(h, letters, offsets)
        out, boxes = light_pipeline(b, h, letters, offsets, 0)
    check_against_oracle(prob, 0, *out)
    check_boxes(prob, 0, boxes)
