"""The seeded input generator follows the recipe the workloads are stated
with: sizes, families, scoring, alphabets, length distributions, the
substitution and indel rates, and the helpers that draw reference samples
and training pairs."""
import numpy as np
import pytest

from seqgen import (WORKLOADS, generate, scoring, reference_sample, training_pairs,
                    STANDARD_AA, DNA_LETTERS)
from seqgen import synth


def test_workload_table():
    expect = {
        "plain_protein_200": (200, "protein", 1, 11, 1),
        "batched_uneven_10k": (10_000, "protein", 5, 11, 1),
        "learned_center_50k": (50_000, "protein", 20, 11, 1),
        "similar_dna_100k": (100_000, "dna", 1, 5, 2),
        "short_peptides_1m": (1_000_000, "protein", 1, 11, 1),
    }
    assert set(WORKLOADS) == set(expect)
    for name, (n, kind, fams, o, e) in expect.items():
        w = WORKLOADS[name]
        assert (w.n, w.kind, w.families, w.gap_open, w.gap_extend) == (n, kind, fams, o, e)
    assert [w.seed for w in WORKLOADS.values()] == [17041, 17042, 17043, 17044, 17045]


def test_deterministic_and_in_alphabet():
    for name, emit in [("batched_uneven_10k", STANDARD_AA), ("similar_dna_100k", DNA_LETTERS)]:
        a = generate(name, n=300, seed=5)
        b = generate(name, n=300, seed=5)
        assert all((x == y).all() for x, y in zip((a[0], a[1], a[3]), (b[0], b[1], b[3])))
        letters, offsets = a[0], a[1]
        assert offsets[0] == 0 and (np.diff(offsets) > 0).all() and offsets[-1] == letters.size
        assert set(bytes(letters).decode()) <= set(emit)


@pytest.mark.parametrize("name,median", [("batched_uneven_10k", 350), ("short_peptides_1m", 90)])
def test_lognormal_lengths(name, median):
    letters, offsets, w, fam = generate(name, n=4000, seed=9)
    lens = np.diff(offsets)
    if w.center_seq:
        assert lens[0] == w.ancestor_len and fam[0] == 0
        lens = lens[1:]
    # indels at a few percent move a window's length by little
    assert abs(np.median(lens) / median - 1) < 0.1
    lo, hi = w.length[3], w.length[4]
    assert lens.min() >= 0.6 * lo and lens.max() <= 1.2 * hi


def test_uniform_lengths_and_families():
    letters, offsets, w, fam = generate("learned_center_50k", n=3000, seed=2,
                                        length=("uniform", 200, 400))
    lens = np.diff(offsets)
    assert 180 <= lens.min() and lens.max() <= 440
    assert set(np.unique(fam)) == set(range(w.families))


def test_substitution_and_indel_rates():
    w = WORKLOADS["plain_protein_200"]
    letters, mat, emit, bg = scoring(w.kind)
    cdf = synth._sub_cdf(mat, letters, emit, bg)
    bg_cdf = np.cumsum(bg)
    bg_cdf[-1] = 1.0
    rng = np.random.default_rng(3)
    seq = np.searchsorted(bg_cdf, rng.random(20000), side="right")
    no_indel = synth.Workload(**{**w.__dict__, "p_indel": 0.0})
    out = synth._mutate(rng, seq, no_indel, cdf, bg_cdf)
    assert out.size == seq.size
    assert abs((out != seq).mean() - w.p_sub) < 0.015   # a substitution never keeps the residue
    no_sub = synth.Workload(**{**w.__dict__, "p_sub": 0.0})
    out = synth._mutate(rng, seq, no_sub, cdf, bg_cdf)
    # geometric(0.5) indels: mean length 2, insertions and deletions equally likely
    assert abs(out.size - seq.size) < 0.02 * seq.size


def test_reference_sample_and_training_pairs():
    r = reference_sample(1000, 37, seed=9)
    assert r.size == 37 and (np.diff(r) > 0).all() and r.min() >= 0 and r.max() < 1000
    assert (r == reference_sample(1000, 37, seed=9)).all()
    assert reference_sample(10, 37, seed=1).size == 10
    fam = np.random.default_rng(0).integers(0, 5, size=800)
    p = training_pairs(800, 2000, fam, seed=4)
    assert p.shape == (2000, 2) and (p >= 0).all() and (p < 800).all()
    assert (p[:, 0] != p[:, 1]).all()
    within = (fam[p[:1000, 0]] == fam[p[:1000, 1]]).mean()
    assert within > 0.95
