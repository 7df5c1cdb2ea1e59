"""Seeded synthetic sequence sets with the shapes of the paper's workloads.

The paper evaluates on BAliBASE 4 R10 proteins, human mitochondrial genomes and
16S rRNA (Table 1); none of those files are available, so every workload here is
generated: ancestors drawn from background residue frequencies, a window of each
sequence's length cut from its family ancestor, then substitutions and indels.

Substitution picks b != a with probability proportional to p_b * 2^(M[a][b]/2)
(the substitution matrix read as half-bit log-odds).  An indel starts after
each position with the given rate; it is an insertion or a deletion with
probability 1/2 each, with a geometric(p) length or a uniform {lo..hi} length.

This module draws random numbers only.  It holds none of the alignment
arithmetic; the CUDA path and the oracle both take its arrays as inputs.
"""
from dataclasses import dataclass, field
import numpy as np

from .matrices import (blosum62, dna_matrix, aa_background, STANDARD_AA,
                       PROTEIN_LETTERS, DNA_LETTERS)


@dataclass
class Workload:
    name: str
    kind: str                      # "protein" | "dna"
    n: int
    length: tuple                  # ("uniform", lo, hi) | ("lognormal", median, sigma, lo, hi)
    families: int
    p_sub: float
    p_indel: float
    indel: tuple                   # ("geom", p) | ("uniform", lo, hi)
    gap_open: int
    gap_extend: int
    seed: int
    ancestor_len: int              # length of each family ancestor
    center_seq: bool = False       # prepend the (unmutated) ancestor as sequence 0
    extra: dict = field(default_factory=dict)


# The five workloads (seeds 1704*10 + k).
WORKLOADS = {
    "plain_protein_200": Workload(
        "plain_protein_200", "protein", 200, ("uniform", 200, 400), 1, 0.30, 0.03,
        ("geom", 0.5), 11, 1, 17041, 400),
    "batched_uneven_10k": Workload(
        "batched_uneven_10k", "protein", 10_000, ("lognormal", 350, 0.6, 50, 2000), 5,
        0.40, 0.05, ("geom", 0.5), 11, 1, 17042, 2000),
    "learned_center_50k": Workload(
        "learned_center_50k", "protein", 50_000, ("lognormal", 300, 0.6, 50, 2000), 20,
        0.40, 0.05, ("geom", 0.5), 11, 1, 17043, 2000,
        extra={"train_pairs": 200_000}),
    "similar_dna_100k": Workload(
        "similar_dna_100k", "dna", 100_000, ("uniform", 1400, 1600), 1, 0.02, 0.005,
        ("uniform", 1, 3), 5, 2, 17044, 1600),
    "short_peptides_1m": Workload(
        "short_peptides_1m", "protein", 1_000_000, ("lognormal", 90, 0.6, 30, 200), 1,
        0.30, 0.03, ("geom", 0.5), 11, 1, 17045, 500, center_seq=True),
}


def scoring(kind):
    """(letters, int8 matrix, letters the generator emits, their background)."""
    if kind == "protein":
        letters, mat = blosum62()
        return letters, mat, STANDARD_AA, aa_background()
    letters, mat = dna_matrix(2, -3)
    return letters, mat, DNA_LETTERS, np.full(4, 0.25)


def _sub_cdf(mat, letters, emit, bg):
    """Row a: cumulative P(b | a), b != a, over the emitted residues."""
    idx = np.array([letters.index(ch) for ch in emit])
    sub = mat[np.ix_(idx, idx)].astype(np.float64)
    w = bg[None, :] * np.power(2.0, sub / 2.0)
    np.fill_diagonal(w, 0.0)
    w /= w.sum(axis=1, keepdims=True)
    cdf = np.cumsum(w, axis=1)
    cdf[:, -1] = 1.0
    return cdf


def _lengths(rng, spec, n):
    if spec[0] == "uniform":
        return rng.integers(spec[1], spec[2] + 1, size=n)
    _, median, sigma, lo, hi = spec
    raw = np.exp(rng.normal(np.log(median), sigma, size=n))
    return np.clip(np.rint(raw), lo, hi).astype(np.int64)


def _indel_len(rng, spec):
    if spec[0] == "geom":
        return int(rng.geometric(spec[1]))
    return int(rng.integers(spec[1], spec[2] + 1))


def _mutate(rng, seq, w, cdf, bg_cdf):
    """Substitutions then indels; `seq` holds indices into the emitted letters."""
    seq = seq.copy()
    n = seq.size
    hit = rng.random(n) < w.p_sub
    if hit.any():
        a = seq[hit]
        u = rng.random(a.size)
        seq[hit] = (cdf[a] < u[:, None]).sum(axis=1)
    events = np.nonzero(rng.random(n) < w.p_indel)[0]
    if events.size == 0:
        return seq
    pieces, pos = [], 0
    for p in events:
        if p < pos:                      # inside an earlier deletion
            continue
        k = _indel_len(rng, w.indel)
        if rng.random() < 0.5:           # insertion after position p
            pieces.append(seq[pos:p + 1])
            pieces.append(np.searchsorted(bg_cdf, rng.random(k), side="right"))
            pos = p + 1
        else:                            # deletion of positions p .. p+k-1
            pieces.append(seq[pos:p])
            pos = p + k
    pieces.append(seq[pos:])
    out = np.concatenate(pieces).astype(np.int64)
    if out.size == 0:
        out = seq[:1]
    return out


def generate(name_or_workload, n=None, seed=None, length=None):
    """Return (letters_ascii uint8[total], offsets int64[n+1], workload, family int64[n]).

    `n` and `seed` override the workload's count and seed (same distributions);
    `length` overrides the length distribution (same tuple form as Workload).
    """
    w = WORKLOADS[name_or_workload] if isinstance(name_or_workload, str) else name_or_workload
    n = w.n if n is None else int(n)
    rng = np.random.default_rng(w.seed if seed is None else seed)
    letters, mat, emit, bg = scoring(w.kind)
    cdf = _sub_cdf(mat, letters, emit, bg)
    bg_cdf = np.cumsum(bg)
    bg_cdf[-1] = 1.0
    emit_ascii = np.frombuffer(emit.encode(), dtype=np.uint8)

    ancestors = [np.searchsorted(bg_cdf, rng.random(w.ancestor_len), side="right")
                 for _ in range(w.families)]
    n_gen = n - 1 if w.center_seq else n
    lens = _lengths(rng, w.length if length is None else tuple(length), n_gen)
    fams = rng.integers(0, w.families, size=n_gen)
    seqs = []
    if w.center_seq:
        seqs.append(ancestors[0])
        fams = np.concatenate([[0], fams])
    for L, f in zip(lens, fams[1:] if w.center_seq else fams):
        anc = ancestors[f]
        L = int(min(L, anc.size))
        start = int(rng.integers(0, anc.size - L + 1))
        seqs.append(_mutate(rng, anc[start:start + L], w, cdf, bg_cdf))
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.size for s in seqs])
    flat = emit_ascii[np.concatenate(seqs)] if seqs else np.zeros(0, np.uint8)
    return np.ascontiguousarray(flat, dtype=np.uint8), offsets, w, fams.astype(np.int64)


def random_sequences(rng, n, lo, hi, alphabet_size):
    """Uniform random index sequences (for small pin tests), list of int arrays."""
    return [rng.integers(0, alphabet_size, size=int(rng.integers(lo, hi + 1)))
            for _ in range(n)]


def reference_sample(n, r, seed):
    """Seeded reference subset (sorted indices) for the sampled exact center."""
    rng = np.random.default_rng(seed)
    r = min(r, n)
    return np.sort(rng.choice(n, size=r, replace=False)).astype(np.int64)


def training_pairs(n, count, families_of, seed):
    """Half within-family, half uniformly random pairs (i != j), int64[count, 2]."""
    rng = np.random.default_rng(seed)
    fam = np.asarray(families_of)
    out = np.empty((count, 2), dtype=np.int64)
    half = count // 2
    out[half:, 0] = rng.integers(0, n, size=count - half)
    out[half:, 1] = (out[half:, 0] + rng.integers(1, n, size=count - half)) % n
    order = np.argsort(fam, kind="stable")
    starts = np.searchsorted(fam[order], np.arange(fam.max() + 1))
    ends = np.searchsorted(fam[order], np.arange(fam.max() + 1), side="right")
    a = rng.integers(0, n, size=half)
    f = fam[a]
    size = ends[f] - starts[f]
    b = order[starts[f] + (rng.random(half) * size).astype(np.int64)]
    same = b == a
    b[same] = (b[same] + 1) % n
    out[:half, 0], out[:half, 1] = a, b
    return out


def split_sequences(letters, offsets):
    """List of per-sequence ASCII byte arrays."""
    return [letters[offsets[i]:offsets[i + 1]] for i in range(offsets.size - 1)]


def pack_sequences(seqs):
    """Inverse of split_sequences for lists of uint8 arrays or bytes."""
    arrs = [np.frombuffer(s, dtype=np.uint8) if isinstance(s, (bytes, bytearray))
            else np.asarray(s, dtype=np.uint8) for s in seqs]
    offsets = np.zeros(len(arrs) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([a.size for a in arrs])
    flat = np.concatenate(arrs) if arrs else np.zeros(0, np.uint8)
    return np.ascontiguousarray(flat, dtype=np.uint8), offsets
