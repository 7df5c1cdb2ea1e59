"""Helpers for the GPU parity tests: contexts built through the C ABI and the
matching oracle problems, from the same seeded inputs."""
import numpy as np

import oracle
from seqgen import generate, scoring, pack_sequences


def binding():
    from paper_1704_00878_gb300 import binding as b
    b.lib()
    return b


def workload(name, n=None, seed=None):
    letters, offsets, w, fam = generate(name, n=n, seed=seed)
    alph, M, _, _ = scoring(w.kind)
    return letters, offsets, w, alph, M


def make_ctx(alph, M, o, e, **kw):
    b = binding()
    return b.Context(M, alph, o, e, **kw)


def oracle_problem(letters, offsets, alph, M, o, e):
    return oracle.Problem(letters, offsets, alph, M, o, e)


def random_set(rng, n, lo, hi, alph, emit=None):
    emit = emit or alph
    pool = np.frombuffer(emit.encode(), dtype=np.uint8)
    seqs = [rng.choice(pool, size=int(rng.integers(lo, hi + 1))) for _ in range(n)]
    return pack_sequences(seqs)
