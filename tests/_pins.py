"""Independent restatements used to pin the oracle (pure Python, tiny inputs).

None of these shares code with the oracle: brute-force enumeration of every
local alignment, the literal cubic form of Eq. (2), and textbook linear-gap
Smith-Waterman.
"""
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def _paths(la, lb):
    """Every global alignment of lengths la, lb as a string over M/I/D
    (M: residue pair, I: sequence residue vs gap, D: center residue vs gap)."""
    if la == 0 and lb == 0:
        return ("",)
    out = []
    if la and lb:
        out += ["M" + p for p in _paths(la - 1, lb - 1)]
    if lb:
        out += ["I" + p for p in _paths(la, lb - 1)]
    if la:
        out += ["D" + p for p in _paths(la - 1, lb)]
    return tuple(out)


def score_path(A, B, ops, M, o, e):
    """Affine score of one alignment: each maximal run of k gaps of one kind
    costs o + (k-1)e."""
    i = j = 0
    total = 0
    prev = None
    for op in ops:
        if op == "M":
            total += int(M[A[i]][B[j]])
            i += 1
            j += 1
        elif op == "I":
            total -= e if prev == "I" else o
            j += 1
        else:
            total -= e if prev == "D" else o
            i += 1
        prev = op
    return total


def brute_local(A, B, M, o, e):
    """(best score, dict cell -> best score of alignments ending exactly there).

    Local score = max(0, max over substrings A[a0:a1], B[b0:b1] and every
    global alignment of them).  Cell (a1, b1) collects alignments that end
    there, which is what H[a1][b1] holds in the DP."""
    best = 0
    ending = {}
    for a0 in range(len(A) + 1):
        for a1 in range(a0, len(A) + 1):
            for b0 in range(len(B) + 1):
                for b1 in range(b0, len(B) + 1):
                    if a1 == a0 and b1 == b0:
                        continue
                    sa, sb = A[a0:a1], B[b0:b1]
                    v = max(score_path(sa, sb, p, M, o, e) for p in _paths(len(sa), len(sb)))
                    best = max(best, v)
                    if v > ending.get((a1, b1), 0):
                        ending[(a1, b1)] = v
    return best, ending


def eq2_literal(A, B, M, o, e):
    """Eq. (2) as printed: gap terms maximised over every gap length k, l."""
    n, m = len(A), len(B)
    H = np.zeros((n + 1, m + 1), dtype=np.int64)
    for i in range(1, n + 1):
        for j in range(1, m + 1):
            v = max(0, H[i - 1, j - 1] + int(M[A[i - 1]][B[j - 1]]))
            for k in range(1, i + 1):
                v = max(v, H[i - k, j] - (o + (k - 1) * e))
            for l in range(1, j + 1):
                v = max(v, H[i, j - l] - (o + (l - 1) * e))
            H[i, j] = v
    return H


def linear_sw(A, B, M, g):
    """Textbook Smith-Waterman with a linear gap penalty g per residue."""
    n, m = len(A), len(B)
    H = np.zeros((n + 1, m + 1), dtype=np.int64)
    for i in range(1, n + 1):
        for j in range(1, m + 1):
            H[i, j] = max(0, H[i - 1, j - 1] + int(M[A[i - 1]][B[j - 1]]),
                          H[i - 1, j] - g, H[i, j - 1] - g)
    return int(H.max())


def first_argmax(H):
    """Smallest i, then smallest j, among the maxima of H (0,0 if max is 0)."""
    best = H.max()
    if best == 0:
        return 0, 0
    idx = np.argwhere(H == best)
    idx = sorted(map(tuple, idx))
    return int(idx[0][0]), int(idx[0][1])


def pairwise_columns(ins, occ, lc, ls):
    """The pairwise alignment (center index | None, seq index | None), 1-based,
    that a row's inserted-space entry describes."""
    cols = []
    k = 1
    for j in range(lc + 1):
        for _ in range(int(ins[j])):
            cols.append((None, k))
            k += 1
        if j < lc:
            if occ[j + 1]:
                cols.append((j + 1, k))
                k += 1
            else:
                cols.append((j + 1, None))
    assert k == ls + 1
    return cols


def rescore_segment(cols, c, s, seg, M, o, e):
    """Affine score of the columns from pair (i1+1, j1+1) to pair (i2, j2)."""
    i1, j1, i2, j2 = seg
    if i2 == 0:
        return 0
    start = cols.index((i1 + 1, j1 + 1))
    stop = cols.index((i2, j2))
    total, prev = 0, None
    for ci, si in cols[start:stop + 1]:
        if ci is not None and si is not None:
            total += int(M[c[ci - 1]][s[si - 1]])
            prev = "M"
        elif ci is None:
            total -= e if prev == "I" else o
            prev = "I"
        else:
            total -= e if prev == "D" else o
            prev = "D"
    return total
