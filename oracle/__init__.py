"""Plain CPU oracle for the center-star MSA hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
never does.  It shares no code with the CUDA library.

The arithmetic lives in ``msa_oracle.c`` (plain scalar C, full DP matrices);
this module compiles it with gcc, marshals arrays, and encodes letters to
alphabet indices.  Parity is pinned by the ``-m "not gpu"`` tests
(brute-force enumeration, the literal cubic form of Eq. 2, invariants and
hand-worked fixtures).
"""
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle into liboracle.so (plain -O2, no SIMD flags)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.orc_sw.restype = i32
        L.orc_sw.argtypes = [P, i32, P, i32, P, i32, i32, i32, P, P]
        L.orc_traceback.restype = ctypes.c_int
        L.orc_traceback.argtypes = [P, i32, i32, i32, i32, i32, P, P, P]
        L.orc_pair_scores.restype = ctypes.c_int
        L.orc_pair_scores.argtypes = [P, P, P, i64, P, i32, i32, i32, P, ctypes.c_int]
        L.orc_align_all.restype = ctypes.c_int
        L.orc_align_all.argtypes = [P, P, i64, i64, P, i32, i32, i32, P, P, P, ctypes.c_int]
        L.orc_merge_width.restype = i64
        L.orc_merge_width.argtypes = [P, i64, i32, P]
        L.orc_write_rows.restype = ctypes.c_int
        L.orc_write_rows.argtypes = [P, P, i64, i32, P, P, P, i64, ctypes.c_char_p, P]
        L.orc_sp_pairwise.restype = i64
        L.orc_sp_pairwise.argtypes = [P, i64, i64]
        L.orc_sp_columns.restype = i64
        L.orc_sp_columns.argtypes = [P, i64, i64]
        L.orc_center_rowsums.restype = ctypes.c_int
        L.orc_center_rowsums.argtypes = [P, P, i64, P, i64, P, i64, P, i32, i32, i32, P,
                                         ctypes.c_int]
        L.orc_exact_center.restype = i64
        L.orc_exact_center.argtypes = [P, P, i64, P, i64, P, i32, i32, i32, P, ctypes.c_int]
        L.orc_anchored.restype = ctypes.c_int
        L.orc_anchored.argtypes = [P, i32, P, i32, P, i32, i32, i32, i32, P, P, P]
        L.orc_anchored_all.restype = ctypes.c_int
        L.orc_anchored_all.argtypes = [P, P, i64, i64, P, i32, i32, i32, i32, P, P, P, ctypes.c_int]
        L.orc_default_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads():
    return lib().orc_default_threads()


# ---------------------------------------------------------------- encoding

def encode(letters_ascii, alphabet):
    """ASCII bytes -> alphabet indices (uint8); raises on a letter not in it."""
    lut = np.full(256, 255, dtype=np.uint8)
    for k, ch in enumerate(alphabet):
        lut[ord(ch)] = k
    arr = np.frombuffer(bytes(letters_ascii), dtype=np.uint8) \
        if isinstance(letters_ascii, (bytes, bytearray)) else np.asarray(letters_ascii, np.uint8)
    out = lut[arr]
    if out.size and out.max() == 255:
        raise ValueError("letter not in alphabet")
    return out


class Problem:
    """Encoded sequence set + scoring scheme (the oracle's view of the inputs)."""

    def __init__(self, letters_ascii, offsets, alphabet, matrix, gap_open, gap_extend):
        self.alphabet = alphabet
        self.res = np.ascontiguousarray(encode(letters_ascii, alphabet))
        self.off = np.ascontiguousarray(offsets, dtype=np.int64)
        self.M = np.ascontiguousarray(matrix, dtype=np.int8)
        self.K = int(self.M.shape[0])
        self.o, self.e = int(gap_open), int(gap_extend)
        self.n = self.off.size - 1

    def seq(self, i):
        return self.res[self.off[i]:self.off[i + 1]]

    def length(self, i):
        return int(self.off[i + 1] - self.off[i])


# ---------------------------------------------------------------- pairwise

def sw(c, s, M, o, e, codes=False):
    """Score (and optionally Lc x Ls codes, best cell) of one local alignment."""
    c = np.ascontiguousarray(c, dtype=np.uint8)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    M = np.ascontiguousarray(M, dtype=np.int8)
    end = np.zeros(2, dtype=np.int32)
    cb = np.zeros((c.size, s.size), dtype=np.uint8) if codes else None
    v = lib().orc_sw(_p(c), c.size, _p(s), s.size, _p(M), M.shape[0], o, e,
                     _p(cb) if codes else None, _p(end))
    if v < 0:
        raise MemoryError("oracle sw")
    if codes:
        return int(v), cb, (int(end[0]), int(end[1]))
    return int(v)


def traceback(codes, best, end):
    """(ins uint16[Lc+1], occ uint8[Lc+1], (i1, j1, i2, j2)) from codes."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    lc, ls = codes.shape
    ins = np.zeros(lc + 1, dtype=np.uint16)
    occ = np.zeros(lc + 1, dtype=np.uint8)
    seg = np.zeros(4, dtype=np.int32)
    rc = lib().orc_traceback(_p(codes), lc, ls, int(best), int(end[0]), int(end[1]),
                             _p(ins), _p(occ), _p(seg))
    if rc != 0:
        raise RuntimeError("inconsistent traceback codes")
    return ins, occ, tuple(int(x) for x in seg)


def pair_scores(prob, pairs, threads=0):
    pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    out = np.zeros(pairs.shape[0], dtype=np.int32)
    rc = lib().orc_pair_scores(_p(prob.res), _p(prob.off), _p(pairs), pairs.shape[0],
                               _p(prob.M), prob.K, prob.o, prob.e, _p(out), threads)
    if rc != 0:
        raise MemoryError("oracle pair scores")
    return out


def align_all(prob, center, threads=0):
    """Per row: seg int32[n,5] = (score,i1,j1,i2,j2), ins uint16[n,Lc+1], occ uint8[n,Lc+1]."""
    lc = prob.length(center)
    ins = np.zeros((prob.n, lc + 1), dtype=np.uint16)
    occ = np.zeros((prob.n, lc + 1), dtype=np.uint8)
    seg = np.zeros((prob.n, 5), dtype=np.int32)
    rc = lib().orc_align_all(_p(prob.res), _p(prob.off), prob.n, int(center), _p(prob.M),
                             prob.K, prob.o, prob.e, _p(ins), _p(occ), _p(seg), threads)
    if rc != 0:
        raise RuntimeError("oracle align_all failed")
    return seg, ins, occ


def merge(prob, center, ins, occ):
    """(G int32[Lc+1], W, msa uint8[n, W]) from the inserted-space matrix."""
    lc = prob.length(center)
    ins = np.ascontiguousarray(ins, dtype=np.uint16)
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    G = np.zeros(lc + 1, dtype=np.int32)
    W = int(lib().orc_merge_width(_p(ins), prob.n, lc, _p(G)))
    msa = np.zeros((prob.n, W), dtype=np.uint8)
    rc = lib().orc_write_rows(_p(prob.res), _p(prob.off), prob.n, lc, _p(ins), _p(occ),
                              _p(G), W, prob.alphabet.encode(), _p(msa))
    if rc != 0:
        raise RuntimeError("oracle rows inconsistent")
    return G, W, msa


def sp_pairwise(msa):
    msa = np.ascontiguousarray(msa, dtype=np.uint8)
    return int(lib().orc_sp_pairwise(_p(msa), msa.shape[0], msa.shape[1]))


def sp_columns(msa):
    msa = np.ascontiguousarray(msa, dtype=np.uint8)
    return int(lib().orc_sp_columns(_p(msa), msa.shape[0], msa.shape[1]))


def avg_sp(msa):
    n = msa.shape[0]
    return sp_columns(msa) / (n * (n - 1) / 2) if n > 1 else 0.0


def exact_center(prob, refs=None, threads=0):
    """(center, rowsum int64[n]); refs=None means every sequence."""
    rowsum = np.zeros(prob.n, dtype=np.int64)
    if refs is None:
        c = lib().orc_exact_center(_p(prob.res), _p(prob.off), prob.n, None, prob.n,
                                   _p(prob.M), prob.K, prob.o, prob.e, _p(rowsum), threads)
    else:
        refs = np.ascontiguousarray(refs, dtype=np.int64)
        c = lib().orc_exact_center(_p(prob.res), _p(prob.off), prob.n, _p(refs), refs.size,
                                   _p(prob.M), prob.K, prob.o, prob.e, _p(rowsum), threads)
    if c < 0:
        raise MemoryError("oracle exact center")
    return int(c), rowsum


def center_rowsums(prob, cands, refs=None, threads=0):
    """Row sums sum_{r in refs} d(c, r) of the listed candidates (refs=None:
    every sequence), int64[len(cands)]."""
    cands = np.ascontiguousarray(cands, dtype=np.int64)
    out = np.zeros(cands.size, dtype=np.int64)
    if refs is None:
        rp, nr = None, prob.n
    else:
        refs = np.ascontiguousarray(refs, dtype=np.int64)
        rp, nr = _p(refs), refs.size
    rc = lib().orc_center_rowsums(_p(prob.res), _p(prob.off), prob.n, _p(cands), cands.size,
                                  rp, nr, _p(prob.M), prob.K, prob.o, prob.e, _p(out), threads)
    if rc != 0:
        raise MemoryError("oracle center row sums")
    return out


def anchored(c, x, M, o, e, k):
    """Anchored alignment of x to the center c (the trie path for similar
    sequences): (ins uint16[Lc+1], occ uint8[Lc+1], seg (score, i1, j1, i2, j2))."""
    c = np.ascontiguousarray(c, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    M = np.ascontiguousarray(M, dtype=np.int8)
    ins = np.zeros(c.size + 1, dtype=np.uint16)
    occ = np.zeros(c.size + 1, dtype=np.uint8)
    seg = np.zeros(5, dtype=np.int32)
    rc = lib().orc_anchored(_p(c), c.size, _p(x), x.size, _p(M), M.shape[0], o, e, k,
                            _p(ins), _p(occ), _p(seg))
    if rc != 0:
        raise RuntimeError("oracle anchored alignment failed")
    return ins, occ, tuple(int(v) for v in seg)


def anchored_all(prob, center, k, threads=0):
    """Every row aligned to the center by the anchored path: (seg, ins, occ)."""
    lc = prob.length(center)
    ins = np.zeros((prob.n, lc + 1), dtype=np.uint16)
    occ = np.zeros((prob.n, lc + 1), dtype=np.uint8)
    seg = np.zeros((prob.n, 5), dtype=np.int32)
    rc = lib().orc_anchored_all(_p(prob.res), _p(prob.off), prob.n, int(center), _p(prob.M),
                                prob.K, prob.o, prob.e, int(k), _p(ins), _p(occ), _p(seg),
                                threads)
    if rc != 0:
        raise RuntimeError("oracle anchored alignment failed")
    return seg, ins, occ


def msa(prob, center, threads=0):
    """The whole path for a given center: (seg, ins, occ, G, W, msa)."""
    seg, ins, occ = align_all(prob, center, threads)
    G, W, rows = merge(prob, center, ins, occ)
    return seg, ins, occ, G, W, rows
