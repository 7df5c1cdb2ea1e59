"""ctypes binding of libmsa.so (include/msa.h): argument marshalling only.

Every function has the name of its C entry point.  Arrays may be numpy arrays
(host) or torch tensors (host or CUDA); outputs are returned as numpy arrays
unless a caller-provided `out` buffer is given.  Errors raise MSAError with the
library's message.  There is no CPU fallback: importing this module on a
machine without the built library raises.
"""
import ctypes
import os

import numpy as np

from . import _build

MSA_OK, MSA_EINVAL, MSA_ENOMEM, MSA_ECUDA, MSA_ETIMEOUT, MSA_ESTATE, MSA_ERANGE = 0, -1, -2, -3, -4, -5, -6
MSA_AUTO, MSA_INT16, MSA_INT32 = 0, 1, 2
MSA_CENTER_EXACT, MSA_CENTER_EXACT_SAMPLED, MSA_CENTER_LEARNED, MSA_CENTER_FIRST = 0, 1, 2, 3
MSA_CENTER_LEARNED_REFINED = 4
MSA_MAX_LEN = 8192
MSA_ALIGN_FULL, MSA_ALIGN_BOX = 0, 1

STAGES = ("encode", "center", "align_dp", "traceback", "merge", "rows", "sp", "center_kernels",
          "align_kernels", "selector", "tree", "light_score", "light_corner", "light_box")


class MSAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class msa_train_cfg(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch_pairs", ctypes.c_int32),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_uint64), ("target_scale", ctypes.c_float)]


class msa_params(ctypes.Structure):
    _fields_ = [("matrix", ctypes.c_void_p), ("alphabet", ctypes.c_int32),
                ("letters", ctypes.c_char_p), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("sat_limit", ctypes.c_int32)]


_lib = None
_SIGS = {
    "msa_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(msa_params), ctypes.c_void_p]),
    "msa_destroy": (None, [ctypes.c_void_p]),
    "msa_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "msa_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "msa_pair_scores": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "msa_select_center": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "msa_select_center_refined": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_center_rowsums": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_align_anchored": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "msa_align_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "msa_center_partial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "msa_center_combine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "msa_align_to_center": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "msa_alignment_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_debug_codes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "msa_merge_gaps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_sp_score": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_insert_maxima": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_merge_gaps_with": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_dims": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "msa_memory": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_set_memory_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "msa_set_codes_budget": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "msa_set_align_group": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "msa_debug_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_tree_distances": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_set_align_threads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "msa_set_align_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "msa_align_boxes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_nj": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                              ctypes.c_void_p]),
    "msa_nj_tree": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_nj_cluster_tree": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "msa_probe_int_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_selector_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64]),
    "msa_selector_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "msa_selector_targets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                            ctypes.c_void_p]),
    "msa_selector_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "msa_selector_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.POINTER(msa_train_cfg), ctypes.c_void_p]),
    "msa_selector_embed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "msa_save_selector": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "msa_load_selector": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "msa_pair_scores_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                               ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
}


def library_path():
    return _build.LIB


def lib():
    """Load libmsa.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libmsa.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(x))


def _check(ctx, rc):
    if rc != MSA_OK:
        msg = lib().msa_last_error(ctx)
        raise MSAError(rc, msg.decode() if msg else "error")


def msa_create(matrix, letters, gap_open, gap_extend, precision=MSA_AUTO, sat_limit=0, stream=None):
    """Returns a context handle.  stream: a torch.cuda.Stream, an int handle, or None."""
    M = np.ascontiguousarray(matrix, dtype=np.int8)
    p = msa_params(ctypes.c_void_p(M.ctypes.data), int(M.shape[0]), letters.encode(),
                   int(gap_open), int(gap_extend), int(precision), int(sat_limit))
    h = ctypes.c_void_p()
    st = getattr(stream, "cuda_stream", stream)
    rc = lib().msa_create(ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(st) if st else None)
    if rc != MSA_OK:
        raise MSAError(rc, "msa_create rejected its parameters")
    return h


def msa_destroy(ctx):
    lib().msa_destroy(ctx)


def msa_last_error(ctx):
    m = lib().msa_last_error(ctx)
    return m.decode() if m else ""


def msa_load(ctx, letters, offsets):
    """letters: uint8 ASCII (numpy, or torch host/CUDA); offsets: int64[n+1] host."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(ctx, lib().msa_load(ctx, _ptr(letters), _ptr(off), off.size - 1))


def msa_autotune(ctx):
    """Measured cells/s per (length bucket, center variant): float64[buckets, variants]."""
    rates = np.zeros((32, 32), np.float64)
    dims = np.zeros(2, np.int32)
    _check(ctx, lib().msa_autotune(ctx, _ptr(rates), _ptr(dims)))
    nb, nv = int(dims[0]), int(dims[1])
    return rates.ravel()[:nb * nv].reshape(nb, nv)


def msa_dims(ctx):
    d = np.zeros(4, np.int64)
    _check(ctx, lib().msa_dims(ctx, _ptr(d)))
    return tuple(int(x) for x in d)


def msa_pair_scores(ctx, pairs, out=None):
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    res = np.zeros(pr.shape[0], np.int32) if out is None else out
    _check(ctx, lib().msa_pair_scores(ctx, _ptr(pr), pr.shape[0], _ptr(res)))
    return res


def msa_pair_scores_noalloc(residues, offsets, pairs, max_len, matrix, gap_open, gap_extend,
                            scores_out, stream=None):
    """Allocation-free pair scores for callers that cannot allocate device
    memory: every array is a CUDA tensor the caller owns (residues uint8
    alphabet indices, offsets int64[n+1], pairs int64[npairs, 2], scores_out
    int32[npairs]); matrix is a host array.  Raises MSAError on failure."""
    import torch
    for name, t, dt in (("residues", residues, torch.uint8), ("offsets", offsets, torch.int64),
                        ("pairs", pairs, torch.int64), ("scores_out", scores_out, torch.int32)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if t.dtype != dt:
            raise TypeError("%s must be %s, got %s" % (name, dt, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape [npairs, 2]")
    if offsets.dim() != 1 or offsets.numel() < 2:
        raise ValueError("offsets must hold n + 1 >= 2 entries")
    if scores_out.numel() < pairs.shape[0]:
        raise ValueError("scores_out holds fewer entries than there are pairs")
    M = np.ascontiguousarray(matrix, dtype=np.int8)
    st = getattr(stream, "cuda_stream", stream)
    rc = lib().msa_pair_scores_noalloc(_ptr(residues), _ptr(offsets), offsets.numel() - 1,
                                       _ptr(pairs), pairs.shape[0], int(max_len), _ptr(M),
                                       int(M.shape[0]), int(gap_open), int(gap_extend),
                                       _ptr(scores_out), ctypes.c_void_p(st) if st else None)
    if rc != MSA_OK:
        raise MSAError(rc, "msa_pair_scores_noalloc failed")
    return scores_out


def msa_select_center(ctx, mode, refs=None, candidates=0):
    """Returns (center, winning row sum of distances).  candidates: the
    number of network candidates LEARNED_REFINED checks exactly (0 = 32)."""
    c = np.zeros(1, np.int64)
    s = np.zeros(1, np.int64)
    r = None if refs is None else np.ascontiguousarray(refs, dtype=np.int64)
    nref = r.size if r is not None else int(candidates)
    _check(ctx, lib().msa_select_center(ctx, int(mode), _ptr(r), nref, _ptr(c), _ptr(s)))
    return int(c[0]), int(s[0])


def msa_select_center_refined(ctx, candidates=0, refs=None):
    """Returns (center, winning row sum of distances): the selector's
    `candidates` best sequences (0 = 32) ranked by exact row sums over refs
    (None = every sequence)."""
    c = np.zeros(1, np.int64)
    s = np.zeros(1, np.int64)
    r = None if refs is None else np.ascontiguousarray(refs, dtype=np.int64)
    _check(ctx, lib().msa_select_center_refined(ctx, int(candidates), _ptr(r),
                                                0 if r is None else r.size, _ptr(c), _ptr(s)))
    return int(c[0]), int(s[0])


def msa_align_anchored(ctx, center, k, scores=None):
    """Anchored alignment to `center` (segments of k residues); returns the
    number of sequences the Smith-Waterman path aligned instead."""
    fb = ctypes.c_int64(0)
    _check(ctx, lib().msa_align_anchored(ctx, int(center), int(k), _ptr(scores),
                                         ctypes.byref(fb)))
    return int(fb.value)


ALIGN_LANES = (1, 2, 4, 8, 16, 32)  # lanes per subject group of the alignment kernels


def msa_align_autotune(ctx, center):
    """(rates double[3, 6] = [packed, int32, packed in 384-thread CTAs] x
    [1, 2, 4, 8, 16, 32] lanes, (lanes, packed, threads per CTA))."""
    rates = np.zeros((3, len(ALIGN_LANES)), np.float64)
    choice = np.zeros(3, np.int32)
    _check(ctx, lib().msa_align_autotune(ctx, int(center), _ptr(rates), _ptr(choice)))
    return rates, (int(choice[0]), bool(choice[1]), int(choice[2]))


def msa_set_align_threads(ctx, threads):
    """Threads per CTA of the packed alignment kernel (256 or 384; 0 = 256)."""
    rc = lib().msa_set_align_threads(ctx, int(threads))
    if rc != MSA_OK:
        raise MSAError(rc, "align threads must be 0, 256 or 384")


def msa_center_partial(ctx, shard, nshards, refs=None, out=None):
    """This shard's partial similarity sums of the exact center (uint64[n])."""
    n = msa_dims(ctx)[0]
    res = np.zeros(n, np.uint64) if out is None else out
    if refs is None:
        _check(ctx, lib().msa_center_partial(ctx, None, 0, int(shard), int(nshards), _ptr(res)))
    else:
        r = np.ascontiguousarray(refs, dtype=np.int64)
        _check(ctx, lib().msa_center_partial(ctx, _ptr(r), r.size, int(shard), int(nshards),
                                             _ptr(res)))
    return res


def msa_center_combine(ctx, sums, nref=0):
    """(center, its row sum) from the summed partial sums; sets the row sums."""
    sm = np.ascontiguousarray(sums, dtype=np.uint64)
    c = ctypes.c_int64(0)
    v = ctypes.c_int64(0)
    _check(ctx, lib().msa_center_combine(ctx, _ptr(sm), int(nref), ctypes.byref(c),
                                         ctypes.byref(v)))
    return int(c.value), int(v.value)


def msa_center_rowsums(ctx, out=None):
    n = msa_dims(ctx)[0]
    res = np.zeros(n, np.int64) if out is None else out
    _check(ctx, lib().msa_center_rowsums(ctx, _ptr(res)))
    return res


def msa_align_to_center(ctx, center, scores_out=None):
    _check(ctx, lib().msa_align_to_center(ctx, int(center), _ptr(scores_out)))
    return scores_out


def msa_alignment_info(ctx):
    """(seg int32[n,5], ins uint16[n,Lc+1], occ uint8[n,Lc+1])."""
    n, _, lc, _ = msa_dims(ctx)
    seg = np.zeros((n, 5), np.int32)
    ins = np.zeros((n, lc + 1), np.uint16)
    occ = np.zeros((n, lc + 1), np.uint8)
    _check(ctx, lib().msa_alignment_info(ctx, _ptr(seg), _ptr(ins), _ptr(occ)))
    return seg, ins, occ


def msa_debug_codes(ctx, seq, ls):
    _, _, lc, _ = msa_dims(ctx)
    out = np.zeros((lc, int(ls)), np.uint8)
    _check(ctx, lib().msa_debug_codes(ctx, int(seq), _ptr(out)))
    return out


def msa_merge_gaps(ctx, out=None, want_rows=True):
    """Returns (msa uint8[n, W] or the given out buffer or None, W)."""
    w = np.zeros(1, np.int64)
    _check(ctx, lib().msa_merge_gaps(ctx, None, _ptr(w)))
    W = int(w[0])
    if not want_rows:
        return None, W
    n = msa_dims(ctx)[0]
    res = np.zeros((n, W), np.uint8) if out is None else out
    _check(ctx, lib().msa_merge_gaps(ctx, _ptr(res), _ptr(w)))
    return res, W


def msa_insert_maxima(ctx):
    lc = msa_dims(ctx)[2]
    G = np.zeros(lc + 1, np.int32)
    _check(ctx, lib().msa_insert_maxima(ctx, _ptr(G)))
    return G


def msa_merge_gaps_with(ctx, G, out=None):
    """(rows uint8[n, W], W) merged with the given slot widths."""
    g = np.ascontiguousarray(G, dtype=np.int32)
    w = np.zeros(1, np.int64)
    _check(ctx, lib().msa_merge_gaps_with(ctx, _ptr(g), None, _ptr(w)))
    W = int(w[0])
    res = np.zeros((msa_dims(ctx)[0], W), np.uint8) if out is None else out
    _check(ctx, lib().msa_merge_gaps_with(ctx, _ptr(g), _ptr(res), _ptr(w)))
    return res, W


def msa_sp_score(ctx):
    v = np.zeros(1, np.int64)
    _check(ctx, lib().msa_sp_score(ctx, _ptr(v)))
    return int(v[0])


def msa_tree_distances(ctx, out=None):
    """Fixed-point p-distances int64[n, n] of the merged MSA's rows."""
    n = msa_dims(ctx)[0]
    d = np.zeros((n, n), np.int64) if out is None else out
    _check(ctx, lib().msa_tree_distances(ctx, _ptr(d)))
    return d


def msa_nj(ctx, dist):
    """Neighbour joining of an int64[n, n] matrix (host array or device
    tensor): (joins int32[n-1, 2], lengths float64[n-1, 2])."""
    n = int(dist.shape[0])
    joins = np.zeros((max(n - 1, 0), 2), np.int32)
    lengths = np.zeros((max(n - 1, 0), 2), np.float64)
    if isinstance(dist, np.ndarray):
        dist = np.ascontiguousarray(dist, dtype=np.int64)
    elif getattr(dist, "dtype", None) is not None and str(dist.dtype) != "torch.int64":
        raise ValueError("distances must be int64")
    _check(ctx, lib().msa_nj(ctx, _ptr(dist), n, _ptr(joins), _ptr(lengths)))
    return joins, lengths


def msa_nj_tree(ctx):
    """The neighbour-joining tree of the merged MSA: (joins, lengths) as msa_nj."""
    n = msa_dims(ctx)[0]
    joins = np.zeros((max(n - 1, 0), 2), np.int32)
    lengths = np.zeros((max(n - 1, 0), 2), np.float64)
    _check(ctx, lib().msa_nj_tree(ctx, _ptr(joins), _ptr(lengths)))
    return joins, lengths


def msa_nj_cluster_tree(ctx, sample, cap):
    """The clustered tree of the merged MSA: (joins int32[n-1, 2], lengths
    float64[n-1, 2], cluster int32[n])."""
    n = msa_dims(ctx)[0]
    smp = np.ascontiguousarray(sample, dtype=np.int64)
    joins = np.zeros((max(n - 1, 0), 2), np.int32)
    lengths = np.zeros((max(n - 1, 0), 2), np.float64)
    cluster = np.zeros(n, np.int32)
    _check(ctx, lib().msa_nj_cluster_tree(ctx, _ptr(smp), smp.size, int(cap), _ptr(joins),
                                          _ptr(lengths), _ptr(cluster)))
    return joins, lengths, cluster


def msa_memory(ctx):
    """(bytes held now, peak bytes) of the context's device buffers."""
    cur = np.zeros(1, np.int64)
    peak = np.zeros(1, np.int64)
    _check(ctx, lib().msa_memory(ctx, _ptr(cur), _ptr(peak)))
    return int(cur[0]), int(peak[0])


def msa_set_memory_limit(ctx, limit_bytes):
    _check(ctx, lib().msa_set_memory_limit(ctx, int(limit_bytes)))


def msa_set_align_group(ctx, lanes):
    """Lanes per subject group of the alignment kernels (1, 2, 4, 8, 16, 32; 0 = modelled)."""
    rc = lib().msa_set_align_group(ctx, int(lanes))
    if rc != MSA_OK:
        raise MSAError(rc, "align group must be 0 or one of %s" % (ALIGN_LANES,))


def msa_set_align_mode(ctx, mode):
    """MSA_ALIGN_FULL (codes of every cell) or MSA_ALIGN_BOX (traceback-light)."""
    rc = lib().msa_set_align_mode(ctx, int(mode))
    if rc != MSA_OK:
        raise MSAError(rc, "align mode must be MSA_ALIGN_FULL or MSA_ALIGN_BOX")


def msa_align_boxes(ctx, n, out=None):
    """int32[n, 4] {i0, j0, i2, j2} per sequence of the last MSA_ALIGN_BOX alignment."""
    res = np.zeros((n, 4), np.int32) if out is None else out
    _check(ctx, lib().msa_align_boxes(ctx, _ptr(res)))
    return res


def msa_set_codes_budget(ctx, nbytes):
    """Bytes of traceback codes the alignment holds at once (its batch size)."""
    rc = lib().msa_set_codes_budget(ctx, int(nbytes))
    if rc != MSA_OK:
        raise MSAError(rc, "codes budget must be >= 1 byte")


def msa_debug_wait_timeout(ctx):
    """True when the tensor-core convolution reported its bounded waits running out."""
    out = np.zeros(1, np.int32)
    _check(ctx, lib().msa_debug_wait_timeout(ctx, _ptr(out)))
    return bool(out[0])


def msa_stage_times(ctx):
    """({stage: ms}, {"center_cells", "align_cells", "launches"})."""
    ms = np.zeros(len(STAGES), np.float32)
    cnt = np.zeros(3, np.int64)
    _check(ctx, lib().msa_stage_times(ctx, _ptr(ms), len(STAGES), _ptr(cnt)))
    return (dict(zip(STAGES, (float(x) for x in ms))),
            {"center_cells": int(cnt[0]), "align_cells": int(cnt[1]), "launches": int(cnt[2])})


def msa_selector_init(ctx, seed=0, params=None):
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, lib().msa_selector_init(ctx, int(seed), _ptr(p), 0 if p is None else p.size))


def msa_selector_params(ctx):
    cnt = np.zeros(1, np.int64)
    _check(ctx, lib().msa_selector_params(ctx, None, _ptr(cnt)))
    out = np.zeros(int(cnt[0]), np.float32)
    _check(ctx, lib().msa_selector_params(ctx, _ptr(out), _ptr(cnt)))
    return out


DEFAULT_TARGET_SCALE = 1e-3


def msa_selector_targets(ctx, pairs, scale=DEFAULT_TARGET_SCALE):
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    out = np.zeros(pr.shape[0], np.float32)
    _check(ctx, lib().msa_selector_targets(ctx, _ptr(pr), pr.shape[0], float(scale), _ptr(out)))
    return out


def msa_selector_grad(ctx, pairs, targets):
    """(loss, gradient float32[count])."""
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    t = np.ascontiguousarray(targets, dtype=np.float32)
    cnt = np.zeros(1, np.int64)
    _check(ctx, lib().msa_selector_params(ctx, None, _ptr(cnt)))
    g = np.zeros(int(cnt[0]), np.float32)
    loss = np.zeros(1, np.float32)
    _check(ctx, lib().msa_selector_grad(ctx, _ptr(pr), _ptr(t), pr.shape[0], _ptr(g), _ptr(loss)))
    return float(loss[0]), g


def msa_selector_train(ctx, pairs, targets=None, steps=3000, batch_pairs=256, lr=3e-4,
                       beta1=0.9, beta2=0.999, eps=1e-8, seed=0, target_scale=0.0):
    """Returns the per-step batch losses (float32[steps])."""
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.float32)
    cfg = msa_train_cfg(int(steps), int(batch_pairs), float(lr), float(beta1), float(beta2),
                        float(eps), int(seed), float(target_scale))
    losses = np.zeros(max(1, int(steps)), np.float32)
    _check(ctx, lib().msa_selector_train(ctx, _ptr(pr), _ptr(t), pr.shape[0], ctypes.byref(cfg),
                                         _ptr(losses)))
    return losses[:int(steps)]


def msa_selector_embed(ctx, out=None):
    n = msa_dims(ctx)[0]
    res = np.zeros((n, 64), np.float32) if out is None else out
    _check(ctx, lib().msa_selector_embed(ctx, _ptr(res)))
    return res


def msa_save_selector(ctx, path):
    _check(ctx, lib().msa_save_selector(ctx, str(path).encode()))


def msa_load_selector(ctx, path):
    _check(ctx, lib().msa_load_selector(ctx, str(path).encode()))


MSA_PROBE_VIADDMAX_S16X2, MSA_PROBE_VIMAX3_S16X2, MSA_PROBE_VIADDMAX_S32, MSA_PROBE_PRMT = 0, 1, 2, 3


def msa_probe_int_rate(op):
    """(instructions/s, instructions per clock per SM) of one integer op."""
    r = np.zeros(2, np.float64)
    rc = lib().msa_probe_int_rate(int(op), _ptr(r[:1]), _ptr(r[1:]))
    if rc != MSA_OK:
        raise MSAError(rc, "probe failed")
    return float(r[0]), float(r[1])


class Context:
    """Owns one msa_ctx; `with Context(...) as h:` destroys it on exit."""

    def __init__(self, matrix, letters, gap_open, gap_extend, **kw):
        self.h = msa_create(matrix, letters, gap_open, gap_extend, **kw)

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self.h:
            msa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
