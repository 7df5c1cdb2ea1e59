"""The allocation-free pair-score entry point (msa_pair_scores_noalloc) gives
the same scores as msa_pair_scores, on two calls in a row.

It is meant for callers that cannot allocate device memory (for example code
running while a CUDA graph is captured), so every buffer here is allocated by
the test itself.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_pair_scores_match_the_context_path():
    import torch
    from seqgen import generate, scoring
    from tests._gpu import binding
    b = binding()
    letters, offsets, w, _ = generate("batched_uneven_10k", n=160, seed=21)
    alph, M, _, _ = scoring(w.kind)
    lens = np.diff(offsets)
    assert lens.max() > 512          # several 512-row passes use the fixed scratch
    rng = np.random.default_rng(4)
    pairs = rng.integers(0, lens.size, size=(700, 2)).astype(np.int64)
    pairs[:20, 1] = pairs[:20, 0]    # self pairs
    pairs[20:40, 0] = int(np.argmax(lens))
    with b.Context(M, alph, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        expected = b.msa_pair_scores(h, pairs)
    lut = np.full(256, 255, np.uint8)
    for k, ch in enumerate(alph):
        lut[ord(ch)] = k
    dres = torch.from_numpy(lut[letters]).cuda()
    doff = torch.from_numpy(offsets.astype(np.int64)).cuda()
    dpairs = torch.from_numpy(pairs).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((pairs.shape[0],), -7, dtype=torch.int32, device="cuda")
        b.msa_pair_scores_noalloc(dres, doff, dpairs, int(lens.max()), M, w.gap_open,
                                  w.gap_extend, out, stream=stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert (got == expected).all(), "call %d differs" % call
    # a pair touching a sequence longer than max_len is refused, not computed
    out = torch.zeros(pairs.shape[0], dtype=torch.int32, device="cuda")
    with pytest.raises(b.MSAError) as ei:
        b.msa_pair_scores_noalloc(dres, doff, dpairs, 64, M, w.gap_open, w.gap_extend, out,
                                  stream=stream)
    assert ei.value.code == b.MSA_ERANGE
