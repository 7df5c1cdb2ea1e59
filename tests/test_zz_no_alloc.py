"""The allocation-free pair-score entry point (msa_pair_scores_noalloc) gives
the oracle's scores, the same as msa_pair_scores, on two calls in a row.

It is meant for callers that cannot allocate device memory (plug-ins whose
host application owns the GPU's memory, processes whose memory comes from
another framework's pool), so every buffer here is allocated by the test
itself.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs():
    from seqgen import generate, scoring
    letters, offsets, w, _ = generate("batched_uneven_10k", n=160, seed=21)
    alph, M, _, _ = scoring(w.kind)
    lens = np.diff(offsets)
    assert lens.max() > 512          # several 512-row passes use the fixed scratch
    rng = np.random.default_rng(4)
    pairs = rng.integers(0, lens.size, size=(700, 2)).astype(np.int64)
    pairs[:20, 1] = pairs[:20, 0]    # self pairs
    pairs[20:40, 0] = int(np.argmax(lens))
    return letters, offsets, w, alph, M, lens, pairs


def _device_inputs(letters, offsets, alph, pairs):
    import torch
    lut = np.full(256, 255, np.uint8)
    for k, ch in enumerate(alph):
        lut[ord(ch)] = k
    dres = torch.from_numpy(lut[letters]).cuda()
    doff = torch.from_numpy(offsets.astype(np.int64)).cuda()
    dpairs = torch.from_numpy(pairs).cuda()
    return dres, doff, dpairs


def test_noalloc_pair_scores_match_the_oracle():
    import torch
    import oracle
    from tests._gpu import binding
    b = binding()
    letters, offsets, w, alph, M, lens, pairs = _inputs()
    prob = oracle.Problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    expected = oracle.pair_scores(prob, pairs)
    with b.Context(M, alph, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        assert (b.msa_pair_scores(h, pairs) == expected).all()
    dres, doff, dpairs = _device_inputs(letters, offsets, alph, pairs)
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


def test_noalloc_rejects_a_residue_outside_the_alphabet():
    """A residue byte >= alphabet (here 255, an unmapped letter) is caught on
    the GPU before it indexes shared memory: its pairs get -1, the call
    returns MSA_EINVAL, and the next call on the same array is correct."""
    import torch
    import oracle
    from tests._gpu import binding
    b = binding()
    letters, offsets, w, alph, M, lens, pairs = _inputs()
    prob = oracle.Problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    expected = oracle.pair_scores(prob, pairs)
    dres, doff, dpairs = _device_inputs(letters, offsets, alph, pairs)
    bad_seq = int(pairs[50, 1])
    dbad = dres.clone()
    dbad[int(offsets[bad_seq]) + lens[bad_seq] // 2] = 255
    stream = torch.cuda.current_stream()
    out = torch.zeros(pairs.shape[0], dtype=torch.int32, device="cuda")
    with pytest.raises(b.MSAError) as ei:
        b.msa_pair_scores_noalloc(dbad, doff, dpairs, int(lens.max()), M, w.gap_open,
                                  w.gap_extend, out, stream=stream)
    assert ei.value.code == b.MSA_EINVAL
    got = out.cpu().numpy()
    touched = (pairs[:, 0] == bad_seq) | (pairs[:, 1] == bad_seq)
    assert (got[touched] == -1).all()
    assert (got[~touched] == expected[~touched]).all()
    out = torch.zeros(pairs.shape[0], dtype=torch.int32, device="cuda")
    b.msa_pair_scores_noalloc(dres, doff, dpairs, int(lens.max()), M, w.gap_open, w.gap_extend,
                              out, stream=stream)
    assert (out.cpu().numpy() == expected).all()


def test_noalloc_binding_checks_its_tensors():
    """The binding refuses a tensor of the wrong type or place before the call."""
    import torch
    from tests._gpu import binding
    b = binding()
    letters, offsets, w, alph, M, lens, pairs = _inputs()
    dres, doff, dpairs = _device_inputs(letters, offsets, alph, pairs)
    out = torch.zeros(pairs.shape[0], dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        b.msa_pair_scores_noalloc(dres, doff.int(), dpairs, 64, M, w.gap_open, w.gap_extend, out)
    with pytest.raises(TypeError):
        b.msa_pair_scores_noalloc(dres.cpu(), doff, dpairs, 64, M, w.gap_open, w.gap_extend, out)
    with pytest.raises(ValueError):
        b.msa_pair_scores_noalloc(dres, doff, dpairs, 64, M, w.gap_open, w.gap_extend, out[:10])
