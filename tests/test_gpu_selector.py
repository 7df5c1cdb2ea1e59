"""The learned center selector on the GPU vs the fp64 oracle: embeddings,
loss, gradients and an Adam step (bf16 tolerance), exact training targets,
and what training gains over choosing the center without the network."""
import os

import numpy as np
import pytest

import oracle
from oracle import net
from tests._gpu import binding, workload, make_ctx, oracle_problem

pytestmark = pytest.mark.gpu

# bf16 operands (8 mantissa bits) through four layers: a few 1e-2 relative
EMB_TOL, LOSS_TOL, GRAD_TOL = 3e-2, 6e-2, 8e-2


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def setup_small(seed=2, n=14):
    letters, offsets, w, alph, M = workload("learned_center_50k", n=n, seed=seed)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    seqs = [prob.seq(i) for i in range(prob.n)]
    return letters, offsets, w, alph, M, prob, seqs


def test_embeddings_loss_and_gradients_match_oracle():
    b = binding()
    letters, offsets, w, alph, M, prob, seqs = setup_small()
    rng = np.random.default_rng(5)
    pairs = rng.integers(0, prob.n, size=(10, 2))
    targets = rng.uniform(0.2, 0.9, size=10).astype(np.float32)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        b.msa_selector_init(h, seed=7)
        flat = b.msa_selector_params(h).astype(np.float64)
        emb = b.msa_selector_embed(h)
        loss, grad = b.msa_selector_grad(h, pairs, targets)
    params = net.unflatten(flat)
    oemb = net.embed_all(params, seqs)
    assert rel_err(emb, oemb) < EMB_TOL
    oloss, og = net.loss_and_grad(params, seqs, pairs, targets.astype(np.float64))
    assert abs(loss - oloss) <= LOSS_TOL * abs(oloss)
    ogflat = net.flatten(og)
    assert rel_err(grad, ogflat) < GRAD_TOL
    # every tensor, not only the total (b4's true gradient is exactly zero: a
    # bias shared by all embeddings cancels in e_A - e_B, so its error is
    # measured against the whole gradient)
    at, total = 0, np.linalg.norm(ogflat)
    for name, shape in net.SHAPES:
        size = int(np.prod(shape))
        g, o = grad[at:at + size], ogflat[at:at + size]
        scale = max(np.linalg.norm(o), 1e-2 * total)
        assert np.linalg.norm(g - o) / scale < GRAD_TOL, name
        at += size


def test_embeddings_many_tiles_sampled():
    """Enough rows that every persistent tensor-core CTA walks many 128-row
    tiles through both of its input buffers: sampled embeddings against the
    fp64 oracle."""
    b = binding()
    letters, offsets, w, alph, M = workload("learned_center_50k", n=1500, seed=9)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        b.msa_selector_init(h, seed=13)
        params = net.unflatten(b.msa_selector_params(h).astype(np.float64))
        emb = b.msa_selector_embed(h)
    pick = np.random.default_rng(4).choice(prob.n, size=24, replace=False)
    pick[:2] = [0, prob.n - 1]
    oemb = np.stack([net.forward(params, prob.seq(int(i)))[0] for i in pick])
    assert rel_err(emb[pick], oemb) < EMB_TOL


def test_one_adam_step_matches_oracle():
    b = binding()
    letters, offsets, w, alph, M, prob, seqs = setup_small(seed=3)
    pairs = np.array([(i, (i * 5 + 3) % prob.n) for i in range(prob.n)])
    targets = np.linspace(0.3, 0.8, len(pairs)).astype(np.float32)
    lr = 1e-3
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        b.msa_selector_init(h, seed=11)
        before = b.msa_selector_params(h).astype(np.float64)
        b.msa_selector_train(h, pairs, targets, steps=1, batch_pairs=len(pairs), lr=lr)
        after = b.msa_selector_params(h).astype(np.float64)
    params = net.unflatten(before)
    _, og = net.loss_and_grad(params, seqs, pairs, targets.astype(np.float64))
    net.adam(params, og, {}, 1, lr, 0.9, 0.999, 1e-8)
    exp = net.flatten(params)
    # a first Adam step moves every weight by ~lr * sign(g): compare moves
    step_gpu, step_orc = after - before, exp - before
    big = np.abs(og_flat := net.flatten(og)) > 1e-3 * np.abs(og_flat).max()
    agree = np.sign(step_gpu[big]) == np.sign(step_orc[big])
    assert agree.mean() > 0.97
    assert np.abs(step_gpu - step_orc).max() <= 2.05 * lr


def test_targets_are_scaled_exact_distances():
    b = binding()
    letters, offsets, w, alph, M, prob, seqs = setup_small(seed=4, n=30)
    rng = np.random.default_rng(6)
    pairs = rng.integers(0, prob.n, size=(50, 2))
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        t = b.msa_selector_targets(h, pairs, scale=1e-3)
    S = oracle.pair_scores(prob, pairs)
    Sa = oracle.pair_scores(prob, np.stack([pairs[:, 0], pairs[:, 0]], 1))
    Sb = oracle.pair_scores(prob, np.stack([pairs[:, 1], pairs[:, 1]], 1))
    assert np.allclose(t, net.distance_targets(S, Sa, Sb, 1e-3), rtol=1e-6, atol=1e-6)


def test_training_gains_over_the_method_without_it(tmp_path):
    """Trained on exact-kernel distances, the selector ranks the exact center
    among its best candidates: refining its top 64 with exact row sums gives
    the exact center's row sum and avg SP (0 % loss), where the untrained
    network and the first sequence (the nucleotide path's center) do worse,
    at a fraction of the exact all-pairs cost."""
    b = binding()
    from seqgen import generate, training_pairs
    letters, offsets, w, fam = generate("learned_center_50k", n=1200, seed=31)
    alph, M = workload("learned_center_50k", n=2)[3:5]
    pairs = training_pairs(1200, 24000, fam, seed=8)

    def avg_sp(h, center):
        b.msa_align_to_center(h, center)
        b.msa_merge_gaps(h, want_rows=False)
        return b.msa_sp_score(h) / (1200 * 1199 / 2)

    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        exact, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        rowsum = b.msa_center_rowsums(h).astype(np.float64)
        exact_ms = b.msa_stage_times(h)[0]["center"]
        b.msa_selector_init(h, seed=1)
        untrained, _ = b.msa_select_center(h, b.MSA_CENTER_LEARNED_REFINED, candidates=64)
        losses = b.msa_selector_train(h, pairs, steps=4000, batch_pairs=256, lr=3e-4, seed=3)
        top1, _ = b.msa_select_center(h, b.MSA_CENTER_LEARNED)
        refined, rs = b.msa_select_center(h, b.MSA_CENTER_LEARNED_REFINED, candidates=64)
        st = b.msa_stage_times(h)[0]
        refined_ms = st["selector"] + st["center"]
        sp = {name: avg_sp(h, c) for name, c in
              [("exact", exact), ("refined", refined), ("top1", top1), ("untrained", untrained),
               ("first", 0)]}
        path = os.path.join(str(tmp_path), "sel.bin")
        b.msa_save_selector(h, path)
        saved = b.msa_selector_params(h)
    excess = {name: rowsum[c] / rowsum[exact] - 1 for name, c in
              [("refined", refined), ("top1", top1), ("untrained", untrained), ("first", 0)]}
    print("avg SP", sp, "row-sum excess", excess, "loss", float(losses[:20].mean()), "->",
          float(losses[-20:].mean()), "exact ms", exact_ms, "refined ms", refined_ms)
    assert rs == rowsum[refined]
    assert losses[-50:].mean() < 0.1 * losses[:10].mean()
    assert excess["top1"] < excess["first"] and excess["top1"] < 0.5 * excess["untrained"]
    assert excess["refined"] < 0.01
    assert sp["refined"] <= 1.01 * sp["exact"]
    assert refined_ms < exact_ms
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h2:
        b.msa_load(h2, letters, offsets)
        b.msa_load_selector(h2, path)
        assert (b.msa_selector_params(h2) == saved).all()
        assert b.msa_select_center(h2, b.MSA_CENTER_LEARNED)[0] == top1


@pytest.mark.parametrize("k", [400, 24])
def test_refined_over_references_is_the_sampled_row_sum(k):
    """Candidates ranked by their row sums over a reference sample (the
    candidates and the references meet as a view of the set): the winner's
    sum is the oracle's sampled row sum; with every sequence a candidate the
    winner is the sampled exact center, and with 24 no candidate beats it."""
    b = binding()
    from seqgen import reference_sample
    letters, offsets, w, alph, M = workload("learned_center_50k", n=400, seed=3)
    prob = oracle_problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    refs = reference_sample(400, 37, seed=9)
    oc, orow = oracle.exact_center(prob, refs=refs)
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        b.msa_selector_init(h, seed=1)
        c, s = b.msa_select_center_refined(h, candidates=k, refs=refs)
        emb = b.msa_selector_embed(h).astype(np.float64)
        with pytest.raises(b.MSAError):
            b.msa_select_center_refined(h, candidates=k, refs=np.array([3, 3]))
    assert s == orow[c]
    if k == 400:
        assert c == oc
        return
    d = ((emb - emb.mean(0)) ** 2).sum(1)
    order = np.argsort(d, kind="stable")
    # the device ranks in fp32: allow a near-tie at the k-th place
    assert c in set(order[:k + 2].tolist())
    for q in order[:k - 2]:
        assert orow[q] > orow[c] or (orow[q] == orow[c] and q >= c)
