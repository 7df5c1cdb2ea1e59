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
    # every tensor, not only the total
    at = 0
    for name, shape in net.SHAPES:
        size = int(np.prod(shape))
        assert rel_err(grad[at:at + size], ogflat[at:at + size]) < GRAD_TOL, name
        at += size


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


def test_targets_are_exact_normalised_distances():
    b = binding()
    letters, offsets, w, alph, M, prob, seqs = setup_small(seed=4, n=30)
    rng = np.random.default_rng(6)
    pairs = rng.integers(0, prob.n, size=(50, 2))
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        t = b.msa_selector_targets(h, pairs)
    S = oracle.pair_scores(prob, pairs)
    Sa = oracle.pair_scores(prob, np.stack([pairs[:, 0], pairs[:, 0]], 1))
    Sb = oracle.pair_scores(prob, np.stack([pairs[:, 1], pairs[:, 1]], 1))
    assert np.allclose(t, net.distance_targets(S, Sa, Sb), atol=1e-6)


def test_training_gains_over_the_method_without_it(tmp_path):
    """Trained on exact-kernel distances, the selector's center gives a lower
    (better) avg SP than the untrained network's and than the first
    sequence (the nucleotide path's center), and the embedding pass is far
    cheaper than the exact all-pairs selection it replaces."""
    b = binding()
    from seqgen import generate, training_pairs
    letters, offsets, w, fam = generate("learned_center_50k", n=1200, seed=31)
    alph, M = workload("learned_center_50k", n=2)[3:5]
    pairs = training_pairs(1200, 24000, fam, seed=8)

    def avg_sp(h, center):
        b.msa_align_to_center(h, center)
        _, W = b.msa_merge_gaps(h, want_rows=False)
        return b.msa_sp_score(h) / (1200 * 1199 / 2)

    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h:
        b.msa_load(h, letters, offsets)
        exact, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        exact_ms = b.msa_stage_times(h)[0]["center"]
        b.msa_selector_init(h, seed=1)
        untrained, _ = b.msa_select_center(h, b.MSA_CENTER_LEARNED)
        losses = b.msa_selector_train(h, pairs, steps=400, batch_pairs=256, lr=1e-3, seed=3)
        learned, _ = b.msa_select_center(h, b.MSA_CENTER_LEARNED)
        learned_ms = b.msa_stage_times(h)[0]["selector"]
        sp = {name: avg_sp(h, c) for name, c in
              [("exact", exact), ("learned", learned), ("untrained", untrained), ("first", 0)]}
        path = os.path.join(str(tmp_path), "sel.bin")
        b.msa_save_selector(h, path)
        saved = b.msa_selector_params(h)
    print("avg SP", sp, "loss", float(losses[:20].mean()), "->", float(losses[-20:].mean()),
          "exact ms", exact_ms, "learned ms", learned_ms)
    assert losses[-50:].mean() < 0.5 * losses[:10].mean()
    assert sp["learned"] <= sp["first"] and sp["learned"] <= sp["untrained"]
    assert sp["learned"] <= 1.05 * sp["exact"]
    assert learned_ms < exact_ms
    with make_ctx(alph, M, w.gap_open, w.gap_extend) as h2:
        b.msa_load(h2, letters, offsets)
        b.msa_load_selector(h2, path)
        assert (b.msa_selector_params(h2) == saved).all()
        assert b.msa_select_center(h2, b.MSA_CENTER_LEARNED)[0] == learned
