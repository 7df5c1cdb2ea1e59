"""Pins for the fp64 oracle of the learned center selector (CPU only)."""
import numpy as np
import pytest

from oracle import net


def small_params(rng, scale=0.3):
    return {name: rng.normal(0, scale / np.sqrt(np.prod(shape[:-1]) if len(shape) > 1 else 1), shape)
            for name, shape in net.SHAPES}


def test_conv9_matches_library_correlation():
    """Every (input, output) channel pair of conv9 is numpy's 'valid'
    correlation of the zero-padded input with that pair's 9 taps."""
    rng = np.random.default_rng(0)
    L, cin, cout = 13, 3, 2
    x = rng.normal(size=(L, cin))
    W = rng.normal(size=(net.TAPS, cin, cout))
    b = rng.normal(size=cout)
    out = net.conv9(x, W, b)
    for co in range(cout):
        exp = np.full(L, b[co])
        for ci in range(cin):
            xp = np.concatenate([np.zeros(4), x[:, ci], np.zeros(4)])
            exp += np.correlate(xp, W[:, ci, co], mode="valid")
        assert np.allclose(out[:, co], exp)


def test_bias_only_network_gives_closed_form_loss():
    rng = np.random.default_rng(1)
    p = {name: np.zeros(shape) for name, shape in net.SHAPES}
    p["b4"] = rng.normal(size=net.DIM)
    seqs = [rng.integers(0, 20, size=5) for _ in range(4)]
    e, _ = net.forward(p, seqs[0])
    assert np.allclose(e, p["b4"] * np.sqrt(5))    # sum of 5 rows / sqrt(5)
    t = np.array([0.2, 0.5, 0.9])
    loss, g = net.loss_and_grad(p, seqs, [(0, 1), (1, 2), (3, 0)], t)
    assert np.isclose(loss, np.mean(t ** 2))
    # equal embeddings: the loss does not move with b4 or W4
    assert np.allclose(g["b4"], 0) and np.allclose(g["W4"], 0)


@pytest.mark.parametrize("seed", range(2))
def test_gradients_match_central_differences(seed):
    rng = np.random.default_rng(10 + seed)
    p = small_params(rng)
    seqs = [rng.integers(0, 24, size=int(rng.integers(2, 12))) for _ in range(5)]
    pairs = [(0, 1), (2, 3), (4, 0), (1, 1)]
    t = rng.uniform(0, 1, size=len(pairs))
    _, g = net.loss_and_grad(p, seqs, pairs, t)
    h = 1e-6
    for name, shape in net.SHAPES:
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in shape)
            if name == "W1":  # make the tap/channel hit a residue that occurs
                idx = (idx[0], int(seqs[0][0]), idx[2])
            old = p[name][idx]
            p[name][idx] = old + h
            lp, _ = net.loss_and_grad(p, seqs, pairs, t)
            p[name][idx] = old - h
            lm, _ = net.loss_and_grad(p, seqs, pairs, t)
            p[name][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 + 1e-5 * abs(fd), (name, idx, fd, g[name][idx])


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(3)
    p = small_params(rng)
    g = {name: rng.normal(size=shape) for name, shape in net.SHAPES}
    before = {k: v.copy() for k, v in p.items()}
    lr, eps = 1e-3, 1e-8
    net.adam(p, g, {}, 1, lr, 0.9, 0.999, eps)
    for name, _ in net.SHAPES:
        # bias-corrected first step: m_hat = g, v_hat = g^2
        exp = before[name] - lr * g[name] / (np.abs(g[name]) + eps)
        assert np.allclose(p[name], exp)


def test_flatten_roundtrip_and_center_rule():
    rng = np.random.default_rng(4)
    p = small_params(rng)
    flat = net.flatten(p)
    assert flat.size == net.n_params()
    q = net.unflatten(flat)
    assert all(np.array_equal(p[k], q[k]) for k in p)
    emb = np.array([[0.0, 0.0], [1.0, 0.0], [-1.0, 0.0], [0.0, 3.0]])
    assert net.center_of(emb) == 0
    # the exact center's distance 2^16 - floor(2^16 S_ab / max(S_aa, S_bb)), 0 when
    # both self scores are 0: 5 of 10 -> 32768; 0 of 6 -> 65536; 1 of 3 -> 65536 -
    # 21845; no self score -> 0
    t = net.distance_targets([5, 0, 1, 0], [10, 4, 3, 0], [10, 6, 2, 0], 0.01)
    assert np.allclose(t, [327.68, 655.36, 436.91, 0.0])


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 9, 40])
def test_pooled_output_layer_on_window_sums(L):
    """The GPU embedding runs the output layer on nine window sums per
    sequence: P_0 = sum of padded rows 0 .. L-1 (row i = a3[i - 4], zero
    outside), P_{t+1} = P_t - row t + row L + t, and
    sum_r y4[r] = sum_t P_t W4_t + L b4.  Checked against the oracle's
    convolution followed by the sum over positions, down to one residue."""
    rng = np.random.default_rng(L)
    a3 = np.maximum(rng.normal(size=(L, net.WIDTH)), 0)
    W = rng.normal(size=(net.TAPS, net.WIDTH, net.DIM))
    b = rng.normal(size=net.DIM)
    pad = np.vstack([np.zeros((net.HALF, net.WIDTH)), a3, np.zeros((net.HALF, net.WIDTH))])
    P = [pad[0:L].sum(axis=0)]
    for t in range(net.TAPS - 1):
        P.append(P[-1] - pad[t] + pad[L + t])
    window = sum(P[t] @ W[t] for t in range(net.TAPS)) + L * b
    assert np.allclose(window, net.conv9(a3, W, b).sum(axis=0), rtol=1e-12, atol=1e-9)
