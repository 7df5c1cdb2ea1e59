"""fp64 oracle of the learned center selector (test infrastructure only).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
path.

The paper selects the center with Smith-Waterman scores; the learned selector
replaces that O(n^2) pass with an embedding network whose squared distances
are trained to follow the scaled alignment distance
t(A,B) = scale * d(A,B), with d the exact center's distance,
d(A,B) = 2^16 - floor(2^16 S(A,B) / max(S(A,A), S(B,B))),
so that argmin_i sum_j ||e_i - e_j||^2 tracks the exact center's
argmin_i sum_j d(i,j).
Architecture (a reading; the paper has no network):
  x0  = one-hot(residues) over KP = 32 channels            [L, 32]
  a1  = relu(conv9(x0, W1, b1))                             [L, 128]
  a2  = relu(conv9(a1, W2, b2))                             [L, 128]
  a3  = relu(conv9(a2, W3, b3))                             [L, 128]
  y4  = conv9(a3, W4, b4)                                   [L, 64]
  e   = (sum over the L positions of y4) / sqrt(L)          [64]
(the sum over positions is divided by sqrt(L), not by L: a mean makes the
embedding nearly blind to the length, which the distance depends on.)
conv9(x, W, b)[p] = b + sum_{k=0..8} xpad[p + k] @ W[k], xpad = x with four
zero rows before and after (the sequence ends are zero-padded).
Loss over a batch of pairs: mean over pairs of (||e_A - e_B||^2 - t)^2.
Adam (Kingma & Ba 2015) with bias correction.

Parameters are a dict of float64 arrays: W1 [9,32,128], b1 [128], W2 [9,128,128],
b2, W3 [9,128,128], b3, W4 [9,128,64], b4 [64]; flat order W1 b1 W2 b2 W3 b3 W4 b4.
"""
import numpy as np

KP, WIDTH, DIM, TAPS, HALF = 32, 128, 64, 9, 4
SHAPES = [("W1", (TAPS, KP, WIDTH)), ("b1", (WIDTH,)), ("W2", (TAPS, WIDTH, WIDTH)),
          ("b2", (WIDTH,)), ("W3", (TAPS, WIDTH, WIDTH)), ("b3", (WIDTH,)),
          ("W4", (TAPS, WIDTH, DIM)), ("b4", (DIM,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, at = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = flat[at:at + size].reshape(shape).copy()
        at += size
    assert at == flat.size
    return out


def flatten(params):
    return np.concatenate([params[name].ravel() for name, _ in SHAPES])


def conv9(x, W, b):
    """out[p] = b + sum_k xpad[p + k] @ W[k] (xpad: 4 zero rows each side)."""
    L = x.shape[0]
    xp = np.vstack([np.zeros((HALF, x.shape[1])), x, np.zeros((HALF, x.shape[1]))])
    out = np.tile(b, (L, 1)).astype(np.float64)
    for k in range(TAPS):
        out += xp[k:k + L] @ W[k]
    return out


def conv9_backward(x, W, dout):
    """Gradients of conv9 with respect to x, W and b, given d(out)."""
    L = x.shape[0]
    xp = np.vstack([np.zeros((HALF, x.shape[1])), x, np.zeros((HALF, x.shape[1]))])
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for k in range(TAPS):
        dW[k] = xp[k:k + L].T @ dout
        dxp[k:k + L] += dout @ W[k].T
    return dxp[HALF:HALF + L], dW, dout.sum(axis=0)


def onehot(res):
    x = np.zeros((len(res), KP))
    x[np.arange(len(res)), np.asarray(res, dtype=np.int64)] = 1.0
    return x


def forward(params, res):
    """Embedding of one encoded sequence and the activations for backward."""
    x0 = onehot(res)
    z1 = conv9(x0, params["W1"], params["b1"]); a1 = np.maximum(z1, 0)
    z2 = conv9(a1, params["W2"], params["b2"]); a2 = np.maximum(z2, 0)
    z3 = conv9(a2, params["W3"], params["b3"]); a3 = np.maximum(z3, 0)
    y4 = conv9(a3, params["W4"], params["b4"])
    return y4.sum(axis=0) / np.sqrt(len(res)), (x0, a1, a2, a3)


def backward(params, cache, de):
    """Parameter gradients of one sequence's embedding, given d(e)."""
    x0, a1, a2, a3 = cache
    L = x0.shape[0]
    g = {}
    dy4 = np.tile(de / np.sqrt(L), (L, 1))
    da3, g["W4"], g["b4"] = conv9_backward(a3, params["W4"], dy4)
    dz3 = da3 * (a3 > 0)
    da2, g["W3"], g["b3"] = conv9_backward(a2, params["W3"], dz3)
    dz2 = da2 * (a2 > 0)
    da1, g["W2"], g["b2"] = conv9_backward(a1, params["W2"], dz2)
    dz1 = da1 * (a1 > 0)
    _, g["W1"], g["b1"] = conv9_backward(x0, params["W1"], dz1)
    return g


def embed_all(params, seqs):
    return np.stack([forward(params, s)[0] for s in seqs])


def loss_and_grad(params, seqs, pairs, targets):
    """Mean pair loss and its gradient (dict like params)."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    targets = np.asarray(targets, dtype=np.float64)
    used = np.unique(pairs)
    emb, caches = {}, {}
    for i in used:
        emb[i], caches[i] = forward(params, seqs[i])
    de = {i: np.zeros(DIM) for i in used}
    loss = 0.0
    m = pairs.shape[0]
    for (a, b), t in zip(pairs, targets):
        diff = emb[a] - emb[b]
        r = float(diff @ diff) - t
        loss += r * r / m
        g = 4.0 * r * diff / m
        de[a] += g
        de[b] -= g
    grads = {name: np.zeros(shape) for name, shape in SHAPES}
    for i in used:
        gi = backward(params, caches[i], de[i])
        for name in grads:
            grads[name] += gi[name]
    return loss, grads


def adam(params, grads, state, step, lr, beta1, beta2, eps):
    """One Adam update in place; state = dict of (m, v); step counts from 1."""
    for name, _ in SHAPES:
        m, v = state.setdefault(name, (np.zeros_like(params[name]), np.zeros_like(params[name])))
        g = grads[name]
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        state[name] = (m, v)
        mh = m / (1 - beta1 ** step)
        vh = v / (1 - beta2 ** step)
        params[name] = params[name] - lr * mh / (np.sqrt(vh) + eps)
    return params


def center_of(emb):
    """argmin_i ||e_i - mean(e)||^2 (lowest index on ties)."""
    mu = emb.mean(axis=0)
    return int(np.argmin(((emb - mu) ** 2).sum(axis=1)))


def distance_targets(S_ab, S_aa, S_bb, scale):
    """scale * d(A,B), d = 2^16 - floor(2^16 S_ab / max(S_aa, S_bb)) (0 when
    that max is 0): the exact center's distance of the pair."""
    S_ab = np.asarray(S_ab, np.int64)
    m = np.maximum(np.asarray(S_aa, np.int64), np.asarray(S_bb, np.int64))
    d = np.where(m > 0, 65536 - (S_ab * 65536) // np.maximum(m, 1), 0)
    return scale * d.astype(np.float64)
