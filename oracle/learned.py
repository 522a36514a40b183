"""Learned sketch proposal (oracle side): features, the scoring MLP, the proposal
distribution, Gumbel-top-tau selection, the per-coordinate training labels and
Adam.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper samples blocks uniformly or with probabilities proportional to the
diagonal of A (Section 6, importance sampling of single columns); the scored
proposal below replaces those fixed probabilities by ones a small network
predicts from per-coordinate features. The paper fixes neither the features nor
the network; the readings used here:

* chunks: the proposal is evaluated once per chunk of L iterations, from the
  residual and the visit ages at the chunk's first iteration k0; every iteration
  k of the chunk draws its own sample from it.
* raw features of coordinate j: x0 = ln A_jj; x1 = ln(1 + |r_j| / rms(r)),
  rms(r) = ||r|| / sqrt(m) (x1 = 0 when r = 0); x2 = ln ||A[:, j]||_2;
  x3 = ln(1 + age_j), age_j = k0 - (last iteration before k0 whose sample held j),
  k0 + 1 when j was never drawn. Each feature is standardised over the m
  coordinates: z = (x - mean) / (std + 1e-6), std the population deviation.
* network: h1 = relu(W1 z + b1) (64), h2 = relu(W2 h1 + b2) (64),
  s = w3 . h2 + b3. In BF16 mode the weights hold bfloat16 values and h1, h2 are
  rounded to bfloat16 before the next layer (a bfloat16-operand pipeline with
  wide accumulation).
* proposal: p_j = (1 - eps) softmax(s)_j + eps / m.
* selection for iteration k: u_j = (hi32(draw(seed, k, 4, j)) + 1/2) / 2^32,
  g_j = -ln(-ln u_j), key_j = ln p_j + g_j; the sample C_k is the tau coordinates
  with the largest keys (ties: smaller index first), in increasing index order.
  The tau largest of ln p_j + Gumbel noise are a draw of tau coordinates without
  replacement from p (the Gumbel-top-k construction).
* label: without momentum one step lowers ||w - w*||_A^2 by exactly r_C . delta
  (delta = M^+ r_C, M = A[C, C]; the projection identity of Section 3). The part
  of coordinate C_p is a_p = r_{C_p} delta_p (for a single coordinate it is the
  whole one-coordinate decrease r_j^2 / A_jj); its target is
  y_p = (1/2) ln(m max(a_p, 0) / ||e_k||_A^2 + 1e-3), ||e_k||_A^2 = (w_k - w*) . r_k,
  so that softmax(s) puts mass on a coordinate in proportion to the square root
  of its measured share of the decrease. The network regresses y on the
  chunk-start features of the drawn coordinate with the loss mean (s - y)^2 / 2.
* optimiser: Adam (Kingma and Ba, 2015) with bias correction.

Parameter vector (4545 entries): W1 (64 x 4, row-major), b1 (64), W2 (64 x 64,
row-major: W2[o, i]), b2 (64), w3 (64), b3 (1).
"""
from __future__ import annotations

import numpy as np

from .rng import draw
from .solver import least_norm_solution

H = 64
NF = 4
N_PARAMS = H * NF + H + H * H + H + H + 1
EPS_STD = 1e-6


def unpack(theta):
    """(W1, b1, W2, b2, w3, b3) views of a flat parameter vector."""
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = t[o:o + H * NF].reshape(H, NF); o += H * NF
    b1 = t[o:o + H]; o += H
    W2 = t[o:o + H * H].reshape(H, H); o += H * H
    b2 = t[o:o + H]; o += H
    w3 = t[o:o + H]; o += H
    b3 = t[o]
    return W1, b1, W2, b2, w3, b3


def bf16(x):
    """Values rounded to the nearest bfloat16 (ties to even), via float32."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def standardise(x):
    """z = (x - mean) / (std + 1e-6) over the coordinates (population std)."""
    x = np.asarray(x, dtype=np.float64)
    return (x - x.mean()) / (x.std() + EPS_STD)


def static_features(A):
    """Standardised ln A_jj and ln ||A[:, j]||_2 (computed once)."""
    A = np.asarray(A, dtype=np.float64)
    return standardise(np.log(np.diag(A))), standardise(np.log(np.linalg.norm(A, axis=0)))


def features(static, r, age):
    """m x 4 standardised features from the static pair, the residual and the ages."""
    r = np.asarray(r, dtype=np.float64)
    m = r.shape[0]
    rms = np.linalg.norm(r) / np.sqrt(m)
    x1 = np.log1p(np.abs(r) / rms) if rms > 0 else np.zeros(m)
    x3 = np.log1p(np.asarray(age, dtype=np.float64))
    return np.stack([static[0], standardise(x1), static[1], standardise(x3)], axis=1)


def forward(theta, Z, bf16_mode: bool = False, cache: bool = False):
    """Scores s (n) of feature rows Z (n x 4); with cache, also the layer values."""
    W1, b1, W2, b2, w3, b3 = unpack(bf16(theta) if bf16_mode else theta)
    Z = np.asarray(Z, dtype=np.float64)
    a1 = Z @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    if bf16_mode:
        h1 = bf16(h1)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    if bf16_mode:
        h2 = bf16(h2)
    s = h2 @ w3 + b3
    if cache:
        return s, dict(a1=a1, h1=h1, a2=a2, h2=h2)
    return s


def loss_grad(theta, Z, y, bf16_mode: bool = False):
    """Mean loss (s - y)^2 / 2 over the rows and its gradient w.r.t. theta (the
    bfloat16 roundings, in BF16 mode, pass gradients straight through)."""
    W1, b1, W2, b2, w3, b3 = unpack(bf16(theta) if bf16_mode else theta)
    Z = np.asarray(Z, dtype=np.float64)
    n = Z.shape[0]
    s, c = forward(theta, Z, bf16_mode, cache=True)
    ds = (s - np.asarray(y, dtype=np.float64)) / n
    loss = 0.5 * np.mean((s - y) ** 2)
    g_w3 = c["h2"].T @ ds
    g_b3 = ds.sum()
    dh2 = np.outer(ds, w3) * (c["a2"] > 0)
    g_W2 = dh2.T @ c["h1"]
    g_b2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (c["a1"] > 0)
    g_W1 = dh1.T @ Z
    g_b1 = dh1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def adam_step(theta, grad, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; state = dict(m, v, t) (created when empty)."""
    if not state:
        state.update(m=np.zeros_like(theta), v=np.zeros_like(theta), t=0)
    state["t"] += 1
    t = state["t"]
    state["m"] = b1 * state["m"] + (1 - b1) * grad
    state["v"] = b2 * state["v"] + (1 - b2) * grad * grad
    mh = state["m"] / (1 - b1 ** t)
    vh = state["v"] / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps)


def label(a, e2: float, m: int):
    """Targets y_p = (1/2) ln(m max(a_p, 0) / e2 + 1e-3) of the drawn coordinates."""
    return 0.5 * np.log(m * np.maximum(np.asarray(a, dtype=np.float64), 0.0) / e2 + 1e-3)


def log_proposal(s, eps: float):
    """ln p_j with p = (1 - eps) softmax(s) + eps / m."""
    s = np.asarray(s, dtype=np.float64)
    m = s.shape[0]
    e = np.exp(s - s.max())
    return np.log((1.0 - eps) * e / e.sum() + eps / m)


def gumbel(seed: int, k: int, m: int):
    """g_j = -ln(-ln u_j), u_j = (hi32(draw(seed, k, 4, j)) + 1/2) / 2^32."""
    hi = (draw(seed, k, 4, np.arange(m, dtype=np.uint64)) >> np.uint64(32)).astype(np.float64)
    u = (hi + 0.5) / 4294967296.0
    return -np.log(-np.log(u))


def select(logp, seed: int, k: int, tau: int):
    """The tau coordinates with the largest ln p_j + g_j (ties: smaller index),
    in increasing index order; also the keys."""
    keys = np.asarray(logp, dtype=np.float64) + gumbel(seed, k, len(logp))
    order = np.lexsort((np.arange(len(keys)), -keys))
    return np.sort(order[:tau]), keys


def solve_learned(A, b, theta, tau: int, seed: int, tol: float, max_iters: int, eps: float = 0.1,
                  chunk: int = 50, bf16_mode: bool = True, w_star=None, collect: bool = False):
    """Sketch-and-project (Algorithm 2, no momentum) with subsample sketches drawn
    from the learned proposal, re-evaluated at the start of every chunk. theta =
    None draws uniformly (p_j = 1 / m: the same Gumbel keys, constant ln p).
    Returns dict(w, hist, iters, samples[, data]); with collect (needs w_star) the
    training pairs (chunk-start features of each drawn coordinate, target)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = b.shape[0]
    static = static_features(A)
    w = np.zeros(m)
    r = -b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    samples = []
    last = np.full(m, -1, dtype=np.int64)
    feats, targets = [], []
    k = 0
    while k < max_iters and np.linalg.norm(r) / r0 > tol:
        k0 = k
        age = k0 - last
        Z = features(static, r, age)
        logp = (log_proposal(forward(theta, Z, bf16_mode), eps) if theta is not None
                else np.full(m, -np.log(m)))
        for _ in range(chunk):
            if k >= max_iters or np.linalg.norm(r) / r0 <= tol:
                break
            C, _ = select(logp, seed, k, tau)
            rC = r[C]
            M = A[np.ix_(C, C)]
            delta = least_norm_solution(M, rC)
            if collect:
                e2 = float((w - w_star) @ r)
                a = rC * delta
                feats.append(Z[C])
                targets.append(label(a, e2, m))
            w = w.copy()
            w[C] -= delta
            r = r - A[:, C] @ delta
            last[C] = k
            samples.append(C)
            k += 1
            hist.append(np.linalg.norm(r) / r0)
    out = dict(w=w, hist=hist, iters=k, samples=samples)
    if collect:
        out["data"] = (np.concatenate(feats), np.concatenate(targets))
    return out
