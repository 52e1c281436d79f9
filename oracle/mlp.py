"""FP64 CPU oracle of the learned warm start for Alg. 2 (§3).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library and imports nothing from it.

The paper starts Alg. 2 at x⁰ = 0 and maps a start point with y⁰ = x⁰·√H_ii
(Eq. Rescaling, Fig. 2).  A learned start point is not in the paper; this
module defines the one the library implements, in plain numpy float64:

  features   u = [ (q/‖q‖ − μ)/σ ; z ],  z_j = (log s_j − mean log s)/std log s
             (q is the scaled linear term of Eq. NQPQ for one right-hand side,
             s_j = √H_jj; μ_j, σ_j are the mean and standard deviation of
             q_j/‖q‖ over the training set (σ_j := 1 if 0); z depends on A
             only, std := 1 if it is 0; the q-part is q/‖q‖ = 0 when q = 0)
  network    h1 = relu(W1 u + b1),  h2 = relu(W2 h1 + b2),  o = W3 h2 + b3,
             o = [ ŷ ; ℓ ]  (ŷ and the logits ℓ have n entries each)
  start      direction d = relu(ŷ)·[ℓ > 0], then the exact line search of
             Alg. 2 along it from 0: y⁰ = α*·d, α* = max(0, −qᵀd / dᵀQd)
             (0 when dᵀQd = 0).  So f(y⁰) = ½y⁰ᵀQy⁰ + qᵀy⁰ ≤ f(0): the start is
             never worse than x⁰ = 0, and y⁰ = 0 when the direction does not
             descend.
  loss       L = mean (ŷ − y*/(τ‖q‖))² + mean BCE(ℓ, [y* > 0]), both means over
             the batch and the n outputs; BCE(ℓ, c) = log(1 + e^ℓ) − c·ℓ;
             τ = RMS of y*/‖q‖ over the training set (1 if 0)
  training   Adam (Kingma & Ba 2015) with bias correction.

Parameters are a dict {W1, b1, W2, b2, W3, b3}; W_l has shape (out, in).  The
normalisation statistics (μ, σ, τ) are a dict {mu, sd, tau}; None means
μ = 0, σ = 1, τ = 1.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def _unit(q):
    qn = np.linalg.norm(q, axis=1)
    qpart = np.zeros_like(q)
    nz = qn > 0
    qpart[nz] = q[nz] / qn[nz, None]
    return qpart, qn


def stats(q, Y):
    """μ, σ of q/‖q‖ per entry and τ = RMS of y*/‖q‖, over a training set."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    qpart, qn = _unit(q)
    sd = qpart.std(axis=0)
    sd[sd == 0] = 1.0
    T, _ = targets(Y, qn)
    tau = float(np.sqrt(np.mean(T ** 2)))
    return {"mu": qpart.mean(axis=0), "sd": sd, "tau": tau if tau > 0 else 1.0}


def features(q, s, st=None):
    """u = [(q/‖q‖ − μ)/σ ; z] for a batch of q (B, n) and scale factors s (n,)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    s = np.asarray(s, dtype=np.float64)
    qpart, qn = _unit(q)
    if st is not None:
        qpart = (qpart - st["mu"]) / st["sd"]
    ls = np.log(s)
    sd = ls.std()
    z = (ls - ls.mean()) / (sd if sd > 0 else 1.0)
    return np.hstack([qpart, np.broadcast_to(z, q.shape)]), qn


def init_params(n_in, hidden, n_out, seed=0):
    """He-uniform weights, zero biases (any start is valid for the oracle)."""
    r = np.random.default_rng(seed)
    p = {}
    dims = [(hidden, n_in), (hidden, hidden), (n_out, hidden)]
    for l, (o, i) in enumerate(dims, 1):
        lim = np.sqrt(6.0 / i)
        p[f"W{l}"] = r.uniform(-lim, lim, (o, i))
        p[f"b{l}"] = np.zeros(o)
    return p


def forward(p, U):
    """The network on a batch U (B, 2n); returns the output and the cache."""
    Z1 = U @ p["W1"].T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    O = H2 @ p["W3"].T + p["b3"]
    return O, (U, Z1, H1, Z2, H2)


def bce(logit, c):
    """log(1 + e^ℓ) − c·ℓ, evaluated without overflow."""
    return np.maximum(logit, 0.0) - logit * c + np.log1p(np.exp(-np.abs(logit)))


def loss(p, U, T, C):
    """L for targets T = y*/‖q‖ and classes C = [y* > 0], both (B, n)."""
    O, _ = forward(p, U)
    n = T.shape[1]
    yh, lg = O[:, :n], O[:, n:]
    return float(np.mean((yh - T) ** 2) + np.mean(bce(lg, C)))


def loss_and_grad(p, U, T, C):
    """L and its gradient with respect to every parameter (backpropagation)."""
    O, (U, Z1, H1, Z2, H2) = forward(p, U)
    B, n = T.shape
    yh, lg = O[:, :n], O[:, n:]
    L = float(np.mean((yh - T) ** 2) + np.mean(bce(lg, C)))
    m = B * n
    dO = np.hstack([2.0 * (yh - T) / m, (1.0 / (1.0 + np.exp(-lg)) - C) / m])
    g = {"W3": dO.T @ H2, "b3": dO.sum(axis=0)}
    dH2 = dO @ p["W3"]
    dZ2 = dH2 * (Z2 > 0)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ p["W2"]
    dZ1 = dH1 * (Z1 > 0)
    g["W1"] = dZ1.T @ U
    g["b1"] = dZ1.sum(axis=0)
    return L, g


def adam_init(p):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()},
            "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p, g, st, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place: m, v moving averages, bias-corrected."""
    st["t"] += 1
    t = st["t"]
    for k in p:
        st["m"][k] = beta1 * st["m"][k] + (1 - beta1) * g[k]
        st["v"][k] = beta2 * st["v"][k] + (1 - beta2) * g[k] ** 2
        mh = st["m"][k] / (1 - beta1 ** t)
        vh = st["v"][k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def targets(Y, qn, tau=1.0):
    """T = y*/(τ‖q‖) (0 where q = 0) and C = [y* > 0]."""
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    T = np.zeros_like(Y)
    nz = qn > 0
    T[nz] = Y[nz] / (tau * qn[nz, None])
    return T, (Y > 0).astype(np.float64)


def predict(p, q, s, Q, st=None):
    """Start points y⁰ (B, n) in the scaled space: the predicted direction
    scaled by the exact line search from 0 (α* ≥ 0)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    U, _ = features(q, s, st)
    O, _ = forward(p, U)
    n = q.shape[1]
    d = np.maximum(O[:, :n], 0.0) * (O[:, n:] > 0)
    num = -np.einsum("bi,bi->b", q, d)
    den = np.einsum("bi,ij,bj->b", d, Q, d)
    alpha = np.zeros(len(q))
    ok = (num > 0) & (den > 0)
    alpha[ok] = num[ok] / den[ok]
    return alpha[:, None] * d


def train(p, Qs, Ys, s, epochs=1, batch=256, lr=1e-3, seed=0, st=None):
    """Minibatch Adam over (q, y*) pairs; returns the mean loss of each epoch.
    ``st`` (normalisation statistics) defaults to stats(Qs, Ys)."""
    if st is None:
        st = stats(Qs, Ys)
    U, qn = features(Qs, s, st)
    T, C = targets(Ys, qn, st["tau"])
    ad = adam_init(p)
    r = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        perm = r.permutation(len(U))
        tot, cnt = 0.0, 0
        for i in range(0, len(U), batch):
            idx = perm[i:i + batch]
            L, g = loss_and_grad(p, U[idx], T[idx], C[idx])
            adam_step(p, g, ad, lr=lr)
            tot += L * len(idx)
            cnt += len(idx)
        hist.append(tot / cnt)
    return hist
