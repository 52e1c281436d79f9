"""FP64 CPU oracle of the learned warm start for Alg. 2 (§3).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library and imports nothing from it.

The paper starts Alg. 2 at x⁰ = 0 and maps a start point with y⁰ = x⁰·√H_ii
(Eq. Rescaling, Fig. 2).  A learned start point is not in the paper; this
module defines the one the library implements, in plain numpy float64.  For a
fixed A (so a fixed scaled matrix Q of Eq. NQPQ) and a right-hand side with
scaled linear term q:

  direction  z = −Q⁻¹q, the unconstrained minimiser of ½yᵀQy + qᵀy (Q is
             positive definite when A has full column rank)
  features   u = [ (q/‖q‖ − μ)/σ ; (z/‖q‖ − μz)/σz ]  (μ, σ, μz, σz per entry
             over the training set, σ := 1 where 0; both parts are 0 when
             q = 0)
  network    h1 = relu(W1 u + b1),  h2 = relu(W2 h1 + b2),  o = W3 h2 + b3,
             o = [ r ; ℓ′ ]  (n entries each), and per-entry skips from the
             direction in the target's scale, ẑ = z/(τ‖q‖):
             ŷ = r + e ⊙ ẑ,   ℓ = ℓ′ + f ⊙ ẑ
  start      d = relu(ŷ)·[ℓ > 0], then the exact line search of Alg. 2 along
             it from 0: y⁰ = α*·d, α* = max(0, −qᵀd / dᵀQd) (0 when
             dᵀQd = 0), so f(y⁰) ≤ f(0) and y⁰ = 0 when d does not descend
  loss       L = mean (ŷ − y*/(τ‖q‖))² + mean BCE(ℓ, [y* > 0]), means over the
             batch and the n outputs; BCE(ℓ, c) = log(1 + e^ℓ) − c·ℓ;
             τ = RMS of y*/‖q‖ over the training set (1 if 0)
  training   Adam (Kingma & Ba 2015) with bias correction, every parameter
             (W1, b1, W2, b2, W3, b3, e, f).

The inverse Q⁻¹ is computed once per A (``numpy.linalg.inv`` here); it is a
feature transform, not a parameter.  Parameters are a dict {W1, b1, W2, b2, W3,
b3, e, f}; W_l has shape (out, in).  The normalisation statistics are a dict
{mu, sd, muz, sdz, tau}; None means μ = μz = 0, σ = σz = 1, τ = 1.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "e", "f")
SKIP_INIT = (1.0, 4.0)  # e, f at initialisation: ŷ follows ẑ, ℓ its sign


def _unit(q):
    qn = np.linalg.norm(q, axis=1)
    inv = np.zeros_like(qn)
    nz = qn > 0
    inv[nz] = 1.0 / qn[nz]
    return qn, inv


def direction(q, Qinv):
    """z = −Q⁻¹q for a batch of q (B, n)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    return -(q @ np.asarray(Qinv, dtype=np.float64).T)


def stats(q, Y, Qinv):
    """μ, σ of q/‖q‖, μz, σz of z/‖q‖ per entry and τ = RMS of y*/‖q‖ over a
    training set."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    qn, inv = _unit(q)
    qp = q * inv[:, None]
    zp = direction(q, Qinv) * inv[:, None]
    sd = qp.std(axis=0)
    sd[sd == 0] = 1.0
    sdz = zp.std(axis=0)
    sdz[sdz == 0] = 1.0
    T, _ = targets(Y, qn)
    tau = float(np.sqrt(np.mean(T ** 2)))
    return {"mu": qp.mean(axis=0), "sd": sd, "muz": zp.mean(axis=0), "sdz": sdz,
            "tau": tau if tau > 0 else 1.0}


def features(q, Qinv, st=None):
    """(u, ‖q‖, ẑ) for a batch of q (B, n): u = [(q/‖q‖ − μ)/σ ; (z/‖q‖ − μz)/σz]
    and the skip input ẑ = z/(τ‖q‖) (0 where q = 0)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    qn, inv = _unit(q)
    qp = q * inv[:, None]
    zp = direction(q, Qinv) * inv[:, None]
    tau = 1.0
    if st is not None:
        qp = (qp - st["mu"]) / st["sd"]
        zp_n = (zp - st["muz"]) / st["sdz"]
        tau = st["tau"]
    else:
        zp_n = zp
    qp[qn == 0] = 0.0
    zp_n[qn == 0] = 0.0
    return np.hstack([qp, zp_n]), qn, zp / tau


def init_params(n_in, hidden, n_out, seed=0):
    """He-uniform weights, zero biases, skips at SKIP_INIT (any start is valid
    for the oracle)."""
    r = np.random.default_rng(seed)
    p = {}
    dims = [(hidden, n_in), (hidden, hidden), (n_out, hidden)]
    for l, (o, i) in enumerate(dims, 1):
        lim = np.sqrt(6.0 / i)
        p[f"W{l}"] = r.uniform(-lim, lim, (o, i))
        p[f"b{l}"] = np.zeros(o)
    n = n_out // 2
    p["e"] = np.full(n, SKIP_INIT[0])
    p["f"] = np.full(n, SKIP_INIT[1])
    return p


def forward(p, U, zt):
    """The network on a batch U (B, 2n) with skip input zt (B, n); returns
    o = [ŷ ; ℓ] (skips included) and the cache."""
    Z1 = U @ p["W1"].T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    O = H2 @ p["W3"].T + p["b3"]
    n = O.shape[1] // 2
    O = np.hstack([O[:, :n] + p["e"] * zt, O[:, n:] + p["f"] * zt])
    return O, (U, Z1, H1, Z2, H2)


def bce(logit, c):
    """log(1 + e^ℓ) − c·ℓ, evaluated without overflow."""
    return np.maximum(logit, 0.0) - logit * c + np.log1p(np.exp(-np.abs(logit)))


def loss(p, U, zt, T, C):
    """L for targets T = y*/(τ‖q‖) and classes C = [y* > 0], both (B, n)."""
    O, _ = forward(p, U, zt)
    n = T.shape[1]
    yh, lg = O[:, :n], O[:, n:]
    return float(np.mean((yh - T) ** 2) + np.mean(bce(lg, C)))


def loss_and_grad(p, U, zt, T, C):
    """L and its gradient with respect to every parameter (backpropagation)."""
    O, (U, Z1, H1, Z2, H2) = forward(p, U, zt)
    B, n = T.shape
    yh, lg = O[:, :n], O[:, n:]
    L = float(np.mean((yh - T) ** 2) + np.mean(bce(lg, C)))
    m = B * n
    dy = 2.0 * (yh - T) / m
    dl = (1.0 / (1.0 + np.exp(-lg)) - C) / m
    dO = np.hstack([dy, dl])
    g = {"W3": dO.T @ H2, "b3": dO.sum(axis=0),
         "e": (dy * zt).sum(axis=0), "f": (dl * zt).sum(axis=0)}
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


def predict(p, q, Qinv, Q, st=None):
    """Start points y⁰ (B, n) in the scaled space: the predicted direction
    scaled by the exact line search from 0 (α* ≥ 0)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    U, _, zt = features(q, Qinv, st)
    O, _ = forward(p, U, zt)
    n = q.shape[1]
    d = np.maximum(O[:, :n], 0.0) * (O[:, n:] > 0)
    num = -np.einsum("bi,bi->b", q, d)
    den = np.einsum("bi,ij,bj->b", d, Q, d)
    alpha = np.zeros(len(q))
    ok = (num > 0) & (den > 0)
    alpha[ok] = num[ok] / den[ok]
    return alpha[:, None] * d


def train(p, Qs, Ys, Qinv, epochs=1, batch=256, lr=1e-3, seed=0, st=None):
    """Minibatch Adam over (q, y*) pairs; returns the mean loss of each epoch.
    ``st`` (normalisation statistics) defaults to stats(Qs, Ys, Qinv)."""
    if st is None:
        st = stats(Qs, Ys, Qinv)
    U, qn, zt = features(Qs, Qinv, st)
    T, C = targets(Ys, qn, st["tau"])
    ad = adam_init(p)
    r = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        perm = r.permutation(len(U))
        tot, cnt = 0.0, 0
        for i in range(0, len(U), batch):
            idx = perm[i:i + batch]
            L, g = loss_and_grad(p, U[idx], zt[idx], T[idx], C[idx])
            adam_step(p, g, ad, lr=lr)
            tot += L * len(idx)
            cnt += len(idx)
        hist.append(tot / cnt)
    return hist
