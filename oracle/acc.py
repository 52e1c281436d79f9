"""FP64 CPU oracle of Anti+Acc (§5): Nesterov's accelerated projected
gradient applied to the anti-lopsided problem of Alg. 1.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library and imports nothing from it.

§5 lists Anti+Acc among the compared methods: the scaling steps of Alg. 1
(Q, q of Eq. NQPQ), then a Nesterov accelerated method, the one the paper
cites for its "Accer" baseline (the optimal gradient method of Guan et al.,
2012).  The paper gives no update rule; this module reads it as that method
for f(y) = ½yᵀQy + qᵀy over y ⪰ 0 with the constant step 1/L:

    x_k     = [Y_k − ∇f(Y_k)/L]₊
    α_{k+1} = (1 + √(4α_k² + 1)) / 2
    Y_{k+1} = x_k + ((α_k − 1)/α_{k+1}) (x_k − x_{k−1})

from Y_0 = x_{−1} = y⁰ (the start point, 0 by default) and α_0 = 1 (so the
first two steps carry no momentum: Y_0 = y⁰, Y_1 = x_0).  Because
f is quadratic, ∇f(Y_{k+1}) = (1 + β)∇f(x_k) − β∇f(x_{k−1}) with
β = (α_k − 1)/α_{k+1}; the oracle forms ∇f(Y) = QY + q directly.

Further readings (each also listed in the design notes):
  * L is the largest eigenvalue of Q, estimated by the power iteration of
    ``power_iteration`` (fixed start vector, Rayleigh quotient, stop when two
    successive quotients agree to 1e-7 relative, at most 500 products).  The
    quotient never exceeds λ_max(Q).  When it is 0 (Q = 0) the step is 1.
  * The stop rule is that of Alg. 2, tested at the start point and at every
    iterate x_k: P(x) and ḡ as in §3, stop when P = ∅ or ‖ḡ‖² < ε,
    ε = (tol·‖min(q, 0)‖)².  The iteration count is the number of steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import nnls as O

POWER_TOL = 1e-7
POWER_MAX = 500


def power_start(n):
    """Start vector of the power iteration: v_i = 1 + (i mod 5)/8, normalised."""
    v = 1.0 + (np.arange(n) % 5) / 8.0
    return v / np.linalg.norm(v)


def power_iteration(Q, tol=POWER_TOL, max_steps=POWER_MAX):
    """λ_max(Q) estimate: u = Qv, ρ = vᵀu (‖v‖ = 1), v ← u/‖u‖; stop when
    |ρ_t − ρ_{t−1}| ≤ tol·|ρ_t| or after max_steps products.  Returns
    (ρ, products)."""
    Q = np.asarray(Q, dtype=np.float64)
    v = power_start(Q.shape[0])
    rho_prev = None
    for t in range(1, max_steps + 1):
        u = Q @ v
        rho = float(v @ u)
        nu = float(np.linalg.norm(u))
        if rho_prev is not None and abs(rho - rho_prev) <= tol * abs(rho):
            return rho, t
        if nu == 0.0:
            return rho, t
        v = u / nu
        rho_prev = rho
    return rho, max_steps


def step_constant(rho):
    """L used for the step 1/L: the power-iteration quotient, or 1 when it is
    not positive (then Q = 0 on the orthant's reachable directions)."""
    return rho if rho > 0.0 else 1.0


def projected_step(Q, q, Y, L):
    """x = [Y − ∇f(Y)/L]₊ with ∇f(Y) = QY + q (the gradient step with step
    1/L, projected onto the orthant)."""
    return np.maximum(Y - (Q @ Y + q) / L, 0.0)


def momentum_next(alpha):
    """α_{k+1} = (1 + √(4α_k² + 1)) / 2."""
    return (1.0 + np.sqrt(4.0 * alpha * alpha + 1.0)) / 2.0


def extrapolate(x, x_prev, alpha, alpha_next):
    """Y_{k+1} = x_k + ((α_k − 1)/α_{k+1}) (x_k − x_{k−1})."""
    return x + ((alpha - 1.0) / alpha_next) * (x - x_prev)


@dataclass
class AccResult:
    y: np.ndarray
    iters: int
    status: int
    gbar2: float
    alphas: list = field(default_factory=list)    # α_0, α_1, … (traced)
    history: list = field(default_factory=list)   # (k, ‖ḡ(x_k)‖², f(x_k)) (traced)


def solve_nqp_acc(Q, q, L, y0=None, eps=None, tol=None, max_iter=None, trace=False):
    """The accelerated projected gradient above on (Q, q) with step 1/L.

    The stop rule is tested at every x_k, the start point included (k = 0:
    x = y⁰); ``iters`` counts the steps taken.  ``alphas`` traces α_0, α_1, …
    and ``history`` (k, ‖ḡ(x_k)‖², f(x_k))."""
    Q = np.asarray(Q, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[0]
    if max_iter is None:
        max_iter = max(5 * n, 20000)
    if eps is None:
        if tol is None:
            raise ValueError("give eps (absolute on ‖ḡ‖²) or tol (relative KKT)")
        den = O.kkt_denominator(q)
        eps = (tol * den) ** 2 if den > 0 else tol ** 2
    x = np.zeros(n) if y0 is None else np.asarray(y0, dtype=np.float64).copy()
    x_prev = x.copy()                # x_{k−1}; at the start x_{−1} = y⁰
    a_prev, a_cur = 1.0, 1.0         # (α_{k−1}, α_k) of the next extrapolation
    alphas, hist = [1.0], []
    k = 0
    while True:
        g = Q @ x + q
        P = O.passive_mask(x, g)
        gb = np.where(P, g, 0.0)
        gb2 = float(gb @ gb)
        if trace:
            hist.append((k, gb2, O.objective(Q, q, x)))
        if not P.any():
            return AccResult(x, k, O.STATUS_EMPTY_PASSIVE, gb2, alphas, hist)
        if gb2 < eps or gb2 == 0.0:
            return AccResult(x, k, O.STATUS_CONVERGED, gb2, alphas, hist)
        if k >= max_iter:
            return AccResult(x, k, O.STATUS_MAXITER, gb2, alphas, hist)
        Y = extrapolate(x, x_prev, a_prev, a_cur)
        a_prev, a_cur = a_cur, momentum_next(a_cur)
        alphas.append(a_cur)
        x_prev, x = x, projected_step(Q, q, Y, L)
        k += 1


def anti_acc(A, b, tol=1e-10, max_iter=None, x0=None, trace=False):
    """Anti+Acc end to end for one right-hand side: Alg. 1's scaling, L by the
    power iteration, the accelerated method; returns (x, AccResult, s, L)."""
    H, h = O.nqp_from_nnls(A, b)
    Q, q, s = O.antilopsided_scaling(H, h)
    rho, _ = power_iteration(Q)
    L = step_constant(rho)
    y0 = None if x0 is None else O.scale_start(x0, s)
    res = solve_nqp_acc(Q, q, L, y0=y0, tol=tol, max_iter=max_iter, trace=trace)
    return O.unscale(res.y, s), res, s, L
