"""FP64 CPU oracle for the anti-lopsided NNLS method (arXiv 1502.01645).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library and imports nothing from it.

Everything is plain numpy in float64.  Library primitives (matrix product,
``numpy.linalg.solve``) serve as single steps; there is no blocking, fusion or
reordering beyond what the paper states.

Notation follows the paper:
  * Def. 1 / Eq. NNL (§2.1):  min ½‖Ax−b‖²  s.t. x ⪰ 0,  A ∈ R^{d×n}.
  * Eq. NQP (§2.1):           f(x) = ½xᵀHx + hᵀx,  H = AᵀA,  h = −Aᵀb.
  * Alg. 1 (§3):              Q = H / sqrt(diag H diag Hᵀ),  q = h / sqrt(diag H),
                              y = solveNQP(Q, q),  x = y / sqrt(diag H).
  * Eq. Rescaling (§3):       x_i = y_i / sqrt(H_ii); when H_ii = 0, x_i = y_i.
  * Eq. NQPQ (§3):            Q_ij = H_ij / sqrt(H_ii H_jj),  q_i = h_i / sqrt(H_ii).
  * §3, passive set:          P(x) = {i : x_i > 0 or ∇f_i(x) < 0}.
  * Alg. 2 (§3):              x⁰ = 0, ∇f = q; repeat: ḡ = ∇f masked to P;
                              α = ‖ḡ‖² / (ḡᵀQḡ);  x ← [x − αḡ]₊;
                              ∇f ← ∇f + Q(x_{k+1} − x_k); until P = ∅ or ‖ḡ‖² < ε.

Readings where the paper is silent or inconsistent (each also listed in the
design notes):
  * Update sign: the algorithm box of Alg. 2 steps along −ḡ (descent); the prose
    of §3 and §4.1 writes +α∇f̄, which would ascend.  The box is followed.
  * Zero column (H_ii = 0): the scale is taken as 1, so row/column i of Q and
    q_i are 0 and Q_ii = 0; x_i = y_i as Eq. Rescaling says.
  * Ties in the passive test are strict: y_i = 0 and g_i = 0 is not passive.
  * κ = ḡᵀQḡ ≤ 0 with ḡ ≠ 0 cannot happen in exact arithmetic (q lies in the
    range of Q); numerically it ends the loop as "converged".
  * The stopping threshold ε is not given; callers pass either an absolute ε on
    ‖ḡ‖² (the paper's form) or a relative KKT tolerance
    rel = ‖ḡ‖ / ‖min(q, 0)‖ (our reading of the metric).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STATUS_CONVERGED = 0
STATUS_EMPTY_PASSIVE = 1
STATUS_CURVATURE = 2
STATUS_MAXITER = 3


# --------------------------------------------------------------------------
# Eq. NQP and Alg. 1 (transform)
# --------------------------------------------------------------------------
def nqp_from_nnls(A, b):
    """Eq. NQP (§2.1): H = AᵀA, h = −Aᵀb, both in float64.

    ``b`` may be a vector (d,) or a stack of right-hand sides (k, d); h has the
    matching shape (n,) or (k, n)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    H = A.T @ A
    h = -(b @ A)
    return H, h


def antilopsided_scaling(H, h):
    """Alg. 1 (§3) lines forming Q and q; Eq. Rescaling / Eq. NQPQ.

    Returns (Q, q, s) with s_i = sqrt(H_ii) (1 where H_ii = 0, the paper's
    special case), Q_ij = H_ij / (s_i s_j) and q_i = h_i / s_i."""
    H = np.asarray(H, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    diag = np.diag(H).copy()
    s = np.sqrt(diag)
    s[diag == 0.0] = 1.0
    Q = H / np.outer(s, s)
    q = h / s
    return Q, q, s


def unscale(y, s):
    """Alg. 1 final step and Eq. Rescaling: x = y / sqrt(diag H)."""
    return np.asarray(y, dtype=np.float64) / s


def scale_start(x0, s):
    """Map a start point x0 of Eq. NQP to y0 of Eq. NQPQ: y0 = x0 · sqrt(diag H).

    (§3 writes y0_i = x0_i · H_ii once and x0 .* sqrt(diag H) in the caption of
    Fig. 2; Eq. Rescaling fixes the square root.)"""
    return np.asarray(x0, dtype=np.float64) * s


# --------------------------------------------------------------------------
# §3 passive set and Alg. 2
# --------------------------------------------------------------------------
def passive_mask(y, g):
    """§3: P(y) = {i : y_i > 0 or ∇f_i(y) < 0}, strict comparisons."""
    return (y > 0.0) | (g < 0.0)


def projected_gradient(y, g):
    """§3: ∇f̄_i = ∇f_i for i ∈ P(y), otherwise 0."""
    return np.where(passive_mask(y, g), g, 0.0)


def objective(Q, q, y):
    """Eq. NQPQ objective f(y) = ½ yᵀQy + qᵀy."""
    return 0.5 * y @ (Q @ y) + q @ y


def kkt_denominator(q):
    """‖ḡ(0)‖ = ‖min(q, 0)‖: the projected gradient at the start point 0."""
    return float(np.linalg.norm(np.minimum(q, 0.0)))


@dataclass
class SolveResult:
    y: np.ndarray
    iters: int
    status: int
    gbar2: float                       # ‖ḡ‖² at the returned iterate
    history: list = field(default_factory=list)   # (k, ‖ḡ‖², f) per iteration if traced


def solve_nqp(Q, q, y0=None, eps=None, tol=None, max_iter=None, trace=False):
    """Alg. 2 (§3): gradient method with exact line search for the NQP.

    Steps, in the paper's order, per iteration:
      ḡ = ∇f masked to P(y)                         (passive set, §3)
      stop if P = ∅ or ‖ḡ‖² < ε                      (Alg. 2 loop test)
      α = ‖ḡ‖² / (ḡᵀQḡ)                              (exact line search, §3)
      y_{k+1} = [y_k − αḡ]₊                          (projection)
      ∇f ← ∇f + Q(y_{k+1} − y_k)                     (gradient update)

    ``eps`` is the paper's absolute threshold on ‖ḡ‖².  ``tol`` instead sets
    ε = (tol · ‖min(q,0)‖)², i.e. a relative KKT residual.  With a start point
    y0 the initial gradient is Q y0 + q (Alg. 2 starts at 0 with ∇f = q).
    """
    Q = np.asarray(Q, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[0]
    if max_iter is None:
        max_iter = max(5 * n, 20000)          # §5: k = 5n, 2·10^4 in the experiments
    if eps is None:
        if tol is None:
            raise ValueError("give eps (absolute on ‖ḡ‖²) or tol (relative KKT)")
        den = kkt_denominator(q)
        eps = (tol * den) ** 2 if den > 0 else tol ** 2
    if y0 is None:
        y = np.zeros(n)
        g = q.copy()
    else:
        y = np.asarray(y0, dtype=np.float64).copy()
        g = Q @ y + q
    hist = []
    k = 0
    while True:
        P = passive_mask(y, g)
        gbar = np.where(P, g, 0.0)
        gbar2 = float(gbar @ gbar)
        if trace:
            hist.append((k, gbar2, objective(Q, q, y)))
        if not P.any():
            return SolveResult(y, k, STATUS_EMPTY_PASSIVE, gbar2, hist)
        if gbar2 < eps or gbar2 == 0.0:
            return SolveResult(y, k, STATUS_CONVERGED, gbar2, hist)
        if k >= max_iter:
            return SolveResult(y, k, STATUS_MAXITER, gbar2, hist)
        alpha = exact_line_search(Q, gbar, gbar2)
        if alpha is None:
            return SolveResult(y, k, STATUS_CURVATURE, gbar2, hist)
        y_next = projected_update(y, gbar, alpha)
        g = gradient_update(Q, g, y_next, y)
        y = y_next
        k += 1


def exact_line_search(Q, gbar, gbar2):
    """Alg. 2 step size and its derivation in §3: α = ‖ḡ‖² / (ḡᵀQḡ), the
    minimiser of f(y − αḡ) along the projected gradient.  Returns None when the
    curvature ḡᵀQḡ is not positive."""
    curv = float(gbar @ (Q @ gbar))
    if curv <= 0.0:
        return None
    return gbar2 / curv


def projected_update(y, gbar, alpha):
    """Alg. 2: y_{k+1} = [y_k − αḡ]₊ (projection onto the non-negative orthant)."""
    return np.maximum(y - alpha * gbar, 0.0)


def gradient_update(Q, g, y_next, y):
    """Alg. 2: ∇f ← ∇f + Q(y_{k+1} − y_k), exact for the quadratic f."""
    return g + Q @ (y_next - y)


def antilop(A, b, tol=1e-10, max_iter=None, x0=None, trace=False):
    """Alg. 1 (§3) end to end for one right-hand side: returns (x, SolveResult, s)."""
    H, h = nqp_from_nnls(A, b)
    Q, q, s = antilopsided_scaling(H, h)
    y0 = None if x0 is None else scale_start(x0, s)
    res = solve_nqp(Q, q, y0=y0, tol=tol, max_iter=max_iter, trace=trace)
    return unscale(res.y, s), res, s


# --------------------------------------------------------------------------
# FP64 KKT / objective straight from A (defines the reported residual)
# --------------------------------------------------------------------------
def nnls_objective(A, b, x):
    """F(x) = ½‖Ax − b‖² (Def. 1)."""
    r = np.asarray(A, np.float64) @ np.asarray(x, np.float64) - np.asarray(b, np.float64)
    return 0.5 * float(r @ r)


def kkt_residual(A, b, x):
    """Relative KKT residual of x for Def. 1, evaluated from A in float64.

    ∇F = Aᵀ(Ax − b); in scaled variables g = ∇F / s and y = s·x, so g = Qy + q
    (Eq. NQPQ).  ḡ is g masked to P(y) (§3), and the residual is
    ‖ḡ‖ / ‖min(q, 0)‖ with q = −Aᵀb / s (the projected gradient at y = 0).  When
    that denominator is 0 the optimum is x = 0 and the absolute ‖ḡ‖ is returned.
    Returns (rel_kkt, F(x))."""
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    x = np.asarray(x, np.float64)
    col2 = np.einsum("ij,ij->j", A, A)
    s = np.sqrt(col2)
    s[col2 == 0.0] = 1.0
    r = A @ x - b
    g = (A.T @ r) / s
    y = x * s
    gbar = np.where(passive_mask(y, g), g, 0.0)
    q = -(A.T @ b) / s
    den = kkt_denominator(q)
    num = float(np.linalg.norm(gbar))
    return (num / den if den > 0 else num), 0.5 * float(r @ r)


# --------------------------------------------------------------------------
# Reference optimum for parity: exact solve on the identified passive set
# --------------------------------------------------------------------------
def polish(Q, q, y):
    """Exact solve on P = {i : y_i > 0}: Q_PP y_P = −q_P (numpy.linalg.solve).

    Accepted only if the result is a KKT point: y_P > 0 and g_i ≥ 0 off P, where
    g = Qy + q.  Returns the polished y, or None when the test fails."""
    P = np.flatnonzero(y > 0.0)
    yp = np.zeros_like(y)
    if P.size:
        try:
            yp[P] = np.linalg.solve(Q[np.ix_(P, P)], -q[P])
        except np.linalg.LinAlgError:
            return None
        if np.any(yp[P] <= 0.0):
            return None
    g = Q @ yp + q
    off = np.ones(y.shape[0], bool)
    off[P] = False
    scale = max(1.0, float(np.max(np.abs(q))))
    if np.any(g[off] < -1e-12 * scale):
        return None
    return yp


def reference_solution(A, b, tol=1e-12, max_iter=None):
    """The oracle's x* for parity: Alg. 2 to ``tol``, then the passive-set
    polish; if the polish is rejected, Alg. 2 continues to tol 1e-14 and the
    polish is tried once more.  Returns (x*, y*, s, info dict)."""
    H, h = nqp_from_nnls(A, b)
    Q, q, s = antilopsided_scaling(H, h)
    res = solve_nqp(Q, q, tol=tol, max_iter=max_iter)
    yp = polish(Q, q, res.y)
    iters = res.iters
    if yp is None:
        res2 = solve_nqp(Q, q, y0=res.y, tol=1e-14, max_iter=max_iter)
        iters += res2.iters
        yp = polish(Q, q, res2.y)
        if yp is None:
            yp = res2.y
    return unscale(yp, s), yp, s, {"iters": iters, "status": res.status}


# --------------------------------------------------------------------------
# Brute force for tiny n: enumerate every support set
# --------------------------------------------------------------------------
def brute_force_nnls(A, b):
    """Exhaustive NNLS for n ≤ 12: for every support S, solve the normal
    equations A_Sᵀ A_S x_S = A_Sᵀ b and keep feasible KKT points; return the one
    with the smallest objective.  Independent of Alg. 2."""
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    n = A.shape[1]
    if n > 12:
        raise ValueError("brute force is for n ≤ 12")
    best, best_f = np.zeros(n), nnls_objective(A, b, np.zeros(n))
    for mask in range(1, 1 << n):
        S = [i for i in range(n) if mask >> i & 1]
        AS = A[:, S]
        try:
            xs = np.linalg.solve(AS.T @ AS, AS.T @ b)
        except np.linalg.LinAlgError:
            continue
        if np.any(xs <= 0.0):
            continue
        x = np.zeros(n)
        x[S] = xs
        f = nnls_objective(A, b, x)
        if f < best_f:
            best, best_f = x, f
    return best, best_f


# --------------------------------------------------------------------------
# Lemma (§4.1) quantities, used as test invariants
# --------------------------------------------------------------------------
def q_norm_paper(Q):
    """‖Q‖₂ as the Lemma of §4.1 defines it: sqrt(Σ_ij Q_ij²) (Frobenius)."""
    return float(np.sqrt(np.sum(np.asarray(Q, np.float64) ** 2)))
