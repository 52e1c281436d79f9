"""Pins for the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, a
brute-force enumeration, an invariant of Eq. NQPQ / the Lemma of §4.1, a value
printed in the paper, or an independent library routine.  A planted mistake in
the oracle (wrong update sign, dropped scale, wrong passive test) must fail at
least one of them; ``test_planted_mistakes_are_caught`` checks that.
"""
import json
import os

import numpy as np
import pytest

from oracle import nnls as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- worked example
def test_worked_example_scaling_and_iterations():
    """§3, Eq. scaling: H=[[1,.1],[.1,9]], h=[-4,-5], x0=[30,2].  The paper
    reports 3 iterations after the rescaling and more without it."""
    g = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    H = np.array(g["H"])
    h = np.array(g["h"])
    x0 = np.array(g["x0"])
    Q, q, s = O.antilopsided_scaling(H, h)
    # Eq. NQPQ by hand: s = [1, 3]; Q_12 = 0.1/3; q = [-4, -5/3].
    np.testing.assert_allclose(s, [1.0, 3.0], rtol=0, atol=0)
    np.testing.assert_allclose(Q, [[1.0, 0.1 / 3.0], [0.1 / 3.0, 1.0]], rtol=1e-15)
    np.testing.assert_allclose(q, [-4.0, -5.0 / 3.0], rtol=1e-15)

    scaled = O.solve_nqp(Q, q, y0=O.scale_start(x0, s), eps=1e-6)
    unscaled = O.solve_nqp(H, h, y0=x0, eps=1e-6)
    assert scaled.iters == g["paper_iterations_scaled"]
    assert scaled.iters < unscaled.iters
    x_closed = np.array([35.5 / 8.99, 4.6 / 8.99])
    np.testing.assert_allclose(x_closed, g["closed_form_minimiser"]["value"], rtol=1e-15)
    np.testing.assert_allclose(O.unscale(scaled.y, s), x_closed, atol=1e-3)
    # Run to a tight threshold: the iterate reaches the closed form.
    tight = O.solve_nqp(Q, q, y0=O.scale_start(x0, s), eps=1e-26)
    np.testing.assert_allclose(O.unscale(tight.y, s), x_closed, rtol=1e-11)


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("seed", range(8))
def test_matches_brute_force_enumeration(seed):
    """For n ≤ 10 the unique NNLS optimum is found by enumerating supports."""
    r = _rng(seed)
    n = int(r.integers(2, 11))
    d = n + int(r.integers(2, 8))
    A = r.standard_normal((d, n)) if seed % 2 else r.random((d, n))
    b = r.standard_normal(d) * 3.0
    x_bf, f_bf = O.brute_force_nnls(A, b)
    x_or, _, _, _ = O.reference_solution(A, b)
    np.testing.assert_allclose(x_or, x_bf, atol=1e-9 * max(1.0, np.abs(x_bf).max()))
    assert abs(O.nnls_objective(A, b, x_or) - f_bf) <= 1e-10 * max(1.0, f_bf)


# --------------------------------------------------- special cases with closed forms
def test_positive_unconstrained_solution_is_recovered():
    """§2.2: when the unconstrained LS solution is positive it is the NNLS optimum."""
    r = _rng(11)
    A = r.random((60, 12))
    x_true = r.uniform(0.5, 1.5, 12)
    b = A @ x_true
    x, res, _ = O.antilop(A, b, tol=1e-14)
    np.testing.assert_allclose(x, x_true, rtol=1e-8)
    x_ref, _, _, _ = O.reference_solution(A, b)
    np.testing.assert_allclose(x_ref, x_true, rtol=1e-11)


def test_zero_solution_when_Atb_nonpositive():
    """Alg. 2 stop rule P(x) = ∅: with A ≥ 0 and b ≤ 0, Aᵀb ≤ 0 so q ≥ 0 and
    P(0) is empty at once; x = 0 is optimal."""
    r = _rng(12)
    A = r.random((30, 8))
    b = -r.random(30)
    x, res, _ = O.antilop(A, b, tol=1e-12)
    assert res.iters == 0
    assert res.status == O.STATUS_EMPTY_PASSIVE
    assert np.all(x == 0.0)


def test_zero_column_reading():
    """Eq. Rescaling special case H_ii = 0: s_i = 1, row/column i of Q and q_i
    vanish, x_i = 0, and the remaining entries solve the reduced problem."""
    r = _rng(13)
    A = r.random((40, 7))
    A[:, 3] = 0.0
    b = A @ r.random(7) + 0.01 * r.standard_normal(40)
    H, h = O.nqp_from_nnls(A, b)
    Q, q, s = O.antilopsided_scaling(H, h)
    assert s[3] == 1.0 and q[3] == 0.0
    assert np.all(Q[3, :] == 0.0) and np.all(Q[:, 3] == 0.0)
    x, _, _, _ = O.reference_solution(A, b)
    keep = [0, 1, 2, 4, 5, 6]
    x_red, _ = O.brute_force_nnls(A[:, keep], b)
    assert x[3] == 0.0
    np.testing.assert_allclose(x[keep], x_red, atol=1e-10)


# ----------------------------------------------------------- Eq. NQPQ invariants
@pytest.mark.parametrize("seed", [21, 22, 23])
def test_scaled_matrix_invariants(seed):
    """Remark (§3): Q_ii = 1, Q_ij = cos(A_i, A_j); Lemma (§4.1):
    √n ≤ ‖Q‖ ≤ n with ‖Q‖ the Frobenius norm, and Q ⪯ ‖Q‖ I."""
    r = _rng(seed)
    d, n = 80, 30
    A = r.standard_normal((d, n)) * np.exp(r.uniform(-4, 4, n))[None, :]
    b = r.standard_normal(d)
    H, h = O.nqp_from_nnls(A, b)
    Q, q, s = O.antilopsided_scaling(H, h)
    np.testing.assert_allclose(np.diag(Q), 1.0, rtol=1e-14)
    np.testing.assert_array_equal(Q, Q.T)
    assert np.all(np.abs(Q) <= 1.0 + 1e-14)
    # cos(A_i, A_j) computed from the columns directly.
    i, j = 4, 17
    cos = A[:, i] @ A[:, j] / (np.linalg.norm(A[:, i]) * np.linalg.norm(A[:, j]))
    np.testing.assert_allclose(Q[i, j], cos, rtol=1e-12)
    ev = np.linalg.eigvalsh(Q)
    assert ev[0] >= -1e-12                       # PSD
    fro = O.q_norm_paper(Q)
    assert np.sqrt(n) - 1e-12 <= fro <= n + 1e-12
    assert ev[-1] <= fro + 1e-12
    # q_i = h_i / s_i with h = -Aᵀb (Eq. NQP)
    np.testing.assert_allclose(q, -(A.T @ b) / np.linalg.norm(A, axis=0), rtol=1e-12)


def test_column_rescaling_invariance():
    """The point of the transform (§3): positive column scaling of A leaves Q, q,
    y* and the whole Alg. 2 trajectory unchanged, and x* scales inversely."""
    r = _rng(31)
    d, n = 50, 15
    A = r.random((d, n))
    b = A @ np.where(r.random(n) < 0.5, 0.0, r.random(n)) + 0.01 * r.standard_normal(d)
    c = np.exp(r.uniform(np.log(1e-3), np.log(1e3), n))
    Q1, q1, _ = O.antilopsided_scaling(*O.nqp_from_nnls(A, b))
    Q2, q2, _ = O.antilopsided_scaling(*O.nqp_from_nnls(A * c[None, :], b))
    np.testing.assert_allclose(Q2, Q1, atol=1e-13)
    np.testing.assert_allclose(q2, q1, atol=1e-12 * np.abs(q1).max())
    r1 = O.solve_nqp(Q1, q1, tol=1e-8)
    r2 = O.solve_nqp(Q2, q2, tol=1e-8)
    assert abs(r1.iters - r2.iters) <= 2
    x1, _, _, _ = O.reference_solution(A, b)
    x2, _, _, _ = O.reference_solution(A * c[None, :], b)
    np.testing.assert_allclose(x2 * c, x1, atol=1e-9 * np.abs(x1).max())


# -------------------------------------------------------------- KKT at the optimum
def test_kkt_conditions_at_reference_solution():
    """Optimality for Def. 1: x ≥ 0, ∇F ≥ 0, xᵀ∇F = 0 (equivalently ḡ = 0, §3)."""
    r = _rng(41)
    A = r.random((200, 60))
    x_true = np.where(r.random(60) < 0.5, 0.0, r.random(60))
    b = A @ x_true + 0.01 * r.standard_normal(200)
    x, _, _, _ = O.reference_solution(A, b)
    grad = A.T @ (A @ x - b)
    scale = np.abs(A.T @ b).max()
    assert np.all(x >= 0)
    assert np.all(grad >= -1e-10 * scale)
    assert abs(x @ grad) <= 1e-10 * scale * np.abs(x).max()
    rel, F = O.kkt_residual(A, b, x)
    assert rel <= 1e-12
    np.testing.assert_allclose(F, 0.5 * np.sum((A @ x - b) ** 2), rtol=1e-14)


def test_kkt_residual_definition_at_zero():
    """At x = 0 the relative residual is exactly 1: ḡ(0) = min(q, 0)."""
    r = _rng(42)
    A = r.random((30, 10))
    b = A @ r.random(10)
    rel, F = O.kkt_residual(A, b, np.zeros(10))
    np.testing.assert_allclose(rel, 1.0, rtol=1e-14)
    np.testing.assert_allclose(F, 0.5 * b @ b, rtol=1e-14)


def test_agrees_with_lawson_hanson():
    """Independent library cross-check: scipy's active-set NNLS."""
    nnls = pytest.importorskip("scipy.optimize").nnls
    r = _rng(51)
    A = r.random((150, 40))
    b = A @ np.where(r.random(40) < 0.5, 0.0, r.random(40)) + 0.01 * r.standard_normal(150)
    x_ls, _ = nnls(A, b)
    x, _, _, _ = O.reference_solution(A, b)
    np.testing.assert_allclose(x, x_ls, atol=1e-9 * np.abs(x_ls).max())


# ------------------------------------------------------------- convergence rates
def _well_conditioned_case(seed, n=12):
    """Gaussian A with d ≥ 12n: λ_min(Q) ≥ ½ so the Lemma's m = ½ holds."""
    r = _rng(seed)
    A = r.standard_normal((16 * n, n))
    x_true = r.uniform(0.5, 2.0, n)
    b = A @ x_true
    Q, q, s = O.antilopsided_scaling(*O.nqp_from_nnls(A, b))
    return Q, q


def test_rate_theorem_when_lemma_premise_holds():
    """Theorems of §4.1: f(x^{k+1}) − f* ≤ (1 − m/M)^k (f(x⁰) − f*), and with
    m = ½, M = ‖Q‖ (Frobenius) the paper's (1 − 1/(2‖Q‖))^k."""
    Q, q = _well_conditioned_case(61)
    ev = np.linalg.eigvalsh(Q)
    assert ev[0] >= 0.5
    y_star = np.linalg.solve(Q, -q)
    assert np.all(y_star > 0)
    f_star = O.objective(Q, q, y_star)
    res = O.solve_nqp(Q, q, eps=1e-28, trace=True)
    f = np.array([h[2] for h in res.history])
    gap0 = f[0] - f_star
    fro = O.q_norm_paper(Q)
    for k in range(len(f) - 1):
        gap = f[k + 1] - f_star
        assert gap <= (1 - 1 / (2 * fro)) ** k * gap0 + 1e-13
        assert gap <= (1 - ev[0] / ev[-1]) ** k * gap0 + 1e-13


def test_lemma_lower_bound_is_false_in_general():
    """Reading: the Lemma's ½I ⪯ Q does not hold in general — duplicate columns
    make Q singular — so the ½ rate is only tested where λ_min(Q) ≥ ½."""
    r = _rng(62)
    A = r.random((20, 5))
    A[:, 4] = A[:, 0]
    Q, q, s = O.antilopsided_scaling(*O.nqp_from_nnls(A, r.random(20)))
    assert np.linalg.eigvalsh(Q)[0] < 1e-12


# ------------------------------------------------------- planted-mistake detection
def _pins_pass():
    try:
        with np.errstate(all="ignore"):
            test_worked_example_scaling_and_iterations()
            for s in range(4):
                test_matches_brute_force_enumeration(s)
            test_scaled_matrix_invariants(21)
            test_kkt_conditions_at_reference_solution()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible mistake planted in the oracle fails at least one pin."""
    assert _pins_pass()

    good_mask = O.passive_mask
    monkeypatch.setattr(O, "passive_mask", lambda y, g: (y >= 0.0) | (g < 0.0))
    assert not _pins_pass(), "non-strict passive test (every y=0 passive)"
    monkeypatch.setattr(O, "passive_mask", lambda y, g: y > 0.0)
    assert not _pins_pass(), "dropped gradient term of the passive test"
    monkeypatch.setattr(O, "passive_mask", good_mask)

    good_scale = O.antilopsided_scaling

    def no_sqrt(H, h):
        Q, q, s = good_scale(H, h)
        return Q, h / (s * s), s
    monkeypatch.setattr(O, "antilopsided_scaling", no_sqrt)
    assert not _pins_pass(), "q divided by H_ii instead of sqrt(H_ii)"

    def sign_flip(H, h):
        Q, q, s = good_scale(H, h)
        return Q, -q, s
    monkeypatch.setattr(O, "antilopsided_scaling", sign_flip)
    assert not _pins_pass(), "wrong sign of h"
    monkeypatch.setattr(O, "antilopsided_scaling", good_scale)

    good_update = O.projected_update
    monkeypatch.setattr(O, "projected_update",
                        lambda y, gb, a: np.maximum(y + a * gb, 0.0))
    assert not _pins_pass(), "update along +ḡ (the prose's sign)"
    monkeypatch.setattr(O, "projected_update", good_update)

    good_grad = O.gradient_update
    monkeypatch.setattr(O, "gradient_update", lambda Q, g, yn, y: g + (yn - y))
    assert not _pins_pass(), "dropped Q in the gradient update"
    monkeypatch.setattr(O, "gradient_update", lambda Q, g, yn, y: g - Q @ (yn - y))
    assert not _pins_pass(), "wrong sign in the gradient update"
    monkeypatch.setattr(O, "gradient_update", good_grad)

    good_ls = O.exact_line_search
    monkeypatch.setattr(O, "exact_line_search",
                        lambda Q, gb, g2: g2 / float(gb @ gb) if g2 > 0 else None)
    assert not _pins_pass(), "line search without Q (unit step)"
    monkeypatch.setattr(O, "exact_line_search", good_ls)

    good_nqp = O.nqp_from_nnls
    monkeypatch.setattr(O, "nqp_from_nnls",
                        lambda A, b: (good_nqp(A, b)[0], -good_nqp(A, b)[1]))
    assert not _pins_pass(), "h = +Aᵀb"
    monkeypatch.setattr(O, "nqp_from_nnls", good_nqp)
    assert _pins_pass()
