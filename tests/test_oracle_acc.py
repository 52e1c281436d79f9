"""Pins for the Anti+Acc oracle (oracle/acc.py) against what the mathematics
fixes: the spectrum of constructed matrices and numpy's eigensolver for the
power iteration; the Beck–Teboulle convergence bound of the accelerated
projected gradient (Beck & Teboulle 2009, Thm. 4.4); the momentum recursion's
identity; closed forms in one dimension; optima found by brute force or by the
independent Alg. 2 oracle.  ``test_planted_mistakes_are_caught`` plants
plausible mistakes and checks that some pin fails."""
import numpy as np
import pytest

from oracle import acc as AC
from oracle import nnls as O


def _spectral(seed, lam):
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((len(lam), len(lam))))
    return (U * np.asarray(lam)) @ U.T


def _ill(seed, d=60, n=30, cond=1e4):
    """A with prescribed singular values (cond(AᵀA) = cond), sparse x, noise."""
    r = np.random.default_rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((d, n)))
    V, _ = np.linalg.qr(r.standard_normal((n, n)))
    A = (U * np.logspace(0, -np.log10(cond) / 2, n)) @ V.T
    x = np.where(r.random(n) < 0.4, 0.0, r.random(n))
    return A, A @ x + 0.05 * r.standard_normal(d)


# ------------------------------------------------------------- power iteration
def _pin_power():
    lam = np.concatenate([[10.0, 6.0, 3.0], np.linspace(1.0, 0.1, 37)])
    rho, steps = AC.power_iteration(_spectral(3, lam))
    assert rho <= 10.0 + 1e-12          # a Rayleigh quotient never exceeds λ_max
    assert abs(rho - 10.0) <= 1e-5 * 10.0, rho
    rho, steps = AC.power_iteration(np.eye(7))
    assert rho == pytest.approx(1.0, abs=1e-15) and steps == 2
    # a scaled lopsided problem against numpy's symmetric eigensolver
    r = np.random.default_rng(5)
    A = r.random((300, 80)) * np.exp(r.uniform(-3, 3, 80))
    H, h = O.nqp_from_nnls(A, r.random(300))
    Q, q, s = O.antilopsided_scaling(H, h)
    lmax = np.linalg.eigvalsh(Q).max()
    rho, _ = AC.power_iteration(Q)
    assert rho <= lmax * (1 + 1e-14) and rho >= lmax * (1 - 1e-6), (rho, lmax)


def test_power_iteration():
    _pin_power()


# ----------------------------------------------------------- momentum sequence
def _pin_alphas():
    A, b = _ill(7)
    H, h = O.nqp_from_nnls(A, b)
    res = AC.solve_nqp_acc(H, h, np.linalg.eigvalsh(H).max(), tol=1e-14, max_iter=200,
                           trace=True)
    a = np.array(res.alphas)
    assert a[0] == 1.0
    # t_{k+1}² − t_{k+1} = t_k² (the recursion solved for t_{k+1}) and t_k ≥ (k+2)/2
    np.testing.assert_allclose(a[1:] ** 2 - a[1:], a[:-1] ** 2, rtol=1e-12)
    assert np.all(a >= (np.arange(len(a)) + 2) / 2.0 - 1e-12)


def test_momentum_sequence():
    _pin_alphas()


# ------------------------------------------------------- Beck–Teboulle bound
def _pin_rate(seed=1):
    """f(x_k) − f* ≤ 2L‖y⁰ − y*‖²/(k+1)² for every k when L ≥ λ_max(Q)
    (Beck & Teboulle 2009, Thm. 4.4; y⁰ = 0).  f* comes from the Alg. 2
    oracle's polished optimum, an independent method."""
    A, b = _ill(seed)
    H, h = O.nqp_from_nnls(A, b)
    L = np.linalg.eigvalsh(H).max()
    xs, _, _, _ = O.reference_solution(A, b)
    fs = O.objective(H, h, xs)
    res = AC.solve_nqp_acc(H, h, L, tol=1e-13, max_iter=3000, trace=True)
    R2 = float(xs @ xs)
    for k, _, f in res.history:
        if k >= 1:
            assert f - fs <= 2.0 * L * R2 / (k + 1) ** 2 + 1e-12, k


def test_beck_teboulle_bound():
    _pin_rate(1)
    _pin_rate(2)


# ------------------------------------------------------------ closed forms
def _pin_closed_forms():
    # one dimension, f = ½y² − y (y* = 1), L = 2 > λ = 1: x_0 = 1/2; Y_1 = x_0
    # (no momentum yet), x_1 = 3/4; α_1 = φ = (1+√5)/2, α_2 = (1 + √(4φ²+1))/2,
    # Y_2 = x_1 + ((φ − 1)/α_2)(x_1 − x_0), x_2 = Y_2 − (Y_2 − 1)/2
    phi = (1 + np.sqrt(5.0)) / 2
    a2 = (1 + np.sqrt(4 * phi * phi + 1)) / 2
    Y2 = 0.75 + (phi - 1) / a2 * 0.25
    Q, q = np.array([[1.0]]), np.array([-1.0])
    for k, want in ((1, 0.5), (2, 0.75), (3, Y2 - (Y2 - 1.0) / 2)):
        r = AC.solve_nqp_acc(Q, q, 2.0, eps=1e-300, max_iter=k)
        assert r.iters == k and r.y[0] == pytest.approx(want, rel=1e-15), (k, r.y, want)
    # L = λ: one step reaches y* = max(0, −q), then the stop rule holds
    r = AC.solve_nqp_acc(Q, np.array([-3.0]), 1.0, tol=1e-12)
    assert r.iters == 1 and r.y[0] == 3.0 and r.status == O.STATUS_CONVERGED
    # q > 0: y = 0 is optimal and no index is passive at the start
    r = AC.solve_nqp_acc(Q, np.array([2.0]), 1.0, tol=1e-12)
    assert r.iters == 0 and r.status == O.STATUS_EMPTY_PASSIVE


def test_closed_forms():
    _pin_closed_forms()


# ------------------------------------------------------------------- optima
def _pin_optima():
    r = np.random.default_rng(11)
    for t in range(6):
        d, n = 9, 6
        A = r.standard_normal((d, n))
        b = r.standard_normal(d)
        x, res, s, L = AC.anti_acc(A, b, tol=1e-11, max_iter=200000)
        xb, _ = O.brute_force_nnls(A, b)
        assert res.status in (O.STATUS_CONVERGED, O.STATUS_EMPTY_PASSIVE)
        np.testing.assert_allclose(x, xb, atol=1e-7 * max(1.0, np.abs(xb).max()))
    A, b = _ill(13, 120, 50, 1e3)
    x, res, s, L = AC.anti_acc(A, b, tol=1e-10, max_iter=200000)
    rel, _ = O.kkt_residual(A, b, x)
    assert rel <= 1e-10
    xs, _, _, _ = O.reference_solution(A, b)
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)


def test_optima_match_independent_solvers():
    _pin_optima()


# ------------------------------------------------------------ planted mistakes
def _pins_pass():
    try:
        _pin_power()
        _pin_alphas()
        _pin_rate(1)
        _pin_closed_forms()
        _pin_optima()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    good = AC.extrapolate
    for label, bad in [
        ("momentum sign flipped", lambda x, xp, a, an: x - ((a - 1) / an) * (x - xp)),
        ("no momentum", lambda x, xp, a, an: x),
        ("coefficient α_k/α_{k+1}", lambda x, xp, a, an: x + (a / an) * (x - xp)),
        ("extrapolation from x_{k−1}", lambda x, xp, a, an: xp + ((a - 1) / an) * (x - xp)),
    ]:
        monkeypatch.setattr(AC, "extrapolate", bad)
        assert not _pins_pass(), label
    monkeypatch.setattr(AC, "extrapolate", good)

    good_m = AC.momentum_next
    monkeypatch.setattr(AC, "momentum_next", lambda a: (1 + np.sqrt(a * a + 1)) / 2)
    assert not _pins_pass(), "α recursion without the factor 4"
    monkeypatch.setattr(AC, "momentum_next", lambda a: a + 1.0)
    assert not _pins_pass(), "α_k = k + 1"
    monkeypatch.setattr(AC, "momentum_next", good_m)

    good_s = AC.projected_step
    monkeypatch.setattr(AC, "projected_step", lambda Q, q, Y, L: Y - (Q @ Y + q) / L)
    assert not _pins_pass(), "projection dropped"
    monkeypatch.setattr(AC, "projected_step",
                        lambda Q, q, Y, L: np.maximum(Y - (Q @ Y - q) / L, 0.0))
    assert not _pins_pass(), "wrong sign of q in the gradient"
    monkeypatch.setattr(AC, "projected_step",
                        lambda Q, q, Y, L: np.maximum(Y - (Q.T @ Y + q) * L, 0.0))
    assert not _pins_pass(), "step L instead of 1/L"
    monkeypatch.setattr(AC, "projected_step", good_s)

    good_p = AC.power_iteration
    monkeypatch.setattr(AC, "power_iteration", lambda Q, **k: (float(np.abs(Q).sum(1).max()), 1))
    assert not _pins_pass(), "row-sum bound instead of the power iteration"
    monkeypatch.setattr(AC, "power_iteration", good_p)
    assert _pins_pass()
