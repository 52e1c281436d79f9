"""Pins for the ANLS oracle (oracle/nmf.py): the block-minimisation property
(the objective never rises), exact recovery of a non-negative factorisation
from a nearby start, each half-step against brute-force NNLS, the KKT
conditions of every sub-problem at the end, and planted mistakes."""
import numpy as np
import pytest

from oracle import nmf as N
from oracle import nnls as O


def _exact(seed, m, n, r):
    g = np.random.default_rng(seed)
    W = g.random((m, r)) * (g.random((m, r)) < 0.7)
    H = g.random((r, n)) * (g.random((r, n)) < 0.7)
    return W, H, W @ H


def _pin_monotone():
    g = np.random.default_rng(3)
    V = g.random((30, 24))
    W0, H0 = g.random((30, 4)), g.random((4, 24))
    W, H, objs = N.anls(V, W0, H0, outer=6, tol=1e-11)
    assert objs[0] <= N.objective(V, W0, H0) + 1e-9
    assert all(b <= a * (1 + 1e-9) + 1e-12 for a, b in zip(objs, objs[1:])), objs
    assert np.all(W >= 0) and np.all(H >= 0)
    assert objs[-1] == pytest.approx(N.objective(V, W, H), rel=1e-12)


def _pin_objective():
    # ½‖V − WH‖²: a 1×1 case by hand, and the sum of the W-step's
    # sub-problem objectives ½‖Hᵀw_i − v_i‖² from the NNLS oracle
    assert N.objective(np.array([[2.0]]), np.array([[1.0]]), np.array([[1.0]])) == 0.5
    g = np.random.default_rng(4)
    V, W, H = g.random((7, 5)), g.random((7, 2)), g.random((2, 5))
    tot = sum(O.nnls_objective(H.T, V[i, :], W[i, :]) for i in range(7))
    assert N.objective(V, W, H) == pytest.approx(tot, rel=1e-12)


def _pin_recovery():
    W, H, V = _exact(5, 25, 20, 3)
    g = np.random.default_rng(6)
    W0 = W + 0.05 * g.random(W.shape)
    _, _, objs = N.anls(V, W0, np.ones_like(H), outer=30, tol=1e-12)
    # ANLS converges linearly: after 30 outer iterations from a 5% perturbed
    # W the residual is ~1e-7 of ½‖V‖² (a wrong half-step stalls far above)
    assert objs[-1] <= 1e-6 * N.objective(V, np.zeros_like(W), H), objs[-1]


def _pin_half_steps():
    g = np.random.default_rng(8)
    V = g.standard_normal((9, 5)) + 1.0
    W = g.random((9, 4))
    H = g.random((4, 5))
    Hn = N.h_step(V, W, H, 1e-12)
    for j in range(5):
        xb, _ = O.brute_force_nnls(W, V[:, j])
        np.testing.assert_allclose(Hn[:, j], xb, atol=1e-8)
    Wn = N.w_step(V, W, Hn, 1e-12)
    for i in range(9):
        xb, _ = O.brute_force_nnls(Hn.T, V[i, :])
        np.testing.assert_allclose(Wn[i, :], xb, atol=1e-8)


def _pin_kkt():
    g = np.random.default_rng(9)
    V = g.random((40, 30))
    W, H, _ = N.anls(V, g.random((40, 5)), g.random((5, 30)), outer=3, tol=1e-10)
    # the last half-step (W) is optimal for the final H, row by row
    for i in range(40):
        rel, _ = O.kkt_residual(H.T, V[i, :], W[i, :])
        assert rel <= 1e-9
    # one more H-step against the final W gives KKT points column by column
    H2 = N.h_step(V, W, H, 1e-10)
    for j in range(30):
        rel, _ = O.kkt_residual(W, V[:, j], H2[:, j])
        assert rel <= 1e-9


def test_objective_never_rises():
    _pin_monotone()


def test_exact_factorisation_is_recovered():
    _pin_recovery()


def test_objective_definition():
    _pin_objective()


def test_half_steps_match_brute_force():
    _pin_half_steps()


def test_final_subproblems_meet_kkt():
    _pin_kkt()


def _pins_pass():
    try:
        _pin_objective()
        _pin_monotone()
        _pin_recovery()
        _pin_half_steps()
        _pin_kkt()
    except (AssertionError, ValueError):
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    good_h = N.h_step
    monkeypatch.setattr(N, "h_step", lambda V, W, H, tol: np.maximum(
        np.linalg.lstsq(W, V, rcond=None)[0], 0.0))
    assert not _pins_pass(), "H-step as clipped least squares"
    monkeypatch.setattr(N, "h_step", good_h)
    good_w = N.w_step

    monkeypatch.setattr(N, "w_step", lambda V, W, H, tol: good_w(V, W, H[::-1], tol))
    assert not _pins_pass(), "W-step against H with its rows permuted"
    monkeypatch.setattr(N, "w_step", good_w)
    good_obj = N.objective
    monkeypatch.setattr(N, "objective", lambda V, W, H: float(np.sum((V - W @ H) ** 2)))
    assert not _pins_pass(), "objective without the ½"
    monkeypatch.setattr(N, "objective", good_obj)
    assert _pins_pass()
