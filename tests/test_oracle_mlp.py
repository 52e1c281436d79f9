"""Pins of the warm-start MLP oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: central finite differences of the loss, the
closed form of Adam's first steps, limits of the loss terms, the feature
normalisation, the unconstrained minimiser behind the direction feature, and
the fallback rule of the start point."""
import numpy as np
import pytest

from oracle import mlp as M


def _spd(n, seed=0, d=None):
    r = np.random.default_rng(seed)
    A = np.abs(r.normal(size=(d or 4 * n, n)))
    H = A.T @ A
    sc = np.sqrt(np.diag(H))
    return A, H / np.outer(sc, sc), sc


def _tiny(seed=0, n=3, hidden=5, B=4):
    r = np.random.default_rng(seed)
    p = M.init_params(2 * n, hidden, 2 * n, seed=seed)
    for k in ("b1", "b2", "b3"):
        p[k] = r.normal(0, 0.1, p[k].shape)
    p["e"] = r.normal(1.0, 0.3, n)
    p["f"] = r.normal(2.0, 0.5, n)
    _, Q, _ = _spd(n, seed)
    q = r.normal(size=(B, n))
    U, qn, zt = M.features(q, np.linalg.inv(Q))
    Y = np.maximum(r.normal(size=(B, n)), 0.0)
    T, C = M.targets(Y, qn)
    return p, U, zt, T, C


def _fd_check(p, U, zt, T, C, h=1e-4, per_tensor=6, seed=1):
    """Relative error of the analytic gradient against central differences on
    random entries of every parameter tensor."""
    _, g = M.loss_and_grad(p, U, zt, T, C)
    r = np.random.default_rng(seed)
    worst = 0.0
    for k in M.PARAM_NAMES:
        flat = p[k].reshape(-1)
        for idx in r.choice(flat.size, size=min(per_tensor, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, U, zt, T, C)
            flat[idx] = old - h
            lm = M.loss(p, U, zt, T, C)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            worst = max(worst, abs(fd - an) / max(abs(fd), abs(an), 1e-8))
    return worst


def test_gradient_matches_central_differences():
    p, U, zt, T, C = _tiny()
    _, (_, Z1, _, Z2, _) = M.forward(p, U, zt)
    # keep every pre-activation away from the ReLU kink by more than h (1e-4)
    assert np.abs(Z1).min() > 1e-2 and np.abs(Z2).min() > 1e-2
    assert np.abs(zt).min() > 1e-3   # the skips see a non-zero input
    assert _fd_check(p, U, zt, T, C) <= 1e-6


def _wrong_grad(drop_relu=False, swap_skips=False):
    def grad(p_, U_, zt_, T_, C_):
        O, (U_, Z1, H1, Z2, H2) = M.forward(p_, U_, zt_)
        B, n = T_.shape
        m = B * n
        dy = 2.0 * (O[:, :n] - T_) / m
        dl = (1.0 / (1.0 + np.exp(-O[:, n:])) - C_) / m
        dO = np.hstack([dy, dl])
        g = {"W3": dO.T @ H2, "b3": dO.sum(0)}
        g["e"], g["f"] = ((dl * zt_).sum(0), (dy * zt_).sum(0)) if swap_skips else \
            ((dy * zt_).sum(0), (dl * zt_).sum(0))
        dZ2 = (dO @ p_["W3"]) * (Z2 > 0)
        g["W2"], g["b2"] = dZ2.T @ H1, dZ2.sum(0)
        dZ1 = dZ2 @ p_["W2"]
        if not drop_relu:
            dZ1 = dZ1 * (Z1 > 0)
        g["W1"], g["b1"] = dZ1.T @ U_, dZ1.sum(0)
        return M.loss(p_, U_, zt_, T_, C_), g
    return grad


def test_gradient_check_catches_a_dropped_relu_mask(monkeypatch):
    monkeypatch.setattr(M, "loss_and_grad", _wrong_grad(drop_relu=True))
    p, U, zt, T, C = _tiny(seed=3, hidden=8)
    _, (_, Z1, _, _, _) = M.forward(p, U, zt)
    assert (Z1 < 0).any()
    assert _fd_check(p, U, zt, T, C, per_tensor=40) > 1e-3


def test_gradient_check_catches_swapped_skip_gradients(monkeypatch):
    monkeypatch.setattr(M, "loss_and_grad", _wrong_grad(swap_skips=True))
    p, U, zt, T, C = _tiny(seed=5)
    assert _fd_check(p, U, zt, T, C) > 1e-3


def test_direction_is_the_unconstrained_minimiser():
    """z = −Q⁻¹q solves Qz + q = 0 (the gradient of ½yᵀQy + qᵀy vanishes),
    for Q = I it is −q, and for a diagonal Q it is −q/diag Q."""
    r = np.random.default_rng(6)
    n = 9
    _, Q, _ = _spd(n, 6)
    q = r.normal(size=(5, n))
    z = M.direction(q, np.linalg.inv(Q))
    np.testing.assert_allclose(z @ Q.T + q, 0.0, atol=1e-10)
    np.testing.assert_allclose(M.direction(q, np.eye(n)), -q)
    dg = r.uniform(0.5, 2.0, n)
    np.testing.assert_allclose(M.direction(q, np.diag(1.0 / dg)), -q / dg)


def test_positive_unconstrained_minimiser_is_the_start():
    """A network whose skip passes ẑ straight through (W3 = 0, e = 1, f = 0,
    logits +5) predicts d = relu(z); when z > 0 it is the NNLS solution of the
    problem (the bound is inactive), and the line search keeps α* = 1."""
    n = 6
    A, Q, sc = _spd(n, 7, d=40)
    x_true = np.linspace(0.5, 2.0, n)
    b = A @ x_true
    q = -(A.T @ b) / sc
    Qinv = np.linalg.inv(Q)
    z = M.direction(q, Qinv)[0]
    assert np.all(z > 0)
    p = M.init_params(2 * n, 4, 2 * n, seed=0)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    p["b3"][n:] = 5.0
    p["e"][:] = 1.0
    p["f"][:] = 0.0
    y0 = M.predict(p, q, Qinv, Q)[0]
    np.testing.assert_allclose(y0, x_true * sc, rtol=1e-9)


def test_loss_limits():
    # BCE at ℓ = 0 is log 2 whatever the class; huge logits do not overflow
    assert M.bce(np.array(0.0), 1.0) == pytest.approx(np.log(2.0))
    assert M.bce(np.array(0.0), 0.0) == pytest.approx(np.log(2.0))
    big = M.bce(np.array([1000.0, -1000.0]), np.array([1.0, 0.0]))
    assert np.all(np.isfinite(big)) and np.all(big < 1e-300 + 1e-12)
    assert M.bce(np.array(-1000.0), 1.0) == pytest.approx(1000.0)
    # a network that outputs the targets exactly and confident logits: L → 0
    n = 3
    T = np.array([[0.2, 0.0, 0.5]])
    C = (T > 0).astype(float)
    p = {"W1": np.zeros((4, 2 * n)), "b1": np.ones(4), "W2": np.eye(4), "b2": np.zeros(4),
         "W3": np.zeros((2 * n, 4)), "b3": np.zeros(2 * n), "e": np.zeros(n),
         "f": np.zeros(n)}
    p["b3"] = np.concatenate([T[0], np.where(C[0] > 0, 60.0, -60.0)])
    L = M.loss(p, np.zeros((1, 2 * n)), np.zeros((1, n)), T, C)
    assert L < 1e-25
    # the skips alone reproduce the targets when ẑ equals them
    p["b3"][:n] = 0.0
    p["e"][:] = 1.0
    L2 = M.loss(p, np.zeros((1, 2 * n)), T.copy(), T, C)
    assert L2 < 1e-25


def test_adam_first_steps_closed_form():
    # with m = v = 0, bias correction makes the first step −lr·g/(|g| + ε)
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    st = M.adam_init(p)
    M.adam_step(p, g, st, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p["w"], [1.0, -2.0, 3.0] - 0.1 * g["w"] / (np.abs(g["w"]) + 1e-8))
    # a constant gradient keeps the same step size in later steps
    before = p["w"].copy()
    M.adam_step(p, g, st, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p["w"] - before, -0.1 * g["w"] / (np.abs(g["w"]) + 1e-8),
                               rtol=1e-12)


def test_features_normalisation():
    r = np.random.default_rng(4)
    n = 7
    q = r.normal(size=(3, n))
    _, Q, _ = _spd(n, 4)
    Qinv = np.linalg.inv(Q)
    U, qn, zt = M.features(q, Qinv)
    np.testing.assert_allclose(qn, np.linalg.norm(q, axis=1))
    np.testing.assert_allclose(np.linalg.norm(U[:, :n], axis=1), 1.0)
    np.testing.assert_allclose(U[:, n:] * qn[:, None], M.direction(q, Qinv), rtol=1e-12)
    np.testing.assert_allclose(zt, U[:, n:])      # τ = 1 without statistics
    # scale invariance of both parts; ẑ scales with nothing either
    U2, _, zt2 = M.features(5.0 * q, Qinv)
    np.testing.assert_allclose(U2, U, rtol=1e-12)
    np.testing.assert_allclose(zt2, zt, rtol=1e-12)
    # q = 0: zero features and zero skip input
    U4, qn4, zt4 = M.features(np.zeros((1, n)), Qinv)
    assert qn4[0] == 0.0 and np.all(U4 == 0.0) and np.all(zt4 == 0.0)


def _identity_net(n, sign):
    """h1 = relu(sign·q/‖q‖) on the first n units, ŷ = h1[:n], logits 5,
    skips off."""
    hidden = 2 * n
    p = {"W1": np.zeros((2 * n, 2 * n)), "b1": np.zeros(2 * n),
         "W2": np.eye(2 * n), "b2": np.zeros(2 * n),
         "W3": np.zeros((2 * n, hidden)), "b3": np.zeros(2 * n),
         "e": np.zeros(n), "f": np.zeros(n)}
    p["W1"][:n, :n] = sign * np.eye(n)
    p["W3"][:n, :n] = np.eye(n)
    p["b3"][n:] = 5.0
    return p


def test_predict_line_search_rule():
    n = 4
    Q = np.eye(n)
    q = -np.array([[1.0, 2.0, 0.5, 3.0]])
    # direction −q/‖q‖ with Q = I: the exact line search lands on y* = −q
    p = _identity_net(n, -1.0)
    np.testing.assert_allclose(M.predict(p, q, Q, Q)[0], -q[0])
    # the start does not depend on the predicted magnitude
    p10 = dict(p, W3=10.0 * p["W3"])
    np.testing.assert_allclose(M.predict(p10, q, Q, Q), M.predict(p, q, Q, Q))
    # a direction that does not descend (qᵀd ≥ 0) gives y⁰ = 0
    assert np.all(M.predict(_identity_net(n, 1.0), -q, Q, Q) == 0.0)
    # logits ≤ 0 switch every entry off
    p["b3"][n:] = -5.0
    assert np.all(M.predict(p, q, Q, Q) == 0.0)


def test_predict_is_the_best_point_on_its_ray():
    """f(y⁰) ≤ f(α·d) for every α ≥ 0 on a grid, and f(y⁰) ≤ 0 = f(0)."""
    r = np.random.default_rng(8)
    n = 12
    A, Q, sc = _spd(n, 8, d=40)
    Qinv = np.linalg.inv(Q)
    q = -(r.random((16, n)) @ A.T @ A) / sc + 0.3 * r.normal(size=(16, n))
    p = M.init_params(2 * n, 32, 2 * n, seed=9)
    p["b3"][n:] = 2.0
    y0 = M.predict(p, q, Qinv, Q)
    U, _, zt = M.features(q, Qinv)
    O, _ = M.forward(p, U, zt)
    d = np.maximum(O[:, :n], 0.0) * (O[:, n:] > 0)

    def f(y, qq):
        return 0.5 * y @ Q @ y + qq @ y

    for b in range(len(q)):
        fy = f(y0[b], q[b])
        assert fy <= 1e-14
        for a in np.linspace(0.0, 3.0, 61) * max(np.abs(y0[b]).max(), 1e-3) / max(
                np.abs(d[b]).max(), 1e-12):
            assert fy <= f(a * d[b], q[b]) + 1e-12


def test_normalisation_statistics():
    r = np.random.default_rng(10)
    n, m = 5, 300
    q = r.normal(size=(m, n)) + np.array([3.0, 0, 0, 0, -1.0])
    Y = np.maximum(r.normal(size=(m, n)), 0.0) * 7.0
    _, Q, _ = _spd(n, 10)
    Qinv = np.linalg.inv(Q)
    st = M.stats(q, Y, Qinv)
    U, qn, zt = M.features(q, Qinv, st)
    np.testing.assert_allclose(U.mean(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(U.std(axis=0), 1.0, rtol=1e-12)
    T, _ = M.targets(Y, qn, st["tau"])
    assert abs(np.sqrt(np.mean(T ** 2)) - 1.0) < 1e-12
    # the skip input is z in the targets' scale
    np.testing.assert_allclose(zt * st["tau"] * qn[:, None], M.direction(q, Qinv), rtol=1e-12)


def test_training_lowers_the_loss():
    r = np.random.default_rng(5)
    n, m = 6, 256
    A = np.abs(r.normal(size=(30, n)))
    s = np.linalg.norm(A, axis=0)
    Q = (A.T @ A) / np.outer(s, s)
    X = np.maximum(r.normal(size=(m, n)), 0.0)
    Ys = X * s
    Qs = -(X @ A.T @ A) / s     # q = −D⁻¹Aᵀb with b = A x (noise-free)
    p = M.init_params(2 * n, 32, 2 * n, seed=1)
    hist = M.train(p, Qs, Ys, np.linalg.inv(Q), epochs=100, batch=32, lr=3e-3)
    assert hist[-1] < 0.45 * hist[0]
    assert hist[-1] < hist[len(hist) // 3]
