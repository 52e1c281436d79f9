"""Pins for the CSC oracle (oracle/sparse.py): a matrix written out by hand,
scipy's own CSC → dense conversion, the structure rules, the single-entry
Gram and Aᵀb against the dense products, and planted mistakes."""
import numpy as np
import pytest

from oracle import nnls as O
from oracle import sparse as S


def _random_csc(seed, d, n, density):
    g = np.random.default_rng(seed)
    M = g.standard_normal((d, n)) * (g.random((d, n)) < density)
    col_ptr = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        nz = np.flatnonzero(M[:, j])
        rows.extend(nz.tolist())
        vals.extend(M[nz, j].tolist())
        col_ptr[j + 1] = len(rows)
    return M, col_ptr, np.array(rows, np.int32), np.array(vals, np.float64)


def _pin_hand():
    # [[1 0 2], [0 0 3], [4 5 0]] stored column by column
    cp = np.array([0, 2, 3, 5], np.int64)
    ri = np.array([0, 2, 2, 0, 1], np.int32)
    v = np.array([1.0, 4.0, 5.0, 2.0, 3.0])
    A = S.csc_to_dense(3, 3, cp, ri, v)
    np.testing.assert_array_equal(A, [[1, 0, 2], [0, 0, 3], [4, 5, 0]])
    # H = AᵀA by hand: columns (1,0,4), (0,0,5), (2,3,0)
    assert S.gram_entry(cp, ri, v, 0, 0) == 17.0
    assert S.gram_entry(cp, ri, v, 0, 1) == 20.0
    assert S.gram_entry(cp, ri, v, 0, 2) == 2.0
    assert S.gram_entry(cp, ri, v, 1, 2) == 0.0
    assert S.atb_entry(cp, ri, v, np.array([1.0, 1.0, 1.0]), 2) == 5.0


def _pin_scipy():
    sp = pytest.importorskip("scipy.sparse")
    for seed, (d, n, dens) in enumerate([(40, 30, 0.2), (7, 50, 0.6), (65, 3, 0.05)]):
        M, cp, ri, v = _random_csc(seed, d, n, dens)
        ref = sp.csc_matrix((v, ri, cp), shape=(d, n)).toarray()
        np.testing.assert_array_equal(S.csc_to_dense(d, n, cp, ri, v), ref)
        np.testing.assert_array_equal(ref, M)


def _pin_entries():
    M, cp, ri, v = _random_csc(11, 50, 20, 0.3)
    b = np.random.default_rng(12).standard_normal(50)
    H = M.T @ M
    h = M.T @ b
    for i, j in [(0, 0), (3, 7), (19, 2), (5, 5)]:
        assert S.gram_entry(cp, ri, v, i, j) == pytest.approx(H[i, j], rel=1e-13, abs=1e-13)
    for j in (0, 9, 19):
        assert S.atb_entry(cp, ri, v, b, j) == pytest.approx(h[j], rel=1e-13, abs=1e-13)
    Q, q, s = S.scaled_problem_csc(50, 20, cp, ri, v, b)
    Qd, qd, sd = O.antilopsided_scaling(H, h)
    np.testing.assert_allclose(Q, Qd, atol=1e-14)
    np.testing.assert_allclose(s, sd, rtol=1e-14)


def _pin_kkt_csc():
    # the CSC residual against the dense oracle's on the expanded matrix, at
    # random points, the origin and the optimum, with an empty column
    M, cp, ri, v = _random_csc(21, 60, 25, 0.3)
    M[:, 7] = 0.0
    cp, ri, v = _csc_of(M)
    g = np.random.default_rng(22)
    b = M @ np.abs(g.standard_normal(25)) + 0.1 * g.standard_normal(60)
    x_star, _, _, _ = O.reference_solution(M, b)
    for x in (np.zeros(25), np.abs(g.standard_normal(25)) * (g.random(25) < 0.5), x_star):
        rel, F = S.kkt_residual_csc(60, 25, cp, ri, v, b, x)
        rel_d, F_d = O.kkt_residual(M, b, x)
        assert rel == pytest.approx(rel_d, rel=1e-10, abs=1e-14)
        assert F == pytest.approx(F_d, rel=1e-12)
    assert S.kkt_residual_csc(60, 25, cp, ri, v, b, np.zeros(25))[0] == pytest.approx(1.0)
    assert S.kkt_residual_csc(60, 25, cp, ri, v, b, x_star)[0] <= 1e-10


def _csc_of(M):
    n = M.shape[1]
    cp = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        nz = np.flatnonzero(M[:, j])
        rows.extend(nz.tolist())
        vals.extend(M[nz, j].tolist())
        cp[j + 1] = len(rows)
    return cp, np.array(rows, np.int32), np.array(vals, np.float64)


def test_kkt_residual_from_csc_matches_dense():
    _pin_kkt_csc()


def test_hand_matrix():
    _pin_hand()


def test_matches_scipy_conversion():
    _pin_scipy()


def test_single_entries_match_dense_products():
    _pin_entries()


@pytest.mark.parametrize("cp,ri,why", [
    ([0, 2, 1], [0, 1], "col_ptr decreases"),
    ([1, 2, 2], [0, 1], r"col_ptr\[0\] must be 0"),
    ([0, 2, 2], [1, 0], "strictly increasing"),
    ([0, 2, 2], [1, 1], "strictly increasing"),
    ([0, 1, 2], [0, 3], "out of range"),
    ([0, 1, 2], [0, -1], "out of range"),
])
def test_structure_rules(cp, ri, why):
    with pytest.raises(ValueError, match=why):
        S.check_csc(3, 2, np.array(cp, np.int64), np.array(ri, np.int32), np.ones(len(ri)))


def test_empty_columns_and_empty_matrix():
    A = S.csc_to_dense(4, 3, np.array([0, 0, 1, 1], np.int64), np.array([2], np.int32),
                       np.array([5.0]))
    np.testing.assert_array_equal(A[:, [0, 2]], 0.0)
    assert A[2, 1] == 5.0
    Z = S.csc_to_dense(4, 2, np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros(0))
    np.testing.assert_array_equal(Z, 0.0)


def _pins_pass():
    try:
        _pin_hand()
        _pin_scipy()
        _pin_entries()
        _pin_kkt_csc()
    except (AssertionError, ValueError, IndexError):
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    good = S.csc_to_dense

    def transposed(d, n, cp, ri, v):  # row and column roles swapped
        A = np.zeros((d, n))
        for j in range(n):
            for t in range(int(cp[j]), int(cp[j + 1])):
                if int(ri[t]) < n and j < d:
                    A[j, int(ri[t])] = v[t]
        return A
    monkeypatch.setattr(S, "csc_to_dense", transposed)
    assert not _pins_pass(), "rows and columns swapped"

    def off_by_one(d, n, cp, ri, v):  # column j read from col_ptr[j+1]
        A = np.zeros((d, n))
        for j in range(n - 1):
            for t in range(int(cp[j + 1]), int(cp[j + 2])):
                A[int(ri[t]), j] = v[t]
        return A
    monkeypatch.setattr(S, "csc_to_dense", off_by_one)
    assert not _pins_pass(), "column offsets shifted"
    monkeypatch.setattr(S, "csc_to_dense", good)
    good_g = S.gram_entry
    monkeypatch.setattr(S, "gram_entry", lambda cp, ri, v, i, j: good_g(cp, ri, v, i, j) +
                        (good_g(cp, ri, v, i, i) if i != j else 0.0))
    assert not _pins_pass(), "Gram entry with an extra term"
    monkeypatch.setattr(S, "gram_entry", good_g)
    good_k = S.kkt_residual_csc

    def no_mask(d, n, cp, ri, v, b, x):  # ḡ without the passive-set mask
        saved = O.passive_mask
        O.passive_mask = lambda y, g: np.ones_like(g, dtype=bool)
        try:
            return good_k(d, n, cp, ri, v, b, x)
        finally:
            O.passive_mask = saved
    monkeypatch.setattr(S, "kkt_residual_csc", no_mask)
    assert not _pins_pass(), "KKT residual without the passive-set mask"
    monkeypatch.setattr(S, "kkt_residual_csc", good_k)
    assert _pins_pass()
