"""The §5 test-case generators (Table 1): sign, sparsity, column lengths and
b = A x*, checked on reduced sizes (the recipe does not depend on n, d)."""
import numpy as np
import pytest

from paper_1502_01645_gb300 import workloads as W


@pytest.mark.parametrize("kind", sorted(W.TCASES))
@pytest.mark.parametrize("sub", [0, 2, 4])
def test_tcase_recipe(kind, sub):
    P = W.tcase(kind, sub, n=400, d=600, dtype=np.float64)
    sign, length = W.TCASES[kind]
    A, b, x = P.A, P.B[0], P.x_true[0]
    assert A.shape == (600, 400) and A.flags.f_contiguous and b.shape == (600,)
    frac = W.TCASE_SPARSITY[sub]
    # sparsity of A and x*
    assert abs(np.mean(A == 0.0) - frac) <= 0.01
    assert abs(np.mean(x == 0.0) - frac) <= 0.06
    # signs
    if sign == "+":
        assert A.min() >= 0.0 and x.min() >= 0.0
    else:
        assert (A < 0).any() and (x < 0).any() and (A > 0).any()
    # column lengths
    L = np.linalg.norm(A, axis=0)
    nz = L > 0
    if length == "SAM":
        np.testing.assert_allclose(L[nz], 1.0, rtol=1e-12)
    elif length == "RAN":
        assert L[nz].max() <= 1.0 + 1e-12 and L[nz].min() > 0.0
        assert L[nz].std() > 0.2                       # U(0, 1]: sd ≈ 0.29
    else:
        assert L[nz].max() / L[nz].min() >= 50.0       # 10^U[−1, 1]
        assert L[nz].max() <= 10.0 * (1 + 1e-12) and L[nz].min() >= 0.1 * (1 - 1e-12)
    # b = A x*, no noise
    np.testing.assert_allclose(b, A @ x, rtol=0, atol=1e-12 * np.abs(A @ x).max())


def test_tcase_is_deterministic_and_cases_differ():
    a = W.tcase("T4", 1, n=50, d=75)
    b = W.tcase("T4", 1, n=50, d=75)
    c = W.tcase("T4", 2, n=50, d=75)
    np.testing.assert_array_equal(a.A, b.A)
    np.testing.assert_array_equal(a.B, b.B)
    assert not np.array_equal(a.A, c.A)
    assert a.A.dtype == np.float32 and a.meta["kind"] == "T4"
