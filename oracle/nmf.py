"""FP64 CPU oracle of non-negative matrix factorisation by alternating NNLS.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library and imports nothing from it.

The paper motivates fast NNLS with NMF and tensor factorisation (§1), and
notes that Bro's method reuses work across the many right-hand sides such a
factorisation produces (§2.2).  It does not spell out the outer loop; this
module reads it as the standard alternating non-negative least squares
(ANLS): for V ≈ W·H with W (m×r) ⪰ 0 and H (r×n) ⪰ 0, each outer iteration

    H-step: h_j = argmin_{h ⪰ 0} ½‖W h − v_j‖²         for every column j of V
    W-step: w_i = argmin_{w ⪰ 0} ½‖Hᵀ w − (v_i)ᵀ‖²     for every row i of V

each sub-problem solved by Alg. 1 + Alg. 2 (``oracle.nnls.antilop``) to the
given relative KKT tolerance, warm-started from the previous outer
iteration's column or row.  The objective after outer iteration t is
½‖V − W H‖_F² (the sum of the W-step's sub-problem objectives).
"""
from __future__ import annotations

import numpy as np

from . import nnls as O


def objective(V, W, H):
    """½‖V − W H‖_F²."""
    R = np.asarray(V, np.float64) - np.asarray(W, np.float64) @ np.asarray(H, np.float64)
    return 0.5 * float(np.sum(R * R))


def h_step(V, W, H, tol):
    """Every column of H from the NNLS problem with matrix W and right-hand
    side the matching column of V, warm-started from H's column."""
    V = np.asarray(V, np.float64)
    W = np.asarray(W, np.float64)
    Hn = np.empty_like(np.asarray(H, np.float64))
    for j in range(V.shape[1]):
        x, _, _ = O.antilop(W, V[:, j], tol=tol, x0=H[:, j])
        Hn[:, j] = x
    return Hn


def w_step(V, W, H, tol):
    """Every row of W from the NNLS problem with matrix Hᵀ and right-hand
    side the matching row of V, warm-started from W's row."""
    V = np.asarray(V, np.float64)
    Ht = np.asarray(H, np.float64).T
    Wn = np.empty_like(np.asarray(W, np.float64))
    for i in range(V.shape[0]):
        x, _, _ = O.antilop(Ht, V[i, :], tol=tol, x0=W[i, :])
        Wn[i, :] = x
    return Wn


def anls(V, W0, H0, outer, tol=1e-10):
    """``outer`` ANLS iterations (H-step, then W-step) from (W0, H0); returns
    (W, H, objectives after each outer iteration)."""
    W = np.array(W0, dtype=np.float64)
    H = np.array(H0, dtype=np.float64)
    objs = []
    for _ in range(outer):
        H = h_step(V, W, H, tol)
        W = w_step(V, W, H, tol)
        objs.append(objective(V, W, H))
    return W, H, objs
