"""FP64 CPU oracle of Alg. 1 for a matrix given in compressed sparse column
(CSC) form.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library and imports nothing from it.

The paper's test matrices include sparse ``A`` (§5: sub-tests with 0–40% of
the entries of ``A_k`` set to zero).  Sparsity changes how ``A`` is stored,
not what Alg. 1 computes: ``H = AᵀA``, ``h = Aᵀb``, ``D = diag(√H_ii)``,
``Q = D⁻¹HD⁻¹``, ``q = −D⁻¹h`` (Eq. NQP, Eq. NQPQ).  So the oracle is the
definition written out: expand the CSC arrays to the dense matrix they
denote, then the dense Alg. 1 of ``oracle.nnls``.

The CSC form read here: ``col_ptr`` (n+1 offsets, ``col_ptr[0] = 0``,
non-decreasing), and for column ``j`` the entries ``t`` with
``col_ptr[j] ≤ t < col_ptr[j+1]``: value ``vals[t]`` in row ``row_idx[t]``,
rows in ``[0, d)`` and strictly increasing within a column.
"""
from __future__ import annotations

import numpy as np

from . import nnls as O


def check_csc(d, n, col_ptr, row_idx, vals):
    """Raise ValueError unless the arrays are a well-formed CSC matrix d×n."""
    col_ptr = np.asarray(col_ptr)
    row_idx = np.asarray(row_idx)
    vals = np.asarray(vals)
    if col_ptr.shape != (n + 1,):
        raise ValueError("col_ptr must have n+1 entries")
    if col_ptr[0] != 0:
        raise ValueError("col_ptr[0] must be 0")
    nnz = int(col_ptr[n])
    if row_idx.shape[0] < nnz or vals.shape[0] < nnz:
        raise ValueError("row_idx and vals need col_ptr[n] entries")
    for j in range(n):
        p0, p1 = int(col_ptr[j]), int(col_ptr[j + 1])
        if p1 < p0:
            raise ValueError(f"col_ptr decreases at column {j}")
        prev = -1
        for t in range(p0, p1):
            r = int(row_idx[t])
            if r < 0 or r >= d:
                raise ValueError(f"row {r} out of range in column {j}")
            if r <= prev:
                raise ValueError(f"rows not strictly increasing in column {j}")
            prev = r


def csc_to_dense(d, n, col_ptr, row_idx, vals):
    """The dense d×n FP64 matrix the CSC arrays denote (entries not stored
    are zero)."""
    check_csc(d, n, col_ptr, row_idx, vals)
    A = np.zeros((d, n), dtype=np.float64)
    for j in range(n):
        for t in range(int(col_ptr[j]), int(col_ptr[j + 1])):
            A[int(row_idx[t]), j] = float(vals[t])
    return A


def scaled_problem_csc(d, n, col_ptr, row_idx, vals, b):
    """(Q, q, s) of Alg. 1 (Eq. NQPQ) for the CSC matrix and right-hand side b."""
    A = csc_to_dense(d, n, col_ptr, row_idx, vals)
    H, h = O.nqp_from_nnls(A, np.asarray(b, np.float64))
    return O.antilopsided_scaling(H, h)


def gram_entry(col_ptr, row_idx, vals, i, j):
    """H_ij = A_iᵀA_j from the two stored columns (rows matched one by one):
    a single entry, for checks at sizes where the dense matrix is too large."""
    ri = {int(row_idx[t]): float(vals[t]) for t in range(int(col_ptr[i]), int(col_ptr[i + 1]))}
    return sum(ri.get(int(row_idx[t]), 0.0) * float(vals[t])
               for t in range(int(col_ptr[j]), int(col_ptr[j + 1])))


def atb_entry(col_ptr, row_idx, vals, b, j):
    """(Aᵀb)_j from the stored entries of column j."""
    return sum(float(vals[t]) * float(b[int(row_idx[t])])
               for t in range(int(col_ptr[j]), int(col_ptr[j + 1])))


def kkt_residual_csc(d, n, col_ptr, row_idx, vals, b, x):
    """The relative KKT residual and objective of ``oracle.nnls.kkt_residual``
    (Def. 1 in the scaled variables of Eq. NQPQ) evaluated from the stored
    entries, for matrices too large to expand: r = Ax − b accumulated entry
    by entry, ∇F_j = A_jᵀr and s_j = ‖A_j‖ per column (s_j = 1 for an empty
    column), g = ∇F/s, ḡ = g on P(y = s·x), q = −Aᵀb/s; returns
    (‖ḡ‖/‖min(q, 0)‖ — or ‖ḡ‖ when that is 0 — and ½‖r‖²)."""
    check_csc(d, n, col_ptr, row_idx, vals)
    cp = np.asarray(col_ptr, np.int64)
    ri = np.asarray(row_idx, np.int64)
    v = np.asarray(vals, np.float64)
    b = np.asarray(b, np.float64)
    x = np.asarray(x, np.float64)
    cols = np.repeat(np.arange(n), np.diff(cp[:n + 1]))
    nnz = int(cp[n])
    ri, v = ri[:nnz], v[:nnz]
    r = np.bincount(ri, weights=v * x[cols], minlength=d) - b
    grad = np.bincount(cols, weights=v * r[ri], minlength=n)
    col2 = np.bincount(cols, weights=v * v, minlength=n)
    s = np.sqrt(col2)
    s[col2 == 0.0] = 1.0
    g = grad / s
    y = x * s
    gbar = np.where(O.passive_mask(y, g), g, 0.0)
    q = -np.bincount(cols, weights=v * b[ri], minlength=n) / s
    den = O.kkt_denominator(q)
    num = float(np.linalg.norm(gbar))
    return (num / den if den > 0 else num), 0.5 * float(r @ r)
