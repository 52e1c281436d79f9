"""Seeded synthetic NNLS inputs shaped like the paper's large-matrix workloads.

This module only draws random numbers and assembles ``b = A x_true + noise``;
it contains none of the solver's arithmetic, so both the CUDA path and the CPU
oracle may consume what it produces.  The paper generates its test cases the
same way (§5, "Experimental Evaluation": random ``A`` and ``x*``, then
``b = A x*``), but its saved cases were never published, so these recipes stand
in for them.

Every generator takes a seed and returns numpy arrays.  ``A`` is column-major in
the sense the library expects: ``A.T`` is C-contiguous, i.e. the returned array
is Fortran-ordered ``(d, n)`` so that each column ``A_i`` is contiguous.
Right-hand sides are returned as ``(k, d)`` C-contiguous (each RHS contiguous).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "uniform_small",
    "lopsided_single",
    "shared_multi_rhs",
    "uneven_batch",
    "warmstart_family",
    "TCASES",
    "tcase",
    "nmf_matrix",
    "SparseProblem",
    "banded_tall",
    "to_csc",
    "CONFIGS",
]


@dataclass
class Problem:
    """One NNLS instance ``min ½‖Ax−b‖²  s.t. x ≥ 0`` (possibly many RHS)."""

    A: np.ndarray            # (d, n), Fortran order, float32 or float64
    B: np.ndarray            # (k, d), C order; row c is the c-th right-hand side
    x_true: np.ndarray       # (k, n) generating solution (not the NNLS optimum)
    tol: float               # relative KKT tolerance the workload is solved to
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]

    @property
    def k(self) -> int:
        return self.B.shape[0]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _sparse_rows(rng, k, n, zero_frac, draw):
    """k rows of length n with round(zero_frac*n) zeros at random positions."""
    X = draw((k, n))
    nz = int(round(zero_frac * n))
    for c in range(k):
        X[c, rng.permutation(n)[:nz]] = 0.0
    return X


def _noisy_rhs(rng, A64, X, rel_noise):
    """b_c = A x_c + rel_noise * (‖A x_c‖/√d) * N(0, I), per column c."""
    d = A64.shape[0]
    clean = X @ A64.T                                   # (k, d)
    scale = rel_noise * np.linalg.norm(clean, axis=1, keepdims=True) / np.sqrt(d)
    return clean + scale * rng.standard_normal(clean.shape)


def uniform_small(d=1000, n=200, zero_frac=0.5, noise_sd=0.01, seed=1001, tol=1e-10):
    """Plain FP64 single-RHS case: A ~ U[0,1], x_true half zeros, rest U[0,1],
    b = A x_true + N(0, noise_sd²) (absolute noise)."""
    rng = _rng(seed)
    A = np.asfortranarray(rng.random((d, n)))
    x = _sparse_rows(rng, 1, n, zero_frac, lambda s: rng.random(s))
    b = x @ A.T + noise_sd * rng.standard_normal((1, d))
    return Problem(A, np.ascontiguousarray(b), x, tol, "uniform_small",
                   {"d": d, "n": n, "dtype": "f64"})


def _lopsided_A(rng, d, n, lo=1e-2, hi=1e2):
    """A ~ U[0,1] with every column multiplied by a log-uniform factor in [lo, hi]."""
    A = rng.random((d, n))
    scale = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    return A * scale[None, :]


def lopsided_single(d=20000, n=5000, zero_frac=0.7, seed=1002, tol=1e-6):
    """Single large RHS with lopsided column scaling (FP32 inputs):
    x_true 70% zeros with Exp(1) nonzeros, b = A x_true + 1% Gaussian noise."""
    rng = _rng(seed)
    A64 = _lopsided_A(rng, d, n)
    A = np.asfortranarray(A64.astype(np.float32))
    x = _sparse_rows(rng, 1, n, zero_frac, lambda s: rng.exponential(1.0, s))
    b = _noisy_rhs(rng, A.astype(np.float64), x, 0.01).astype(np.float32)
    return Problem(A, np.ascontiguousarray(b), x, tol, "lopsided_single",
                   {"d": d, "n": n, "dtype": "f32"})


def shared_multi_rhs(d=10000, n=1000, k=4096, zero_frac=0.8, seed=1003, tol=1e-6):
    """Many RHS sharing one A (NMF inner-solve shape): A ~ U[0,1] FP32,
    X_true 80% zeros with Gamma(2,1) nonzeros, B = A X_true + 1% noise per column."""
    rng = _rng(seed)
    A = np.asfortranarray(rng.random((d, n)).astype(np.float32))
    X = _sparse_rows(rng, k, n, zero_frac, lambda s: rng.gamma(2.0, 1.0, s))
    B = _noisy_rhs(rng, A.astype(np.float64), X, 0.01).astype(np.float32)
    return Problem(A, np.ascontiguousarray(B), X, tol, "shared_multi_rhs",
                   {"d": d, "n": n, "k": k, "dtype": "f32"})


def uneven_batch(count=512, n_lo=32, n_hi=1024, zero_frac=0.6, seed=1004, tol=1e-6):
    """Independent problems of uneven size: n log-uniform in [n_lo, n_hi],
    d = n * U{2,3,4}, A = |N(0,1)| FP32, x_true 60% zeros with U[0,1] nonzeros,
    b with 1% noise.  Problem p draws from seed + p."""
    probs = []
    for p in range(count):
        rng = _rng(seed * 100003 + p)
        n = int(np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        n = max(n_lo, min(n, n_hi))
        d = n * int(rng.integers(2, 5))
        A = np.asfortranarray(np.abs(rng.standard_normal((d, n))).astype(np.float32))
        x = _sparse_rows(rng, 1, n, zero_frac, lambda s: rng.random(s))
        b = _noisy_rhs(rng, A.astype(np.float64), x, 0.01).astype(np.float32)
        probs.append(Problem(A, np.ascontiguousarray(b), x, tol, f"uneven_{p}",
                             {"d": d, "n": n, "dtype": "f32"}))
    return probs


def warmstart_family(d=8000, n=2000, k=1024, support=(50, 400), seed=1005, rhs_seed=None,
                     tol=1e-6):
    """Fixed lopsided A (U[0,1] times log-uniform column scales, FP32) with k RHS
    whose x_true has a random support size in [support] and Exp(1) values;
    b = A x_true + 1% noise.  ``rhs_seed`` selects a disjoint RHS stream so the
    training and held-out sets share A but not right-hand sides."""
    rng = _rng(seed)
    A = np.asfortranarray(_lopsided_A(rng, d, n).astype(np.float32))
    r2 = _rng(seed if rhs_seed is None else rhs_seed)
    if rhs_seed is None:
        r2 = rng
    X = np.zeros((k, n))
    for c in range(k):
        m = int(r2.integers(support[0], support[1] + 1))
        idx = r2.permutation(n)[:m]
        X[c, idx] = r2.exponential(1.0, m)
    B = _noisy_rhs(r2, A.astype(np.float64), X, 0.01).astype(np.float32)
    return Problem(A, np.ascontiguousarray(B), X, tol, "warmstart_family",
                   {"d": d, "n": n, "k": k, "dtype": "f32"})


def warmstart_family_device(d=8000, n=2000, k=1024, support=(50, 400), seed=1005,
                            rhs_seed=None, device="cuda"):
    """The warm-start family with its right-hand sides formed on a torch
    device, for training sets of hundreds of thousands of columns (the numpy
    path's dense FP64 product takes minutes there).  A is the numpy path's
    for the same seed (bit for bit).  The supports and values of x_true come
    from the same numpy stream as the numpy path; b = A x_true is formed in
    FP32 on the device and the 1% noise (standard deviation 0.01·‖Ax‖/√d per
    column) from a torch generator seeded from the stream, so the columns
    follow the same recipe but are not bitwise the numpy path's.  Returns
    (A as numpy FP32 Fortran, B as a (k, d) FP32 device tensor)."""
    import torch
    rng = _rng(seed)
    A = np.asfortranarray(_lopsided_A(rng, d, n).astype(np.float32))
    r2 = rng if rhs_seed is None else _rng(rhs_seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(r2.integers(0, 2 ** 62)))
    At = torch.from_numpy(np.ascontiguousarray(A.T)).to(device)      # (n, d)
    B = torch.empty((k, d), dtype=torch.float32, device=device)
    step = 16384
    top = support[1]
    for c0 in range(0, k, step):
        kc = min(step, k - c0)
        # support: the m smallest of n uniform keys per column (a uniform
        # random m-subset), values Exp(1)
        sizes = r2.integers(support[0], support[1] + 1, size=kc)
        keys = r2.random((kc, n))
        part = np.argpartition(keys, top - 1, axis=1)[:, :top]
        order = np.take_along_axis(part, np.argsort(np.take_along_axis(keys, part, 1), 1), 1)
        vals = r2.exponential(1.0, (kc, top))
        take = np.arange(top)[None, :] < sizes[:, None]
        X = np.zeros((kc, n), dtype=np.float32)
        rows = np.broadcast_to(np.arange(kc)[:, None], order.shape)
        X[rows[take], order[take]] = vals[take]
        Xc = torch.from_numpy(X).to(device)
        clean = Xc @ At
        scale = 0.01 * torch.linalg.vector_norm(clean, dim=1, keepdim=True) / np.sqrt(d)
        noise = torch.randn(clean.shape, generator=gen, device=device, dtype=torch.float32)
        B[c0:c0 + kc] = clean + scale * noise
    return A, B


# §5, Table 1: the six test-case kinds — sign of A and x* (+ non-negative,
# ± mixed) and the lengths of the vectors A_k (SAM same, RAN random, VAR
# various).
TCASES = {
    "T1": ("+", "SAM"), "T2": ("±", "RAN"), "T3": ("+", "VAR"),
    "T4": ("±", "SAM"), "T5": ("+", "RAN"), "T6": ("±", "VAR"),
}
TCASE_SPARSITY = (0.0, 0.1, 0.2, 0.3, 0.4)   # the five sub-tests of each case


def tcase(kind="T1", sub=0, n=4000, d=6000, seed=1006, dtype=np.float32):
    """One sub-test of the paper's test-case design (§5, Table 1): n = 4000,
    d = 1.5n, b = A x* with no noise.

    Readings (the paper prints the design, not the generator):
      * entries of A and x*: U[0, 1] for "+", U[−1, 1] for "±";
      * sparsity of sub-test ``sub`` (0…4): 0, 10, …, 40% of the entries of
        every column A_k and of x* set to zero;
      * the vectors A_k are the columns (Table 1 indexes them by k, and the
        method's scaling acts on column lengths): SAM rescales every column
        to length 1, RAN to a length U(0, 1], VAR to 10^U[−1, 1] (two
        decades: the lopsided case the scaling is for).  A column left all
        zero by the sparsity stays zero.
    Problem p's draws come from seed·100003 + 10·case + sub."""
    sign, length = TCASES[kind]
    frac = TCASE_SPARSITY[sub]
    rng = _rng(seed * 100003 + 10 * int(kind[1]) + sub)
    if sign == "+":
        A = rng.random((d, n))
        x = rng.random(n)
    else:
        A = rng.uniform(-1.0, 1.0, (d, n))
        x = rng.uniform(-1.0, 1.0, n)
    if frac > 0.0:
        A[rng.random((d, n)) < frac] = 0.0
        x[rng.random(n) < frac] = 0.0
    norms = np.linalg.norm(A, axis=0)
    if length == "SAM":
        target = np.ones(n)
    elif length == "RAN":
        target = 1.0 - rng.random(n)               # (0, 1]
    else:
        target = 10.0 ** rng.uniform(-1.0, 1.0, n)
    scale = np.where(norms > 0.0, target / np.where(norms > 0.0, norms, 1.0), 0.0)
    A = np.asfortranarray((A * scale[None, :]).astype(dtype))
    b = A.astype(np.float64) @ x                   # b = A x* for the A returned
    return Problem(A, np.ascontiguousarray(b.astype(dtype))[None, :], x[None, :], 1e-6,
                   f"{kind}_s{int(round(frac * 100))}",
                   {"d": d, "n": n, "kind": kind, "sign": sign, "length": length,
                    "sparsity": frac, "dtype": np.dtype(dtype).name})


def nmf_matrix(m=4096, n=4096, r=64, seed=1007, noise=0.01):
    """A non-negative data matrix for NMF: V = W* H* + noise, W* (m×r) and
    H* (r×n) with 70% non-zero U[0,1] entries, Gaussian noise of ``noise`` ×
    the RMS entry of W*H*, clipped at 0; FP32, column-major.  Also returns a
    seeded non-negative start (W0, H0) of U[0,1] entries (FP64, column-major)
    scaled so that W0·H0 has V's mean."""
    rng = _rng(seed)
    Ws = rng.random((m, r)) * (rng.random((m, r)) < 0.7)
    Hs = rng.random((r, n)) * (rng.random((r, n)) < 0.7)
    V = Ws @ Hs
    V = V + noise * np.sqrt(np.mean(V * V)) * rng.standard_normal((m, n))
    V = np.asfortranarray(np.maximum(V, 0.0).astype(np.float32))
    W0 = rng.random((m, r))
    H0 = rng.random((r, n))
    c = np.sqrt(V.astype(np.float64).mean() / (W0 @ H0).mean())
    return V, np.asfortranarray(W0 * c), np.asfortranarray(H0 * c)


@dataclass
class SparseProblem:
    """An NNLS instance with A (d×n) in compressed sparse column form:
    ``col_ptr`` int64 (n+1), ``row_idx`` int32 (strictly increasing within a
    column), ``vals`` of the problem's dtype; B (k, d) as in ``Problem``."""

    d: int
    n: int
    col_ptr: np.ndarray
    row_idx: np.ndarray
    vals: np.ndarray
    B: np.ndarray
    x_true: np.ndarray
    tol: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_ptr[-1])

    def dense(self) -> np.ndarray:
        """The same matrix stored densely (Fortran order, the values' dtype)."""
        A = np.zeros((self.d, self.n), dtype=self.vals.dtype, order="F")
        cols = np.repeat(np.arange(self.n), np.diff(self.col_ptr))
        A[self.row_idx, cols] = self.vals
        return A


def to_csc(A) -> tuple:
    """(col_ptr, row_idx, vals) of the non-zero entries of a dense (d, n) array."""
    n = A.shape[1]
    col_ptr = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        nz = np.flatnonzero(A[:, j])
        rows.append(nz.astype(np.int32))
        vals.append(np.asarray(A[nz, j]))
        col_ptr[j + 1] = col_ptr[j] + nz.size
    return col_ptr, np.concatenate(rows), np.concatenate(vals).astype(A.dtype)


def banded_tall(d=200000, n=5000, band=6000, density=0.1, zero_frac=0.7, seed=1008, tol=1e-6,
                dtype=np.float32):
    """A tall sparse A whose columns' supports drift down the rows: column j
    holds round(density·band) entries at distinct random rows of the window
    [r_j, r_j + band), r_j = round(j·(d − band)/(n − 1)) — the structure of a
    design matrix of local, overlapping features (e.g. shifted copies of a
    kernel in a deconvolution).  Values U(0, 1] times a log-uniform column
    factor in [10⁻², 10²] (lopsided, as in ``lopsided_single``); x_true 70%
    zeros with Exp(1) non-zeros; b = A x_true + 1% Gaussian noise."""
    rng = _rng(seed)
    per = max(1, int(round(density * band)))
    col_ptr = np.arange(n + 1, dtype=np.int64) * per
    row_idx = np.empty(n * per, np.int32)
    vals = np.empty(n * per, np.float64)
    scale = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), size=n))
    for j in range(n):
        r0 = int(round(j * (d - band) / max(n - 1, 1)))
        rows = np.sort(rng.choice(band, size=per, replace=False)) + r0
        row_idx[j * per:(j + 1) * per] = rows
        vals[j * per:(j + 1) * per] = (1.0 - rng.random(per)) * scale[j]
    vals = vals.astype(dtype)
    x = _sparse_rows(rng, 1, n, zero_frac, lambda s: rng.exponential(1.0, s))
    cols = np.repeat(np.arange(n), per)
    clean = np.bincount(row_idx, weights=vals.astype(np.float64) * x[0, cols], minlength=d)
    b = clean + 0.01 * np.linalg.norm(clean) / np.sqrt(d) * rng.standard_normal(d)
    return SparseProblem(d, n, col_ptr, row_idx, vals, np.ascontiguousarray(b.astype(dtype))[None, :],
                         x, tol, "banded_tall",
                         {"d": d, "n": n, "band": band, "density": density, "nnz": n * per,
                          "dtype": np.dtype(dtype).name})


CONFIGS = {
    "uniform_small_1000x200_f64": uniform_small,
    "lopsided_single_20000x5000_f32": lopsided_single,
    "shared_multi_rhs_10000x1000_k4096_f32": shared_multi_rhs,
    "uneven_batch_512": uneven_batch,
    "warmstart_8000x2000": warmstart_family,
}
