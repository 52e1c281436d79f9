"""Thin ctypes binding of libaln (include/aln.h).

The functions keep the C names and do argument marshalling only: every step of
the solver runs in the CUDA library.  Array arguments may be torch tensors
(device or host) or numpy arrays; their data pointers are passed through.
Loading fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libaln.so")

OK = 0
ERR_INVALID_ARG, ERR_NOT_PREPARED, ERR_NONFINITE = 1, 2, 3
ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = 4, 5, 6, 7
PREC_FP64, PREC_SPLIT_BF16 = 0, 1
ALG_ANTILOP, ALG_ANTI_ACC = 0, 1
DTYPE_F32, DTYPE_F64 = 0, 1
RHS_CONVERGED, RHS_EMPTY_PASSIVE, RHS_CURVATURE = 0, 1, 2
RHS_MAXITER, RHS_NONFINITE, RHS_STAGNATED = 3, 4, 5

# Every symbol include/aln.h declares (checked by the CPU test suite).
EXPORTS = (
    "aln_default_options", "aln_create", "aln_prepare", "aln_solve", "aln_kkt_residual",
    "aln_export_scaled", "aln_get_stats", "aln_destroy", "aln_status_string", "aln_version",
    "aln_kkt_residual_noalloc", "aln_prepare_grouped", "aln_default_train_opts",
    "aln_warmstart_init", "aln_warmstart_params", "aln_warmstart_grad", "aln_warmstart_train",
    "aln_warmstart_predict", "aln_nmf", "aln_prepare_csc", "aln_set_wait_limit",
    "aln_l2_read_bandwidth",
)


class AlnOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_refine", ctypes.c_int32),
                ("persist_blocks", ctypes.c_int32), ("row_groups", ctypes.c_int32),
                ("stagnation", ctypes.c_int32), ("iter_kernel", ctypes.c_int32),
                ("batch_min", ctypes.c_int32), ("refine_gain", ctypes.c_int32),
                ("gram_split", ctypes.c_int32), ("group_cluster", ctypes.c_int32),
                ("algorithm", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("test_barrier_skew", ctypes.c_int32), ("group_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("autotune_cache", ctypes.c_char_p)]


class AlnSolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("refine_rounds", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rel_kkt", ctypes.c_double), ("objective", ctypes.c_double)]


class AlnStats(ctypes.Structure):
    _fields_ = [("prepare_ms", ctypes.c_double), ("gram_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("kkt_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("iterate_ms", ctypes.c_double), ("passive_rows", ctypes.c_int64),
                ("clipped_rows", ctypes.c_int64), ("persist_blocks", ctypes.c_int32),
                ("clipped_iterations", ctypes.c_int32), ("phase_us", ctypes.c_double * 5),
                ("product_bytes", ctypes.c_double), ("lipschitz", ctypes.c_double),
                ("power_products", ctypes.c_int64), ("iter_kernel", ctypes.c_int32),
                ("reserved2", ctypes.c_int32)]


class AlnProblem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("d", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64)]


class AlnTrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("hidden", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("seed", ctypes.c_uint64)]


class AlnError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where} failed: {status_string(code)} ({code})")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libaln (once).  Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libaln is not built ({p} missing); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    lib.aln_default_options.argtypes = [ctypes.POINTER(AlnOptions)]
    lib.aln_default_options.restype = None
    lib.aln_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(AlnOptions), vp]
    lib.aln_create.restype = ctypes.c_int
    lib.aln_prepare.argtypes = [vp, vp, i64, i64, i64, i32, vp, i64, i64]
    lib.aln_prepare.restype = ctypes.c_int
    lib.aln_prepare_csc.argtypes = [vp, i64, i64, vp, vp, vp, i32, vp, i64, i64]
    lib.aln_prepare_csc.restype = ctypes.c_int
    lib.aln_solve.argtypes = [vp, ctypes.c_double, i32, dp, i64, dp, ctypes.POINTER(AlnSolveInfo)]
    lib.aln_solve.restype = ctypes.c_int
    lib.aln_kkt_residual.argtypes = [vp, dp, i64, dp, dp]
    lib.aln_kkt_residual.restype = ctypes.c_int
    lib.aln_export_scaled.argtypes = [vp, dp, i64, dp, i64, dp]
    lib.aln_export_scaled.restype = ctypes.c_int
    lib.aln_get_stats.argtypes = [vp, ctypes.POINTER(AlnStats)]
    lib.aln_get_stats.restype = ctypes.c_int
    lib.aln_destroy.argtypes = [vp]
    lib.aln_destroy.restype = None
    lib.aln_status_string.argtypes = [ctypes.c_int]
    lib.aln_status_string.restype = ctypes.c_char_p
    lib.aln_version.argtypes = []
    lib.aln_version.restype = i32
    lib.aln_kkt_residual_noalloc.argtypes = [vp, i64, i64, i64, i32, vp, dp, dp, vp]
    lib.aln_kkt_residual_noalloc.restype = ctypes.c_int
    lib.aln_prepare_grouped.argtypes = [vp, i32, ctypes.POINTER(AlnProblem), i32]
    lib.aln_prepare_grouped.restype = ctypes.c_int
    lib.aln_default_train_opts.argtypes = [ctypes.POINTER(AlnTrainOpts)]
    lib.aln_default_train_opts.restype = None
    lib.aln_warmstart_init.argtypes = [vp, i32, ctypes.c_uint64]
    lib.aln_warmstart_init.restype = ctypes.c_int
    lib.aln_warmstart_params.argtypes = [vp, i32] + [vp] * 13
    lib.aln_warmstart_params.restype = ctypes.c_int
    lib.aln_warmstart_grad.argtypes = [vp, dp, dp, i64, dp] + [vp] * 8
    lib.aln_warmstart_grad.restype = ctypes.c_int
    lib.aln_warmstart_train.argtypes = [vp, dp, dp, i64, ctypes.POINTER(AlnTrainOpts), dp]
    lib.aln_warmstart_train.restype = ctypes.c_int
    lib.aln_warmstart_predict.argtypes = [vp, dp, i64, vp]
    lib.aln_warmstart_predict.restype = ctypes.c_int
    lib.aln_nmf.argtypes = [vp, vp, i64, i64, i64, i64, dp, i64, dp, i64, i32, ctypes.c_double,
                            i32, dp]
    lib.aln_nmf.restype = ctypes.c_int
    lib.aln_set_wait_limit.argtypes = [vp, i32, i32]
    lib.aln_set_wait_limit.restype = ctypes.c_int
    lib.aln_l2_read_bandwidth.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_double)]
    lib.aln_l2_read_bandwidth.restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().aln_status_string(code).decode()
    except Exception:  # pragma: no cover - only for messages
        return f"status {code}"


def _check(code: int, where: str):
    if code != OK:
        raise AlnError(code, where)


def _ptr(a):
    """Raw data pointer of a torch tensor or numpy array (None → NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _dtype_code(a) -> int:
    name = str(a.dtype)
    if name.endswith("float64"):
        return DTYPE_F64
    if name.endswith("float32"):
        return DTYPE_F32
    raise ValueError(f"unsupported dtype {a.dtype}")


# ------------------------------------------------------------------ C-named calls
def aln_default_options() -> AlnOptions:
    o = AlnOptions()
    load().aln_default_options(ctypes.byref(o))
    return o


def aln_create(opt: AlnOptions | None = None, stream: int | None = None) -> int:
    ctx = ctypes.c_void_p()
    _check(load().aln_create(ctypes.byref(ctx), ctypes.byref(opt) if opt is not None else None,
                             stream or None), "aln_create")
    return ctx.value


def aln_prepare(ctx, A, d, n, lda, dtype, B, k, ldb) -> None:
    _check(load().aln_prepare(ctx, _ptr(A), d, n, lda, dtype, _ptr(B), k, ldb), "aln_prepare")


def aln_prepare_csc(ctx, d, n, col_ptr, row_idx, vals, dtype, B, k, ldb) -> None:
    _check(load().aln_prepare_csc(ctx, d, n, _ptr(col_ptr), _ptr(row_idx), _ptr(vals), dtype,
                                  _ptr(B), k, ldb), "aln_prepare_csc")


def aln_prepare_grouped(ctx, problems, dtype) -> None:
    """problems: a ctypes array of AlnProblem, or a sequence of AlnProblem."""
    arr = problems if isinstance(problems, ctypes.Array) else (AlnProblem * len(problems))(
        *problems)
    _check(load().aln_prepare_grouped(ctx, len(arr), arr, dtype), "aln_prepare_grouped")


def aln_solve(ctx, tol, max_iter, X, ldx, X0, k) -> list:
    info = (AlnSolveInfo * k)()
    _check(load().aln_solve(ctx, tol, max_iter, _ptr(X), ldx, _ptr(X0), info), "aln_solve")
    return list(info)


def aln_kkt_residual(ctx, X, ldx, rel, obj) -> None:
    _check(load().aln_kkt_residual(ctx, _ptr(X), ldx, _ptr(rel), _ptr(obj)), "aln_kkt_residual")


def aln_export_scaled(ctx, Q, ldq, q, ldqv, s) -> None:
    _check(load().aln_export_scaled(ctx, _ptr(Q), ldq, _ptr(q), ldqv, _ptr(s)),
           "aln_export_scaled")


def aln_default_train_opts() -> AlnTrainOpts:
    o = AlnTrainOpts()
    load().aln_default_train_opts(ctypes.byref(o))
    return o


def aln_warmstart_init(ctx, hidden, seed) -> None:
    _check(load().aln_warmstart_init(ctx, hidden, seed), "aln_warmstart_init")


def aln_warmstart_params(ctx, set_, tensors) -> None:
    _check(load().aln_warmstart_params(ctx, set_, *[_ptr(t) for t in tensors]),
           "aln_warmstart_params")


def aln_warmstart_grad(ctx, Qb, Yb, count, loss, grads) -> None:
    _check(load().aln_warmstart_grad(ctx, _ptr(Qb), _ptr(Yb), count, _ptr(loss),
                                     *[_ptr(g) for g in grads]), "aln_warmstart_grad")


def aln_warmstart_train(ctx, Qt, Yt, count, opts, epoch_loss) -> None:
    _check(load().aln_warmstart_train(ctx, _ptr(Qt), _ptr(Yt), count, ctypes.byref(opts),
                                      _ptr(epoch_loss)), "aln_warmstart_train")


def aln_nmf(ctx, V, m, n, ldv, r, W, ldw, H, ldh, outer, tol, max_iter, objective) -> None:
    _check(load().aln_nmf(ctx, _ptr(V), m, n, ldv, r, _ptr(W), ldw, _ptr(H), ldh, outer, tol,
                          max_iter, _ptr(objective)), "aln_nmf")


def aln_warmstart_predict(ctx, X0, ldx, kept) -> None:
    _check(load().aln_warmstart_predict(ctx, _ptr(X0), ldx, _ptr(kept)), "aln_warmstart_predict")


def aln_set_wait_limit(ctx, wait_limit_us, test_barrier_skew=0) -> None:
    _check(load().aln_set_wait_limit(ctx, wait_limit_us, test_barrier_skew),
           "aln_set_wait_limit")


def aln_l2_read_bandwidth(nbytes=64 << 20, reps=20) -> float:
    """Measured L2 read bandwidth of the current device (GB/s)."""
    v = ctypes.c_double()
    _check(load().aln_l2_read_bandwidth(nbytes, reps, ctypes.byref(v)), "aln_l2_read_bandwidth")
    return v.value


def aln_get_stats(ctx) -> AlnStats:
    st = AlnStats()
    _check(load().aln_get_stats(ctx, ctypes.byref(st)), "aln_get_stats")
    return st


def aln_destroy(ctx) -> None:
    if ctx:
        load().aln_destroy(ctx)


def aln_version() -> int:
    return load().aln_version()


def aln_kkt_residual_noalloc(A, d, n, lda, dtype, b, x, out, stream=None) -> None:
    """Allocation-free FP64 KKT residual of one solution (device pointers only)."""
    _check(load().aln_kkt_residual_noalloc(_ptr(A), d, n, lda, dtype, _ptr(b), _ptr(x), _ptr(out),
                                           stream or None), "aln_kkt_residual_noalloc")


# --------------------------------------------------------------- convenience class
@dataclass
class SolveInfo:
    iters: int
    status: int
    refine_rounds: int
    rel_kkt: float
    objective: float


class Solver:
    """One library context.  ``A`` is (d, n) column-major — a Fortran-ordered
    numpy array, or a torch tensor whose transpose is contiguous; ``B`` is
    (k, d) row-major (one right-hand side per row).  Inputs on the host are
    copied by the library; device inputs must stay alive while in use."""

    def __init__(self, precision: str = "split_bf16", stream=None, **opts):
        o = aln_default_options()
        o.precision = {"fp64": PREC_FP64, "split_bf16": PREC_SPLIT_BF16}[precision]
        for k, v in opts.items():
            if k == "autotune_cache" and isinstance(v, str):
                v = v.encode()
                self._cache_path = v   # keep the bytes alive with the context
            setattr(o, k, v)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        self.ctx = aln_create(o, stream)
        self.precision = precision
        self._keep = ()
        self.n = self.k = 0
        self.sizes = None  # per-problem n after prepare_grouped

    def prepare(self, A, B):
        d, n = A.shape
        lda = _col_major_ld(A)
        if B.ndim == 1:
            B = B.reshape(1, -1)
        k, dB = B.shape
        if dB != d:
            raise ValueError("B rows must have length d")
        ldb = _row_major_ld(B)
        self._keep = (A, B)
        aln_prepare(self.ctx, A, d, n, lda, _dtype_code(A), B, k, ldb)
        self.n, self.k = n, k
        self.sizes = None

    def prepare_csc(self, d, col_ptr, row_idx, vals, B):
        """A (d × n) in compressed sparse column form: col_ptr int64 (n+1),
        row_idx int32 (strictly increasing within a column), vals float32 or
        float64 — all three on the host or all on the device; B as in
        prepare."""
        n = int(col_ptr.shape[0]) - 1
        if str(col_ptr.dtype).split(".")[-1] != "int64" or \
                str(row_idx.dtype).split(".")[-1] != "int32":
            raise ValueError("col_ptr must be int64 and row_idx int32")
        if B.ndim == 1:
            B = B.reshape(1, -1)
        k, dB = B.shape
        if dB != d:
            raise ValueError("B rows must have length d")
        ldb = _row_major_ld(B)
        nnz = int(row_idx.shape[0])
        self._keep = (col_ptr, row_idx, vals, B)
        aln_prepare_csc(self.ctx, d, n, col_ptr, row_idx if nnz else None,
                        vals if nnz else None, _dtype_code(vals), B, k, ldb)
        self.n, self.k = n, k
        self.sizes = None

    @staticmethod
    def grouped_records(problems):
        """Marshal (A, b) pairs — A (d_p, n_p) column-major, b (d_p,), one dtype
        for all — into the C records once; the result can be passed to
        prepare_grouped repeatedly while the arrays stay alive."""
        recs, keep = [], []
        dtype = None
        for A, b in problems:
            d, n = A.shape
            if b.shape[-1] != d:
                raise ValueError("b must have length d")
            code = _dtype_code(A)
            if dtype is None:
                dtype = code
            elif code != dtype or _dtype_code(b) != dtype:
                raise ValueError("all problems must share one dtype")
            recs.append(AlnProblem(_ptr(A), _ptr(b), d, n, _col_major_ld(A)))
            keep.append((A, b))
        arr = (AlnProblem * len(recs))(*recs)
        return arr, dtype, [int(r.n) for r in recs], tuple(keep)

    def prepare_grouped(self, problems=None, records=None):
        """Independent problems (A_p, b_p) of uneven size in one context;
        solutions come back as a list of vectors."""
        if records is None:
            records = self.grouped_records(problems)
        arr, dtype, sizes, keep = records
        self._keep = keep
        aln_prepare_grouped(self.ctx, arr, dtype)
        self.sizes = sizes
        self.n, self.k = sum(sizes), len(sizes)

    def _split(self, X):
        out, o = [], 0
        for n in self.sizes:
            out.append(X[o:o + n])
            o += n
        return out

    def solve(self, tol=1e-6, max_iter=0, X=None, X0=None):
        if self.sizes is not None:  # grouped: packed vectors
            Xp = np.zeros(self.n) if X is None else X
            X0p = None if X0 is None else (np.concatenate(X0) if isinstance(X0, (list, tuple))
                                           else X0)
            info = aln_solve(self.ctx, tol, max_iter, Xp, self.n, X0p, self.k)
            return (self._split(Xp) if X is None else Xp,
                    [SolveInfo(i.iters, i.status, i.refine_rounds, i.rel_kkt, i.objective)
                     for i in info])
        if X is None:
            X = np.zeros((self.k, self.n))
        info = aln_solve(self.ctx, tol, max_iter, X, _row_major_ld(X), X0, self.k)
        return X, [SolveInfo(i.iters, i.status, i.refine_rounds, i.rel_kkt, i.objective)
                   for i in info]

    def kkt(self, X):
        if self.sizes is not None and isinstance(X, (list, tuple)):
            X = np.concatenate([np.asarray(x, dtype=np.float64) for x in X])
        rel = np.zeros(self.k)
        obj = np.zeros(self.k)
        ld = self.n if self.sizes is not None else _row_major_ld(X)
        aln_kkt_residual(self.ctx, X, ld, rel, obj)
        return rel, obj

    def export(self):
        if self.sizes is not None:  # grouped: per-problem blocks
            Qp = np.zeros(sum(n * n for n in self.sizes))
            q = np.zeros(self.n)
            s = np.zeros(self.n)
            aln_export_scaled(self.ctx, Qp, 0, q, 0, s)
            Qs, o = [], 0
            for n in self.sizes:
                Qs.append(Qp[o:o + n * n].reshape(n, n))
                o += n * n
            return Qs, self._split(q), self._split(s)
        Q = np.zeros((self.n, self.n))
        q = np.zeros((self.k, self.n))
        s = np.zeros(self.n)
        aln_export_scaled(self.ctx, Q, self.n, q, self.n, s)
        return Q, q, s

    def set_wait_limit(self, wait_limit_us, test_barrier_skew=0):
        aln_set_wait_limit(self.ctx, wait_limit_us, test_barrier_skew)

    def stats(self) -> AlnStats:
        return aln_get_stats(self.ctx)

    # ------------------------------------------------------------ warm start
    def warmstart_shapes(self, hidden):
        n2 = 2 * self.n
        return [(hidden, n2), (hidden,), (hidden, hidden), (hidden,), (n2, hidden), (n2,),
                (self.n,), (self.n,)]

    def warmstart_init(self, hidden=1024, seed=0):
        aln_warmstart_init(self.ctx, hidden, seed)
        self.hidden = hidden

    _WS_PARAMS = ("W1", "b1", "W2", "b2", "W3", "b3", "e", "f")
    _WS_KEYS = _WS_PARAMS + ("mu", "sd", "muz", "sdz", "tau")

    def warmstart_set(self, params):
        """params: dict with any of W1, b1, W2, b2, W3, b3, e, f (oracle
        shapes), mu, sd, muz, sdz (n) and tau (scalar); missing keys are left
        as they are."""
        ts = []
        for k in self._WS_KEYS:
            v = params.get(k)
            ts.append(None if v is None else
                      np.ascontiguousarray(np.atleast_1d(v), dtype=np.float32))
        aln_warmstart_params(self.ctx, 1, ts)

    def warmstart_get(self):
        shapes = self.warmstart_shapes(self.hidden) + [(self.n,)] * 4 + [(1,)]
        ts = [np.zeros(sh, np.float32) for sh in shapes]
        aln_warmstart_params(self.ctx, 0, ts)
        out = dict(zip(self._WS_KEYS, ts))
        out["tau"] = float(out["tau"][0])
        return out

    def warmstart_grad(self, Qb, Yb):
        Qb = np.ascontiguousarray(Qb, dtype=np.float64)
        Yb = np.ascontiguousarray(Yb, dtype=np.float64)
        loss = np.zeros(1)
        gs = [np.zeros(sh, np.float32) for sh in self.warmstart_shapes(self.hidden)]
        aln_warmstart_grad(self.ctx, Qb, Yb, Qb.shape[0], loss, gs)
        return float(loss[0]), dict(zip(self._WS_PARAMS, gs))

    def warmstart_train(self, Qt, Yt, **opts):
        o = aln_default_train_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        self.hidden = o.hidden if not hasattr(self, "hidden") else self.hidden
        if isinstance(Qt, np.ndarray):
            Qt = np.ascontiguousarray(Qt, dtype=np.float64)
            Yt = np.ascontiguousarray(Yt, dtype=np.float64)
        hist = np.zeros(max(o.epochs, 1))
        aln_warmstart_train(self.ctx, Qt, Yt, Qt.shape[0], o, hist)
        return hist[:o.epochs]

    def warmstart_predict(self, X0=None):
        if X0 is None:
            X0 = np.zeros((self.k, self.n))
        kept = np.zeros(self.k, np.int32)
        aln_warmstart_predict(self.ctx, X0, _row_major_ld(X0), kept)
        return X0, kept

    def nmf(self, V, W0, H0, outer=10, tol=1e-6, max_iter=0):
        """V ≈ W·H by alternating NNLS (aln_nmf).  V (m, n) float32 and the
        starts W0 (m, r), H0 (r, n) float64 are column-major (Fortran numpy
        arrays or transposed-contiguous tensors).  Returns (W, H, objective
        after each outer iteration); W0 and H0 are not modified."""
        m, n = V.shape
        r = W0.shape[1]
        if W0.shape[0] != m or H0.shape != (r, n):
            raise ValueError("W0 must be (m, r) and H0 (r, n)")
        if isinstance(W0, np.ndarray):
            W = np.asfortranarray(W0, dtype=np.float64).copy(order="F")
            H = np.asfortranarray(H0, dtype=np.float64).copy(order="F")
        else:
            W = W0.detach().t().contiguous().t().clone()
            H = H0.detach().t().contiguous().t().clone()
        obj = np.zeros(outer)
        self._keep = (V, W, H)
        aln_nmf(self.ctx, V, m, n, _col_major_ld(V), r, W, _col_major_ld(W), H,
                _col_major_ld(H), outer, tol, max_iter, obj)
        self.n, self.k = r, m
        self.sizes = None
        return W, H, obj

    def close(self):
        aln_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        if getattr(self, "ctx", None):
            try:
                self.close()
            except Exception:
                pass


def _col_major_ld(A) -> int:
    """Leading dimension of a (d, n) column-major array (stride of dim 1)."""
    if isinstance(A, np.ndarray):
        s0, s1 = A.strides[0] // A.itemsize, A.strides[1] // A.itemsize
    else:
        s0, s1 = A.stride()
    if A.shape[1] == 1:
        if s0 != 1 and A.shape[0] > 1:
            raise ValueError("A must be column-major (Fortran order / transposed contiguous)")
        return max(s1, A.shape[0])
    if s0 != 1:
        raise ValueError("A must be column-major (Fortran order / transposed contiguous)")
    return s1


def _row_major_ld(B) -> int:
    if B.size == 0:
        return max(1, B.shape[-1])
    if isinstance(B, np.ndarray):
        s0, s1 = B.strides[0] // B.itemsize, B.strides[1] // B.itemsize
    else:
        s0, s1 = B.stride()
    if s1 != 1:
        raise ValueError("rows must be contiguous")
    return s0 if B.shape[0] > 1 else max(s0, B.shape[1])
