/*
 * aln.h — C ABI of the anti-lopsided NNLS library (libaln).
 *
 * Solves the non-negative least squares problem of Def. 1 (§2.1, Eq. NNL):
 *
 *     minimise ½‖A x − b‖²   subject to  x ⪰ 0,   A ∈ R^{d×n}, b ∈ R^d,
 *
 * by the paper's anti-lopsided method:
 *   Alg. 1 (§3):  H = AᵀA, h = −Aᵀb (Eq. NQP), rescale to the unit-diagonal
 *                 problem Q_ij = H_ij/√(H_ii H_jj), q_i = h_i/√H_ii (Eq. NQPQ),
 *                 solve it, then x_i = y_i/√H_ii (Eq. Rescaling).
 *   Alg. 2 (§3):  projected gradient with exact line search on (Q, q):
 *                 passive set P = {y_i > 0 or g_i < 0}, ḡ = g on P,
 *                 α = ‖ḡ‖²/(ḡᵀQḡ), y ← [y − αḡ]₊, g ← g + Q(y_new − y).
 *
 * Also: the Anti+Acc variant of §5 (aln_options.algorithm), non-negative
 * matrix factorisation by alternating NNLS on the multi-RHS solver (aln_nmf),
 * and a learned start point for families of right-hand sides that share A
 * (aln_warmstart_*).
 *
 * Sign convention: q is the paper's, q = −D⁻¹Aᵀb with D = diag(‖A_i‖), so the
 * gradient of ½yᵀQy + qᵀy is g = Qy + q.
 *
 * Memory: every pointer argument may be device memory or host memory; the
 * library detects which (cudaPointerGetAttributes) and copies host data
 * through its own device buffers.  Matrices are column-major: element (t, i)
 * of A is A[t + i*lda]; right-hand side c is B[c*ldb + t]; solution c is
 * X[c*ldx + i].  The caller owns A, B, X and X0.  The context owns every
 * derived array (scale factors, Q, q, split copies of A, iteration state).
 *
 * Lifetime: when A was passed as a DEVICE pointer, the context keeps that
 * pointer (it is needed for the FP64 KKT evaluation and refinement) and the
 * caller must keep A and B alive and unchanged until the last aln_solve or
 * aln_kkt_residual on this context returns.  Host inputs are copied.
 *
 * Streams: all work is ordered on the stream given to aln_create (NULL means
 * the legacy default stream).  Calls return after the work they launched has
 * finished on that stream, because the solve loop reads convergence flags on
 * the host.
 *
 * Errors: every call returns an aln_status; no C++ exception crosses this
 * boundary.  After ALN_ERR_CUDA the context should be destroyed.
 * Thread safety: a context must not be used from two threads at once.
 */
#ifndef ALN_H
#define ALN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ALN_VERSION 201

typedef enum aln_status {
    ALN_OK = 0,
    ALN_ERR_INVALID_ARG = 1,   /* null pointer, negative size, ld too small, bad enum */
    ALN_ERR_NOT_PREPARED = 2,  /* aln_solve / aln_kkt_residual before aln_prepare */
    ALN_ERR_NONFINITE = 3,     /* NaN or Inf found in A, B or X0 */
    ALN_ERR_OUT_OF_MEMORY = 4, /* a workspace allocation failed */
    ALN_ERR_CUDA = 5,          /* a CUDA runtime call or kernel launch failed */
    ALN_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    ALN_ERR_UNSUPPORTED = 7    /* combination not built (e.g. no sm_103a device) */
} aln_status;

/* Arithmetic of the Gram formation and the iteration. */
typedef enum aln_precision {
    /* H = AᵀA in FP64, Alg. 2 in FP64: the plain method. */
    ALN_PREC_FP64 = 0,
    /* H from tensor-core products of the exact three-term BF16 split of A
     * (a = h + m + l; hh + hm + mh + mm + hl + lh, FP32 accumulation), Alg. 2 in
     * FP32, scale factors / KKT / refinement in FP64.  With many right-hand
     * sides the scaled matrix comes from an FP64-accurate (Dot2) product. */
    ALN_PREC_SPLIT_BF16 = 1
} aln_precision;

typedef enum aln_dtype { ALN_DTYPE_F32 = 0, ALN_DTYPE_F64 = 1 } aln_dtype;

/* Solver run after the scaling of Alg. 1 (§3). */
typedef enum aln_algorithm {
    /* Alg. 2 (§3): projected gradient on the passive set with the exact line
     * search α = ‖ḡ‖²/ḡᵀQḡ (the paper's method; default). */
    ALN_ALG_ANTILOP = 0,
    /* Anti+Acc (§5): Nesterov's accelerated projected gradient with the
     * constant step 1/L, L = λ_max(Q) from a power iteration; the paper names
     * it as a compared variant without printing its update rule, which is
     * read as the optimal gradient method it cites (Guan et al., 2012):
     * x_k = [Y_k − ∇f(Y_k)/L]₊, α_{k+1} = (1 + √(4α_k² + 1))/2,
     * Y_{k+1} = x_k + ((α_k − 1)/α_{k+1})(x_k − x_{k−1}), α_0 = 1.  Same stop
     * rule and FP64 refinement as Alg. 2 (a refinement round restarts the
     * momentum); since ‖ḡ‖ of this method is not monotone, an FP32 inner run
     * takes 10 × stagnation iterations without a new best ‖ḡ‖² to stagnate,
     * and the FP64 iteration never stagnates.  Single-problem path only (aln_prepare with fewer than
     * batch_min right-hand sides, or FP64), and only while x_k, x_{k−1}, both
     * gradients (and in SPLIT_BF16 the low parts of the double-float x and
     * the step) fit in one SM's shared memory (n up to about 7 500 in
     * SPLIT_BF16, 6 000 in FP64); otherwise aln_solve returns
     * ALN_ERR_UNSUPPORTED. */
    ALN_ALG_ANTI_ACC = 1
} aln_algorithm;

/* Per right-hand-side outcome, reported in aln_solve_info.status. */
typedef enum aln_rhs_status {
    ALN_RHS_CONVERGED = 0,     /* ‖ḡ‖ ≤ tol·‖min(q,0)‖ in the FP64 check */
    ALN_RHS_EMPTY_PASSIVE = 1, /* P(y) = ∅: y is a KKT point (Alg. 2 stop rule) */
    ALN_RHS_CURVATURE = 2,     /* ḡᵀQḡ ≤ 0 with ḡ ≠ 0: numerically converged */
    ALN_RHS_MAXITER = 3,       /* max_iter reached; X holds the last iterate */
    ALN_RHS_NONFINITE = 4,     /* the iteration produced NaN/Inf */
    ALN_RHS_STAGNATED = 5      /* no new smallest ‖ḡ‖² within the stagnation window and
                                  the FP64 check still above tol (the paper's
                                  experimental stop rule, §5) */
} aln_rhs_status;

typedef struct aln_options {
    int32_t precision;    /* aln_precision */
    int32_t max_refine;   /* FP64 refinement rounds after the first FP32
                             convergence (SPLIT_BF16 only); default 8 */
    int32_t persist_blocks; /* blocks of the persistent Alg. 2 kernel; 0 = one
                             per SM (capped by co-residency and work items) */
    int32_t row_groups;   /* row groups of the single-RHS matvec; 0 = auto */
    int32_t stagnation;   /* stop an inner run after this many iterations without a
                             new smallest ‖ḡ‖² (§5 stop rule); 0 = default 100 */
    int32_t iter_kernel;  /* persistent Alg. 2 kernel: 0 auto (FP64 with n up to
                             about 460: one thread-block cluster holding Q in
                             shared memory; else replicated state when the
                             vectors fit in shared memory; else tiled),
                             1 tiled, 2 replicated, 3 one cluster (FP64 only,
                             falls back to 0's choice where Q does not fit) */
    int32_t batch_min;    /* SPLIT_BF16 with at least this many right-hand sides
                             runs the batched solver (all columns advance together,
                             tcgen05 products Q·Ḡ); 0 = default 8 */
    int32_t refine_gain;  /* progressive refinement: each inner FP32 run stops
                             when its relative KKT residual is this many decades
                             below the last FP64 one (the first run: below 1),
                             but not below tol/2 (first run) or tol/4 (later
                             runs); < 0 = every run aims at tol; 0 = automatic:
                             3 for the batched solver, off for the single-problem
                             and grouped solvers (measured fastest on each) */
    int32_t gram_split;   /* BF16 terms of the split-BF16 Gram: 3 = exact split of
                             the FP32 input (six products), 2 = h + m (three
                             products, half the tensor work); 0 = default 3 */
    int32_t group_cluster; /* grouped solver: blocks of the thread-block cluster
                             that solves each large problem (n ≥ 512 and Q_p
                             larger than one block's shared memory) while
                             single blocks take the rest; 1 = no clusters, 2, 4
                             or 8; 0 = default 4 */
    int32_t algorithm;    /* aln_algorithm; default ALN_ALG_ANTILOP */
    int32_t wait_limit_us; /* limit of one device-side wait of the persistent
                             solver kernels (a grid barrier), in microseconds;
                             when it expires the kernel stops every block,
                             leaves no work in flight and aln_solve returns
                             ALN_ERR_TIMEOUT (the context stays usable);
                             0 = default 2 000 000 (2 s) */
    int32_t test_barrier_skew; /* FOR TESTS ONLY, 0 in normal use: every grid
                             barrier of the persistent solver kernels waits for
                             this many arrivals more than the grid provides, so
                             the first wait expires after wait_limit_us and the
                             timeout path runs (no fault, no hang); must be
                             0..1024 */
    int32_t group_graph;  /* grouped solver: 1 = run each aln_solve as one CUDA graph
                             (captured on the first solve of a layout, replayed by
                             later ones with the same tol, max_iter and start
                             kind): the refinement rounds become max_refine fixed
                             rounds that pass over finished problems, with the same
                             results problem by problem; 0 = host-driven rounds */
    int32_t autotune;     /* launch geometry chosen per shape by measurement, kept
                             in the JSON file autotune_cache: 0 off; 1 use the
                             cached choice of the shape (the options above
                             where there is none); 2 as 1, and on a miss the
                             first aln_solve of the shape measures the
                             candidates (whole solves, or a 64-iteration probe
                             for one problem), records the fastest and then
                             solves.  Tuned per shape: blocks and row groups of
                             the persistent Alg. 2 kernel (one problem),
                             group_cluster (grouped problems), the batched
                             solver's iterations per captured chunk and its
                             hand-off of the last running columns; an autotuned
                             choice replaces persist_blocks and group_cluster.
                             Results remain Alg. 2's; only the geometry moves */
    const char* autotune_cache; /* path of the JSON cache file (copied by aln_create;
                             required when autotune > 0, else
                             ALN_ERR_INVALID_ARG); written by renaming a
                             temporary file next to it */
} aln_options;

typedef struct aln_solve_info {
    int32_t iters;         /* Alg. 2 iterations, summed over refinement rounds */
    int32_t status;        /* aln_rhs_status */
    int32_t refine_rounds; /* FP64 refinement rounds used */
    int32_t reserved;
    double rel_kkt;        /* FP64 relative KKT residual ‖ḡ‖/‖min(q,0)‖ from A */
    double objective;      /* ½‖A x − b‖² in FP64 */
} aln_solve_info;

typedef struct aln_ctx aln_ctx;

/* Fill *opt with the defaults (precision SPLIT_BF16, max_refine 8, automatic
 * persistent grid and row groups, stagnation window 100). */
void aln_default_options(aln_options* opt);

/* Create a context on the current CUDA device.  `stream` is a cudaStream_t
 * (NULL = legacy default stream).  opt may be NULL (defaults).
 * Errors: INVALID_ARG (ctx NULL or bad option), UNSUPPORTED (device is not
 * compute capability 10.3 when precision is SPLIT_BF16), CUDA. */
aln_status aln_create(aln_ctx** ctx, const aln_options* opt, void* stream);

/* Alg. 1 up to the solve: scale factors s_i = ‖A_i‖ (FP64; s_i := 1 for a zero
 * column, Eq. Rescaling's special case), Q = D⁻¹AᵀAD⁻¹ (Eq. NQPQ) and
 * q_c = −D⁻¹Aᵀb_c for each of the k right-hand sides.
 *   A    d×n, column-major, leading dimension lda ≥ d, dtype aln_dtype.
 *   B    k right-hand sides, B[c*ldb + t], ldb ≥ d, same dtype as A.
 * Requires d ≥ 1, n ≥ 1, k ≥ 1.  SPLIT_BF16 requires dtype F32 or F64 (F64 is
 * rounded to F32 before splitting).  Errors: INVALID_ARG, NONFINITE (NaN/Inf
 * in A or B), OUT_OF_MEMORY, CUDA. */
aln_status aln_prepare(aln_ctx* ctx, const void* A, int64_t d, int64_t n, int64_t lda,
                       int32_t dtype, const void* B, int64_t k, int64_t ldb);

/* Alg. 1 as aln_prepare, for A given in compressed sparse column form:
 *   col_ptr  n+1 offsets (int64): column j holds entries col_ptr[j] ≤ t <
 *            col_ptr[j+1]; col_ptr[0] = 0, non-decreasing, nnz = col_ptr[n].
 *   row_idx  nnz row indices (int32), in [0, d), strictly increasing within a
 *            column (no duplicates).
 *   vals     nnz values of dtype aln_dtype.
 *   B        k right-hand sides as in aln_prepare (dense).
 * The three CSC arrays are all host memory or all device memory; row_idx and
 * vals may be NULL when nnz = 0.  Only the stored entries are read: the column
 * statistics and Aᵀb come from them, and with SPLIT_BF16 and a single-RHS
 * solver the Gram multiplies, per pair of 128-column tiles, only the 64-row
 * blocks stored in both — the Q of the dense matrix up to the grouping of its
 * FP32 sums, for work proportional to the occupied block pairs.  With F32
 * values, SPLIT_BF16, a single-RHS solver and k ≤ 4, no dense copy of A is
 * made: the FP64 KKT pass reads the CSC arrays and the packed blocks (whose
 * split terms add up exactly to the entries), so device CSC arrays are kept
 * by pointer and must stay valid until the next prepare or aln_destroy.  Otherwise (F64 values, FP64
 * precision, the many-right-hand-side solver, k > 4) a dense column-major copy
 * of A (d·n elements) is made on the device.  The call synchronises the
 * stream twice (structure check; sizing of the packed blocks).  Afterwards
 * the context is prepared as by aln_prepare.
 * Errors: INVALID_ARG (also a malformed structure), NONFINITE, OUT_OF_MEMORY,
 * TIMEOUT, CUDA. */
aln_status aln_prepare_csc(aln_ctx* ctx, int64_t d, int64_t n, const int64_t* col_ptr,
                           const int32_t* row_idx, const void* vals, int32_t dtype,
                           const void* B, int64_t k, int64_t ldb);

/* One problem of a grouped batch: min ½‖A x − b‖², x ⪰ 0 (Def. 1), with its
 * own A (d×n, column-major, lda ≥ d) and b (d entries).  A and b may be host
 * or device memory, independently per problem. */
typedef struct aln_problem {
    const void* A;
    const void* b;
    int64_t d, n, lda;
} aln_problem;

/* Alg. 1 for `count` independent problems of different sizes at once (one
 * Gram launch over every problem's tiles, one persistent Alg. 2 launch whose
 * blocks take problems largest first).  All problems share `dtype`.
 * Requires 1 ≤ count ≤ 2^20, and per problem d ≥ 1 and 1 ≤ n ≤ 4096 (larger
 * problems go through aln_prepare, whose solver spans the whole GPU).
 * After this call the context is in grouped mode until the next prepare:
 *   - vectors are PACKED: problem p occupies entries [o_p, o_p + n_p) of X,
 *     X0, q and s, with o_p = Σ_{r<p} n_r; ldx and ldqv are ignored;
 *   - info, rel_kkt and objective hold `count` entries, one per problem;
 *   - aln_export_scaled writes Q as packed row-major n_p×n_p blocks starting
 *     at Σ_{r<p} n_r² (ldq ignored).
 * Device inputs are kept by pointer (same lifetime rule as aln_prepare).
 * Errors: INVALID_ARG, NONFINITE, OUT_OF_MEMORY, TIMEOUT, UNSUPPORTED (no
 * sm_103a device for SPLIT_BF16), CUDA. */
aln_status aln_prepare_grouped(aln_ctx* ctx, int32_t count, const aln_problem* probs,
                               int32_t dtype);

/* Alg. 2 on every prepared right-hand side, then x = y/s (Alg. 1).
 *   tol       relative KKT tolerance: stop when ‖ḡ‖ ≤ tol·‖min(q,0)‖ (FP64,
 *             evaluated from A); must be > 0.
 *   max_iter  cap on Alg. 2 iterations per right-hand side (≤ 0: max(5n, 20000),
 *             the paper's experimental cap).
 *   X         output, FP64, X[c*ldx + i], ldx ≥ n.
 *   X0        optional start point in x-space (FP64, same layout, ≥ 0), or NULL
 *             for Alg. 2's x⁰ = 0.  Mapped to y0 = x0·s.
 *   info      optional array of k records (host memory).
 * Errors: NOT_PREPARED, INVALID_ARG, NONFINITE (X0), TIMEOUT, UNSUPPORTED
 * (ALN_ALG_ANTI_ACC outside the single-problem path, or n too large for its
 * shared-memory state), CUDA.  Hitting max_iter is not an error; it is
 * reported per right-hand side. */
aln_status aln_solve(aln_ctx* ctx, double tol, int32_t max_iter, double* X, int64_t ldx,
                     const double* X0, aln_solve_info* info);

/* FP64 KKT residual and objective of given solutions, from A directly:
 * r = Ax − b, ∇F = Aᵀr, g = ∇F/s, ḡ = g on P(s·x), rel = ‖ḡ‖/‖min(q,0)‖
 * (absolute ‖ḡ‖ when ‖min(q,0)‖ = 0), objective = ½‖r‖².
 *   X          k solutions, FP64, X[c*ldx + i].
 *   rel_kkt    k doubles out (host or device).  objective: k doubles out or NULL.
 * Errors: NOT_PREPARED, INVALID_ARG, CUDA. */
aln_status aln_kkt_residual(aln_ctx* ctx, const double* X, int64_t ldx, double* rel_kkt,
                            double* objective);

/* Copy the prepared scaled problem out as FP64 (for inspection and tests):
 *   Q  n×n, Q[i*ldq + j] (symmetric), ldq ≥ n; may be NULL.
 *   q  k×n, q[c*ldqv + i], ldqv ≥ n; may be NULL.
 *   s  n scale factors; may be NULL.
 * Errors: NOT_PREPARED, INVALID_ARG, CUDA. */
aln_status aln_export_scaled(aln_ctx* ctx, double* Q, int64_t ldq, double* q, int64_t ldqv,
                             double* s);

/* ---------------------------------------------------------------------------
 * Learned start point (not in the paper: Alg. 2 starts at x⁰ = 0 in §3, and a
 * given x⁰ maps to y⁰ = x⁰·√H_ii by Eq. Rescaling).  A network predicts y⁰ in
 * the scaled space from q for a fixed A (a fixed scaled matrix Q):
 *   z  = −Q⁻¹q, the unconstrained minimiser of ½yᵀQy + qᵀy (Q⁻¹ formed once
 *        per network on the GPU by a Newton–Schulz iteration in FP32)
 *   u  = [ (q/‖q‖ − μ)/σ ; (z/‖q‖ − μz)/σz ],  μ, σ, μz, σz per entry over
 *        the training set (both parts 0 when q = 0)
 *   h1 = relu(W1 u + b1), h2 = relu(W2 h1 + b2), [r ; ℓ′] = W3 h2 + b3
 *   ŷ  = r + e ⊙ ẑ,  ℓ = ℓ′ + f ⊙ ẑ,  ẑ = z/(τ‖q‖)  (per-entry skips)
 *   d  = relu(ŷ)·[ℓ > 0], y⁰ = α*·d with α* = max(0, −qᵀd/dᵀQd), the exact
 *        line search of Alg. 2 from 0 along d, so f(y⁰) ≤ f(0) = 0
 * W1 is hidden×2n, W2 hidden×hidden, W3 2n×hidden (row-major), e and f have
 * n entries (FP32 master copies; the layer products in BF16 on the tensor
 * cores with FP32 accumulation, z in FP32).
 * Training minimises mean (ŷ − y* / (τ‖q‖))² + mean BCE(ℓ, [y* > 0]) with
 * Adam over every parameter; τ is the RMS of y* / ‖q‖ over the training set.
 * All calls need a context prepared with aln_prepare (not grouped); the
 * network belongs to that A (its n and Q⁻¹) and survives later aln_prepare
 * calls with new right-hand sides.
 * ------------------------------------------------------------------------- */
typedef struct aln_train_opts {
    int32_t epochs;   /* passes over the training pairs; default 10 */
    int32_t batch;    /* pairs per Adam step; default 1024 */
    int32_t hidden;   /* width of both hidden layers (used when the network is
                         created by this call); default 1024 */
    int32_t reserved;
    double lr;        /* Adam step size; default 1e-3 */
    double beta1;     /* default 0.9 */
    double beta2;     /* default 0.999 */
    double eps;       /* default 1e-8 */
    uint64_t seed;    /* initial weights and shuffling; default 0 */
} aln_train_opts;

void aln_default_train_opts(aln_train_opts* opts);

/* Create (or re-create) the network for the prepared A: He-uniform weights
 * from `seed`, zero biases, skips e = 1 and f = 4 (ŷ follows ẑ and ℓ its
 * sign), and Q⁻¹ of the prepared Q (Newton–Schulz from I/‖Q‖∞ until
 * ‖I − Q·X‖_F < 1e-4 or stops falling; Q must be positive definite, as it is
 * for A of full column rank).  hidden ≥ 1.
 * Errors: INVALID_ARG, NOT_PREPARED, NONFINITE (the iteration diverged: Q
 * singular), OUT_OF_MEMORY, CUDA. */
aln_status aln_warmstart_init(aln_ctx* ctx, int32_t hidden, uint64_t seed);

/* Copy the FP32 parameters in (set = 1) or out (set = 0); any pointer may be
 * NULL to skip that tensor; host or device memory.  Shapes as above, biases
 * of length hidden, hidden, 2n, skips e, f of length n; mu, sd, muz, sdz (n
 * each) and tau (1) are the feature and target normalisation (defaults 0, 1,
 * 0, 1, 1; the first aln_warmstart_train sets them from its training set
 * unless they were set here).
 * Errors: INVALID_ARG (no network), CUDA. */
aln_status aln_warmstart_params(aln_ctx* ctx, int32_t set, float* W1, float* b1, float* W2,
                                float* b2, float* W3, float* b3, float* e, float* f, float* mu,
                                float* sd, float* muz, float* sdz, float* tau);

/* One forward and backward pass without an update, on `count` pairs:
 * Qb (count×n, the scaled q of each right-hand side, row-major FP64) and Yb
 * (count×n, the scaled solutions y* = s·x*).  Writes the loss and the
 * gradients (same shapes as the parameters; NULL skips).  For tests.
 * Errors: INVALID_ARG, TIMEOUT, OUT_OF_MEMORY, CUDA. */
aln_status aln_warmstart_grad(aln_ctx* ctx, const double* Qb, const double* Yb, int64_t count,
                              double* loss, float* gW1, float* gb1, float* gW2, float* gb2,
                              float* gW3, float* gb3, float* ge, float* gf);

/* Train on `count` pairs (Qtrain, Ytrain as in aln_warmstart_grad; host or
 * device).  Creates the network first when there is none.  epoch_loss: NULL
 * or `epochs` doubles, the mean loss of each epoch.
 * Errors: INVALID_ARG, NOT_PREPARED, TIMEOUT, OUT_OF_MEMORY, CUDA. */
aln_status aln_warmstart_train(aln_ctx* ctx, const double* Qtrain, const double* Ytrain,
                               int64_t count, const aln_train_opts* opts, double* epoch_loss);

/* Start points for the prepared right-hand sides: X0 (k×n, X0[c*ldx + i],
 * x-space, ready for aln_solve) and, when kept is not NULL, kept[c] = 1 if
 * α* > 0 and 0 if the start is 0 (the direction does not descend).
 * Errors: INVALID_ARG (no network, or n differs), NOT_PREPARED, TIMEOUT, CUDA. */
aln_status aln_warmstart_predict(aln_ctx* ctx, double* X0, int64_t ldx, int32_t* kept);

/* Non-negative matrix factorisation V ≈ W·H (W m×r ⪰ 0, H r×n ⪰ 0) by
 * alternating NNLS, the use the paper motivates its solver with (§1; §2.2 on
 * the many right-hand sides of such factorisations).  Each of `outer`
 * iterations runs Alg. 1 + Alg. 2 (this context's options: precision,
 * algorithm, refinement) twice:
 *   H-step: matrix W, the n columns of V as right-hand sides, started from
 *           the previous H;
 *   W-step: matrix Hᵀ, the m rows of V as right-hand sides, started from the
 *           previous W;
 * each sub-problem to relative KKT tolerance `tol` (max_iter per sub-problem,
 * 0 = default).  With n, m ≥ batch_min both steps take the batched solver.
 *   V         FP32, column-major m×n (V[i + j*ldv]), host or device; read only.
 *   W         FP64, column-major m×r (ldw ≥ m): the start on entry (negative
 *             entries are taken as 0), the result on return.  Host or device.
 *   H         FP64, column-major r×n (ldh ≥ r): likewise.
 *   objective host array of `outer` doubles or NULL: ½‖V − W·H‖_F² after each
 *             outer iteration (the sum of the W-step's FP64 sub-problem
 *             objectives).
 * The context's prepared problem is replaced (it ends prepared with the last
 * W-step); work buffers are kept in the context for later calls.
 * Errors: INVALID_ARG (null pointer, r > min(m, n), r > 4096, ld too small,
 * outer < 1, tol not positive), NONFINITE, UNSUPPORTED (as aln_solve),
 * OUT_OF_MEMORY, TIMEOUT, CUDA. */
aln_status aln_nmf(aln_ctx* ctx, const float* V, int64_t m, int64_t n, int64_t ldv, int64_t r,
                   double* W, int64_t ldw, double* H, int64_t ldh, int32_t outer, double tol,
                   int32_t max_iter, double* objective);

/* Device-time breakdown of the last calls, measured with CUDA events on the
 * context's stream, and counters (for benchmarks and tracing). */
typedef struct aln_stats {
    double prepare_ms;       /* last aln_prepare */
    double gram_ms;          /*   of which the Gram kernel (H → Q) */
    double solve_ms;         /* last aln_solve, all right-hand sides */
    double kkt_ms;           /*   of which the FP64 KKT passes */
    int64_t kernel_launches; /* kernels this context launched since creation */
    int64_t iterations;      /* Alg. 2 iterations in the last aln_solve */
    double iterate_ms;       /* of solve_ms: the persistent Alg. 2 kernel(s) */
    int64_t passive_rows;    /* Σ_k |P_k| over those iterations (rows of Q read for Qḡ) */
    int64_t clipped_rows;    /* Σ_k |C_k| (rows of Q read for the clipped correction) */
    int32_t persist_blocks;  /* grid of the persistent kernel */
    int32_t clipped_iterations; /* iterations that needed the clipped correction Qe */
    double phase_us[5];      /* block 0's time in the persistent kernel, per phase:
                                product Qḡ, grid barrier, update (with the
                                gather of Qḡ and the new mask), clipped
                                correction (with its mask), 0 (replicated-state
                                kernel);
                                batched solver: [0] the batched chunks, [1] the
                                per-column tail, summed over rounds */
    double product_bytes;    /* algorithmic bytes of Q the Alg. 2 products of the
                                last aln_solve read: Σ_k n·(|P_k| + |C_k|)·sizeof
                                (summed over problems in grouped mode) */
    double lipschitz;        /* ALN_ALG_ANTI_ACC: L = λ_max(Q) estimate of the power
                                iteration for the prepared Q (0 before the first solve) */
    int64_t power_products;  /* products Qv that power iteration took */
    int32_t iter_kernel;     /* single-problem path of the last prepare: the kernel
                                aln_solve runs (1 tiled, 2 replicated state, 3 one
                                cluster, FP64; 0 for the batched and grouped paths) */
    int32_t reserved2;
} aln_stats;

/* Change the device-wait options of an existing context (aln_options'
 * wait_limit_us and test_barrier_skew, same meaning and ranges); they apply
 * from the next launch on.  Not in the paper: the bounded waits are how the
 * persistent kernels of this library report a stalled grid instead of
 * hanging.  Errors: INVALID_ARG. */
aln_status aln_set_wait_limit(aln_ctx* ctx, int32_t wait_limit_us, int32_t test_barrier_skew);

/* Copy the statistics of this context into *out.  Errors: INVALID_ARG. */
aln_status aln_get_stats(aln_ctx* ctx, aln_stats* out);

/* Scratch of aln_kkt_residual_noalloc, in doubles (16 MiB). */
#define ALN_NOALLOC_SCRATCH_DOUBLES (1 << 21)

/* FP64 KKT residual and objective of ONE solution, allocating nothing.
 * The paper has no counterpart: this is a deployment variant of
 * aln_kkt_residual for callers that cannot call cudaMalloc — code that runs
 * under a fixed device-memory budget, a callback invoked while the caller's
 * own memory pool is exhausted or locked, or a hot path where an allocation
 * (which can synchronize the device or fail) is not allowed.  It needs no
 * context: every intermediate (column norms, r = Ax − b, partial sums) lives in
 * a fixed array of ALN_NOALLOC_SCRATCH_DOUBLES doubles compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  The same quantities as aln_kkt_residual are computed:
 *   out[0] = ‖ḡ‖/‖min(q,0)‖ (absolute ‖ḡ‖ when ‖min(q,0)‖ = 0),
 *   out[1] = ½‖Ax − b‖².
 *   A      d×n column-major, lda ≥ d, dtype F32 or F64   (device memory)
 *   b      d entries, same dtype                         (device memory)
 *   x      n entries, FP64, x ≥ 0                        (device memory)
 *   out    2 doubles                                     (device memory)
 * Unlike the context calls, this one takes device (or managed) memory only:
 * a host pointer in any of the four gives ALN_ERR_INVALID_ARG before anything
 * is launched.
 *   stream cudaStream_t the work is enqueued on (NULL = legacy stream); the
 *          call returns without synchronizing.
 * Limits: 3n + 2d + 520 ≤ ALN_NOALLOC_SCRATCH_DOUBLES, otherwise
 * ALN_ERR_INVALID_ARG and nothing is launched (use aln_kkt_residual instead).
 * A NaN or Inf in A, b or x makes both outputs NaN (the call still returns
 * ALN_OK: the check runs on the GPU and the call does not synchronize).
 * The first call on each device looks up the device address of the scratch
 * array (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array and each call
 * overwrites it, so calls whose work overlaps on the GPU (different streams
 * with no ordering between them) race and produce wrong results.
 * Errors: INVALID_ARG, CUDA. */
aln_status aln_kkt_residual_noalloc(const void* A, int64_t d, int64_t n, int64_t lda,
                                    int32_t dtype, const void* b, const double* x, double* out,
                                    void* stream);

/* Measurement helper, not in the paper: the L2 read bandwidth of the current
 * device in GB/s, from `reps` streaming reads (16-byte loads cached in L2
 * only, every SM) of a `bytes` buffer that stays resident in L2, timed with
 * CUDA events after three warm-up reads.  The Alg. 2 products read Q from L2
 * once it fits there, so this is their ceiling.  The call allocates and frees
 * its own buffer and stream and synchronizes.  Requires 1 MiB ≤ bytes ≤ ¾ of
 * the L2 size and reps ≥ 1.  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
aln_status aln_l2_read_bandwidth(int64_t bytes, int32_t reps, double* gbs);

/* Destroy a context and free its workspace (NULL is accepted). */
void aln_destroy(aln_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* aln_status_string(aln_status status);

/* ALN_VERSION of the built library. */
int32_t aln_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ALN_H */
