// Host-side launchers of the libaln kernels (one translation unit each).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace aln {

constexpr int MODE_GRAM = 0;
constexpr int MODE_PART = 3;  // raw partial tile of a K range (split-K Gram)
constexpr int MODE_QVEC = 1;
constexpr int MODE_AXPY = 2;

// prep.cu
cudaError_t launch_colstats(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                            const void* B, int kc, int64_t ldb, double* s, double* inv_s,
                            double* q64, int64_t ldq, int* flags, __nv_bfloat16* hi,
                            __nv_bfloat16* mid, __nv_bfloat16* lo, int64_t ldk, cudaStream_t st);
cudaError_t launch_check_finite(const void* X, int32_t dtype, int64_t rows, int64_t cols,
                                int64_t ld, int* flags, cudaStream_t st);
cudaError_t launch_denominators(const double* q64, int64_t n, int64_t ldq, int64_t k, double* den,
                                cudaStream_t st);
// FP64 Gram → Q.  With a workspace (`work`, `work_bytes`) and fewer lower-
// triangle tiles than `num_sms`, the K range is split over several CTAs per
// tile whose partial tiles are added in chunk order by a second kernel
// (deterministic); gram64_split_bytes gives the workspace that needs.
cudaError_t launch_gram64(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                          const double* inv_s, double* Q, int64_t ldq, cudaStream_t st,
                          double* work = nullptr, size_t work_bytes = 0, int num_sms = 0);
size_t gram64_split_bytes(int64_t d, int64_t n, int num_sms);
cudaError_t launch_qvec64(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                          const void* B, int64_t k, int64_t ldb, const double* inv_s, double* q64,
                          int64_t ldq, cudaStream_t st);

cudaError_t launch_gemm64_axpy(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                               int64_t K, int64_t M, int64_t N, const double* add, double* out,
                               int64_t ldo, cudaStream_t st);

// gemm_tc.cu — split-BF16 tensor-core Gram (tcgen05 + TMA)
// Q_ij = (Σ_t hh + hm + mh + mm + hl + lh)_ij · inv_s_i · inv_s_j for the exact
// three-term split a = h + m + l (nsplit = 3), or hh + hm + mh for the two-term
// split a ≈ h + m (nsplit = 2); lower tiles mirrored.
// Tile rows [row0, row1) of Q (all by default).  With split > 1 (and part,
// ticket given) each tile pair's K range runs as `split` chunks on separate
// CTAs: part then needs pairs·split·128² floats and ticket one zeroed counter
// per pair of the launch (left zeroed).  The chunking, and so the rounding of
// every entry, depends only on `split`: launches over different row ranges
// with the same split give the same Q as one launch over all rows.
// sk_part / sk_ticket (nullable; a whole-matrix launch without split K only):
// buffers of gram_sk_bytes for the stream-K pass over the last partial wave.
cudaError_t launch_gram_tc(int nsplit, const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                           const __nv_bfloat16* lo, int64_t d, int64_t n, int64_t ldk,
                           const double* inv_s, float* Q, int64_t ldq, int* timeout_flag,
                           cudaStream_t st, int64_t row0 = 0, int64_t row1 = -1,
                           float* part = nullptr, unsigned int* ticket = nullptr, int split = 1,
                           float* sk_part = nullptr, unsigned int* sk_ticket = nullptr,
                           int num_sms = 0);
// The same over the tile pairs [p0, p1) of the triangle order (pair
// I(I+1)/2 + J is tile (I, J ≤ I)).  Each pair is one CTA's whole K loop (or
// `split` CTAs' chunks), so any partition of the pairs into launches gives the
// same Q; the stream-K pass runs in the launch that ends the triangle when it
// holds the whole tail.
cudaError_t launch_gram_tc_pairs(int nsplit, const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                                 const __nv_bfloat16* lo, int64_t d, int64_t n, int64_t ldk,
                                 const double* inv_s, float* Q, int64_t ldq, int* timeout_flag,
                                 cudaStream_t st, int64_t p0, int64_t p1, float* part,
                                 unsigned int* ticket, int split, float* sk_part,
                                 unsigned int* sk_ticket, int num_sms);
// Stream-K for the Gram's last wave: with `pairs` tile pairs (one CTA per SM
// resident), the pairs past the last full wave (0 if none) are run by one CTA
// per SM, each taking an equal share of their K blocks; a pair split over
// several CTAs is summed from partial tiles (at most gram_sk_maxseg each).
inline int64_t gram_sk_tail(int64_t pairs, int num_sms) {
    if (num_sms <= 0 || pairs <= num_sms) return 0;
    return pairs % num_sms;
}
inline int gram_sk_maxseg(int64_t tail, int num_sms) {
    return tail > 0 ? (int)((num_sms + tail - 1) / tail) + 1 : 0;
}
// Partial tiles, then one ticket per tail pair.
inline size_t gram_sk_part_bytes(int64_t pairs, int num_sms) {
    const int64_t r = gram_sk_tail(pairs, num_sms);
    return (size_t)r * gram_sk_maxseg(r, num_sms) * 128 * 128 * 4;
}
inline size_t gram_sk_bytes(int64_t pairs, int num_sms) {
    const int64_t r = gram_sk_tail(pairs, num_sms);
    return r > 0 ? gram_sk_part_bytes(pairs, num_sms) + (size_t)((r * 4 + 255) / 256 * 256) : 0;
}
// Chunks per tile pair for the Gram of a matrix with `pairs` tile pairs over
// num_kb K blocks: enough CTAs to cover the SMs when the pairs alone do not
// (tall, narrow A), with at least 16 K blocks per chunk.
inline int gram_split_k(int64_t pairs, int64_t num_kb, int num_sms) {
    if (pairs <= 0 || pairs >= num_sms) return 1;
    const int64_t s = std::min<int64_t>(num_sms / pairs, num_kb / 16);
    return (int)std::max<int64_t>(1, s);
}
bool tc_supported(int cc_major, int cc_minor);
// One CTA of the block-sparse Gram: positions [k0, k0 + nk) of the K blocks
// occupied in both column tiles I ≥ J (pair index `pair` in the lower-triangle
// order), chunk c of the pair's S.  With S > 1 the chunk's unscaled partial
// tile goes to slot `slot` and the pair's last chunk to finish adds slots
// slot − c … slot − c + S − 1 in that order and stores the tile of Q.
struct SItem {
    int32_t I, J, k0, nk, S, c, slot, pair;
};
// Block-sparse Gram over the occupied boxes packed by sparse.cu, one CTA per
// work item; tiles of Q without an item stay as they are (zeroed by the caller).
// part: 128·128 floats per slot; ticket: one zeroed counter per pair.
cudaError_t launch_sgram_tc(int nsplit, const SItem* items, int64_t nitems, const uint32_t* occ,
                            int W, const int32_t* wbase, const int64_t* toff,
                            const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                            const __nv_bfloat16* lo, int64_t n, const double* inv_s, float* Q,
                            int64_t ldq, float* part, unsigned int* ticket, int* timeout_flag,
                            cudaStream_t st);

// W = Q·V (mode 0, with per-column curvature partials) or g += Q·V (mode 1)
// over the compacted columns of a batch (batch.cu).
// q, v: the three BF16 split terms (h, m, l) of Q ([n][ldk]) and of the
// compacted columns ([kmax][ldk]).
cudaError_t launch_bgemm_tc(int mode, const __nv_bfloat16* q_hi, const __nv_bfloat16* q_lo,
                            int64_t n, int64_t ldk, const __nv_bfloat16* v_hi,
                            const __nv_bfloat16* v_lo, int64_t kmax, const int* ncols,
                            const int* map, int64_t ldq, float* W, const float* gb, double* kpart,
                            float* g, int* timeout_flag, cudaStream_t st);

// grouped.cu — many independent problems of different sizes.
// Per-problem record, built on the host and read by every grouped kernel.
struct GProb {
    const void* A;     // d×n column-major (device), dtype of the group
    const void* b;     // d entries (device)
    int64_t lda;
    int32_t d, n;
    int32_t T, KB;     // 128-row operand tiles (⌈n/128⌉), 64-wide K blocks (⌈d/64⌉)
    int32_t ldq, pad;  // row length of Q_p and of the iteration vectors (n rounded up to 4)
    int64_t pack;      // first 16 KiB tile of the problem in the hi / lo packs
    int64_t qoff;      // first element of Q_p in the Q pool
    int64_t voff;      // first entry in packed n-vectors (Σ_{q<p} n_q)
    int64_t foff;      // first entry in packed iteration vectors (Σ_{q<p} ldq_q)
    int64_t roff;      // first entry in packed d-vectors (Σ_{q<p} d_q)
    int64_t slot;      // first column slot of the prepare grid (Σ_{q<p} 128·T_q)
};
// Per-problem record of the grouped Alg. 2 kernels (also the batched tail).
struct GStat {
    int32_t iters;        // Alg. 2 iterations, summed over rounds
    int32_t status;       // inner stop reason of the last run (aln_rhs_status,
                          // or kRhsPaused)
    int32_t clip_iters;   // iterations that needed the clipped correction
    int32_t npassive;     // |P| at the end of the last run
    int64_t sum_passive;  // Σ |P_k| (rows of Q read for Qḡ)
    int64_t sum_clip;     // Σ |C_k|
    double gbar2;         // ‖ḡ‖² (iteration precision) at the end of the last run
};
// Inner status of a run stopped by its iteration budget (not a stop rule of
// Alg. 2: the problem continues in the next launch).
constexpr int32_t kRhsPaused = 64;
// One lower-triangle output tile (tm ≥ tn) of one problem's Gram.
struct GTile {
    int32_t p, tm, tn, pad;
};
// Elements of one pre-swizzled operand tile: 128 rows × 64 BF16 (16 KiB).
constexpr int kPackTile = 128 * 64;
// Index of element (row j, K index t) of a problem's operand in the tiled
// pack: tile (j/128, t/64), rows of 128 bytes, the 16-byte chunks of row r
// permuted by chunk ^ (r mod 8) — the image of a 128-byte-swizzled TMA box, so
// a tile copied verbatim into 1024-byte-aligned shared memory is a valid
// tcgen05 K-major SWIZZLE_128B operand.
__host__ __device__ __forceinline__ int64_t pack_index(int64_t tile0, int KB, int j, int t) {
    const int r = j & 127, kk = t & 63;
    const int64_t tile = tile0 + (int64_t)(j >> 7) * KB + (t >> 6);
    return tile * kPackTile + r * 64 + ((((kk >> 3) ^ (r & 7)) << 3) | (kk & 7));
}
cudaError_t launch_ggram_tc(int nsplit, const GProb* gp, const GTile* tiles, int64_t ntiles,
                            const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                            const __nv_bfloat16* lo, const double* inv_s, float* Q,
                            int* timeout_flag, cudaStream_t st);
aln_status group_prepare(aln_ctx* c, int32_t count, const aln_problem* probs, int32_t dtype);
aln_status group_solve(aln_ctx* c, double tol, int max_iter, double* X, const double* X0,
                       aln_solve_info* info);
aln_status group_kkt(aln_ctx* c, const double* X, double* rel_kkt, double* objective);
aln_status group_export(aln_ctx* c, double* Q, double* q, double* s);
void group_free(aln_ctx* c);
// Alg. 2 on columns sharing one FP32 Q by the grouped kernels (one CTA or a
// cluster of cs per column); the batched solver's tail
aln_status tail_launch(aln_ctx* c, const GProb* gp, const int* order, int count, int* queue,
                       const float* Q, int64_t ldq, const double* q64, const double* den,
                       double* y, double* g, GStat* stat, const double* tgt, int max_iter,
                       int budget, int cs);
// Dynamic shared memory of one tail CTA for row length ldq
size_t tail_smem_bytes(int64_t ldq, bool cluster);
// problems, Σ n_p and max n_p of the grouped layout
void group_shape(const aln_ctx* c, int* count, int64_t* sum_n, int64_t* max_n);

// mlp.cu — learned start point
aln_status mlp_init(aln_ctx* c, int hidden, uint64_t seed);
aln_status mlp_params(aln_ctx* c, int set, float* const* t);
aln_status mlp_grad(aln_ctx* c, const double* Qs, const double* Ys, int64_t count, double* loss,
                    float* const* grads);
aln_status mlp_train(aln_ctx* c, const double* Qs, const double* Ys, int64_t count,
                     const aln_train_opts& o, double* epoch_loss);
aln_status mlp_predict(aln_ctx* c, double* X0, int64_t ldx, int* kept);
int mlp_n(const aln_ctx* c);
void mlp_free(aln_ctx* c);
void nmf_free(aln_ctx* c);  // nmf.cu

// batch.cu — Alg. 2 on many right-hand sides sharing A
aln_status batch_prepare(aln_ctx* c);
aln_status batch_solve(aln_ctx* c, double tol, int max_iter, double* X, int64_t ldx,
                       const double* X0, aln_solve_info* info);
void batch_free(aln_ctx* c);

// iter.cu — Alg. 2 on one right-hand side
template <typename T>
cudaError_t launch_iter_setup(aln_ctx* c, const double* q64, const double* x0, double eps,
                              int max_iter);
template <typename T>
cudaError_t launch_iter_refresh_from_g64(aln_ctx* c, double eps, int max_iter);
template <typename T>
cudaError_t launch_unscale(aln_ctx* c, double* x64);
cudaError_t launch_state_reset(aln_ctx* c, double eps, int max_iter);

// persist.cu — the whole Alg. 2 loop as one cooperative persistent kernel
template <typename T>
cudaError_t launch_alg2_persist(aln_ctx* c);
// Anti+Acc (§5) iteration on the prepared state (persist.cu).
template <typename T>
cudaError_t launch_acc_persist(aln_ctx* c);
// Shared memory the Anti+Acc kernel needs for row length ldq (persist.cu).
size_t acc_smem_need(bool f64, int64_t ldq);
// Power iteration for λ_max(Q): out[0] = ρ, out[1] = products (persist.cu).
template <typename T>
cudaError_t launch_power(aln_ctx* c, double tol, int max_steps, double* out);
template <typename T>
int persist_max_blocks(int num_sms, int64_t ldq, int* repl);
size_t persist_sync_bytes();
// small64.cu — the FP64 Alg. 2 loop of one small problem on one cluster
bool small64_fits(const aln_ctx* c, int optin_smem);
cudaError_t launch_alg2_small64(aln_ctx* c);

// sparse.cu — Alg. 1 from a CSC matrix (col_ptr int64[n+1], row_idx int32,
// values of dtype); see the kernels there.
cudaError_t launch_csc_check(const int64_t* cp, const int32_t* ri, const void* v, int32_t dtype,
                             int64_t d, int64_t n, int64_t nnz, int* flags, cudaStream_t st);
cudaError_t launch_csc_colstats(const int64_t* cp, const int32_t* ri, const void* v,
                                int32_t dtype, int64_t n, const void* B, int kc, int64_t ldb,
                                void* A, int64_t lda, double* s, double* inv_s, double* q64,
                                int64_t ldq, uint32_t* occ, int W, cudaStream_t st);
cudaError_t launch_csc_number(const uint32_t* occ, int W, int64_t T, int32_t* wbase, int64_t* cnt,
                              int64_t* toff, cudaStream_t st);
// Work list of the block-sparse Gram: Lp[p] = K blocks occupied in both tiles
// of pair p; pairs with Lp > 0 split into chunks of ≤ KC = max(16, ⌈ΣLp /
// num_sms⌉) blocks.  meta[0] = items written (≤ P + num_sms), meta[1] =
// partial slots used (≤ 2·num_sms).
// Non-zero tiles of Q from the pair counts Lp (T·⌈T/32⌉ words, zeroed here).
cudaError_t launch_csc_qmask(const int32_t* Lp, int64_t T, uint32_t* mask, cudaStream_t st);
cudaError_t launch_csc_worklist(const uint32_t* occ, int W, int64_t T, int num_sms, int32_t* Lp,
                                SItem* items, int64_t* meta, cudaStream_t st);
cudaError_t launch_csc_pack(const int64_t* cp, const int32_t* ri, const void* v, int32_t dtype,
                            int64_t n, const uint32_t* occ, int W, const int32_t* wbase,
                            const int64_t* toff, __nv_bfloat16* hi, __nv_bfloat16* mid,
                            __nv_bfloat16* lo, cudaStream_t st);

// FP64 KKT pass from the CSC arrays and the packed boxes (FP32 values):
// r (d; also as FP32 pairs rh, rl), fpart (⌈d/64⌉ block sums of r²), g64 and
// gpart (n) as in launch_kkt.
cudaError_t launch_csc_kkt(const int64_t* cp, const int32_t* ri, const float* v, int64_t d,
                           int64_t n, const uint32_t* occ, int W, const int32_t* wbase,
                           const int64_t* toff, const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                           const __nv_bfloat16* lo, const double* x, const float* b,
                           const double* s, double* r, float* rh, float* rl, double* fpart,
                           double* g64, double* gpart, cudaStream_t st);

// api.cu — workspace of the single-problem solver and one persistent run
aln_status alloc_workspace(aln_ctx* c);
aln_status run_until_done(aln_ctx* c);

// autotune.cu — launch geometry from the JSON cache, measured on a miss
// (autotune = 2); called by aln_solve before the solver runs
aln_status autotune_solve(aln_ctx* c, double tol, int max_iter, double* X, int64_t ldx,
                          const double* X0);

// ozaki.cu — FP64-accurate out[j·ldo + i] = −inv_s[i]·Σ_t X[i·ldx + t]·Y[j·ldy + t]
// for FP32 X (m columns) and Y (n columns) of d rows, by exact BF16 digit
// products on the tensor cores; work: oz_work_bytes(d, m, n) bytes of device
// memory (digits and exponents).
size_t oz_work_bytes(int64_t d, int64_t m, int64_t n);
cudaError_t launch_oz_atb(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t d,
                          int64_t m, int64_t n, const double* inv_s, double* out, int64_t ldo,
                          void* work, size_t work_bytes, int* timeout_flag, cudaStream_t st);
// Q = D⁻¹AᵀAD⁻¹ (the batched checks' FP64 scaled matrix) by the same exact
// products: exactly symmetric, unit diagonal (0 for a zero column).
cudaError_t launch_oz_gram(const float* A, int64_t lda, int64_t d, int64_t n,
                           const double* inv_s, double* Q, int64_t ldq, void* work,
                           size_t work_bytes, int* timeout_flag, cudaStream_t st);
// The same products for FP32 or FP64 inputs (xtype, ytype: aln_dtype; FP64
// values keep their leading 48 bits): mode 0 writes −C_ij·vec[i], mode 1
// writes C_ij + vec[j·ldo + i] (the FP64 check's g = Q·y + q).
cudaError_t launch_oz_product(int mode, int32_t xtype, const void* X, int64_t ldx,
                              int32_t ytype, const void* Y, int64_t ldy, int64_t d, int64_t m,
                              int64_t n, const double* vec, double* out, int64_t ldo, void* work,
                              size_t work_bytes, int* timeout_flag, cudaStream_t st);

// kkt.cu — FP64 KKT residual straight from A
cudaError_t launch_kkt(aln_ctx* c, const double* x64, const void* b, double den, double* out2);

}  // namespace aln
