// Host-side launchers of the libaln kernels (one translation unit each).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace aln {

constexpr int MODE_GRAM = 0;
constexpr int MODE_QVEC = 1;
constexpr int MODE_AXPY = 2;

// prep.cu
cudaError_t launch_colstats(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                            const void* B, int kc, int64_t ldb, double* s, double* inv_s,
                            double* q64, int64_t ldq, int* flags, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, int64_t ldk, cudaStream_t st);
cudaError_t launch_check_finite(const void* X, int32_t dtype, int64_t rows, int64_t cols,
                                int64_t ld, int* flags, cudaStream_t st);
cudaError_t launch_denominators(const double* q64, int64_t n, int64_t ldq, int64_t k, double* den,
                                cudaStream_t st);
cudaError_t launch_gram64(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                          const double* inv_s, double* Q, int64_t ldq, cudaStream_t st);
cudaError_t launch_qvec64(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                          const void* B, int64_t k, int64_t ldb, const double* inv_s, double* q64,
                          int64_t ldq, cudaStream_t st);

cudaError_t launch_gram32_dot2(const float* A, int64_t d, int64_t n, int64_t lda,
                               const double* inv_s, double* Q, int64_t ldq, cudaStream_t st);
cudaError_t launch_qvec32_dot2(const float* A, int64_t d, int64_t n, int64_t lda, const float* B,
                               int64_t k, int64_t ldb, const double* inv_s, double* q64,
                               int64_t ldq, cudaStream_t st);
cudaError_t launch_gemm64_axpy(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                               int64_t K, int64_t M, int64_t N, const double* add, double* out,
                               int64_t ldo, cudaStream_t st);

// gemm_tc.cu — split-BF16 tensor-core Gram (tcgen05 + TMA)
// Q_ij = (Σ_t hi·hi + hi·lo + lo·hi)_ij · inv_s_i · inv_s_j, lower tiles mirrored.
cudaError_t launch_gram_tc(const __nv_bfloat16* hi, const __nv_bfloat16* lo, int64_t d,
                           int64_t n, int64_t ldk, const double* inv_s, float* Q, int64_t ldq,
                           int* timeout_flag, cudaStream_t st);
bool tc_supported(int cc_major, int cc_minor);
// W = Q·V (mode 0, with per-column curvature partials) or g += Q·V (mode 1)
// over the compacted columns of a batch (batch.cu).
cudaError_t launch_bgemm_tc(int mode, const __nv_bfloat16* q_hi, const __nv_bfloat16* q_lo,
                            int64_t n, int64_t ldk, const __nv_bfloat16* v_hi,
                            const __nv_bfloat16* v_lo, int64_t kmax, const int* ncols,
                            const int* map, int64_t ldq, float* W, const float* gb, double* kpart,
                            float* g, int* timeout_flag, cudaStream_t st);

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
template <typename T>
int persist_max_blocks(int num_sms, int64_t ldq, int* repl);
size_t persist_sync_bytes();

// kkt.cu — FP64 KKT residual straight from A
cudaError_t launch_kkt(aln_ctx* c, const double* x64, const void* b, double den, double* out2);

}  // namespace aln
