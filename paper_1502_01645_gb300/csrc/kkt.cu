// FP64 KKT residual and objective of Def. 1 evaluated from A itself:
//   r = A x − b,  ∇F = Aᵀ r,  g = ∇F / s (= Qy + q in the scaled variables of
//   Eq. NQPQ),  ḡ = g on P(y = s·x) (§3),  rel = ‖ḡ‖ / ‖min(q, 0)‖,  F = ½‖r‖².
// A is read in its input precision and every product is accumulated in FP64,
// so the residual does not inherit the error of the FP32 / split-BF16 Q.
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

constexpr int kKktThreads = 256;

// rpart[cg][t] = Σ_{i ∈ column group cg, x_i ≠ 0} A_ti x_i  (each thread one row
// t, consecutive threads consecutive rows: coalesced column reads).
template <typename TA>
__global__ void __launch_bounds__(kKktThreads) k_kkt_ax(const TA* __restrict__ A, int64_t d,
                                                        int64_t n, int64_t lda,
                                                        const double* __restrict__ x,
                                                        int64_t cols_per_group,
                                                        double* __restrict__ rpart) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * cols_per_group;
    const int64_t i1 = min(n, i0 + cols_per_group);
    double acc = 0.0;
    if (t < d) {
        int64_t i = i0;
        for (; i + 4 <= i1; i += 4) {
            const double x0 = x[i], x1 = x[i + 1], x2 = x[i + 2], x3 = x[i + 3];
            const double a0 = x0 != 0.0 ? (double)A[i * lda + t] : 0.0;
            const double a1 = x1 != 0.0 ? (double)A[(i + 1) * lda + t] : 0.0;
            const double a2 = x2 != 0.0 ? (double)A[(i + 2) * lda + t] : 0.0;
            const double a3 = x3 != 0.0 ? (double)A[(i + 3) * lda + t] : 0.0;
            acc = fma(a0, x0, acc);
            acc = fma(a1, x1, acc);
            acc = fma(a2, x2, acc);
            acc = fma(a3, x3, acc);
        }
        for (; i < i1; ++i) {
            const double xi = x[i];
            if (xi != 0.0) acc = fma((double)A[i * lda + t], xi, acc);
        }
        rpart[(int64_t)blockIdx.y * d + t] = acc;
    }
}

// r_t = Σ_cg rpart[cg][t] − b_t ; block partial of ‖r‖².
template <typename TB>
__global__ void __launch_bounds__(kKktThreads) k_kkt_r(int64_t d, const double* __restrict__ rpart,
                                                       int CG, const TB* __restrict__ b,
                                                       double* __restrict__ r,
                                                       double* __restrict__ fpart) {
    __shared__ double scratch[32];
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < d;
         t += (int64_t)gridDim.x * blockDim.x) {
        double v = -(double)b[t];
        for (int cg = 0; cg < CG; ++cg) v += rpart[(int64_t)cg * d + t];
        r[t] = v;
        acc += v * v;
    }
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) fpart[blockIdx.x] = acc;
}

// One warp per column: ∇F_i = A_iᵀ r, g_i = ∇F_i / s_i, ḡ on P(s·x);
// g64 keeps the full gradient (used by the refinement), gpart ‖ḡ‖² per block.
template <typename TA>
__global__ void __launch_bounds__(kKktThreads) k_kkt_grad(const TA* __restrict__ A, int64_t d,
                                                          int64_t n, int64_t lda,
                                                          const double* __restrict__ r,
                                                          const double* __restrict__ s,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ g64,
                                                          double* __restrict__ gpart) {
    __shared__ double wsum[kKktThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    double gb2 = 0.0;
    if (i < n) {
        const TA* col = A + i * lda;
        double acc0 = 0.0, acc1 = 0.0;
        int64_t t = lane;
        for (; t + 32 < d; t += 64) {
            acc0 = fma((double)col[t], r[t], acc0);
            acc1 = fma((double)col[t + 32], r[t + 32], acc1);
        }
        for (; t < d; t += 32) acc0 = fma((double)col[t], r[t], acc0);
        const double grad = warp_sum(acc0 + acc1);
        if (lane == 0) {
            const double gi = grad / s[i];
            const double yi = x[i] * s[i];
            g64[i] = gi;
            const bool P = yi > 0.0 || gi < 0.0;
            gb2 = P ? gi * gi : 0.0;
        }
    }
    if (lane == 0) wsum[wid] = gb2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += wsum[w];
        gpart[blockIdx.x] = v;
    }
}

__global__ void k_kkt_final(const double* __restrict__ gpart, int ng,
                            const double* __restrict__ fpart, int nf, double den,
                            double* __restrict__ out) {
    if (threadIdx.x < 32) {
        const double gb2 = warp_sum_array(gpart, ng);
        const double r2 = warp_sum_array(fpart, nf);
        if (threadIdx.x == 0) {
            const double num = sqrt(gb2);
            out[0] = den > 0.0 ? num / den : num;
            out[1] = 0.5 * r2;
        }
    }
}

// Workspace layout inside c->kkt_pool (sized by the caller of launch_kkt):
//   r64 (d), rpart (CG·d), g64 (ldq), kkt_part (gparts | fparts), kkt_out (2)
cudaError_t launch_kkt(aln_ctx* c, const double* x64, const void* b, double den, double* out2) {
    const int64_t d = c->d, n = c->n;
    const int CG = c->CG;
    const int64_t cpg = ceil_div(n, CG);
    const dim3 g1((unsigned)ceil_div(d, kKktThreads), (unsigned)CG);
    const int nf = (int)std::min<int64_t>(ceil_div(d, kKktThreads), 512);
    const int ng = (int)ceil_div(n, kKktThreads / 32);
    double* fpart = c->kkt_part;
    double* gpart = c->kkt_part + 512;
    if (c->dtype == ALN_DTYPE_F32) {
        k_kkt_ax<float><<<g1, kKktThreads, 0, c->stream>>>((const float*)c->A, d, n, c->lda, x64,
                                                           cpg, c->rpart);
        k_kkt_r<float><<<nf, kKktThreads, 0, c->stream>>>(d, c->rpart, CG, (const float*)b, c->r64,
                                                          fpart);
        k_kkt_grad<float><<<ng, kKktThreads, 0, c->stream>>>((const float*)c->A, d, n, c->lda,
                                                             c->r64, c->s, x64, c->g64, gpart);
    } else {
        k_kkt_ax<double><<<g1, kKktThreads, 0, c->stream>>>((const double*)c->A, d, n, c->lda, x64,
                                                            cpg, c->rpart);
        k_kkt_r<double><<<nf, kKktThreads, 0, c->stream>>>(d, c->rpart, CG, (const double*)b,
                                                           c->r64, fpart);
        k_kkt_grad<double><<<ng, kKktThreads, 0, c->stream>>>((const double*)c->A, d, n, c->lda,
                                                              c->r64, c->s, x64, c->g64, gpart);
    }
    k_kkt_final<<<1, 32, 0, c->stream>>>(gpart, ng, fpart, nf, den, out2);
    return cudaGetLastError();
}

}  // namespace aln
