// FP64 KKT residual and objective of Def. 1 evaluated from A itself:
//   r = A x − b,  ∇F = Aᵀ r,  g = ∇F / s (= Qy + q in the scaled variables of
//   Eq. NQPQ),  ḡ = g on P(y = s·x) (§3),  rel = ‖ḡ‖ / ‖min(q, 0)‖,  F = ½‖r‖².
// A is read in its input precision and every product is accumulated in FP64,
// so the residual does not inherit the error of the FP32 / split-BF16 Q.
// Both passes are HBM-bound; with 16-byte aligned columns they move four
// elements per load so that enough bytes are in flight per SM.
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

constexpr int kKktThreads = 256;
constexpr int kKktRows = 4 * kKktThreads;  // rows of r per block in k_kkt_ax

// rpart[cg][t] = Σ_{i ∈ column group cg, x_i ≠ 0} A_ti x_i.  Each thread owns
// four consecutive rows; columns with x_i = 0 are skipped (x is sparse at the
// optimum, so only the support of x is read).
template <typename TA, bool VEC>
__global__ void __launch_bounds__(kKktThreads) k_kkt_ax(const TA* __restrict__ A, int64_t d,
                                                        int64_t n, int64_t lda,
                                                        const double* __restrict__ x,
                                                        int64_t cols_per_group,
                                                        double* __restrict__ rpart) {
    const int64_t t0 = ((int64_t)blockIdx.x * kKktThreads + threadIdx.x) * 4;
    const int64_t i0 = (int64_t)blockIdx.y * cols_per_group;
    const int64_t i1 = min(n, i0 + cols_per_group);
    if (t0 >= d) return;
    const bool full = VEC && t0 + 4 <= d;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t i = i0;
    for (; i + 4 <= i1; i += 4) {
        double xi[4], a[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) xi[c] = x[i + c];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const TA* p = A + (i + c) * lda + t0;
            if (xi[c] == 0.0) {
                a[c][0] = a[c][1] = a[c][2] = a[c][3] = 0.0;
            } else if (full) {
                load4(p, a[c]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) a[c][u] = t0 + u < d ? (double)p[u] : 0.0;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(a[c][u], xi[c], acc[u]);
    }
    for (; i < i1; ++i) {
        const double xi = x[i];
        if (xi == 0.0) continue;
        const TA* p = A + i * lda + t0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (t0 + u < d) acc[u] = fma((double)p[u], xi, acc[u]);
    }
    double* out = rpart + (int64_t)blockIdx.y * d + t0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (t0 + u < d) out[u] = acc[u];
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
        acc = fma(v, v, acc);
    }
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) fpart[blockIdx.x] = acc;
}

// One block per column: ∇F_i = A_iᵀ r, g_i = ∇F_i / s_i, ḡ on P(s·x);
// g64 keeps the full gradient (used by the refinement), gpart[i] = ḡ_i².
template <typename TA, bool VEC>
__global__ void __launch_bounds__(kKktThreads) k_kkt_grad(const TA* __restrict__ A, int64_t d,
                                                          int64_t n, int64_t lda,
                                                          const double* __restrict__ r,
                                                          const double* __restrict__ s,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ g64,
                                                          double* __restrict__ gpart) {
    __shared__ double scratch[32];
    const int64_t i = blockIdx.x;
    const TA* col = A + i * lda;
    double acc = 0.0;
    const int64_t d4 = VEC ? d / 4 : 0;
#pragma unroll 4
    for (int64_t q = threadIdx.x; q < d4; q += blockDim.x) {
        double a[4], rr[4];
        load4(col + 4 * q, a);
        load4(r + 4 * q, rr);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = fma(a[u], rr[u], acc);
    }
    for (int64_t t = 4 * d4 + threadIdx.x; t < d; t += blockDim.x)
        acc = fma((double)col[t], r[t], acc);
    const double grad = block_sum(acc, scratch);
    if (threadIdx.x == 0) {
        const double gi = grad / s[i];
        const double yi = x[i] * s[i];
        g64[i] = gi;
        const bool P = yi > 0.0 || gi < 0.0;
        gpart[i] = P ? gi * gi : 0.0;
    }
}

// ---------------------------------------------------------------------------
// FP32 inputs: the same sums on the FP32 pipe with FP64-level accuracy.  x and
// r are split into FP32 pairs (v = hi + lo); each product a·hi is formed
// exactly (TwoProduct by FMA) and accumulated with TwoSum, a·lo goes into the
// compensation term (Dot2, Ogita, Rump & Oishi 2005).  This GPU's FP64 pipe
// made the plain FP64 version of these two passes compute-bound (≈1.5 ms at
// 20000×5000); in FP32 pairs they run at the speed of the A reads.
// ---------------------------------------------------------------------------
__global__ void k_split_pairs(const double* __restrict__ v, int64_t m, float* __restrict__ hi,
                              float* __restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)v[i];
        hi[i] = h;
        lo[i] = (float)(v[i] - (double)h);
    }
}

struct Pair {
    float s = 0.0f, c = 0.0f;
    // += a·(h + l)
    __device__ __forceinline__ void add(float a, float h, float l) {
        const float p = mul_rn(a, h);
        const float ep = fmaf(a, h, -p);
        const float t = s + p;
        const float z = t - s;
        c += ((s - (t - z)) + (p - z)) + fmaf(a, l, ep);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <bool VEC>
__global__ void __launch_bounds__(kKktThreads) k_kkt_ax32(const float* __restrict__ A, int64_t d,
                                                          int64_t n, int64_t lda,
                                                          const float* __restrict__ xh,
                                                          const float* __restrict__ xl,
                                                          int64_t cols_per_group,
                                                          double* __restrict__ rpart) {
    const int64_t t0 = ((int64_t)blockIdx.x * kKktThreads + threadIdx.x) * 4;
    const int64_t i0 = (int64_t)blockIdx.y * cols_per_group;
    const int64_t i1 = min(n, i0 + cols_per_group);
    if (t0 >= d) return;
    const bool full = VEC && t0 + 4 <= d;
    Pair acc[4];
    for (int64_t i = i0; i < i1; ++i) {
        const float h = xh[i], l = xl[i];
        if (h == 0.0f && l == 0.0f) continue;  // only the support of x is read
        const float* p = A + i * lda + t0;
        float a[4];
        if (full) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p));
            a[0] = v.x;
            a[1] = v.y;
            a[2] = v.z;
            a[3] = v.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = t0 + u < d ? p[u] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u].add(a[u], h, l);
    }
    double* out = rpart + (int64_t)blockIdx.y * d + t0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (t0 + u < d) out[u] = acc[u].value();
}

template <bool VEC>
__global__ void __launch_bounds__(kKktThreads) k_kkt_grad32(const float* __restrict__ A, int64_t d,
                                                            int64_t n, int64_t lda,
                                                            const float* __restrict__ rh,
                                                            const float* __restrict__ rl,
                                                            const double* __restrict__ s,
                                                            const double* __restrict__ x,
                                                            double* __restrict__ g64,
                                                            double* __restrict__ gpart) {
    __shared__ double scratch[32];
    const int64_t i = blockIdx.x;
    const float* col = A + i * lda;
    Pair acc;
    const int64_t d4 = VEC ? d / 4 : 0;
#pragma unroll 2
    for (int64_t q = threadIdx.x; q < d4; q += blockDim.x) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(col + 4 * q));
        const float4 h = __ldg(reinterpret_cast<const float4*>(rh + 4 * q));
        const float4 l = __ldg(reinterpret_cast<const float4*>(rl + 4 * q));
        acc.add(a.x, h.x, l.x);
        acc.add(a.y, h.y, l.y);
        acc.add(a.z, h.z, l.z);
        acc.add(a.w, h.w, l.w);
    }
    for (int64_t t = 4 * d4 + threadIdx.x; t < d; t += blockDim.x) acc.add(col[t], rh[t], rl[t]);
    const double grad = block_sum(acc.value(), scratch);
    if (threadIdx.x == 0) {
        const double gi = grad / s[i];
        const double yi = x[i] * s[i];
        g64[i] = gi;
        const bool P = yi > 0.0 || gi < 0.0;
        gpart[i] = P ? gi * gi : 0.0;
    }
}

__global__ void k_kkt_final(const double* __restrict__ gpart, int ng,
                            const double* __restrict__ fpart, int nf, double den,
                            double* __restrict__ out) {
    __shared__ double scratch[32];
    double g = 0.0, f = 0.0;
    for (int i = threadIdx.x; i < ng; i += blockDim.x) g += gpart[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) f += fpart[i];
    g = block_sum(g, scratch);
    f = block_sum(f, scratch);
    if (threadIdx.x == 0) {
        const double num = sqrt(g);
        out[0] = den > 0.0 ? num / den : num;
        out[1] = 0.5 * f;
    }
}

// Workspace inside c->kkt_pool: r64 (d), rpart (CG·d), g64 (ldq),
// kkt_part (512 fparts | n gparts), kkt_out (2).
cudaError_t launch_kkt(aln_ctx* c, const double* x64, const void* b, double den, double* out2) {
    const int64_t d = c->d, n = c->n;
    if (c->csc_kkt) {  // A held as CSC arrays and packed boxes (sparse.cu)
        const __nv_bfloat16* hi = c->A_hi;
        const __nv_bfloat16* mid = (const __nv_bfloat16*)((const uint8_t*)c->A_hi + c->csc_box_bytes);
        const __nv_bfloat16* lo =
            (const __nv_bfloat16*)((const uint8_t*)c->A_hi + 2 * c->csc_box_bytes);
        double* gpart = c->kkt_part + 512;
        float* rh = reinterpret_cast<float*>(c->rpart);  // rpart holds ≥ d doubles
        cudaError_t e = launch_csc_kkt(c->csc_cp, c->csc_ri, c->csc_v, d, n, c->csc_occ, c->csc_W,
                                       c->csc_wbase, c->csc_toff, hi, mid, lo, x64,
                                       (const float*)b, c->s, c->r64, rh, rh + d, c->csc_fpart,
                                       c->g64, gpart, c->stream);
        if (e != cudaSuccess) return e;
        k_kkt_final<<<1, 256, 0, c->stream>>>(gpart, (int)n, c->csc_fpart, (int)ceil_div(d, 64),
                                              den, out2);
        return cudaGetLastError();
    }
    const int CG = c->CG;
    const int64_t cpg = ceil_div(n, CG);
    const dim3 g1((unsigned)ceil_div(d, kKktRows), (unsigned)CG);
    const int nf = (int)std::min<int64_t>(ceil_div(d, kKktThreads), 512);
    double* fpart = c->kkt_part;
    double* gpart = c->kkt_part + 512;
    const size_t esz = c->dtype == ALN_DTYPE_F32 ? 4 : 8;
    const bool vec = aligned16(c->A, c->lda, esz);
#define ALN_KKT(TA, VE)                                                                           \
    do {                                                                                          \
        k_kkt_ax<TA, VE><<<g1, kKktThreads, 0, c->stream>>>((const TA*)c->A, d, n, c->lda, x64,  \
                                                            cpg, c->rpart);                       \
        k_kkt_r<TA><<<nf, kKktThreads, 0, c->stream>>>(d, c->rpart, CG, (const TA*)b, c->r64,    \
                                                       fpart);                                    \
        k_kkt_grad<TA, VE><<<(unsigned)n, kKktThreads, 0, c->stream>>>(                           \
            (const TA*)c->A, d, n, c->lda, c->r64, c->s, x64, c->g64, gpart);                     \
    } while (0)
    if (c->dtype == ALN_DTYPE_F32) {
        // x and r as FP32 pairs (hi, lo) in the tail of rpart
        float* xh = reinterpret_cast<float*>(
            ((uintptr_t)(c->rpart + (int64_t)CG * d) + 255) & ~(uintptr_t)255);
        float* xl = xh + c->ldq;
        float* rh = xl + c->ldq;
        float* rl = rh + d;
        k_split_pairs<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, c->stream>>>(
            x64, n, xh, xl);
        const bool vr = vec && (d % 4 == 0);
        if (vec)
            k_kkt_ax32<true><<<g1, kKktThreads, 0, c->stream>>>((const float*)c->A, d, n, c->lda, xh,
                                                                 xl, cpg, c->rpart);
        else
            k_kkt_ax32<false><<<g1, kKktThreads, 0, c->stream>>>((const float*)c->A, d, n, c->lda,
                                                                  xh, xl, cpg, c->rpart);
        k_kkt_r<float><<<nf, kKktThreads, 0, c->stream>>>(d, c->rpart, CG, (const float*)b, c->r64,
                                                          fpart);
        k_split_pairs<<<(unsigned)std::min<int64_t>(ceil_div(d, 256), 1024), 256, 0, c->stream>>>(
            c->r64, d, rh, rl);
        if (vr)
            k_kkt_grad32<true><<<(unsigned)n, kKktThreads, 0, c->stream>>>(
                (const float*)c->A, d, n, c->lda, rh, rl, c->s, x64, c->g64, gpart);
        else
            k_kkt_grad32<false><<<(unsigned)n, kKktThreads, 0, c->stream>>>(
                (const float*)c->A, d, n, c->lda, rh, rl, c->s, x64, c->g64, gpart);
    } else {
        if (vec) ALN_KKT(double, true);
        else ALN_KKT(double, false);
    }
#undef ALN_KKT
    k_kkt_final<<<1, 256, 0, c->stream>>>(gpart, (int)n, fpart, nf, den, out2);
    return cudaGetLastError();
}

}  // namespace aln
