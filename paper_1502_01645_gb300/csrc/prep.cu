// Prepare-phase kernels of Alg. 1 (§3): scale factors, q = −D⁻¹Aᵀb, the
// split-BF16 copies of A, and the FP64 Gram / AᵀB used by the plain method.
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

__device__ __forceinline__ void load4t(const float* p, float* o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void load4t(const double* p, double* o) { load4(p, o); }

// One 256-thread block per column A_i, one pass over the column:
//   s_i² = Σ_t A_ti²                              — √diag(H) of Alg. 1, Eq. Rescaling
//   c_ci = Σ_t A_ti B_ct, c < kc ≤ 4              — Aᵀb of Eq. NQP
//   s_i  = √s_i², or 1 when s_i² = 0 (Eq. Rescaling's H_ii = 0 case)
//   q_ci = −c_ci / s_i                            — q of Eq. NQPQ
// Sums are accurate to FP64 level (DotAcc) and combined in FP64.
// With SPLIT, also writes the exact three-term split A_ti = hi + mid + lo
// (BF16 each) into the K-major [n][ldk] arrays read by the tensor-core Gram
// (zero padding t ≥ d).
// VEC: the column and B rows are 16-byte aligned, so four consecutive
// elements move per load (the kernel is HBM-bound; wide loads keep enough
// bytes in flight).
template <typename TA, bool SPLIT, bool VEC>
__global__ void __launch_bounds__(256) k_colstats(const TA* __restrict__ A, int64_t d, int64_t n,
                                                  int64_t lda, const TA* __restrict__ B, int kc,
                                                  int64_t ldb, double* __restrict__ s,
                                                  double* __restrict__ inv_s,
                                                  double* __restrict__ q64, int64_t ldq,
                                                  int* __restrict__ flags,
                                                  __nv_bfloat16* __restrict__ hi,
                                                  __nv_bfloat16* __restrict__ mid,
                                                  __nv_bfloat16* __restrict__ lo, int64_t ldk) {
    __shared__ double scratch[32];
    const int64_t i = blockIdx.x;
    const TA* col = A + i * lda;
    DotAcc<TA> sq, dot[4];
    bool bad = false;
    const int64_t d4 = VEC ? d / 4 : 0;
#pragma unroll 2
    for (int64_t q = threadIdx.x; q < d4; q += blockDim.x) {
        TA a[4];
        load4t(col + 4 * q, a);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            sq.add(a[u], a[u]);
            bad |= !isfinite(a[u]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c < kc) {
                TA bb[4];
                load4t(B + (int64_t)c * ldb + 4 * q, bb);
#pragma unroll
                for (int u = 0; u < 4; ++u) dot[c].add(a[u], bb[u]);
            }
        }
        if (SPLIT) {
            __align__(8) __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) split3_bf16((float)a[u], h[u], m[u], l[u]);
            *reinterpret_cast<uint2*>(hi + i * ldk + 4 * q) = *reinterpret_cast<uint2*>(h);
            *reinterpret_cast<uint2*>(mid + i * ldk + 4 * q) = *reinterpret_cast<uint2*>(m);
            *reinterpret_cast<uint2*>(lo + i * ldk + 4 * q) = *reinterpret_cast<uint2*>(l);
        }
    }
    for (int64_t t = 4 * d4 + threadIdx.x; t < d; t += blockDim.x) {
        const TA a = col[t];
        sq.add(a, a);
        bad |= !isfinite(a);
        for (int c = 0; c < kc; ++c) dot[c].add(a, B[(int64_t)c * ldb + t]);
        if (SPLIT) {
            __nv_bfloat16 h, m, l;
            split3_bf16((float)col[t], h, m, l);
            hi[i * ldk + t] = h;
            mid[i * ldk + t] = m;
            lo[i * ldk + t] = l;
        }
    }
    if (SPLIT) {
        const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
        for (int64_t t = d + threadIdx.x; t < ldk; t += blockDim.x) {
            hi[i * ldk + t] = z;
            mid[i * ldk + t] = z;
            lo[i * ldk + t] = z;
        }
    }
    const double s2 = block_sum(sq.value(), scratch);
    double dsum[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) dsum[c] = c < kc ? block_sum(dot[c].value(), scratch) : 0.0;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        const double si = s2 > 0.0 ? sqrt(s2) : 1.0;
        s[i] = si;
        inv_s[i] = 1.0 / si;
        for (int c = 0; c < kc; ++c) q64[(int64_t)c * ldq + i] = -dsum[c] / si;
        if (bad) atomicOr(flags, 1);
    }
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                               int* __restrict__ flags) {
    bool bad = false;
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / rows, r = e - c * rows;
        bad |= !isfinite((double)X[c * ld + r]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

// ‖min(q_c, 0)‖ for each right-hand side: the projected gradient at y = 0.
__global__ void k_denominators(const double* __restrict__ q64, int64_t n, int64_t ldq,
                               double* __restrict__ den) {
    __shared__ double scratch[32];
    const double* q = q64 + (int64_t)blockIdx.x * ldq;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double m = q[i] < 0.0 ? q[i] : 0.0;
        v += m * m;
    }
    v = block_sum(v, scratch);
    if (threadIdx.x == 0) den[blockIdx.x] = sqrt(v);
}

// ---------------------------------------------------------------------------
// FP64 SIMT product  C[i][j] = Σ_t X[t][i] Y[t][j]  (X, Y column-major, K = d)
// 64×64 tile per 256-thread block, 4×4 outputs per thread (strided by 16 so
// shared-memory reads are conflict-free), K staged 16 at a time.
//   MODE_GRAM: X = Y = A, lower-triangle tiles only; writes
//              Q_ij = H_ij / (s_i s_j) and its mirror, Q_ii = 1 (0 for a zero
//              column) — Alg. 1, Eq. NQPQ, Remark of §3.
//   MODE_QVEC: X = A, Y = B; writes q_ci = −(Aᵀb_c)_i / s_i at out[c*ldo + i].
// ---------------------------------------------------------------------------
constexpr int kG64Tile = 64;
constexpr int kG64K = 16;

__device__ __forceinline__ void tri_decode(int64_t t, int& I, int& J) {
    // t = I(I+1)/2 + J with 0 ≤ J ≤ I
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    I = (int)r;
    J = (int)(t - r * (r + 1) / 2);
}

template <typename TX, typename TY, int MODE>
__global__ void __launch_bounds__(256) k_atb64(const TX* __restrict__ X, int64_t ldx,
                                               const TY* __restrict__ Y, int64_t ldy, int64_t K,
                                               int64_t M, int64_t N, int tiles_m,
                                               const double* __restrict__ inv_s,
                                               double* __restrict__ out, int64_t ldo) {
    __shared__ double Xs[kG64K][kG64Tile];
    __shared__ double Ys[kG64K][kG64Tile];
    int tm, tn;
    int64_t kbeg = 0, kend = K;
    if (MODE == MODE_GRAM) {
        tri_decode(blockIdx.x, tm, tn);
    } else if (MODE == MODE_PART) {
        // tiles_m = lower-triangle tiles T, ldo = the K-chunk length
        tri_decode(blockIdx.x % tiles_m, tm, tn);
        kbeg = (int64_t)(blockIdx.x / tiles_m) * ldo;
        kend = min(K, kbeg + ldo);
    } else {
        tm = blockIdx.x % tiles_m;
        tn = blockIdx.x / tiles_m;
    }
    const int64_t i0 = (int64_t)tm * kG64Tile, j0 = (int64_t)tn * kG64Tile;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    for (int64_t k0 = kbeg; k0 < kend; k0 += kG64K) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;
            const int kk = e & 15, ii = e >> 4;
            const int64_t gk = k0 + kk;
            const int64_t gi = i0 + ii, gj = j0 + ii;
            Xs[kk][ii] = (gi < M && gk < kend) ? (double)X[gi * ldx + gk] : 0.0;
            Ys[kk][ii] = (gj < N && gk < kend) ? (double)Y[gj * ldy + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kG64K; ++kk) {
            double xa[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
        }
        __syncthreads();
    }

    if (MODE == MODE_PART) {  // the raw partial tile of this K chunk
        double* t = out + (int64_t)blockIdx.x * kG64Tile * kG64Tile;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) t[(ty + 16 * a) * kG64Tile + tx + 16 * b] = acc[a][b];
        return;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty + 16 * a;
        if (i >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + tx + 16 * b;
            if (j >= N) continue;
            if (MODE == MODE_GRAM) {
                // Lower triangle only (diagonal tiles too), mirrored: Q is
                // exactly symmetric.
                if (j > i) continue;
                double v = acc[a][b] * inv_s[i] * inv_s[j];
                if (i == j) v = acc[a][b] != 0.0 ? 1.0 : 0.0;
                out[i * ldo + j] = v;
                out[j * ldo + i] = v;
            } else if (MODE == MODE_QVEC) {
                out[j * ldo + i] = -acc[a][b] * inv_s[i];
            } else {  // MODE_AXPY: out = X^T Y + add (inv_s carries `add`)
                out[j * ldo + i] = acc[a][b] + inv_s[j * ldo + i];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------
cudaError_t launch_colstats(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                            const void* B, int kc, int64_t ldb, double* s, double* inv_s,
                            double* q64, int64_t ldq, int* flags, __nv_bfloat16* hi,
                            __nv_bfloat16* mid, __nv_bfloat16* lo, int64_t ldk,
                            cudaStream_t st) {
    const dim3 grid((unsigned)n), block(256);
    const bool split = hi != nullptr;
    const size_t esz = dtype == ALN_DTYPE_F32 ? 4 : 8;
    const bool vec = aligned16(A, lda, esz) && (kc == 0 || aligned16(B, ldb, esz));
#define ALN_COLSTATS(TA, SP, VE)                                                              \
    k_colstats<TA, SP, VE><<<grid, block, 0, st>>>((const TA*)A, d, n, lda, (const TA*)B, kc, \
                                                   ldb, s, inv_s, q64, ldq, flags, hi, mid, lo, \
                                                   ldk)
    if (dtype == ALN_DTYPE_F32) {
        if (split) {
            if (vec) ALN_COLSTATS(float, true, true);
            else ALN_COLSTATS(float, true, false);
        } else {
            if (vec) ALN_COLSTATS(float, false, true);
            else ALN_COLSTATS(float, false, false);
        }
    } else {
        if (split) {
            if (vec) ALN_COLSTATS(double, true, true);
            else ALN_COLSTATS(double, true, false);
        } else {
            if (vec) ALN_COLSTATS(double, false, true);
            else ALN_COLSTATS(double, false, false);
        }
    }
#undef ALN_COLSTATS
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const void* X, int32_t dtype, int64_t rows, int64_t cols,
                                int64_t ld, int* flags, cudaStream_t st) {
    const int64_t total = rows * cols;
    const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 4096);
    if (dtype == ALN_DTYPE_F32)
        k_check_finite<float><<<blocks, 256, 0, st>>>((const float*)X, rows, cols, ld, flags);
    else
        k_check_finite<double><<<blocks, 256, 0, st>>>((const double*)X, rows, cols, ld, flags);
    return cudaGetLastError();
}

cudaError_t launch_denominators(const double* q64, int64_t n, int64_t ldq, int64_t k, double* den,
                                cudaStream_t st) {
    k_denominators<<<(unsigned)k, 256, 0, st>>>(q64, n, ldq, den);
    return cudaGetLastError();
}

// Split-K finish: tile t of Q is the sum of its `chunks` partial tiles in
// chunk order, then the MODE_GRAM epilogue (scaling, unit diagonal, mirror).
__global__ void __launch_bounds__(256) k_gram64_finish(const double* __restrict__ part, int T,
                                                        int chunks, int64_t n,
                                                        const double* __restrict__ inv_s,
                                                        double* __restrict__ out, int64_t ldo) {
    int tm, tn;
    tri_decode(blockIdx.x, tm, tn);
    constexpr int kTT = kG64Tile * kG64Tile;
    for (int e = threadIdx.x; e < kTT; e += blockDim.x) {
        const int64_t i = (int64_t)tm * kG64Tile + e / kG64Tile;
        const int64_t j = (int64_t)tn * kG64Tile + e % kG64Tile;
        if (i >= n || j >= n || j > i) continue;
        double acc = 0.0;
        for (int ch = 0; ch < chunks; ++ch) acc += part[((int64_t)ch * T + blockIdx.x) * kTT + e];
        double v = acc * inv_s[i] * inv_s[j];
        if (i == j) v = acc != 0.0 ? 1.0 : 0.0;
        out[i * ldo + j] = v;
        out[j * ldo + i] = v;
    }
}

// K chunks of the split Gram: one wave of CTAs over the lower-triangle tiles,
// each chunk at least 64 rows of A; 1 (no split) when the tiles fill the GPU.
static int gram64_chunks(int64_t d, int64_t n, int num_sms) {
    const int64_t tm = ceil_div(n, kG64Tile);
    const int64_t T = tm * (tm + 1) / 2;
    if (num_sms <= 0 || 2 * T > num_sms) return 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms / T, ceil_div(d, 64)));
}

size_t gram64_split_bytes(int64_t d, int64_t n, int num_sms) {
    const int ch = gram64_chunks(d, n, num_sms);
    if (ch <= 1) return 0;
    const int64_t tm = ceil_div(n, kG64Tile);
    return (size_t)ch * (size_t)(tm * (tm + 1) / 2) * kG64Tile * kG64Tile * sizeof(double);
}

cudaError_t launch_gram64(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                          const double* inv_s, double* Q, int64_t ldq, cudaStream_t st,
                          double* work, size_t work_bytes, int num_sms) {
    const int64_t tm = ceil_div(n, kG64Tile);
    const int64_t tiles = tm * (tm + 1) / 2;
    const int chunks = gram64_chunks(d, n, num_sms);
    if (chunks > 1 && work && work_bytes >= gram64_split_bytes(d, n, num_sms)) {
        // few tiles (small n): split the K range so that every SM works
        const int64_t kc = round_up(ceil_div(d, (int64_t)chunks), kG64K);
        const int nch = (int)ceil_div(d, kc);
        const unsigned grid = (unsigned)(tiles * nch);
        if (dtype == ALN_DTYPE_F32)
            k_atb64<float, float, MODE_PART><<<grid, 256, 0, st>>>(
                (const float*)A, lda, (const float*)A, lda, d, n, n, (int)tiles, inv_s, work, kc);
        else
            k_atb64<double, double, MODE_PART><<<grid, 256, 0, st>>>(
                (const double*)A, lda, (const double*)A, lda, d, n, n, (int)tiles, inv_s, work, kc);
        k_gram64_finish<<<(unsigned)tiles, 256, 0, st>>>(work, (int)tiles, nch, n, inv_s, Q, ldq);
        return cudaGetLastError();
    }
    if (dtype == ALN_DTYPE_F32)
        k_atb64<float, float, MODE_GRAM><<<(unsigned)tiles, 256, 0, st>>>(
            (const float*)A, lda, (const float*)A, lda, d, n, n, (int)tm, inv_s, Q, ldq);
    else
        k_atb64<double, double, MODE_GRAM><<<(unsigned)tiles, 256, 0, st>>>(
            (const double*)A, lda, (const double*)A, lda, d, n, n, (int)tm, inv_s, Q, ldq);
    return cudaGetLastError();
}

// out[c][i] = Σ_t X[i][t] Y[c][t] + add[c][i]  (FP64; X = Q64 symmetric, so
// this is Q·y_c + q_c for every column c).
cudaError_t launch_gemm64_axpy(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                               int64_t K, int64_t M, int64_t N, const double* add, double* out,
                               int64_t ldo, cudaStream_t st) {
    const int64_t tm = ceil_div(M, kG64Tile), tn = ceil_div(N, kG64Tile);
    k_atb64<double, double, MODE_AXPY><<<(unsigned)(tm * tn), 256, 0, st>>>(
        X, ldx, Y, ldy, K, M, N, (int)tm, add, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_qvec64(const void* A, int32_t dtype, int64_t d, int64_t n, int64_t lda,
                          const void* B, int64_t k, int64_t ldb, const double* inv_s, double* q64,
                          int64_t ldq, cudaStream_t st) {
    const int64_t tm = ceil_div(n, kG64Tile), tn = ceil_div(k, kG64Tile);
    if (dtype == ALN_DTYPE_F32)
        k_atb64<float, float, MODE_QVEC><<<(unsigned)(tm * tn), 256, 0, st>>>(
            (const float*)A, lda, (const float*)B, ldb, d, n, k, (int)tm, inv_s, q64, ldq);
    else
        k_atb64<double, double, MODE_QVEC><<<(unsigned)(tm * tn), 256, 0, st>>>(
            (const double*)A, lda, (const double*)B, ldb, d, n, k, (int)tm, inv_s, q64, ldq);
    return cudaGetLastError();
}

}  // namespace aln
