// FP64-accurate C = XᵀY on the tensor cores (the q = −D⁻¹Aᵀb of Alg. 1 for
// many right-hand sides, Eq. NQPQ), by exact integer products.
//
// Every column of X (and of Y) is written as 2^e · Σ_{s=1..7} d_s 2^{−7s}
// with e the column's exponent (max |x| < 2^e) and integer digits taken by
// rounding to nearest, 7 bits at a time (|d_1| ≤ 128, |d_s| ≤ 64 after it):
// 49 bits below the column's largest entry, the rest (≤ 2^{e−50}) dropped.
// Rounded digits carry both signs, so the dropped parts have no bias.  A digit
// is exact in BF16, a product of two digits (≤ 2^14) is exact in FP32, and a
// sum of up to 1024 of them stays within 2^24, so the tensor core's FP32
// accumulation of digit products is EXACT.  Then
//     C_ij = 2^{e_i + f_j} Σ_{σ=2..8} 2^{−7σ} Σ_{s+u=σ} Σ_t d_s(x_ti) d_u(y_tj)
// keeping the digit pairs with s + u ≤ 8 (28 pairs): the dropped pairs and the
// rounded-off tails each stay below about 2^{−49}·2^{e_i+f_j} per term, the
// error of a Dot2 sum on the FP32 pipe.  This is the fixed-point splitting of
// Ozaki, Ogita, Oishi and Rump (2012) for error-free matrix products, here
// with BF16 digits on tcgen05.
//
// One CTA computes a 128 (columns of X) × 64 (columns of Y) tile.  Per 64-wide
// K block, two half steps:
//   X half: digits 1–4 of X with digits 1–7 of Y (22 pairs, σ = 2..8),
//   Y half: digits 5–7 of X with digits 1–3 of Y (6 pairs, σ = 6..8),
// into TMEM accumulators, one per σ (64 columns each), kept over two K blocks
// (128 products per pair): at most 7 pairs × 128 products of ≤ 2^14, below
// 2^24.  Then eight promotion warps read the accumulators (integers in FP32),
// scale them by 2^{−7σ} (exact) and add them into a double-float
// accumulator (hi + lo, TwoSum), about 48 bits — the FP32 pipe, not this
// GPU's narrow FP64 pipe — while the loads of the next K blocks go on.  The
// epilogue writes the FP64 result.
//
// Roles (320 threads): warp 0 (one lane) loads, warp 1 (one lane) issues the
// MMAs, warps 2–9 promote (warp w: TMEM lanes 32·(w mod 4), output columns
// 32·((w − 2) / 4) + 0..31).  Every wait is bounded; on expiry the CTA sets
// *timeout_flag, drains its own copies and MMAs, frees tensor memory and
// leaves without storing.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <utility>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace aln {
namespace tc {
namespace {

constexpr int kOzS = 7;                    // digits per value
constexpr int kOzBits = 7;                 // bits per digit
constexpr int kOzSig = 8;                  // largest digit-pair order s + u kept
constexpr int kOzXA = 4;                   // digits of X in the X half step (the rest in Y)
constexpr int kOzYB = 3;                   // digits of Y in the Y half step
constexpr int kOzN = 64;                   // output columns per CTA (Y side)
constexpr int kOzThreads = 320;
constexpr int kOzATile = BM * BK * 2;      // 16 KiB: 128 rows × 64 K
constexpr int kOzBTile = kOzN * BK * 2;    // 8 KiB:   64 rows × 64 K
// half-step buffers: X half = 4 A tiles + 7 B tiles, Y half = 3 A + 3 B
constexpr int kOzXBytes = kOzXA * kOzATile + kOzS * kOzBTile;              // 120 KiB
constexpr int kOzYBytes = (kOzS - kOzXA) * kOzATile + kOzYB * kOzBTile;    // 72 KiB
constexpr int kOzSmem = kOzXBytes + kOzYBytes + 1024 + 256;
constexpr uint32_t kOzTmemCols = 512;      // 7 accumulators × 64 columns, rounded up
constexpr int kOzPromo = 4;                // half steps (2 K blocks) per promotion
constexpr int kOzFlush = 4;                // promotions (8 K blocks) per FP64 flush
constexpr int kOzQvec = 0;                 // out = −C·inv_s
constexpr int kOzAxpy = 1;                 // out = C + vec
constexpr int kOzGram = 2;                 // X = Y: out[c·ldo + i] = C·inv_s_i·inv_s_c for
                                           // i ≥ c (diagonal 1, or 0 for a zero column)

struct OzArgs {
    int num_kb;            // 64-wide K blocks
    int64_t m, n;          // columns of X (rows of C), columns of Y
    const int* ex;         // [m] exponents of X's columns
    const int* ey;         // [n] exponents of Y's columns
    const double* vec;     // kOzQvec: inv_s [m]; kOzAxpy: the added term, as out
    double* out;           // at out[j·ldo + i]: −C_ij·inv_s[i] or C_ij + vec[j·ldo + i]
    int64_t ldo;
    int* timeout_flag;
};

struct OzMaps {
    CUtensorMap x[kOzS];   // digits of X, [m][ldk], box 64 × 128
    CUtensorMap y[kOzS];   // digits of Y, [n][ldk], box 64 × 64
};

// x added into the pair (hi, lo) (TwoSum; lo gathers the errors).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

// MMAs of one half step: pairs (s, u) with s in [S0, S1] and s + u ≤ 8,
// digit s of X at a + (s − S0)·A tile, digit u of Y at b + (u − 1)·B tile,
// accumulator σ − 2 at column (σ − 2)·64.  `start` (X half only): the first
// half step of a promotion block, where each accumulator's first MMA
// overwrites it; that MMA is the pair (1, σ − 1), which exists for every
// σ = 2..8.
template <int S0, int S1>
__device__ __forceinline__ void oz_half(uint32_t tmem, uint32_t a, uint32_t b, bool start) {
    constexpr uint32_t idesc = idesc_bf16_f32(BM, kOzN);
#pragma unroll
    for (int s = S0; s <= S1; ++s) {
#pragma unroll
        for (int u = 1; u <= kOzS; ++u) {
            if (s + u > kOzSig) continue;
            const uint32_t d = tmem + (uint32_t)((s + u - 2) * kOzN);
            const uint32_t ab = a + (uint32_t)((s - S0) * kOzATile);
            const uint32_t bb = b + (uint32_t)((u - 1) * kOzBTile);
            const bool fresh = S0 == 1 && s == 1 && start;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                umma_bf16(d, sdesc_sw128(ab + kk * 32), sdesc_sw128(bb + kk * 32), idesc,
                          (fresh && kk == 0) ? 0u : 1u);
            }
        }
    }
}

// TR: X and Y were swapped by the launcher (C is computed transposed), so
// tile row i is output column and tile column c output row.
template <int MODE, bool TR>
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_atb(const __grid_constant__ OzMaps maps,
                                                         OzArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* bufX = smem;
    uint8_t* bufY = smem + kOzXBytes;
    uint64_t* bars = (uint64_t*)(smem + kOzXBytes + kOzYBytes);
    uint64_t* full = bars;         // [2]: X, Y tiles landed
    uint64_t* empty = bars + 2;    // [2]: X, Y tiles consumed by the MMAs
    uint64_t* tfull = bars + 4;    // accumulators ready (one per promotion block)
    uint64_t* tempty = bars + 5;   // accumulators drained (8 promotion warps)
    uint64_t* done = bars + 6;
    uint32_t* tmem_slot = (uint32_t*)(bars + 7);
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * kOzN;
    const int H = 2 * p.num_kb;                      // half steps
    const int NB = (H + kOzPromo - 1) / kOzPromo;    // promotion blocks

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, 8);
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kOzTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    float hi[32], lo[32];
    double acc[32];  // the pairs are flushed here every kOzFlush promotions
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        hi[j] = lo[j] = 0.0f;
        acc[j] = 0.0;
    }

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int h = 0; h < H; ++h) {
            const int t = h & 1, kb = h >> 1;  // t = 0: X half, 1: Y half
            if (h >= 2 && !mbar_wait(&empty[t], ((h >> 1) - 1) & 1)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            uint8_t* buf = t == 0 ? bufX : bufY;
            const int na = t == 0 ? kOzXA : kOzS - kOzXA;  // digits of X
            const int s0 = t == 0 ? 0 : kOzXA;
            const int nb = t == 0 ? kOzS : kOzYB;           // digits of Y
            mbar_expect_tx(&full[t], na * kOzATile + nb * kOzBTile);
            const int x = kb * BK;
            for (int si = 0; si < na; ++si)
                tma_load_2d(buf + si * kOzATile, &maps.x[s0 + si], &full[t], x, (int)m0);
            for (int u = 0; u < nb; ++u)
                tma_load_2d(buf + na * kOzATile + u * kOzBTile, &maps.y[u], &full[t], x,
                            (int)n0);
            ++issued;
        }
        // our own copies in flight: the last two (bounded wait)
        for (int h = max(0, issued - 2); h < issued; ++h)
            if (!mbar_wait(&full[h & 1], (h >> 1) & 1)) s_abort = 1;
    } else if (warp == 1 && lane == 0) {
        int h = 0;
        for (; h < H; ++h) {
            const int t = h & 1, blk = h / kOzPromo;
            const bool start = h % kOzPromo == 0;
            if (!mbar_wait(&full[t], (h >> 1) & 1) ||
                (start && blk >= 1 && !mbar_wait(tempty, (blk - 1) & 1))) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            tc_fence_after();
            const uint32_t a = smem_u32(t == 0 ? bufX : bufY);
            if (t == 0)
                oz_half<1, kOzXA>(tmem, a, a + kOzXA * kOzATile, start);
            else
                oz_half<kOzXA + 1, kOzS>(tmem, a, a + (kOzS - kOzXA) * kOzATile, false);
            umma_commit(&empty[t]);
            if (h % kOzPromo == kOzPromo - 1 || h == H - 1) umma_commit(tfull);
        }
        if (h > 0) umma_commit(done);
    } else if (warp >= 2) {
        const int q = warp & 3, half = (warp - 2) >> 2;
        const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * half);
        for (int blk = 0; blk < NB; ++blk) {
            if (!mbar_wait(tfull, blk & 1)) {
                s_abort = 1;
                break;
            }
            tc_fence_after();
            // accumulators σ = 2..8 (every order occurs in each block)
            for (int sg = 2; sg <= kOzSig; ++sg) {
                const float scale = __int_as_float((127 - kOzBits * sg) << 23);  // 2^{−7σ}
                float v[32];
                tmem_ld16(tb + (uint32_t)((sg - 2) * kOzN), v);
                tmem_ld16(tb + (uint32_t)((sg - 2) * kOzN + 16), v + 16);
#pragma unroll
                for (int j = 0; j < 32; ++j) df_add(hi[j], lo[j], v[j] * scale);
            }
            if ((blk + 1) % kOzFlush == 0) {
                // FP64 flush: the pair's own rounding stays that of a few
                // K blocks (a handful of FP64 adds per K block, off the MMA
                // path)
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    acc[j] += (double)hi[j] + (double)lo[j];
                    hi[j] = lo[j] = 0.0f;
                }
            } else {
                // renormalise the pairs once per promotion
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float s = hi[j] + lo[j];
                    lo[j] = lo[j] - (s - hi[j]);
                    hi[j] = s;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
            if (*(volatile int*)&s_abort) break;
        }
    }
    __syncwarp();
    if (warp == 1 && H > 0) {
        if (!mbar_wait(done, 0)) s_abort = 1;  // no MMA in flight past this point
    }
    tc_fence_after();
    __syncthreads();
    const bool ok = !s_abort;
    if (ok && warp >= 2) {
        const int q = warp & 3, half = (warp - 2) >> 2;
        const int64_t i = m0 + 32 * q + lane;
        if (i < p.m) {
            const int ei = p.ex[i];
            const double f = (MODE == kOzQvec && !TR) ? -p.vec[i] : 1.0;
            (void)f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int64_t c = n0 + 32 * half + j;
                if (c < p.n) {
                    const double v = ldexp(acc[j] + ((double)hi[j] + (double)lo[j]), ei + p.ey[c]);
                    const int64_t o = TR ? i * p.ldo + c : c * p.ldo + i;
                    if (MODE == kOzQvec)
                        p.out[o] = v * (TR ? -p.vec[c] : f);
                    else if (MODE == kOzAxpy)
                        p.out[o] = v + p.vec[o];
                    else if (i >= c)  // kOzGram: one triangle, mirrored afterwards
                        p.out[o] = i == c ? (v != 0.0 ? 1.0 : 0.0) : v * p.vec[i] * p.vec[c];
                }
            }
        }
    } else if (!ok && threadIdx.x == 0) {
        atomicExch(p.timeout_flag, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, kOzTmemCols);
}

// Column exponents and digits: one block per column of X (d rows, stride
// ld): e = the exponent with max |x| < 2^e (0 for a zero column), then the
// seven 7-bit digits of x·2^{−e}, each rounded to nearest (the remainder
// stays in [−1/2, 1/2]), written K-major [col][ldk] per digit (zero beyond
// d).
template <typename T>
__global__ void __launch_bounds__(256) k_oz_split(const T* __restrict__ X, int64_t ld, int64_t d,
                                                  int64_t ldk, int* __restrict__ ex,
                                                  __nv_bfloat16* __restrict__ dig,
                                                  int64_t dstride) {
    __shared__ T smax[8];
    const int64_t col = blockIdx.x;
    const T* x = X + col * ld;
    T mx = T(0);
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) mx = fmax(mx, fabs(x[t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) mx = fmax(mx, smax[w]);
    int e = 0;
    if (mx > T(0)) (void)frexp(mx, &e);  // mx = m·2^e, m in [0.5, 1)
    if (threadIdx.x == 0) ex[col] = e;
    // digits in the input's own precision: every step is exact (|v| ≤ 1
    // times 128, rounding to an integer, subtraction of that integer)
    for (int64_t t = threadIdx.x; t < ldk; t += blockDim.x) {
        T v = t < d ? ldexp(x[t], -e) : T(0);
#pragma unroll
        for (int s = 0; s < kOzS; ++s) {
            v *= T(1 << kOzBits);
            const T dv = rint(v);
            v -= dv;
            dig[(int64_t)s * dstride + col * ldk + t] = __float2bfloat16_rn((float)dv);
        }
    }
}

// K-major BF16 digits [rows][ldk], box 64 (K) × box_rows.
bool oz_map(CUtensorMap* m, const __nv_bfloat16* base, int64_t K, int64_t rows, int64_t ld,
            int box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace
}  // namespace tc

size_t oz_work_bytes(int64_t d, int64_t m, int64_t n) {
    const int64_t ldk = round_up(d, tc::BK);
    return (size_t)(tc::kOzS * (m + n) * ldk * 2) + (size_t)round_up((m + n) * 4, 256) + 1024;
}

cudaError_t launch_oz_product(int mode, int32_t xtype, const void* X, int64_t ldx,
                              int32_t ytype, const void* Y, int64_t ldy, int64_t d, int64_t m,
                              int64_t n, const double* vec, double* out, int64_t ldo, void* work,
                              size_t work_bytes, int* timeout_flag, cudaStream_t st) {
    using namespace tc;
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (!work || work_bytes < oz_work_bytes(d, m, n) ||
        (mode != kOzQvec && mode != kOzAxpy && mode != kOzGram))
        return cudaErrorInvalidValue;
    // a narrow X (fewer columns than a 128-row tile) and a wide Y: compute Cᵀ,
    // so the wide side fills the 128-row tiles
    const bool tr = mode != kOzGram && m < BM && n >= BM;
    if (tr) {
        std::swap(X, Y);
        std::swap(ldx, ldy);
        std::swap(xtype, ytype);
        std::swap(m, n);
    }
    const int64_t ldk = round_up(d, BK);
    uint8_t* w = (uint8_t*)(((uintptr_t)work + 255) & ~(uintptr_t)255);
    __nv_bfloat16* dx = (__nv_bfloat16*)w;                 // kOzS × [m][ldk]
    __nv_bfloat16* dy = dx + kOzS * m * ldk;               // kOzS × [n][ldk]
    int* ex = (int*)(dy + kOzS * n * ldk);
    int* ey = ex + m;
    if (xtype == ALN_DTYPE_F32)
        k_oz_split<float><<<(unsigned)m, 256, 0, st>>>((const float*)X, ldx, d, ldk, ex, dx,
                                                         m * ldk);
    else
        k_oz_split<double><<<(unsigned)m, 256, 0, st>>>((const double*)X, ldx, d, ldk, ex, dx,
                                                          m * ldk);
    if (ytype == ALN_DTYPE_F32)
        k_oz_split<float><<<(unsigned)n, 256, 0, st>>>((const float*)Y, ldy, d, ldk, ey, dy,
                                                         n * ldk);
    else
        k_oz_split<double><<<(unsigned)n, 256, 0, st>>>((const double*)Y, ldy, d, ldk, ey, dy,
                                                          n * ldk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    OzMaps maps;
    for (int s = 0; s < kOzS; ++s)
        if (!oz_map(&maps.x[s], dx + s * m * ldk, ldk, m, ldk, BM) ||
            !oz_map(&maps.y[s], dy + s * n * ldk, ldk, n, ldk, kOzN))
            return cudaErrorInvalidValue;
    static bool attr[3][2] = {{false, false}, {false, false}, {false, false}};
    const auto fn = mode == kOzQvec  ? (tr ? k_oz_atb<kOzQvec, true> : k_oz_atb<kOzQvec, false>)
                    : mode == kOzGram ? k_oz_atb<kOzGram, false>
                                      : (tr ? k_oz_atb<kOzAxpy, true> : k_oz_atb<kOzAxpy, false>);
    if (!attr[mode][tr]) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
        if (e != cudaSuccess) return e;
        attr[mode][tr] = true;
    }
    OzArgs a;
    a.num_kb = (int)(ldk / BK);
    a.m = m;
    a.n = n;
    a.ex = ex;
    a.ey = ey;
    a.vec = vec;
    a.out = out;
    a.ldo = ldo;
    a.timeout_flag = timeout_flag;
    const dim3 grid((unsigned)ceil_div(m, BM), (unsigned)ceil_div(n, kOzN));
    fn<<<grid, kOzThreads, kOzSmem, st>>>(maps, a);
    return cudaGetLastError();
}

namespace tc {
namespace {
// Q[i][j] = Q[j][i] for i < j (the lower triangle written by kOzGram: entry
// (row c, column i ≥ c) at out[c·ldo + i]).
__global__ void k_oz_mirror(double* __restrict__ Q, int64_t n, int64_t ldq) {
    const int64_t i = blockIdx.x;
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) Q[j * ldq + i] = Q[i * ldq + j];
}
}  // namespace
}  // namespace tc

cudaError_t launch_oz_gram(const float* A, int64_t lda, int64_t d, int64_t n,
                           const double* inv_s, double* Q, int64_t ldq, void* work,
                           size_t work_bytes, int* timeout_flag, cudaStream_t st) {
    cudaError_t e = launch_oz_product(tc::kOzGram, ALN_DTYPE_F32, A, lda, ALN_DTYPE_F32, A, lda,
                                      d, n, n, inv_s, Q, ldq, work, work_bytes, timeout_flag, st);
    if (e != cudaSuccess || n <= 1) return e;
    tc::k_oz_mirror<<<(unsigned)n, 256, 0, st>>>(Q, n, ldq);
    return cudaGetLastError();
}

cudaError_t launch_oz_atb(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t d,
                          int64_t m, int64_t n, const double* inv_s, double* out, int64_t ldo,
                          void* work, size_t work_bytes, int* timeout_flag, cudaStream_t st) {
    return launch_oz_product(tc::kOzQvec, ALN_DTYPE_F32, X, ldx, ALN_DTYPE_F32, Y, ldy, d, m, n,
                             inv_s, out, ldo, work, work_bytes, timeout_flag, st);
}

}  // namespace aln
