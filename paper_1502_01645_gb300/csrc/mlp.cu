// Learned start point for Alg. 2 (§3).  The paper starts at x⁰ = 0 and maps
// a given start with y⁰ = x⁰·√H_ii (Eq. Rescaling, Fig. 2); this file adds a
// small network that predicts y⁰ from the scaled right-hand side q of a fixed
// A (so a fixed scaled matrix Q):
//
//   z  = −Q⁻¹q, the unconstrained minimiser of ½yᵀQy + qᵀy; Q⁻¹ is formed
//        once per network by a Newton–Schulz iteration (FP32 GEMMs)
//   u  = [ (q/‖q‖ − μ)/σ ; (z/‖q‖ − μz)/σz ],  μ, σ, μz, σz per entry over
//        the training set
//   h1 = relu(W1 u + b1),  h2 = relu(W2 h1 + b2),  [r ; ℓ′] = W3 h2 + b3,
//   ŷ  = r + e ⊙ ẑ,  ℓ = ℓ′ + f ⊙ ẑ  with ẑ = z/(τ‖q‖) (per-entry skips)
//   d  = relu(ŷ)·[ℓ > 0],  y⁰ = α*·d with the exact line search of Alg. 2
//        from 0, α* = max(0, −qᵀd/dᵀQd), so f(y⁰) ≤ f(0)
//
// trained with Adam on L = mean (ŷ − y*/(τ‖q‖))² + mean BCE(ℓ, [y* > 0]),
// τ = RMS of y*/‖q‖ over the training set.
//
// The network's products are one tcgen05 GEMM kernel, D = A·Bᵀ with both
// operands K-major BF16 (TMA, 128-byte swizzle, 4-stage ring, FP32
// accumulation in tensor memory) and a fused epilogue: bias + ReLU (+
// transposed copy), bias only (FP32), ReLU-masked gradient (+ transposed
// copy), or plain FP32.  The backward products need Aᵀ-shaped operands; they
// are produced by the epilogues (transposed copies) and by the Adam kernel
// (Wᵀ next to W), so every product keeps K contiguous.  Master weights and
// Adam moments are FP32.  The direction z needs more than BF16 (Q has
// condition numbers in the thousands): Q⁻¹ and z come from an FP32 SIMT GEMM.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace aln {
namespace {
using namespace tc;

constexpr int kMStages = 4;
constexpr int kMTile = BM * BK * 2;                 // one 128×64 BF16 box, 16 KiB
constexpr int kMStageBytes = 2 * kMTile;            // A box + B box
constexpr int kMSmem = kMStages * kMStageBytes + 1024 + 256;

constexpr int EPI_RELU = 0;    // out = relu(acc + bias) → BF16 (+ transposed)
constexpr int EPI_LINEAR = 1;  // out = acc + bias → FP32
constexpr int EPI_DRELU = 2;   // out = acc · [act > 0] → BF16 (+ transposed)
constexpr int EPI_F32 = 3;     // out = acc → FP32

struct GemmArgs {
    int64_t M, N;
    int num_kb;
    const float* bias;
    const __nv_bfloat16* act;
    int64_t ld_act;
    __nv_bfloat16* out_h;
    int64_t ld_h;
    __nv_bfloat16* out_t;
    int64_t ld_t;
    float* out_f;
    int64_t ld_f;
    int* timeout_flag;
};

// D[M×N] = A[M×K] · B[N×K]ᵀ, one 128×128 tile per CTA (warp 0: TMA producer,
// warp 1: MMA issuer, 4 warps: epilogue).  Waits are bounded (1 s); on expiry
// the CTA raises *timeout_flag, drains its own copies, frees TMEM and exits.
template <int EPI>
__global__ void __launch_bounds__(128, 1)
    k_mlp_gemm(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
               GemmArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + kMStages * kMStageBytes);
    uint64_t* empty = full + kMStages;
    uint64_t* done = empty + kMStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    __shared__ float s_bias[BM];
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kMStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const int64_t j = n0 + threadIdx.x;
        s_bias[threadIdx.x] =
            ((EPI == EPI_RELU || EPI == EPI_LINEAR) && j < p.N) ? p.bias[j] : 0.0f;
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int kb = 0; kb < p.num_kb; ++kb) {
            const int s = kb % kMStages;
            if (kb >= kMStages && !mbar_wait(&empty[s], ((kb / kMStages) & 1) ^ 1)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            uint8_t* sb = smem + s * kMStageBytes;
            mbar_expect_tx(&full[s], kMStageBytes);
            tma_load_2d(sb, &ma, &full[s], kb * BK, (int)m0);
            tma_load_2d(sb + kMTile, &mb, &full[s], kb * BK, (int)n0);
            ++issued;
        }
        for (int kb = max(0, issued - kMStages); kb < issued; ++kb)
            if (!mbar_wait(&full[kb % kMStages], (kb / kMStages) & 1)) s_abort = 1;
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16_f32(BM, BM);
        for (int kb = 0; kb < p.num_kb; ++kb) {
            const int s = kb % kMStages;
            if (!mbar_wait(&full[s], (kb / kMStages) & 1)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * kMStageBytes);
            const uint32_t b = a + kMTile;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                umma_bf16(tmem, sdesc_sw128(a + kk * 32), sdesc_sw128(b + kk * 32), idesc,
                          (kb | kk) != 0 ? 1u : 0u);
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    __syncwarp();

    const bool ok = mbar_wait(done, 0);
    tc_fence_after();
    if (!ok) s_abort = 1;
    __syncthreads();
    if (!s_abort) {
        const int64_t m = m0 + warp * 32 + lane;
        const bool mv = m < p.M;
        const int cols = (int)(p.N - n0 < (int64_t)BM ? p.N - n0 : (int64_t)BM);
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < cols; c0 += 16) {
            float v[16];
            tmem_ld16(tbase + c0, v);
            const int64_t nb = n0 + c0;
            const bool fullc = c0 + 16 <= cols;
            if (EPI == EPI_RELU || EPI == EPI_LINEAR) {
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] += s_bias[c0 + t];
            }
            if (EPI == EPI_RELU) {
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] = fmaxf(v[t], 0.0f);
            }
            if (EPI == EPI_DRELU && mv) {
                const __nv_bfloat16* ar = p.act + m * p.ld_act + nb;
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (c0 + t < cols && !(__bfloat162float(ar[t]) > 0.0f)) v[t] = 0.0f;
            }
            if (mv) {
                if (EPI == EPI_RELU || EPI == EPI_DRELU) {
                    __nv_bfloat16* dst = p.out_h + m * p.ld_h + nb;
                    if (fullc && (p.ld_h & 7) == 0) {
                        __align__(16) __nv_bfloat16 hv[16];
#pragma unroll
                        for (int t = 0; t < 16; ++t) hv[t] = __float2bfloat16_rn(v[t]);
                        reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(hv)[0];
                        reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(hv)[1];
                    } else {
                        for (int t = 0; t < cols - c0 && t < 16; ++t)
                            dst[t] = __float2bfloat16_rn(v[t]);
                    }
                } else {
                    float* dst = p.out_f + m * p.ld_f + nb;
                    if (fullc && (p.ld_f & 3) == 0) {
#pragma unroll
                        for (int t = 0; t < 16; t += 4)
                            *reinterpret_cast<float4*>(dst + t) =
                                make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
                    } else {
                        for (int t = 0; t < cols - c0 && t < 16; ++t) dst[t] = v[t];
                    }
                }
            }
            if ((EPI == EPI_RELU || EPI == EPI_DRELU) && p.out_t != nullptr && mv) {
                // transposed copy: the 32 lanes write 32 consecutive rows of it
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (c0 + t < cols) p.out_t[(nb + t) * p.ld_t + m] = __float2bfloat16_rn(v[t]);
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(p.timeout_flag, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Element-wise and reduction kernels
// ---------------------------------------------------------------------------
// Split-mix 64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the finaliser of a Weyl sequence, used as a
// counter-based generator for the initial weights.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// He-uniform weights U(−√(6/fan_in), √(6/fan_in)), zero biases.
__global__ void k_mlp_init(float* __restrict__ W, int64_t rows, int64_t cols, float lim,
                           uint64_t seed) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = splitmix64(seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(e + 1)));
        const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
        W[e] = (float)((2.0 * u - 1.0) * lim);
    }
}

// C = α·A·B + β·Cin for row-major FP32 matrices (A M×K, B K×N), on the FP32
// pipe: 128×128 tiles, K steps of 8 through shared memory, 8×8 outputs per
// thread (rows ty·4 + {0..3} and +64, columns tx·4 + {0..3} and +64).
constexpr int kSgT = 128;
constexpr int kSgK = 8;
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, float alpha,
                                               const float* __restrict__ A, int64_t lda,
                                               const float* __restrict__ B, int64_t ldb,
                                               float beta, const float* __restrict__ Cin,
                                               int64_t ldcin, float* __restrict__ C,
                                               int64_t ldc) {
    __shared__ __align__(16) float As[kSgK][kSgT];
    __shared__ __align__(16) float Bs[kSgK][kSgT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * kSgT, n0 = (int64_t)blockIdx.x * kSgT;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kSgK) {
        // A tile 128×8 (stored transposed), B tile 8×128: 4 values each per thread
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;
            const int ar = e >> 3, ak = e & 7;
            const int64_t gm = m0 + ar;
            const int gk = k0 + ak;
            As[ak][ar] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.f;
            const int bk = e >> 7, bc = e & 127;
            const int64_t gn = n0 + bc;
            const int gk2 = k0 + bk;
            Bs[bk][bc] = (gn < N && gk2 < K) ? B[(int64_t)gk2 * ldb + gn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kSgK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t cc = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
            if (cc >= N) continue;
            float v = alpha * acc[i][j];
            if (beta != 0.f) v = fmaf(beta, Cin[r * ldcin + cc], v);
            C[r * ldc + cc] = v;
        }
    }
}

// Q (FP32 or FP64, row stride ldq) → dense FP32 n×n, and the row sums of
// |Q| (one block per row) for the Newton–Schulz start.
template <typename T>
__global__ void __launch_bounds__(256) k_q_to_f32(const T* __restrict__ Q, int64_t ldq, int n,
                                                  float* __restrict__ out,
                                                  double* __restrict__ rowabs) {
    __shared__ double scratch[32];
    const int i = blockIdx.x;
    double a = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = (double)Q[(int64_t)i * ldq + j];
        out[(int64_t)i * n + j] = (float)v;
        a += fabs(v);
    }
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) rowabs[i] = a;
}

// X = I/‖Q‖∞ (‖Q‖∞ = the largest row sum of |Q|, ≥ λ_max for symmetric Q),
// the Newton–Schulz start; one grid over the n×n entries.
__global__ void k_ns_start(const double* __restrict__ rowabs, int n, float* __restrict__ X) {
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, rowabs[i]);
        s_inv = m > 0.0 ? 1.0 / m : 1.0;
    }
    __syncthreads();
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        X[e] = (e / n == e % n) ? (float)s_inv : 0.f;
}

// R = I − T in place, and per-block partial sums of ‖R‖_F² (one block per row).
__global__ void __launch_bounds__(256) k_ns_resid(float* __restrict__ T, int n,
                                                  double* __restrict__ part) {
    __shared__ double scratch[32];
    const int i = blockIdx.x;
    double a = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float r = (i == j ? 1.f : 0.f) - T[(int64_t)i * n + j];
        T[(int64_t)i * n + j] = r;
        a = fma((double)r, (double)r, a);
    }
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) part[i] = a;
}

// Σ part[0..np) in a fixed order (one block).
__global__ void k_sum_parts(const double* __restrict__ part, int np, double* __restrict__ out) {
    __shared__ double scratch[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) *out = a;
}

// First half of the features for the rows idx[b] of Q (FP64, row stride ldq):
// qn[b] = ‖q_b‖, u_b[0..n) = (q_b/‖q_b‖ − μ)/σ in BF16, and the FP32 unit
// row q_b/‖q_b‖ (0 when q_b = 0) for the direction product.  One block per row.
__global__ void __launch_bounds__(256) k_mlp_features(const double* __restrict__ Qs, int64_t ldq,
                                                      const int* __restrict__ idx, int n,
                                                      const float* __restrict__ mu,
                                                      const float* __restrict__ sd,
                                                      __nv_bfloat16* __restrict__ U, int64_t ldu,
                                                      float* __restrict__ qn,
                                                      float* __restrict__ Qn, int64_t ldqn) {
    __shared__ double scratch[32];
    __shared__ double s_inv;
    const int b = blockIdx.x;
    const double* q = Qs + (int64_t)(idx ? idx[b] : b) * ldq;
    double a = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) a = fma(q[j], q[j], a);
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) {
        const double nr = sqrt(a);
        qn[b] = (float)nr;
        s_inv = nr > 0.0 ? 1.0 / nr : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    __nv_bfloat16* u = U + (int64_t)b * ldu;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float qv = (float)(q[j] * inv);
        u[j] = __float2bfloat16_rn(inv > 0.0 ? (qv - mu[j]) / sd[j] : 0.f);
        if (Qn) Qn[(int64_t)b * ldqn + j] = qv;
    }
}

// Second half of the features from the direction rows zp_b = z_b/‖q_b‖ (the
// rows idx[b] of Zp, or row b): u_b[n..2n) = (zp − μz)/σz in BF16 (0 when
// q_b = 0), and the skip input ẑ_b = zp_b/τ (FP32).
__global__ void __launch_bounds__(256) k_mlp_zfeatures(const float* __restrict__ Zp,
                                                       int64_t ldz, const int* __restrict__ idx,
                                                       int n, const float* __restrict__ qn,
                                                       const float* __restrict__ muz,
                                                       const float* __restrict__ sdz,
                                                       float inv_tau,
                                                       __nv_bfloat16* __restrict__ U, int64_t ldu,
                                                       float* __restrict__ Zt, int64_t ldzt) {
    const int b = blockIdx.x;
    const float* z = Zp + (int64_t)(idx ? idx[b] : b) * ldz;
    const bool live = qn[b] > 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float zv = live ? z[j] : 0.f;
        U[(int64_t)b * ldu + n + j] = __float2bfloat16_rn(live ? (zv - muz[j]) / sdz[j] : 0.f);
        Zt[(int64_t)b * ldzt + j] = zv * inv_tau;
    }
}

// Per-entry skips: o_b[j] += e_j·ẑ_bj, o_b[n + j] += f_j·ẑ_bj.
__global__ void k_mlp_skip(float* __restrict__ O, int64_t ldo, const float* __restrict__ Zt,
                           int64_t ldzt, const float* __restrict__ e, const float* __restrict__ f,
                           int B, int n) {
    const int64_t total = (int64_t)B * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / n), j = (int)(t - (int64_t)b * n);
        const float zt = Zt[(int64_t)b * ldzt + j];
        O[(int64_t)b * ldo + j] += e[j] * zt;
        O[(int64_t)b * ldo + n + j] += f[j] * zt;
    }
}

// Column sums of the direction rows over a chunk (FP64, one thread per column,
// rows in order), added to the running sums s1 (Σ zp) and s2 (Σ zp²).
__global__ void k_zmoments(const float* __restrict__ Zp, int64_t ldz, int rows, int n,
                           const float* __restrict__ qn, double* __restrict__ s1,
                           double* __restrict__ s2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double a = 0.0, c = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double z = qn[r] > 0.f ? (double)Zp[(int64_t)r * ldz + j] : 0.0;
        a += z;
        c = fma(z, z, c);
    }
    s1[j] += a;
    s2[j] += c;
}

// μz = s1/count, σz = sqrt(s2/count − μz²) (σz := 1 when 0).
__global__ void k_zmoments_final(const double* __restrict__ s1, const double* __restrict__ s2,
                                 int64_t count, int n, float* __restrict__ muz,
                                 float* __restrict__ sdz) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double m = s1[j] / (double)count;
    const double v = fmax(s2[j] / (double)count - m * m, 0.0);
    const double sd = sqrt(v);
    muz[j] = (float)m;
    sdz[j] = sd > 0.0 ? (float)sd : 1.f;
}

// out[c][r] = in[r][c] for an R×C BF16 matrix, 32×32 tiles through shared memory.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int64_t ldi, int64_t R,
                                 int64_t C, __nv_bfloat16* __restrict__ out, int64_t ldo) {
    __shared__ __nv_bfloat16 t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < R && c < C) t[k][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < R && c < C) out[c * ldo + r] = t[threadIdx.x][k];
    }
}

// Loss terms and dL/do for a batch: o = [ŷ ; ℓ] (FP32, B × 2n), targets
// y*/(τ‖q‖) from the rows idx[b] of Y (FP64, y* in the scaled space) and qn.  Writes dO in
// BF16 (row-major and transposed) and one loss partial per block.
// With Zt, also the skip gradients' block partials: pe[by·n + j] = Σ_b
// dL/dŷ_bj·ẑ_bj and pf likewise with dL/dℓ_bj, over the block's 32 rows.
__global__ void k_mlp_loss(const float* __restrict__ O, int64_t ldo, const double* __restrict__ Y,
                           int64_t ldy, const int* __restrict__ idx, const float* __restrict__ qn,
                           int B, int n, float inv_m, float tau, __nv_bfloat16* __restrict__ dO,
                           int64_t ldd,
                           __nv_bfloat16* __restrict__ dOT, int64_t lddt,
                           double* __restrict__ part, const float* __restrict__ Zt,
                           int64_t ldzt, float* __restrict__ pe, float* __restrict__ pf) {
    __shared__ float t1[32][33], t2[32][33];
    __shared__ double scratch[32];
    __shared__ float se[8][32], sf[8][32];
    const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 × 8
    double acc = 0.0;
    float ae = 0.0f, af = 0.0f;
    for (int k = ty; k < 32; k += blockDim.y) {
        const int b = b0 + k, j = j0 + tx;
        float d1 = 0.0f, d2 = 0.0f;
        if (b < B && j < n) {
            const float yh = O[(int64_t)b * ldo + j];
            const float lg = O[(int64_t)b * ldo + n + j];
            const double ys = Y[(int64_t)(idx ? idx[b] : b) * ldy + j];
            const float q = qn[b];
            const float t = q > 0.0f ? (float)(ys / ((double)q * (double)tau)) : 0.0f;
            const float c = ys > 0.0 ? 1.0f : 0.0f;
            const float e = yh - t;
            const float bce = fmaxf(lg, 0.0f) - lg * c + log1pf(expf(-fabsf(lg)));
            acc += (double)(e * e) + (double)bce;
            d1 = 2.0f * e * inv_m;
            d2 = (1.0f / (1.0f + expf(-lg)) - c) * inv_m;
            dO[(int64_t)b * ldd + j] = __float2bfloat16_rn(d1);
            dO[(int64_t)b * ldd + n + j] = __float2bfloat16_rn(d2);
            if (Zt) {
                const float zt = Zt[(int64_t)b * ldzt + j];
                ae = fmaf(d1, zt, ae);
                af = fmaf(d2, zt, af);
            }
        }
        t1[k][tx] = d1;
        t2[k][tx] = d2;
    }
    se[ty][tx] = ae;
    sf[ty][tx] = af;
    __syncthreads();
    if (Zt && ty == 0 && j0 + tx < n) {
        float a1 = 0.0f, a2 = 0.0f;
        for (int k = 0; k < 8; ++k) {
            a1 += se[k][tx];
            a2 += sf[k][tx];
        }
        pe[(int64_t)blockIdx.y * n + j0 + tx] = a1;
        pf[(int64_t)blockIdx.y * n + j0 + tx] = a2;
    }
    for (int k = ty; k < 32; k += blockDim.y) {
        const int j = j0 + k, b = b0 + tx;
        if (b < B && j < n) {
            dOT[(int64_t)j * lddt + b] = __float2bfloat16_rn(t1[tx][k]);
            dOT[(int64_t)(n + j) * lddt + b] = __float2bfloat16_rn(t2[tx][k]);
        }
    }
    // block sum of the loss terms (256 threads)
    const int tid = ty * 32 + tx;
    const int lane = tid & 31, wid = tid >> 5;
    double v = warp_sum(acc);
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x * blockDim.y) / 32; ++w) s += scratch[w];
        part[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// Deterministic sum of the loss partials, times 1/m.
__global__ void k_mlp_loss_sum(const double* __restrict__ part, int np, double inv_m,
                               double* __restrict__ out) {
    __shared__ double scratch[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) *out = a * inv_m;
}

// g[j] = Σ_y part[y·n + j] over the row blocks in order (skip gradients).
__global__ void k_colsum_parts(const float* __restrict__ part, int ny, int n,
                               float* __restrict__ g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double a = 0.0;
    for (int y = 0; y < ny; ++y) a += (double)part[(int64_t)y * n + j];
    g[j] = (float)a;
}

// g[r] = Σ_c X[r][c] (bias gradient from a transposed BF16 gradient).
__global__ void __launch_bounds__(256) k_rowsum_bf16(const __nv_bfloat16* __restrict__ X,
                                                     int64_t ld, int64_t C,
                                                     float* __restrict__ g) {
    __shared__ double scratch[32];
    const __nv_bfloat16* x = X + (int64_t)blockIdx.x * ld;
    float a = 0.0f;
    for (int64_t c = threadIdx.x; c < C; c += blockDim.x) a += __bfloat162float(x[c]);
    const double s = block_sum((double)a, scratch);
    if (threadIdx.x == 0) g[blockIdx.x] = (float)s;
}

// One Adam step on an R×C FP32 tensor (gradient G with row stride ldg);
// refreshes the BF16 copy Wh (row stride ldh) and, when WT is set, its
// transpose (row stride ldt), through a 32×32 shared-memory tile.
__global__ void k_adam(float* __restrict__ W, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ G, int64_t ldg, int64_t R, int64_t C, float lr,
                       float beta1, float beta2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ Wh, int64_t ldh, __nv_bfloat16* __restrict__ WT,
                       int64_t ldt) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, cb = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = cb + threadIdx.x;
        if (r < R && c < C) {
            const int64_t e = r * C + c;
            const float g = G[r * ldg + c];
            const float mm = beta1 * m[e] + (1.0f - beta1) * g;
            const float vv = beta2 * v[e] + (1.0f - beta2) * g * g;
            m[e] = mm;
            v[e] = vv;
            const float w = W[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
            W[e] = w;
            const __nv_bfloat16 h = __float2bfloat16_rn(w);
            if (Wh) Wh[r * ldh + c] = h;
            tile[k][threadIdx.x] = h;
        }
    }
    if (WT == nullptr) return;  // uniform over the block
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = cb + k, r = r0 + threadIdx.x;
        if (r < R && c < C) WT[c * ldt + r] = tile[threadIdx.x][k];
    }
}

// BF16 copies of an FP32 tensor and of its transpose (used after init/set).
__global__ void k_to_bf16(const float* __restrict__ W, int64_t R, int64_t C,
                          __nv_bfloat16* __restrict__ Wh, int64_t ldh,
                          __nv_bfloat16* __restrict__ WT, int64_t ldt) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, cb = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = cb + threadIdx.x;
        if (r < R && c < C) {
            const __nv_bfloat16 h = __float2bfloat16_rn(W[r * C + c]);
            Wh[r * ldh + c] = h;
            tile[k][threadIdx.x] = h;
        }
    }
    if (WT == nullptr) return;
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = cb + k, r = r0 + threadIdx.x;
        if (r < R && c < C) WT[c * ldt + r] = tile[threadIdx.x][k];
    }
}

// d = relu(ŷ)·[ℓ > 0]: FP32 and BF16 copies (B × n).
__global__ void k_mlp_post(const float* __restrict__ O, int64_t ldo, int B, int n,
                           float* __restrict__ D, __nv_bfloat16* __restrict__ Dh, int64_t ldy) {
    const int64_t total = (int64_t)B * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), j = (int)(e - (int64_t)b * n);
        const float yh = O[(int64_t)b * ldo + j], lg = O[(int64_t)b * ldo + n + j];
        const float dv = lg > 0.0f ? fmaxf(yh, 0.0f) : 0.0f;
        D[(int64_t)b * ldy + j] = dv;
        Dh[(int64_t)b * ldy + j] = __float2bfloat16_rn(dv);
    }
}

// Exact line search of Alg. 2 from 0 along d: α* = max(0, −qᵀd/dᵀQd)
// (0 when dᵀQd ≤ 0), y⁰ = α*·d, x⁰ = y⁰/s (FP64, row stride ldx).
// QD holds Q·d (FP32).  One block per row.
__global__ void __launch_bounds__(256) k_mlp_linesearch(
    const float* __restrict__ D, const float* __restrict__ QD, int64_t ldy,
    const double* __restrict__ q64, int64_t ldq, const double* __restrict__ s, int n,
    double* __restrict__ X0, int64_t ldx, int* __restrict__ kept) {
    __shared__ double scratch[32];
    __shared__ double s_alpha;
    const int b = blockIdx.x;
    const float* d = D + (int64_t)b * ldy;
    const float* qd = QD + (int64_t)b * ldy;
    const double* q = q64 + (int64_t)b * ldq;
    double num = 0.0, den = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        num -= q[j] * (double)d[j];
        den += (double)d[j] * (double)qd[j];
    }
    num = block_sum(num, scratch);
    den = block_sum(den, scratch);
    if (threadIdx.x == 0) {
        const double a = (num > 0.0 && den > 0.0) ? num / den : 0.0;
        s_alpha = a;
        if (kept) kept[b] = a > 0.0 ? 1 : 0;
    }
    __syncthreads();
    const double a = s_alpha;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        X0[(int64_t)b * ldx + j] = a * (double)d[j] / s[j];
}

// Normalisation statistics of a training set (count rows of q and y*, FP64):
// per-row ‖q‖, then per column Σ u, Σ u², Σ t² with u = q/‖q‖, t = y*/‖q‖,
// in G row groups (partials), then μ, σ and τ.
__global__ void __launch_bounds__(256) k_rownorm(const double* __restrict__ Qs, int64_t count,
                                                 int n, double* __restrict__ qn) {
    __shared__ double scratch[32];
    const double* q = Qs + (int64_t)blockIdx.x * n;
    double a = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) a = fma(q[j], q[j], a);
    a = block_sum(a, scratch);
    if (threadIdx.x == 0) qn[blockIdx.x] = sqrt(a);
}

__global__ void k_colmoments(const double* __restrict__ Qs, const double* __restrict__ Ys,
                             const double* __restrict__ qn, int64_t count, int n,
                             double* __restrict__ part) {
    __shared__ double r1[8][33], r2[8][33], r3[8][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (j < n) {
        for (int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; i < count;
             i += (int64_t)gridDim.y * blockDim.y) {
            const double inv = qn[i] > 0.0 ? 1.0 / qn[i] : 0.0;
            const double u = Qs[i * n + j] * inv, t = Ys[i * n + j] * inv;
            a1 += u;
            a2 = fma(u, u, a2);
            a3 = fma(t, t, a3);
        }
    }
    r1[threadIdx.y][threadIdx.x] = a1;
    r2[threadIdx.y][threadIdx.x] = a2;
    r3[threadIdx.y][threadIdx.x] = a3;
    __syncthreads();
    if (threadIdx.y == 0 && j < n) {
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int k = 0; k < (int)blockDim.y; ++k) {
            s1 += r1[k][threadIdx.x];
            s2 += r2[k][threadIdx.x];
            s3 += r3[k][threadIdx.x];
        }
        double* p = part + ((int64_t)blockIdx.y * n + j) * 3;
        p[0] = s1;
        p[1] = s2;
        p[2] = s3;
    }
}

__global__ void __launch_bounds__(256) k_colstats_final(const double* __restrict__ part, int G,
                                                        int64_t count, int n,
                                                        float* __restrict__ mu,
                                                        float* __restrict__ sd,
                                                        float* __restrict__ tau) {
    __shared__ double scratch[32];
    double t3 = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int g = 0; g < G; ++g) {
            const double* p = part + ((int64_t)g * n + j) * 3;
            s1 += p[0];
            s2 += p[1];
            s3 += p[2];
        }
        const double m = s1 / (double)count;
        const double var = fmax(s2 / (double)count - m * m, 0.0);
        mu[j] = (float)m;
        sd[j] = var > 0.0 ? (float)sqrt(var) : 1.0f;
        t3 += s3;
    }
    t3 = block_sum(t3, scratch);
    if (threadIdx.x == 0) {
        const double r = sqrt(t3 / ((double)count * n));
        *tau = r > 0.0 ? (float)r : 1.0f;
    }
}

__global__ void k_fill(float* __restrict__ p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

template <typename T>
__global__ void k_q_to_bf16(const T* __restrict__ Q, int64_t ldq, int n,
                            __nv_bfloat16* __restrict__ Qh, int64_t ldh) {
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e - i * n;
        Qh[i * ldh + j] = __float2bfloat16_rn((float)Q[i * ldq + j]);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
inline int64_t ld8(int64_t c) { return round_up(std::max<int64_t>(c, 1), 64); }

struct Tensor {
    int64_t R = 0, C = 0;
    float* w = nullptr;         // FP32 master, R×C dense
    float* m = nullptr;
    float* v = nullptr;
    float* g = nullptr;         // gradient, R×C (row stride ldg)
    int64_t ldg = 0;
    __nv_bfloat16* h = nullptr;  // BF16 copy, row stride ldh
    int64_t ldh = 0;
    __nv_bfloat16* t = nullptr;  // BF16 transpose (C×R), row stride ldt
    int64_t ldt = 0;
};

struct Mlp {
    int n = 0, hidden = 0;
    int64_t in = 0, out = 0;     // 2n
    Tensor W[3], b[3];
    Tensor e, f;                 // per-entry skips from ẑ to ŷ and to ℓ (n each)
    float* Minv = nullptr;       // Q⁻¹ (n×n FP32, Newton–Schulz)
    int ns_iters = 0;            // Newton–Schulz iterations it took
    double ns_resid = 0.0;       // ‖I − Q·Q⁻¹‖_F at the end
    float* mu = nullptr;         // feature normalisation (n), σ (n), τ (1)
    float* sd = nullptr;
    float* muz = nullptr;        // direction-feature normalisation (n each)
    float* sdz = nullptr;
    float* tau = nullptr;
    float tau_host = 1.0f;
    bool stats_set = false;      // μ, σ, τ taken from a training set or set
    void* wpool = nullptr;       // weights, moments, gradients, copies
    size_t wbytes = 0;
    int64_t step = 0;            // Adam steps taken

    // activations for a batch of at most Bcap rows
    int Bcap = 0;
    void* apool = nullptr;
    size_t abytes = 0;
    __nv_bfloat16 *U = nullptr, *UT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr,
                  *H2T = nullptr, *dO = nullptr, *dOT = nullptr, *dZ2 = nullptr, *dZ2T = nullptr,
                  *dZ1 = nullptr, *dZ1T = nullptr, *Y0h = nullptr, *Qh = nullptr;
    float *O = nullptr, *Y0 = nullptr, *QY = nullptr, *qn = nullptr;
    float *Qn = nullptr, *Zp = nullptr, *Zt = nullptr;  // unit q rows, z/‖q‖, ẑ (B × ldY)
    float *pe = nullptr, *pf = nullptr;                 // skip-gradient block partials
    double* part = nullptr;
    double* lossv = nullptr;
    int* idx = nullptr;
    int64_t ldU = 0, ldUT = 0, ldH = 0, ldHT = 0, ldO = 0, ldOT = 0, ldY = 0, ldQh = 0;
    int qh_n = -1;
    int* hflag = nullptr;        // pinned
    double* hloss = nullptr;     // pinned
    // prediction outputs kept between calls (no allocation per prediction):
    // the kept flags, and the start points when the caller's X0 is on the host
    int* kept = nullptr;
    int64_t kept_cap = 0;
    double* xtmp = nullptr;
    size_t xtmp_bytes = 0;
};

#define M_TRY(call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) {                             \
            if (e_ == cudaErrorMemoryAllocation) {           \
                cudaGetLastError();                          \
                return ALN_ERR_OUT_OF_MEMORY;                \
            }                                                \
            return ALN_ERR_CUDA;                             \
        }                                                    \
    } while (0)
#define M_CHECK(call)                 \
    do {                              \
        aln_status s_ = (call);       \
        if (s_ != ALN_OK) return s_;  \
    } while (0)

void free_mlp(Mlp* m) {
    if (!m) return;
    if (m->wpool) cudaFree(m->wpool);
    if (m->apool) cudaFree(m->apool);
    if (m->hflag) cudaFreeHost(m->hflag);
    if (m->kept) cudaFree(m->kept);
    if (m->xtmp) cudaFree(m->xtmp);
    delete m;
}

aln_status alloc_weights(aln_ctx* c, Mlp* M) {
    const int64_t dims[3][2] = {{M->hidden, M->in}, {M->hidden, M->hidden}, {M->out, M->hidden}};
    size_t total = 0;
    auto add = [&](size_t bytes) { total += round_up((int64_t)bytes, 256); };
    for (int l = 0; l < 3; ++l) {
        const int64_t R = dims[l][0], C = dims[l][1];
        for (int k = 0; k < 4; ++k) add((size_t)R * C * 4);            // w m v g
        add((size_t)R * ld8(C) * 2);                                    // h
        add((size_t)C * ld8(R) * 2);                                    // t
        for (int k = 0; k < 4; ++k) add((size_t)R * 4);                 // bias w m v g
        add((size_t)ld8(R) * 2);                                        // bias h (unused)
    }
    for (int k = 0; k < 2; ++k)
        for (int t = 0; t < 4; ++t) add((size_t)M->n * 4);           // e, f: w m v g
    add((size_t)M->n * M->n * 4);  // Q⁻¹
    add((size_t)M->n * 4);  // mu
    add((size_t)M->n * 4);  // sd
    add((size_t)M->n * 4);  // muz
    add((size_t)M->n * 4);  // sdz
    add(4);                 // tau
    if (cudaMalloc(&M->wpool, total) != cudaSuccess) {
        cudaGetLastError();
        M->wpool = nullptr;
        return ALN_ERR_OUT_OF_MEMORY;
    }
    M->wbytes = total;
    M_TRY(cudaMemsetAsync(M->wpool, 0, total, c->stream));
    uint8_t* p = (uint8_t*)M->wpool;
    auto take = [&](size_t bytes) {
        void* r = p;
        p += round_up((int64_t)bytes, 256);
        return r;
    };
    for (int l = 0; l < 3; ++l) {
        const int64_t R = dims[l][0], C = dims[l][1];
        Tensor& W = M->W[l];
        W.R = R;
        W.C = C;
        W.w = (float*)take((size_t)R * C * 4);
        W.m = (float*)take((size_t)R * C * 4);
        W.v = (float*)take((size_t)R * C * 4);
        W.g = (float*)take((size_t)R * C * 4);
        W.ldg = C;
        W.ldh = ld8(C);
        W.h = (__nv_bfloat16*)take((size_t)R * W.ldh * 2);
        W.ldt = ld8(R);
        W.t = (__nv_bfloat16*)take((size_t)C * W.ldt * 2);
        Tensor& b = M->b[l];
        b.R = 1;
        b.C = R;
        b.w = (float*)take((size_t)R * 4);
        b.m = (float*)take((size_t)R * 4);
        b.v = (float*)take((size_t)R * 4);
        b.g = (float*)take((size_t)R * 4);
        b.ldg = R;
        b.ldh = ld8(R);
        b.h = (__nv_bfloat16*)take((size_t)b.ldh * 2);
    }
    for (int k = 0; k < 2; ++k) {
        Tensor& T = k == 0 ? M->e : M->f;
        T.R = 1;
        T.C = M->n;
        T.w = (float*)take((size_t)M->n * 4);
        T.m = (float*)take((size_t)M->n * 4);
        T.v = (float*)take((size_t)M->n * 4);
        T.g = (float*)take((size_t)M->n * 4);
        T.ldg = M->n;
    }
    M->Minv = (float*)take((size_t)M->n * M->n * 4);
    M->mu = (float*)take((size_t)M->n * 4);
    M->sd = (float*)take((size_t)M->n * 4);
    M->muz = (float*)take((size_t)M->n * 4);
    M->sdz = (float*)take((size_t)M->n * 4);
    M->tau = (float*)take(4);
    return ALN_OK;
}

aln_status alloc_acts(aln_ctx* c, Mlp* M, int B) {
    if (M->apool && M->Bcap >= B && M->qh_n == M->n) return ALN_OK;
    if (M->apool) cudaFree(M->apool);
    M->apool = nullptr;
    M->Bcap = std::max(B, 128);
    const int64_t Bc = M->Bcap, in = M->in, out = M->out, Hd = M->hidden, n = M->n;
    M->ldU = ld8(in);
    M->ldUT = ld8(Bc);
    M->ldH = ld8(Hd);
    M->ldHT = ld8(Bc);
    M->ldO = ld8(out);
    M->ldOT = ld8(Bc);
    M->ldY = ld8(n);
    M->ldQh = ld8(n);
    const size_t sz[] = {
        (size_t)Bc * M->ldU * 2, (size_t)in * M->ldUT * 2,                      // U UT
        (size_t)Bc * M->ldH * 2, (size_t)Hd * M->ldHT * 2,                      // H1 H1T
        (size_t)Bc * M->ldH * 2, (size_t)Hd * M->ldHT * 2,                      // H2 H2T
        (size_t)Bc * M->ldO * 2, (size_t)out * M->ldOT * 2,                     // dO dOT
        (size_t)Bc * M->ldH * 2, (size_t)Hd * M->ldHT * 2,                      // dZ2 dZ2T
        (size_t)Bc * M->ldH * 2, (size_t)Hd * M->ldHT * 2,                      // dZ1 dZ1T
        (size_t)Bc * M->ldY * 2, (size_t)n * M->ldQh * 2,                       // Y0h Qh
        (size_t)Bc * M->ldO * 4, (size_t)Bc * M->ldY * 4, (size_t)Bc * M->ldY * 4,  // O Y0 QY
        (size_t)Bc * 4,                                                         // qn
        (size_t)Bc * M->ldY * 4, (size_t)Bc * M->ldY * 4, (size_t)Bc * M->ldY * 4,  // Qn Zp Zt
        (size_t)ceil_div(Bc, 32) * n * 4, (size_t)ceil_div(Bc, 32) * n * 4,     // pe pf
        (size_t)ceil_div(n, 32) * ceil_div(Bc, 32) * 8 + 64,                    // part
        64,                                                                     // loss
        (size_t)Bc * 4,                                                         // idx
    };
    size_t total = 0;
    for (size_t b : sz) total += round_up((int64_t)b, 256);
    if (cudaMalloc(&M->apool, total) != cudaSuccess) {
        cudaGetLastError();
        M->apool = nullptr;
        return ALN_ERR_OUT_OF_MEMORY;
    }
    M->abytes = total;
    M_TRY(cudaMemsetAsync(M->apool, 0, total, c->stream));
    uint8_t* p = (uint8_t*)M->apool;
    int k = 0;
    auto take = [&]() {
        void* r = p;
        p += round_up((int64_t)sz[k++], 256);
        return r;
    };
    M->U = (__nv_bfloat16*)take();
    M->UT = (__nv_bfloat16*)take();
    M->H1 = (__nv_bfloat16*)take();
    M->H1T = (__nv_bfloat16*)take();
    M->H2 = (__nv_bfloat16*)take();
    M->H2T = (__nv_bfloat16*)take();
    M->dO = (__nv_bfloat16*)take();
    M->dOT = (__nv_bfloat16*)take();
    M->dZ2 = (__nv_bfloat16*)take();
    M->dZ2T = (__nv_bfloat16*)take();
    M->dZ1 = (__nv_bfloat16*)take();
    M->dZ1T = (__nv_bfloat16*)take();
    M->Y0h = (__nv_bfloat16*)take();
    M->Qh = (__nv_bfloat16*)take();
    M->O = (float*)take();
    M->Y0 = (float*)take();
    M->QY = (float*)take();
    M->qn = (float*)take();
    M->Qn = (float*)take();
    M->Zp = (float*)take();
    M->Zt = (float*)take();
    M->pe = (float*)take();
    M->pf = (float*)take();
    M->part = (double*)take();
    M->lossv = (double*)take();
    M->idx = (int*)take();
    M->qh_n = M->n;
    return ALN_OK;
}

// D = A·Bᵀ: A is M×K (row stride lda), B is N×K (row stride ldb), BF16.
template <int EPI>
aln_status gemm(aln_ctx* c, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* Bm,
                int64_t ldb, int64_t Mr, int64_t N, int64_t K, GemmArgs a) {
    static bool attr = false;
    if (!attr) {
        M_TRY(cudaFuncSetAttribute(k_mlp_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kMSmem));
        attr = true;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, K, Mr, lda) || !make_map(&mb, Bm, K, N, ldb)) return ALN_ERR_CUDA;
    a.M = Mr;
    a.N = N;
    a.num_kb = (int)ceil_div(K, BK);
    a.timeout_flag = c->flags + 1;
    const dim3 grid((unsigned)ceil_div(Mr, BM), (unsigned)ceil_div(N, BM));
    k_mlp_gemm<EPI><<<grid, 128, kMSmem, c->stream>>>(ma, mb, a);
    M_TRY(cudaGetLastError());
    c->launches += 1;
    return ALN_OK;
}

GemmArgs args0() {
    GemmArgs a = {};
    return a;
}

// C = α·A·B + β·Cin (row-major FP32) on the FP32 pipe.
aln_status sgemm(aln_ctx* c, int Mr, int N, int K, float alpha, const float* A, int64_t lda,
                 const float* B, int64_t ldb, float beta, const float* Cin, int64_t ldcin,
                 float* C, int64_t ldc) {
    const dim3 grid((unsigned)ceil_div(N, kSgT), (unsigned)ceil_div(Mr, kSgT));
    k_sgemm<<<grid, 256, 0, c->stream>>>(Mr, N, K, alpha, A, lda, B, ldb, beta, Cin, ldcin, C,
                                         ldc);
    M_TRY(cudaGetLastError());
    c->launches += 1;
    return ALN_OK;
}

// Q⁻¹ of the prepared Q by the Newton–Schulz iteration X ← X(2I − QX)
// (Schulz 1933): with X₀ = I/‖Q‖∞ every eigenvalue of R₀ = I − QX₀ lies in
// [0, 1) for a positive definite Q, and R_{k+1} = R_k², so the residual
// squares every step once it is below 1.  Each step: T = Q·X, R = I − T,
// X ← X + X·R (two FP32 GEMMs).  It stops when ‖R‖_F < 1e-4, when ‖R‖_F has
// stopped falling (the FP32 floor, about cond(Q)·2⁻²⁴·√n), or after 100 steps.
aln_status ns_inverse(aln_ctx* c, Mlp* M) {
    const int n = M->n;
    const size_t nn = (size_t)n * n;
    float *Q32 = nullptr, *T = nullptr, *X2 = nullptr;
    double* part = nullptr;
    aln_status st = ALN_OK;
    if (cudaMalloc(&Q32, nn * 4) != cudaSuccess || cudaMalloc(&T, nn * 4) != cudaSuccess ||
        cudaMalloc(&X2, nn * 4) != cudaSuccess ||
        cudaMalloc(&part, ((size_t)n + 8) * 8) != cudaSuccess) {
        cudaGetLastError();
        st = ALN_ERR_OUT_OF_MEMORY;
    }
    double* rsum = part + n;
    float* X = M->Minv;
    if (st == ALN_OK) {
        if (c->opt.precision == ALN_PREC_FP64)
            k_q_to_f32<double><<<n, 256, 0, c->stream>>>((const double*)c->Q, c->ldq, n, Q32, part);
        else
            k_q_to_f32<float><<<n, 256, 0, c->stream>>>((const float*)c->Q, c->ldq, n, Q32, part);
        k_ns_start<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)nn, 256), 8192), 256, 0,
                     c->stream>>>(part, n, X);
        if (cudaGetLastError() != cudaSuccess) st = ALN_ERR_CUDA;
        c->launches += 2;
    }
    double prev = 1e300;
    int it = 0;
    for (; st == ALN_OK && it < 100; ++it) {
        st = sgemm(c, n, n, n, 1.f, Q32, n, X, n, 0.f, nullptr, 0, T, n);
        if (st != ALN_OK) break;
        k_ns_resid<<<n, 256, 0, c->stream>>>(T, n, part);
        k_sum_parts<<<1, 256, 0, c->stream>>>(part, n, rsum);
        c->launches += 2;
        st = sgemm(c, n, n, n, 1.f, X, n, T, n, 1.f, X, n, X2, n);
        if (st != ALN_OK) break;
        if (cudaMemcpyAsync(M->hloss, rsum, 8, cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(X, X2, nn * 4, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            st = ALN_ERR_CUDA;
            break;
        }
        const double r = std::sqrt(std::max(*M->hloss, 0.0));
        M->ns_resid = r;
        if (!std::isfinite(r)) {
            st = ALN_ERR_NONFINITE;
            break;
        }
        if (r < 1e-4 || (r < 1.0 && r > 0.5 * prev)) {
            ++it;
            break;
        }
        prev = r;
    }
    M->ns_iters = it;
    if (Q32) cudaFree(Q32);
    if (T) cudaFree(T);
    if (X2) cudaFree(X2);
    if (part) cudaFree(part);
    return st;
}

// Forward pass of a batch already in M->U (B rows).  With `train`, also the
// transposed activations the backward products need.
aln_status forward(aln_ctx* c, Mlp* M, int B, bool train) {
    GemmArgs a = args0();
    a.bias = M->b[0].w;
    a.out_h = M->H1;
    a.ld_h = M->ldH;
    a.out_t = train ? M->H1T : nullptr;
    a.ld_t = M->ldHT;
    M_CHECK(gemm<EPI_RELU>(c, M->U, M->ldU, M->W[0].h, M->W[0].ldh, B, M->hidden, M->in, a));
    a = args0();
    a.bias = M->b[1].w;
    a.out_h = M->H2;
    a.ld_h = M->ldH;
    a.out_t = train ? M->H2T : nullptr;
    a.ld_t = M->ldHT;
    M_CHECK(gemm<EPI_RELU>(c, M->H1, M->ldH, M->W[1].h, M->W[1].ldh, B, M->hidden, M->hidden, a));
    a = args0();
    a.bias = M->b[2].w;
    a.out_f = M->O;
    a.ld_f = M->ldO;
    M_CHECK(gemm<EPI_LINEAR>(c, M->H2, M->ldH, M->W[2].h, M->W[2].ldh, B, M->out, M->hidden, a));
    k_mlp_skip<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)B * M->n, 256), 8192), 256, 0,
                 c->stream>>>(M->O, M->ldO, M->Zt, M->ldY, M->e.w, M->f.w, B, M->n);
    M_TRY(cudaGetLastError());
    c->launches += 1;
    return ALN_OK;
}

// Loss and gradients of a batch whose features are in M->U and whose targets
// are the rows idx of Y.  Leaves the gradients in W[l].g, b[l].g and the loss
// in M->lossv (device).
aln_status backward(aln_ctx* c, Mlp* M, int B, const double* Y, int64_t ldy, const int* idx) {
    const int n = M->n;
    const float inv_m = 1.0f / (float)((double)B * n);
    const dim3 lg((unsigned)ceil_div(n, 32), (unsigned)ceil_div(B, 32));
    k_mlp_loss<<<lg, dim3(32, 8), 0, c->stream>>>(M->O, M->ldO, Y, ldy, idx, M->qn, B, n, inv_m,
                                                 M->tau_host, M->dO, M->ldO, M->dOT, M->ldOT,
                                                 M->part, M->Zt, M->ldY, M->pe, M->pf);
    k_mlp_loss_sum<<<1, 256, 0, c->stream>>>(M->part, (int)(lg.x * lg.y), (double)inv_m,
                                            M->lossv);
    k_colsum_parts<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(M->pe, (int)lg.y, n,
                                                                    M->e.g);
    k_colsum_parts<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(M->pf, (int)lg.y, n,
                                                                    M->f.g);
    M_TRY(cudaGetLastError());
    c->launches += 4;
    // layer 3: dW3 = dOᵀ·H2, db3 = Σ_b dO, dZ2 = (dO·W3) ⊙ [h2 > 0]
    GemmArgs a = args0();
    a.out_f = M->W[2].g;
    a.ld_f = M->W[2].ldg;
    M_CHECK(gemm<EPI_F32>(c, M->dOT, M->ldOT, M->H2T, M->ldHT, M->out, M->hidden, B, a));
    k_rowsum_bf16<<<(unsigned)M->out, 256, 0, c->stream>>>(M->dOT, M->ldOT, B, M->b[2].g);
    a = args0();
    a.act = M->H2;
    a.ld_act = M->ldH;
    a.out_h = M->dZ2;
    a.ld_h = M->ldH;
    a.out_t = M->dZ2T;
    a.ld_t = M->ldHT;
    M_CHECK(gemm<EPI_DRELU>(c, M->dO, M->ldO, M->W[2].t, M->W[2].ldt, B, M->hidden, M->out, a));
    // layer 2
    a = args0();
    a.out_f = M->W[1].g;
    a.ld_f = M->W[1].ldg;
    M_CHECK(gemm<EPI_F32>(c, M->dZ2T, M->ldHT, M->H1T, M->ldHT, M->hidden, M->hidden, B, a));
    k_rowsum_bf16<<<(unsigned)M->hidden, 256, 0, c->stream>>>(M->dZ2T, M->ldHT, B, M->b[1].g);
    a = args0();
    a.act = M->H1;
    a.ld_act = M->ldH;
    a.out_h = M->dZ1;
    a.ld_h = M->ldH;
    a.out_t = M->dZ1T;
    a.ld_t = M->ldHT;
    M_CHECK(gemm<EPI_DRELU>(c, M->dZ2, M->ldH, M->W[1].t, M->W[1].ldt, B, M->hidden, M->hidden,
                            a));
    // layer 1 (no input gradient needed)
    a = args0();
    a.out_f = M->W[0].g;
    a.ld_f = M->W[0].ldg;
    M_CHECK(gemm<EPI_F32>(c, M->dZ1T, M->ldHT, M->UT, M->ldUT, M->hidden, M->in, B, a));
    k_rowsum_bf16<<<(unsigned)M->hidden, 256, 0, c->stream>>>(M->dZ1T, M->ldHT, B, M->b[0].g);
    M_TRY(cudaGetLastError());
    c->launches += 3;
    return ALN_OK;
}

// Features of B rows of Q (rows idx[b] of Qs, or row b): u (and its
// transpose for training), ‖q‖ and the skip input ẑ.  The direction rows
// z/‖q‖ come from Zrows (precomputed, same indexing) or, when it is null,
// from one FP32 product −(q/‖q‖)·Q⁻¹ of the batch.
aln_status features(aln_ctx* c, Mlp* M, const double* Qs, int64_t ldq, const int* idx, int B,
                    bool transpose, const float* Zrows = nullptr) {
    k_mlp_features<<<B, 256, 0, c->stream>>>(Qs, ldq, idx, M->n, M->mu, M->sd, M->U, M->ldU,
                                             M->qn, Zrows ? nullptr : M->Qn, M->ldY);
    c->launches += 1;
    M_TRY(cudaGetLastError());
    const float* Z = Zrows;
    int64_t ldz = M->n;
    const int* zidx = idx;
    if (!Z) {
        // Q⁻¹ is symmetric up to its FP32 rounding: rows times Q⁻¹
        M_CHECK(sgemm(c, B, M->n, M->n, -1.f, M->Qn, M->ldY, M->Minv, M->n, 0.f, nullptr, 0,
                      M->Zp, M->ldY));
        Z = M->Zp;
        ldz = M->ldY;
        zidx = nullptr;
    }
    k_mlp_zfeatures<<<B, 256, 0, c->stream>>>(Z, ldz, zidx, M->n, M->qn, M->muz, M->sdz,
                                              1.0f / M->tau_host, M->U, M->ldU, M->Zt, M->ldY);
    c->launches += 1;
    if (transpose) {
        const dim3 grid((unsigned)ceil_div(M->in, 32), (unsigned)ceil_div(B, 32));
        k_transpose_bf16<<<grid, dim3(32, 8), 0, c->stream>>>(M->U, M->ldU, B, M->in, M->UT,
                                                              M->ldUT);
        c->launches += 1;
    }
    M_TRY(cudaGetLastError());
    return ALN_OK;
}

aln_status refresh_copies(aln_ctx* c, Mlp* M) {
    for (int l = 0; l < 3; ++l) {
        const Tensor& W = M->W[l];
        const dim3 g((unsigned)ceil_div(W.C, 32), (unsigned)ceil_div(W.R, 32));
        k_to_bf16<<<g, dim3(32, 8), 0, c->stream>>>(W.w, W.R, W.C, W.h, W.ldh, W.t, W.ldt);
    }
    M_TRY(cudaGetLastError());
    c->launches += 3;
    return ALN_OK;
}

aln_status adam_all(aln_ctx* c, Mlp* M, const aln_train_opts& o) {
    M->step += 1;
    const double t = (double)M->step;
    const float c1 = (float)(1.0 - std::pow(o.beta1, t)), c2 = (float)(1.0 - std::pow(o.beta2, t));
    for (int l = 0; l < 3; ++l) {
        for (int k = 0; k < 2; ++k) {
            Tensor& T = k == 0 ? M->W[l] : M->b[l];
            const dim3 g((unsigned)ceil_div(T.C, 32), (unsigned)ceil_div(T.R, 32));
            k_adam<<<g, dim3(32, 8), 0, c->stream>>>(T.w, T.m, T.v, T.g, T.ldg, T.R, T.C,
                                                     (float)o.lr, (float)o.beta1, (float)o.beta2,
                                                     (float)o.eps, c1, c2, T.h, T.ldh,
                                                     k == 0 ? T.t : nullptr, T.ldt);
        }
    }
    for (int k = 0; k < 2; ++k) {
        Tensor& T = k == 0 ? M->e : M->f;
        const dim3 g((unsigned)ceil_div(T.C, 32), 1);
        k_adam<<<g, dim3(32, 8), 0, c->stream>>>(T.w, T.m, T.v, T.g, T.ldg, T.R, T.C, (float)o.lr,
                                                 (float)o.beta1, (float)o.beta2, (float)o.eps, c1,
                                                 c2, nullptr, 0, nullptr, 0);
    }
    M_TRY(cudaGetLastError());
    c->launches += 8;
    return ALN_OK;
}

bool is_dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device copy of a count×n FP64 row block given on the host (or the device
// pointer itself).
aln_status stage_rows(aln_ctx* c, const double* src, int64_t count, int64_t n, void** tmp,
                      const double** out) {
    if (is_dev_ptr(src)) {
        *out = src;
        return ALN_OK;
    }
    M_TRY(cudaMalloc(tmp, (size_t)count * n * 8));
    M_TRY(cudaMemcpyAsync(*tmp, src, (size_t)count * n * 8, cudaMemcpyHostToDevice, c->stream));
    *out = (const double*)*tmp;
    return ALN_OK;
}

aln_status check_flags(aln_ctx* c) {
    M_TRY(cudaMemcpyAsync(c->flags_host + 1, c->flags + 1, sizeof(int), cudaMemcpyDeviceToHost,
                          c->stream));
    M_TRY(cudaStreamSynchronize(c->stream));
    return c->flags_host[1] ? ALN_ERR_TIMEOUT : ALN_OK;
}

// μ, σ of q/‖q‖ per entry and τ = RMS of y*/‖q‖ over a training set.
aln_status training_stats(aln_ctx* c, Mlp* M, const double* Qd, const double* Yd, int64_t count) {
    const int n = M->n;
    const int G = 64;
    double *qn = nullptr, *part = nullptr;
    M_TRY(cudaMalloc(&qn, (size_t)count * 8));
    if (cudaMalloc(&part, (size_t)G * n * 3 * 8) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(qn);
        return ALN_ERR_OUT_OF_MEMORY;
    }
    k_rownorm<<<(unsigned)count, 256, 0, c->stream>>>(Qd, count, n, qn);
    k_colmoments<<<dim3((unsigned)ceil_div(n, 32), G), dim3(32, 8), 0, c->stream>>>(Qd, Yd, qn,
                                                                                   count, n, part);
    k_colstats_final<<<1, 256, 0, c->stream>>>(part, G, count, n, M->mu, M->sd, M->tau);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(M->hflag + 2, M->tau, 4, cudaMemcpyDeviceToHost,
                                              c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(qn);
    cudaFree(part);
    if (e != cudaSuccess) return ALN_ERR_CUDA;
    std::memcpy(&M->tau_host, M->hflag + 2, 4);
    M->stats_set = true;
    c->launches += 3;
    return ALN_OK;
}

}  // namespace

int mlp_n(const aln_ctx* c) { return c->mlp ? ((const Mlp*)c->mlp)->n : -1; }

void mlp_free(aln_ctx* c) {
    free_mlp((Mlp*)c->mlp);
    c->mlp = nullptr;
}

aln_status mlp_init(aln_ctx* c, int hidden, uint64_t seed) {
    mlp_free(c);
    Mlp* M = new (std::nothrow) Mlp();
    if (!M) return ALN_ERR_OUT_OF_MEMORY;
    c->mlp = M;
    M->n = (int)c->n;
    M->hidden = hidden;
    M->in = M->out = 2 * c->n;
    M_CHECK(alloc_weights(c, M));
    if (cudaMallocHost(&M->hflag, 64) != cudaSuccess) {
        cudaGetLastError();
        M->hflag = nullptr;
        return ALN_ERR_OUT_OF_MEMORY;
    }
    M->hloss = (double*)(M->hflag + 4);
    for (int l = 0; l < 3; ++l) {
        const Tensor& W = M->W[l];
        const float lim = (float)std::sqrt(6.0 / (double)W.C);
        k_mlp_init<<<(unsigned)std::min<int64_t>(ceil_div(W.R * W.C, 256), 4096), 256, 0,
                     c->stream>>>(W.w, W.R, W.C, lim, seed + 0x1000193ull * (uint64_t)(l + 1));
    }
    const unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(M->n, 256), 1024));
    k_fill<<<gn, 256, 0, c->stream>>>(M->sd, M->n, 1.0f);
    k_fill<<<gn, 256, 0, c->stream>>>(M->sdz, M->n, 1.0f);
    k_fill<<<gn, 256, 0, c->stream>>>(M->e.w, M->n, 1.0f);   // ŷ follows ẑ
    k_fill<<<gn, 256, 0, c->stream>>>(M->f.w, M->n, 4.0f);   // ℓ follows its sign
    k_fill<<<1, 32, 0, c->stream>>>(M->tau, 1, 1.0f);
    M->tau_host = 1.0f;
    M_TRY(cudaGetLastError());
    c->launches += 8;
    M_CHECK(refresh_copies(c, M));
    M_CHECK(ns_inverse(c, M));
    M_TRY(cudaStreamSynchronize(c->stream));
    return ALN_OK;
}

// t = {W1, b1, W2, b2, W3, b3, e, f, mu, sd, muz, sdz, tau}; null entries
// are skipped.
aln_status mlp_params(aln_ctx* c, int set, float* const* t) {
    Mlp* M = (Mlp*)c->mlp;
    auto copy = [&](float* p, float* dev, size_t count) -> aln_status {
        if (!p) return ALN_OK;
        const bool d = is_dev_ptr(p);
        if (set)
            M_TRY(cudaMemcpyAsync(dev, p, count * 4,
                                  d ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream));
        else
            M_TRY(cudaMemcpyAsync(p, dev, count * 4,
                                  d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream));
        return ALN_OK;
    };
    for (int l = 0; l < 3; ++l) {
        M_CHECK(copy(t[2 * l], M->W[l].w, (size_t)M->W[l].R * M->W[l].C));
        M_CHECK(copy(t[2 * l + 1], M->b[l].w, (size_t)M->b[l].C));
    }
    M_CHECK(copy(t[6], M->e.w, (size_t)M->n));
    M_CHECK(copy(t[7], M->f.w, (size_t)M->n));
    M_CHECK(copy(t[8], M->mu, (size_t)M->n));
    M_CHECK(copy(t[9], M->sd, (size_t)M->n));
    M_CHECK(copy(t[10], M->muz, (size_t)M->n));
    M_CHECK(copy(t[11], M->sdz, (size_t)M->n));
    M_CHECK(copy(t[12], M->tau, 1));
    if (set && (t[8] || t[9] || t[10] || t[11] || t[12])) M->stats_set = true;
    if (set && t[12]) {
        M_TRY(cudaMemcpyAsync(M->hflag + 2, M->tau, 4, cudaMemcpyDeviceToHost, c->stream));
        M_TRY(cudaStreamSynchronize(c->stream));
        std::memcpy(&M->tau_host, M->hflag + 2, 4);
    }
    if (set) {
        M_CHECK(refresh_copies(c, M));
        for (int l = 0; l < 3; ++l) {
            Tensor& b = M->b[l];
            const dim3 g((unsigned)ceil_div(b.C, 32), 1);
            k_to_bf16<<<g, dim3(32, 8), 0, c->stream>>>(b.w, 1, b.C, b.h, b.ldh, nullptr, 0);
        }
        M_TRY(cudaGetLastError());
        c->launches += 3;
    }
    M_TRY(cudaStreamSynchronize(c->stream));
    return ALN_OK;
}

aln_status mlp_grad(aln_ctx* c, const double* Qs, const double* Ys, int64_t count, double* loss,
                    float* const* grads) {
    Mlp* M = (Mlp*)c->mlp;
    const int n = M->n;
    void *tq = nullptr, *ty = nullptr;
    const double *Qd = nullptr, *Yd = nullptr;
    aln_status st = stage_rows(c, Qs, count, n, &tq, &Qd);
    if (st == ALN_OK) st = stage_rows(c, Ys, count, n, &ty, &Yd);
    if (st == ALN_OK) st = alloc_acts(c, M, (int)count);
    if (st == ALN_OK) {
        M_TRY(cudaMemsetAsync(c->flags + 1, 0, sizeof(int), c->stream));
        st = features(c, M, Qd, n, nullptr, (int)count, true);
    }
    if (st == ALN_OK) st = forward(c, M, (int)count, true);
    if (st == ALN_OK) st = backward(c, M, (int)count, Yd, n, nullptr);
    if (st == ALN_OK) st = check_flags(c);
    if (st == ALN_OK && loss)
        st = cudaMemcpy(loss, M->lossv, 8, cudaMemcpyDeviceToHost) == cudaSuccess ? ALN_OK
                                                                                  : ALN_ERR_CUDA;
    if (st == ALN_OK) {
        const Tensor* ts[8] = {&M->W[0], &M->b[0], &M->W[1], &M->b[1],
                               &M->W[2], &M->b[2], &M->e,    &M->f};
        for (int k = 0; k < 8 && st == ALN_OK; ++k) {
            float* p = grads[k];
            if (!p) continue;
            const Tensor& T = *ts[k];
            if (cudaMemcpy(p, T.g, (size_t)T.R * T.C * 4, cudaMemcpyDefault) != cudaSuccess)
                st = ALN_ERR_CUDA;
        }
    }
    if (tq) cudaFree(tq);
    if (ty) cudaFree(ty);
    return st;
}

aln_status mlp_train(aln_ctx* c, const double* Qs, const double* Ys, int64_t count,
                     const aln_train_opts& o, double* epoch_loss) {
    Mlp* M = (Mlp*)c->mlp;
    const int n = M->n;
    const int B = (int)std::min<int64_t>(o.batch, count);
    void *tq = nullptr, *ty = nullptr;
    const double *Qd = nullptr, *Yd = nullptr;
    aln_status st = stage_rows(c, Qs, count, n, &tq, &Qd);
    if (st == ALN_OK) st = stage_rows(c, Ys, count, n, &ty, &Yd);
    if (st == ALN_OK) st = alloc_acts(c, M, B);
    int* perm_dev = nullptr;
    if (st == ALN_OK && cudaMalloc(&perm_dev, (size_t)count * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        st = ALN_ERR_OUT_OF_MEMORY;
    }
    std::vector<int> perm(count);
    uint64_t rng = o.seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {  // split-mix 64 on the host, for the shuffles
        uint64_t x = (rng += 0x9E3779B97F4A7C15ull);
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        return x ^ (x >> 31);
    };
    if (st == ALN_OK) M_TRY(cudaMemsetAsync(c->flags + 1, 0, sizeof(int), c->stream));
    const bool need_stats = !M->stats_set;
    if (st == ALN_OK && need_stats) st = training_stats(c, M, Qd, Yd, count);
    // The direction rows z/‖q‖ of the whole training set, once (FP32
    // products of Bcap rows at a time), with their column moments when the
    // statistics come from this set.
    float* Ztrain = nullptr;
    double* zs = nullptr;
    if (st == ALN_OK && (cudaMalloc(&Ztrain, (size_t)count * n * 4) != cudaSuccess ||
                         cudaMalloc(&zs, (size_t)2 * n * 8) != cudaSuccess)) {
        cudaGetLastError();
        st = ALN_ERR_OUT_OF_MEMORY;
    }
    if (st == ALN_OK && need_stats &&
        cudaMemsetAsync(zs, 0, (size_t)2 * n * 8, c->stream) != cudaSuccess)
        st = ALN_ERR_CUDA;
    for (int64_t r0 = 0; st == ALN_OK && r0 < count; r0 += M->Bcap) {
        const int rows = (int)std::min<int64_t>(M->Bcap, count - r0);
        k_mlp_features<<<rows, 256, 0, c->stream>>>(Qd + r0 * n, n, nullptr, n, M->mu, M->sd,
                                                    M->U, M->ldU, M->qn, M->Qn, M->ldY);
        c->launches += 1;
        st = sgemm(c, rows, n, n, -1.f, M->Qn, M->ldY, M->Minv, n, 0.f, nullptr, 0,
                   Ztrain + r0 * n, n);
        if (st == ALN_OK && need_stats) {
            k_zmoments<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(Ztrain + r0 * n, n, rows,
                                                                         n, M->qn, zs, zs + n);
            c->launches += 1;
        }
    }
    if (st == ALN_OK && need_stats) {
        k_zmoments_final<<<(unsigned)ceil_div(n, 256), 256, 0, c->stream>>>(zs, zs + n, count, n,
                                                                           M->muz, M->sdz);
        c->launches += 1;
        if (cudaGetLastError() != cudaSuccess) st = ALN_ERR_CUDA;
    }
    std::vector<double> losses;
    for (int ep = 0; st == ALN_OK && ep < o.epochs; ++ep) {
        for (int64_t i = 0; i < count; ++i) perm[i] = (int)i;
        for (int64_t i = count - 1; i > 0; --i) std::swap(perm[i], perm[next() % (uint64_t)(i + 1)]);
        if (cudaMemcpyAsync(perm_dev, perm.data(), (size_t)count * sizeof(int),
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            st = ALN_ERR_CUDA;
            break;
        }
        // per-batch losses accumulate on the device, read once per epoch
        std::vector<double> bl;
        double* dev_losses = nullptr;
        const int64_t nb = ceil_div(count, B);
        if (cudaMalloc(&dev_losses, (size_t)nb * 8) != cudaSuccess) {
            cudaGetLastError();
            st = ALN_ERR_OUT_OF_MEMORY;
            break;
        }
        for (int64_t bi = 0; bi < nb && st == ALN_OK; ++bi) {
            const int64_t off = bi * B;
            const int Bb = (int)std::min<int64_t>(B, count - off);
            st = features(c, M, Qd, n, perm_dev + off, Bb, true, Ztrain);
            if (st == ALN_OK) st = forward(c, M, Bb, true);
            if (st == ALN_OK) st = backward(c, M, Bb, Yd, n, perm_dev + off);
            if (st == ALN_OK) st = adam_all(c, M, o);
            if (st == ALN_OK &&
                cudaMemcpyAsync(dev_losses + bi, M->lossv, 8, cudaMemcpyDeviceToDevice,
                                c->stream) != cudaSuccess)
                st = ALN_ERR_CUDA;
        }
        if (st == ALN_OK) {
            bl.resize(nb);
            if (cudaMemcpyAsync(bl.data(), dev_losses, (size_t)nb * 8, cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                st = ALN_ERR_CUDA;
        }
        cudaFree(dev_losses);
        if (st == ALN_OK) {
            double tot = 0.0;
            for (int64_t bi = 0; bi < nb; ++bi)
                tot += bl[bi] * (double)std::min<int64_t>(B, count - bi * B);
            losses.push_back(tot / (double)count);
        }
    }
    if (st == ALN_OK) st = check_flags(c);
    if (st == ALN_OK && epoch_loss)
        for (size_t i = 0; i < losses.size(); ++i) epoch_loss[i] = losses[i];
    if (perm_dev) cudaFree(perm_dev);
    if (Ztrain) cudaFree(Ztrain);
    if (zs) cudaFree(zs);
    if (tq) cudaFree(tq);
    if (ty) cudaFree(ty);
    return st;
}

aln_status mlp_predict(aln_ctx* c, double* X0, int64_t ldx, int* kept) {
    Mlp* M = (Mlp*)c->mlp;
    const int n = M->n;
    const int64_t k = c->k;
    const int chunk = 4096;
    M_CHECK(alloc_acts(c, M, (int)std::min<int64_t>(k, chunk)));
    // BF16 copy of Q for the line search (Q is symmetric: rows are K-major)
    {
        const unsigned g = (unsigned)std::min<int64_t>(ceil_div((int64_t)n * n, 256), 8192);
        if (c->opt.precision == ALN_PREC_FP64)
            k_q_to_bf16<double><<<g, 256, 0, c->stream>>>((const double*)c->Q, c->ldq, n, M->Qh,
                                                          M->ldQh);
        else
            k_q_to_bf16<float><<<g, 256, 0, c->stream>>>((const float*)c->Q, c->ldq, n, M->Qh,
                                                         M->ldQh);
        M_TRY(cudaGetLastError());
        c->launches += 1;
    }
    const bool x_dev = is_dev_ptr(X0);
    double* xdst = X0;
    if (!x_dev) {
        const size_t bytes = (size_t)k * n * 8;
        if (M->xtmp_bytes < bytes) {
            if (M->xtmp) cudaFree(M->xtmp);
            M->xtmp = nullptr;
            M->xtmp_bytes = 0;
            M_TRY(cudaMalloc(&M->xtmp, bytes));
            M->xtmp_bytes = bytes;
        }
        xdst = M->xtmp;
    }
    const int64_t ldd = x_dev ? ldx : n;
    int* kept_dev = nullptr;
    if (kept) {
        if (M->kept_cap < k) {
            if (M->kept) cudaFree(M->kept);
            M->kept = nullptr;
            M->kept_cap = 0;
            M_TRY(cudaMalloc(&M->kept, (size_t)k * sizeof(int)));
            M->kept_cap = k;
        }
        kept_dev = M->kept;
    }
    M_TRY(cudaMemsetAsync(c->flags + 1, 0, sizeof(int), c->stream));
    aln_status st = ALN_OK;
    for (int64_t b0 = 0; b0 < k && st == ALN_OK; b0 += chunk) {
        const int Bb = (int)std::min<int64_t>(chunk, k - b0);
        st = features(c, M, c->q64 + b0 * c->ldq, c->ldq, nullptr, Bb, false);
        if (st == ALN_OK) st = forward(c, M, Bb, false);
        if (st != ALN_OK) break;
        k_mlp_post<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)Bb * n, 256), 8192), 256, 0,
                     c->stream>>>(M->O, M->ldO, Bb, n, M->Y0, M->Y0h, M->ldY);
        c->launches += 1;
        // Q·d for every row (BF16 operands, FP32 accumulation), then α*
        GemmArgs a = args0();
        a.out_f = M->QY;
        a.ld_f = M->ldY;
        st = gemm<EPI_F32>(c, M->Y0h, M->ldY, M->Qh, M->ldQh, Bb, n, n, a);
        if (st != ALN_OK) break;
        k_mlp_linesearch<<<Bb, 256, 0, c->stream>>>(M->Y0, M->QY, M->ldY, c->q64 + b0 * c->ldq,
                                                   c->ldq, c->s, n, xdst + b0 * ldd, ldd,
                                                   kept_dev ? kept_dev + b0 : nullptr);
        c->launches += 1;
        if (cudaGetLastError() != cudaSuccess) st = ALN_ERR_CUDA;
    }
    if (st == ALN_OK && !x_dev &&
        cudaMemcpy2DAsync(X0, ldx * 8, xdst, n * 8, n * 8, k, cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess)
        st = ALN_ERR_CUDA;
    if (st == ALN_OK && kept &&
        cudaMemcpyAsync(kept, kept_dev, (size_t)k * sizeof(int),
                        is_dev_ptr(kept) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        st = ALN_ERR_CUDA;
    if (st == ALN_OK) st = check_flags(c);
    return st;
}

}  // namespace aln
