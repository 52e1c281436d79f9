// Alg. 2 (§3) on many right-hand sides that share A (the multi-RHS inner
// solve of NMF, §1/§2.2): every column c has its own y_c, g_c, passive set,
// step size and stop state, and one iteration of all running columns is
//
//   k_bmask   (one block per column) ḡ_c = g_c on P(y_c), γ_c = ‖ḡ_c‖²; the
//             stop rules of Alg. 2 per column; running columns are compacted
//             (atomic slot p) and ḡ_c is split into BF16 hi/lo row p;
//   W = Q·Ḡ   (k_bgemm_tc, tcgen05, 3 split products) with the per-column
//             curvature ḡ_cᵀw_c reduced in the epilogue;
//   k_bupdate (one block per running column) α_c = γ_c/κ_c, y⁺ = [y − αḡ]₊,
//             g ← g − α w, e = clipped part; columns with clipping are
//             compacted again and e_c is split;
//   U = Q·E   (k_bgemm_tc) added to g for the clipped columns only.
//
// The FP64 check of every column uses the FP64 scaled matrix Q64 and the
// FP64 q: g64 = Q64 y + q (one FP64-accurate product for all columns, exact
// BF16 digit products on the tensor cores, ozaki.cu), then
// rel_c = ‖ḡ64_c‖/‖min(q_c, 0)‖ and ½‖Ax − b‖² = ½yᵀg64 + ½qᵀy + ½‖b‖².
// Columns above tol restart from y_c with g_c = g64_c (refinement).
#include "blockops.cuh"
#include "dfloat.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

constexpr int kBThreads = 256;
// Tail launches: iterations a column runs before the cluster size is chosen
// again (the last launch, at the largest cluster, has no budget).
constexpr int kTailBudget = 64;

// Q (FP32, [n][ldq]) → hi/lo BF16 [n][ldk], zero-padded columns n..ldk.
__global__ void k_qsplit(const double* __restrict__ Q64, int64_t ldq, int64_t n, int64_t ldk,
                         float* __restrict__ Q32, __nv_bfloat16* __restrict__ hi,
                         __nv_bfloat16* __restrict__ lo) {
    const int64_t i = blockIdx.x;
    for (int64_t j = threadIdx.x; j < ldk; j += blockDim.x) {
        const float v = j < n ? (float)Q64[i * ldq + j] : 0.0f;
        if (j < ldq) Q32[i * ldq + j] = v;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i * ldk + j] = h;
        lo[i * ldk + j] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

__global__ void k_bnorm2(const void* __restrict__ B, int32_t dtype, int64_t d, int64_t ldb,
                         double* __restrict__ out) {
    __shared__ double sc[32];
    const int64_t c = blockIdx.x;
    double v = 0.0;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        const double b = dtype == ALN_DTYPE_F32 ? (double)((const float*)B)[c * ldb + t]
                                                : ((const double*)B)[c * ldb + t];
        v = fma(b, b, v);
    }
    v = block_sum(v, sc);
    if (threadIdx.x == 0) out[c] = v;
}

struct BatchState {
    int64_t n, ldq, ldk, k;
    float* Y;             // [k][ldq]
    float* G;             // [k][ldq]
    float* GB;            // [k][ldq]
    float* E;             // [k][ldq]
    float* W;             // [k][ldq]  (compact rows)
    __nv_bfloat16* Vhi;   // [k][ldk]  (compact rows)
    __nv_bfloat16* Vlo;
    double* kpart;        // [mtiles][k]
    int mtiles;
    int* colst;           // -1 running, otherwise the final aln_rhs_status
    int* iters;
    int* best_iter;
    double* best;
    double* eps;
    double* gamma;
    int* map_act;
    int* map_clip;
    int* counters;        // [0] running columns, [1] clipped columns
    unsigned long long* rows;  // [0] Σ|P|, [1] Σ|C| over the run
    int* limits;          // [0] max_iter, [1] stagnation window (set per solve)
};

__global__ void k_breset(int* counters) {
    counters[0] = 0;
    counters[1] = 0;
}

// Mask and update run one 128-thread block per column: each block's work is a
// short chain of dependent steps (scan, block reduction, one thread's
// decision and atomics, split), so more resident blocks per SM hide more of
// its latency than wider blocks would.  Both read and write the column
// vectors as float4 (ldq is a multiple of 128; entries n..ldq are zero).
constexpr int kBMThreads = 128;
constexpr int kBMWarps = kBMThreads / 32;

// 4 FP32 values → their BF16 hi and lo parts (v = hi + lo + O(2⁻¹⁶|v|)).
__device__ __forceinline__ void split4(float4 v, uint2* hi, uint2* lo) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
    const __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
    uint2 H, L;
    H.x = *reinterpret_cast<const unsigned int*>(&h0);
    H.y = *reinterpret_cast<const unsigned int*>(&h1);
    L.x = *reinterpret_cast<const unsigned int*>(&l0);
    L.y = *reinterpret_cast<const unsigned int*>(&l1);
    *hi = H;
    *lo = L;
}

// Split row p of the compacted operand from v (float4 entries < n4, zero
// beyond, up to ldk).
__device__ __forceinline__ void split_row(const BatchState& s, int p, const float4* v, int n4) {
    uint2* hi = reinterpret_cast<uint2*>(s.Vhi + (int64_t)p * s.ldk);
    uint2* lo = reinterpret_cast<uint2*>(s.Vlo + (int64_t)p * s.ldk);
    const int k4 = (int)(s.ldk >> 2);
    for (int i = threadIdx.x; i < k4; i += kBMThreads)
        split4(i < n4 ? v[i] : make_float4(0.f, 0.f, 0.f, 0.f), hi + i, lo + i);
}

// One block per column: mask, γ, |P|, stop rules, compaction, split of ḡ.
__global__ void __launch_bounds__(kBMThreads) k_bmask(BatchState s) {
    __shared__ double sc[kBMWarps];
    __shared__ int si[kBMWarps];
    __shared__ int s_slot;
    const int64_t c = blockIdx.x;
    if (s.colst[c] >= 0) return;
    // the column's stop state, loaded before the scan so that its latency
    // overlaps it (thread 0 decides)
    int it = 0, best_it = 0, lim_it = 0, lim_win = 0;
    double eps = 0.0, best = 0.0;
    if (threadIdx.x == 0) {
        it = s.iters[c];
        best_it = s.best_iter[c];
        eps = s.eps[c];
        best = s.best[c];
        lim_it = s.limits[0];
        lim_win = s.limits[1];
    }
    const float4* y4 = reinterpret_cast<const float4*>(s.Y + c * s.ldq);
    const float4* g4 = reinterpret_cast<const float4*>(s.G + c * s.ldq);
    float4* gb4 = reinterpret_cast<float4*>(s.GB + c * s.ldq);
    const int n4 = (int)((s.n + 3) >> 2);
    // FP32 partial sums (GB300's FP64 pipe is narrow); thread 0 adds the
    // warp sums in FP64.
    float vf = 0.0f;
    int cnt = 0;
    for (int i = threadIdx.x; i < n4; i += kBMThreads) {
        const float4 y = y4[i], g = g4[i];
        float4 b;
        const bool p0 = y.x > 0.0f || g.x < 0.0f, p1 = y.y > 0.0f || g.y < 0.0f;
        const bool p2 = y.z > 0.0f || g.z < 0.0f, p3 = y.w > 0.0f || g.w < 0.0f;
        b.x = p0 ? g.x : 0.0f;
        b.y = p1 ? g.y : 0.0f;
        b.z = p2 ? g.z : 0.0f;
        b.w = p3 ? g.w : 0.0f;
        gb4[i] = b;
        vf = fmaf(b.x, b.x, vf);
        vf = fmaf(b.y, b.y, vf);
        vf = fmaf(b.z, b.z, vf);
        vf = fmaf(b.w, b.w, vf);
        cnt += (int)p0 + (int)p1 + (int)p2 + (int)p3;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vf += __shfl_xor_sync(0xffffffffu, vf, o);
    cnt = warp_sum_i(cnt);
    if (lane == 0) {
        sc[wid] = (double)vf;
        si[wid] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        int t = 0;
#pragma unroll
        for (int w2 = 0; w2 < kBMWarps; ++w2) {
            t += si[w2];
            v += sc[w2];
        }
        int status = -1;
        if (!isfinite(v)) status = ALN_RHS_NONFINITE;
        else if (t == 0) status = ALN_RHS_EMPTY_PASSIVE;
        else if (v < eps || v == 0.0) status = ALN_RHS_CONVERGED;
        else if (it >= lim_it) status = ALN_RHS_MAXITER;
        else if (it - best_it > lim_win) status = ALN_RHS_STAGNATED;
        int slot = -1;
        if (status >= 0) {
            s.colst[c] = status;
        } else {
            if (v < best) {
                s.best[c] = v;
                s.best_iter[c] = it;
            }
            s.gamma[c] = v;
            slot = atomicAdd(&s.counters[0], 1);
            s.map_act[slot] = (int)c;
            atomicAdd(&s.rows[0], (unsigned long long)t);
        }
        s_slot = slot;
    }
    __syncthreads();  // also orders the ḡ stores above before the split reads them
    const int p = s_slot;
    if (p < 0) return;
    split_row(s, p, gb4, n4);
}

// One block per running column (compact slot p): α, projection, g update, e.
__global__ void __launch_bounds__(kBMThreads) k_bupdate(BatchState s) {
    __shared__ int si[kBMWarps];
    __shared__ int s_slot;
    __shared__ float s_alpha;
    const int p = blockIdx.x;
    if (p >= s.counters[0]) return;
    const int64_t c = s.map_act[p];
    if (threadIdx.x < 32) {
        // κ = Σ of the row tiles' curvature partials, in FP64, lanes in parallel
        const double gam = threadIdx.x == 0 ? s.gamma[c] : 0.0;
        double kp = 0.0;
        for (int m = threadIdx.x; m < s.mtiles; m += 32) kp += s.kpart[(int64_t)m * s.k + p];
        const double kap = warp_sum(kp);
        if (threadIdx.x == 0) {
            float a = 0.0f;
            if (!isfinite(kap)) s.colst[c] = ALN_RHS_NONFINITE;
            else if (kap <= 0.0) s.colst[c] = ALN_RHS_CURVATURE;
            else a = (float)(gam / kap);
            s_alpha = a;
        }
    }
    __syncthreads();
    const float a = s_alpha;
    if (a == 0.0f) return;
    float4* y4 = reinterpret_cast<float4*>(s.Y + c * s.ldq);
    float4* g4 = reinterpret_cast<float4*>(s.G + c * s.ldq);
    float4* e4 = reinterpret_cast<float4*>(s.E + c * s.ldq);
    const float4* gb4 = reinterpret_cast<const float4*>(s.GB + c * s.ldq);
    const float4* w4 = reinterpret_cast<const float4*>(s.W + (int64_t)p * s.ldq);
    const int n4 = (int)((s.n + 3) >> 2);
    int clipped = 0;
    auto step1 = [&](float& y, float& e, float& g, float b, float w) {
        const float st = a * b;
        float yn = y - st;
        e = 0.0f;
        if (yn < 0.0f) {
            e = st - y;
            yn = 0.0f;
            ++clipped;
        }
        y = yn;
        g = g - a * w;
    };
    for (int i = threadIdx.x; i < n4; i += kBMThreads) {
        float4 y = y4[i], g = g4[i], e;
        const float4 b = gb4[i], w = w4[i];
        step1(y.x, e.x, g.x, b.x, w.x);
        step1(y.y, e.y, g.y, b.y, w.y);
        step1(y.z, e.z, g.z, b.z, w.z);
        step1(y.w, e.w, g.w, b.w, w.w);
        y4[i] = y;
        e4[i] = e;
        g4[i] = g;
    }
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int x = warp_sum_i(clipped);
        if (lane == 0) si[wid] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
#pragma unroll
            for (int w2 = 0; w2 < kBMWarps; ++w2) t += si[w2];
            s.iters[c] += 1;
            int slot = -1;
            if (t > 0) {
                slot = atomicAdd(&s.counters[1], 1);
                s.map_clip[slot] = (int)c;
                atomicAdd(&s.rows[1], (unsigned long long)t);
                atomicAdd(&s.rows[2], 1ull);  // column-iterations with a Qe product
            }
            s_slot = slot;
        }
        __syncthreads();
    }
    const int q = s_slot;
    if (q < 0) return;
    split_row(s, q, e4, n4);
}

// Start state of every column: y = s·x0 (0 without a start point), g = q
// (float), running, per-column ε.
__global__ void k_binit(BatchState s, const double* __restrict__ q64, const double* __restrict__ x0,
                        int64_t ldx0, const double* __restrict__ sc, const double* __restrict__ den,
                        double tol_factor, int* __restrict__ rounds) {
    const int64_t c = blockIdx.x;
    for (int64_t i = threadIdx.x; i < s.ldq; i += blockDim.x) {
        const bool in = i < s.n;
        const double y0 = (in && x0) ? x0[c * ldx0 + i] * sc[i] : 0.0;
        const float yh = (float)y0;
        s.Y[c * s.ldq + i] = yh;
        s.G[c * s.ldq + i] = in ? (float)q64[c * s.ldq + i] : 0.0f;
        // the low part of the start (read only by the small-n float-pair path;
        // the batched phase overwrites E with e before using it)
        s.E[c * s.ldq + i] = (float)(y0 - (double)yh);
    }
    if (threadIdx.x == 0) {
        const double t = tol_factor * (den[c] > 0.0 ? den[c] : 1.0);
        s.eps[c] = t * t;
        s.colst[c] = -1;
        s.iters[c] = 0;
        s.best[c] = 1.0 / 0.0;
        s.best_iter[c] = 0;
        rounds[c] = 0;
    }
}

// x = y/s and y in FP64 for the check (Eq. Rescaling).  ylo: the low parts
// of a float-pair iterate (the small-n kernel keeps them in E), or null.
__global__ void k_bunscale(BatchState s, const double* __restrict__ sc, double* __restrict__ X64,
                           double* __restrict__ Y64, const float* __restrict__ ylo) {
    const int64_t c = blockIdx.x;
    for (int64_t i = threadIdx.x; i < s.ldq; i += blockDim.x) {
        const double y = i < s.n ? (double)s.Y[c * s.ldq + i] +
                                       (ylo ? (double)ylo[c * s.ldq + i] : 0.0)
                                 : 0.0;
        Y64[c * s.ldq + i] = y;
        X64[c * s.ldq + i] = i < s.n ? y / sc[i] : 0.0;
    }
}

// One block per column: FP64 check from g64 = Q64 y + q.  Final statuses, or
// refinement (g ← g64, new ε) while rounds remain.
__global__ void __launch_bounds__(kBThreads) k_bcheck(
    BatchState s, const double* __restrict__ G64, const double* __restrict__ Y64,
    const double* __restrict__ q64, const double* __restrict__ bn2, const double* __restrict__ den,
    double tol, double refine_factor, int gain, int max_refine, int* __restrict__ rounds,
    int* __restrict__ final_status, double* __restrict__ rel_out, double* __restrict__ obj_out,
    int* __restrict__ reactivated) {
    __shared__ double sc[32];
    const int64_t c = blockIdx.x;
    if (final_status[c] >= 0) return;
    const double* g = G64 + c * s.ldq;
    const double* y = Y64 + c * s.ldq;
    const double* q = q64 + c * s.ldq;
    double gb2 = 0.0, yg = 0.0, qy = 0.0;
    for (int64_t i = threadIdx.x; i < s.n; i += blockDim.x) {
        const double gi = g[i], yi = y[i];
        const bool P = yi > 0.0 || gi < 0.0;
        if (P) gb2 = fma(gi, gi, gb2);
        yg = fma(yi, gi, yg);
        qy = fma(q[i], yi, qy);
    }
    gb2 = block_sum(gb2, sc);
    yg = block_sum(yg, sc);
    qy = block_sum(qy, sc);
    __shared__ int s_refine;
    if (threadIdx.x == 0) {
        const double num = sqrt(gb2);
        const double rel = den[c] > 0.0 ? num / den[c] : num;
        rel_out[c] = rel;
        // ½‖Ax − b‖² = ½yᵀQy + qᵀy + ½‖b‖² = ½yᵀg64 + ½qᵀy + ½‖b‖²
        obj_out[c] = 0.5 * yg + 0.5 * qy + 0.5 * bn2[c];
        const int inner = s.colst[c];
        int refine = 0;
        if (rel <= tol) {
            final_status[c] = inner == ALN_RHS_EMPTY_PASSIVE ? ALN_RHS_EMPTY_PASSIVE
                                                             : ALN_RHS_CONVERGED;
        } else if (inner == ALN_RHS_NONFINITE || inner == ALN_RHS_MAXITER ||
                   s.iters[c] >= s.limits[0]) {
            final_status[c] = inner == ALN_RHS_NONFINITE ? ALN_RHS_NONFINITE : ALN_RHS_MAXITER;
        } else if (rounds[c] >= max_refine) {
            final_status[c] = inner == ALN_RHS_STAGNATED ? ALN_RHS_STAGNATED : ALN_RHS_MAXITER;
        } else {
            refine = 1;
            rounds[c] += 1;
            const double t =
                inner_target(tol, refine_factor, rel, gain) * (den[c] > 0.0 ? den[c] : 1.0);
            s.eps[c] = t * t;
            s.colst[c] = -1;
            s.best[c] = 1.0 / 0.0;
            s.best_iter[c] = s.iters[c];
            atomicAdd(reactivated, 1);
        }
        s_refine = refine;
    }
    __syncthreads();
    if (s_refine)
        for (int64_t i = threadIdx.x; i < s.n; i += blockDim.x) s.G[c * s.ldq + i] = (float)g[i];
}

// ---------------------------------------------------------------------------
// Small n (≤ 128): one warp per column, the whole Alg. 2 loop in one launch.
// The batched phase above pays several launches and tcgen05 tiles per
// iteration; for n this small each column's products are a few thousand
// FMAs, so a warp runs the loop alone: Q (FP32, n × n) staged in shared
// memory once per block, y and g in registers (VPL entries per lane),
// ḡ_j broadcast by shuffles, the sums of γ and κ as FP32 pairs across lanes
// (normalised double-float: the SM's FP64 unit is narrow, and many columns'
// warps share it), α = γ/κ from the pairs.  The
// iterate is a float pair y = yh + yl (yh in Y, yl in E, which this path
// does not otherwise use): the FP64 refinement then converges below the
// FP32 rounding of y, as in the grouped kernel.
// Same stop rules and per-column state as k_bmask / k_bupdate, so the FP64
// checks and refinement (k_bcheck) follow unchanged.
// Σ_{k < cnt} v[list[k]] · Q[list[k], i] for the lane's rows i = lane + 32u:
// the listed rows of the staged Q, four list entries in flight per step.
template <int VPL>
__device__ __forceinline__ void bsmall_rows(const float* sq, const int* list, const float* vals,
                                            int cnt, int lane, float (&acc)[VPL]) {
    constexpr int NS = VPL * 32;
    float a2[VPL];
#pragma unroll
    for (int u = 0; u < VPL; ++u) a2[u] = 0.0f;
    int k = 0;
    for (; k + 1 < cnt; k += 2) {
        const int j0 = list[k], j1 = list[k + 1];
        const float v0 = vals[j0], v1 = vals[j1];
        const float* r0 = sq + j0 * NS;
        const float* r1 = sq + j1 * NS;
#pragma unroll
        for (int u = 0; u < VPL; ++u) {
            acc[u] = fmaf(r0[lane + 32 * u], v0, acc[u]);
            a2[u] = fmaf(r1[lane + 32 * u], v1, a2[u]);
        }
    }
    if (k < cnt) {
        const int j0 = list[k];
        const float v0 = vals[j0];
        const float* r0 = sq + j0 * NS;
#pragma unroll
        for (int u = 0; u < VPL; ++u) acc[u] = fmaf(r0[lane + 32 * u], v0, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < VPL; ++u) acc[u] += a2[u];
}

// Lane-order list of the indices lane + 32v with x[v] ≠ 0 (increasing), and
// the values by index; returns the count (warp-uniform).
template <int VPL>
__device__ __forceinline__ int bsmall_list(const float (&x)[VPL], int lane, int* list,
                                           float* vals) {
    int base = 0;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const bool nz = x[v] != 0.0f;
        const unsigned int m = __ballot_sync(0xffffffffu, nz);
        if (nz) list[base + __popc(m & ((1u << lane) - 1u))] = lane + 32 * v;
        vals[lane + 32 * v] = x[v];
        base += __popc(m);
    }
    __syncwarp();
    return base;
}

template <int VPL>
__global__ void __launch_bounds__(256) k_bsmall(BatchState s, const float* __restrict__ Q32) {
    constexpr int NS = VPL * 32;  // row stride of the staged Q
    extern __shared__ float sq[];  // NS × NS staged Q, then per warp: list[NS], vals[NS]
    const int n = (int)s.n;
    int* wlist = reinterpret_cast<int*>(sq + NS * NS) + (threadIdx.x >> 5) * 2 * NS;
    float* wvals = reinterpret_cast<float*>(wlist + NS);
    for (int e = threadIdx.x; e < NS * NS; e += blockDim.x) {
        const int j = e / NS, i = e - j * NS;
        sq[e] = (i < n && j < n) ? Q32[(int64_t)j * s.ldq + i] : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // columns are dealt dynamically (counters[2]): a warp that finishes a
    // short column takes the next one, so long columns do not hold others
    for (;;) {
        int64_t c = 0;
        if (lane == 0) c = atomicAdd(&s.counters[2], 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= s.k) break;
        if (s.colst[c] >= 0) continue;  // warp-uniform
        float* Yc = s.Y + c * s.ldq;
        float* Lc = s.E + c * s.ldq;
        float* Gc = s.G + c * s.ldq;
        float y[VPL], yl[VPL], g[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = lane + 32 * v;
            y[v] = i < n ? Yc[i] : 0.0f;
            yl[v] = i < n ? Lc[i] : 0.0f;
            g[v] = i < n ? Gc[i] : 0.0f;
        }
        int it = s.iters[c], best_iter = s.best_iter[c];
        // step scalars as normalised FP32 pairs: the FP64 unit is narrow,
        // and this kernel keeps many columns' warps on each SM
        DF best = sc_of_double<DF>(s.best[c]);
        const DF eps = sc_of_double<DF>(s.eps[c]);
        const int max_iter = s.limits[0], window = s.limits[1];
        unsigned long long rowsP = 0, rowsC = 0, clipIt = 0;
        int status;
        for (;;) {
            float gb[VPL];
            float v2 = 0.0f;
            int cntP = 0;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int i = lane + 32 * v;
                const bool P = i < n && (y[v] > 0.0f || g[v] < 0.0f);
                gb[v] = P ? g[v] : 0.0f;
                v2 = fmaf(gb[v], gb[v], v2);
                cntP += __popc(__ballot_sync(0xffffffffu, P));
            }
            const DF gam = sc_warp_sum(DF{v2, 0.0f});
            status = -1;
            if (!sc_finite(gam)) status = ALN_RHS_NONFINITE;
            else if (cntP == 0) status = ALN_RHS_EMPTY_PASSIVE;
            else if (sc_lt(gam, eps) || sc_zero(gam)) status = ALN_RHS_CONVERGED;
            else if (it >= max_iter) status = ALN_RHS_MAXITER;
            else if (it - best_iter > window) status = ALN_RHS_STAGNATED;
            if (status >= 0) break;
            if (sc_lt(gam, best)) {
                best = gam;
                best_iter = it;
            }
            rowsP += (unsigned long long)cntP;
            // w = Qḡ over the j with ḡ_j ≠ 0 (Q symmetric: row j of the staged Q)
            float w[VPL];
#pragma unroll
            for (int u = 0; u < VPL; ++u) w[u] = 0.0f;
            {
                const int cnt = bsmall_list<VPL>(gb, lane, wlist, wvals);
                bsmall_rows<VPL>(sq, wlist, wvals, cnt, lane, w);
                __syncwarp();
            }
            float kp = 0.0f;
#pragma unroll
            for (int v = 0; v < VPL; ++v) kp = fmaf(gb[v], w[v], kp);
            const DF kap = sc_warp_sum(DF{kp, 0.0f});
            if (!sc_finite(kap)) {
                status = ALN_RHS_NONFINITE;
                break;
            }
            if (sc_nonpos(kap)) {
                status = ALN_RHS_CURVATURE;
                break;
            }
            const float a = df_quotient(gam, kap);
            // y⁺ = [y − αḡ]₊, e on the clipped set, g ← g − αw (+ Qe below)
            float e[VPL];
            int nclip = 0;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                // (yh, yl) − αḡ exactly: TwoSum, then renormalise
                const float step = __fmul_rn(a, gb[v]);
                const float s1 = y[v] - step;
                const float bb = s1 - y[v];
                const float er = (y[v] - (s1 - bb)) + (-step - bb);
                const float t = yl[v] + er;
                float nh = s1 + t, nl = t - ((s1 + t) - s1), ev = 0.0f;
                if (nh < 0.0f) {  // clipped: y⁺ = 0, e = y⁺ − (y − αḡ)
                    ev = -(nh + nl);
                    nh = 0.0f;
                    nl = 0.0f;
                }
                y[v] = nh;
                yl[v] = nl;
                e[v] = ev;
                g[v] = g[v] - a * w[v];
                nclip += __popc(__ballot_sync(0xffffffffu, ev != 0.0f));
            }
            ++it;
            if (nclip > 0) {
                rowsC += (unsigned long long)nclip;
                ++clipIt;
                float qe[VPL];
#pragma unroll
                for (int u = 0; u < VPL; ++u) qe[u] = 0.0f;
                const int cnt = bsmall_list<VPL>(e, lane, wlist, wvals);
                bsmall_rows<VPL>(sq, wlist, wvals, cnt, lane, qe);
                __syncwarp();
#pragma unroll
                for (int u = 0; u < VPL; ++u) g[u] += qe[u];
            }
        }
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = lane + 32 * v;
            if (i < n) {
                Yc[i] = y[v];
                Lc[i] = yl[v];
                Gc[i] = g[v];
            }
        }
        if (lane == 0) {
            s.colst[c] = status;
            s.iters[c] = it;
            s.best[c] = sc_double(best);
            s.best_iter[c] = best_iter;
            atomicAdd(&s.rows[0], rowsP);
            atomicAdd(&s.rows[1], rowsC);
            atomicAdd(&s.rows[2], clipIt);
        }
    }
}

// ---------------------------------------------------------------------------
// Tail of the batched phase.  Once few columns are still running, a batched
// iteration is bound by launch and tile latency (about 30-90 µs whatever the
// count), and the last columns run hundreds of iterations more than the
// median one.  They go to the grouped solver's kernels: each running column
// is one problem (shared Q, its own q, y and stop state), solved by one CTA
// or, as the count drops, by a thread-block cluster that splits each product
// over its CTAs; the launches are cut into iteration budgets so that the
// cluster size can grow as columns finish.
// ---------------------------------------------------------------------------

// Hand-off: y and g of every running column in FP64 (the grouped kernels keep
// y as an FP32 pair and g in FP32), its record, its inner target relative to ‖min(q,0)‖ (so that
// (tgt·den)² is the column's ε), and the list of running columns.
__global__ void k_btail_in(BatchState s, const double* __restrict__ den, double* __restrict__ Y64,
                           double* __restrict__ G64, GStat* __restrict__ st,
                           double* __restrict__ tgt, int* __restrict__ order,
                           int* __restrict__ cnt) {
    const int64_t c = blockIdx.x;
    if (s.colst[c] >= 0) return;
    for (int64_t i = threadIdx.x; i < s.ldq; i += blockDim.x) {
        const bool in = i < s.n;
        Y64[c * s.ldq + i] = in ? (double)s.Y[c * s.ldq + i] : 0.0;
        G64[c * s.ldq + i] = in ? (double)s.G[c * s.ldq + i] : 0.0;
    }
    if (threadIdx.x == 0) {
        GStat z = {};
        z.iters = s.iters[c];
        z.status = -1;
        st[c] = z;
        const double d = den[c] > 0.0 ? den[c] : 1.0;
        tgt[c] = sqrt(s.eps[c]) / d;
        order[atomicAdd(cnt, 1)] = (int)c;
    }
}

// After a tail launch (one block per listed column): y back in FP32; paused
// columns are listed again for the next launch, the others take their final
// inner status and add their row counts.
__global__ void k_btail_out(BatchState s, const double* __restrict__ Y64,
                            const GStat* __restrict__ st, const int* __restrict__ order,
                            int* __restrict__ order2, int* __restrict__ cnt2) {
    const int64_t c = order[blockIdx.x];
    for (int64_t i = threadIdx.x; i < s.n; i += blockDim.x)
        s.Y[c * s.ldq + i] = (float)Y64[c * s.ldq + i];
    if (threadIdx.x == 0) {
        const GStat g = st[c];
        s.iters[c] = g.iters;
        if (g.status == kRhsPaused) {
            order2[atomicAdd(cnt2, 1)] = (int)c;
        } else {
            s.colst[c] = g.status;
            atomicAdd(&s.rows[0], (unsigned long long)g.sum_passive);
            atomicAdd(&s.rows[1], (unsigned long long)g.sum_clip);
            atomicAdd(&s.rows[2], (unsigned long long)g.clip_iters);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Progressive refinement is on by default here: with many columns the FP64
// checks are cheap per column and shorter inner runs cut the column-iterations.
static int batch_gain(const aln_ctx* c) { return c->opt.refine_gain == 0 ? 3 : c->opt.refine_gain; }
// A refinement run of a column stops at this fraction of tol (or its gain
// target, if higher).  The tensor-core path (n > 128) stops close to tol:
// its last columns run hundreds of iterations per tenfold drop of the
// residual, and on the 10000×1000, 4096-column workload 0.75 gave the
// shortest solve (0.25: 62.4 ms, 0.5: 57.5 ms, 0.75: 54.3 ms).  The one-warp
// path for n ≤ 128 keeps 0.25: its refinement rounds cost little, and the
// lower stop keeps an outer loop such as NMF's on the FP64 trajectory.
constexpr double kBatchRefineFactor = 0.75;
constexpr double kSmallRefineFactor = 0.25;

struct BatchWork {
    int64_t k = 0, n = 0, ldq = 0, ldk = 0;
    int mtiles = 0;
    void* pool = nullptr;
    size_t pool_bytes = 0;
    double* Q64 = nullptr;
    __nv_bfloat16* Qhi = nullptr;
    __nv_bfloat16* Qlo = nullptr;
    double* bn2 = nullptr;
    double* X64 = nullptr;
    double* Y64 = nullptr;
    double* G64 = nullptr;
    int* rounds = nullptr;
    int* fin = nullptr;
    double* rel = nullptr;
    double* obj = nullptr;
    int* react = nullptr;
    int* host = nullptr;          // pinned: [0] running count, [1] re-activated
    BatchState s{};
    cudaGraphExec_t graph = nullptr;
    int chunk = 8;
    int small_vpl = 0;            // n ≤ 128: entries per lane of k_bsmall (1, 2, 4), else 0
    // tail (grouped kernels): one problem record per column, records, inner
    // targets, two column lists, counters [0] listed, [1] relisted, [2] queue
    void* tail = nullptr;
    size_t tail_bytes = 0;
    GProb* tgp = nullptr;
    GStat* tstat = nullptr;
    double* ttgt = nullptr;
    int* torder = nullptr;
    int* tcnt = nullptr;
};

static aln_status bw_alloc(aln_ctx* c, BatchWork* b) {
    const int64_t k = c->k, n = c->n, ldq = c->ldq, ldk = round_up(n, 64);
    b->k = k;
    b->n = n;
    b->ldq = ldq;
    b->ldk = ldk;
    b->mtiles = (int)ceil_div(n, 128);
    const size_t f = (size_t)k * ldq * 4, d8 = (size_t)k * ldq * 8;
    // One entry per buffer, in the order they are carved out below; each is
    // rounded to 256 bytes exactly as take() rounds it.
    const size_t sizes[] = {
        (size_t)ldq * ldq * 8,                               // Q64
        (size_t)n * ldk * 2, (size_t)n * ldk * 2,            // Qhi, Qlo
        (size_t)k * 8,                                       // bn2
        d8, d8, d8,                                          // X64, Y64, G64
        f, f, f, f, f,                                       // Y, G, GB, E, W
        (size_t)k * ldk * 2, (size_t)k * ldk * 2,            // Vhi, Vlo
        (size_t)b->mtiles * k * 8,                           // kpart
        (size_t)k * 4, (size_t)k * 4, (size_t)k * 4,         // colst, iters, best_iter
        (size_t)k * 4, (size_t)k * 4, (size_t)k * 4,         // map_act, map_clip, rounds
        (size_t)k * 8, (size_t)k * 8, (size_t)k * 8,         // best, eps, gamma
        (size_t)k * 4, (size_t)k * 8, (size_t)k * 8,         // fin, rel, obj
        64, 64, 64, 64};                                     // counters, rows, limits, react
    size_t total = 0;
    for (size_t x : sizes) total += round_up(x, 256);
    if (b->pool_bytes < total) {
        if (b->pool) cudaFree(b->pool);
        b->pool = nullptr;
        b->pool_bytes = 0;
        if (cudaMalloc(&b->pool, total) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
        b->pool_bytes = total;
    }
    uint8_t* p = (uint8_t*)b->pool;
    uint8_t* const end = p + total;
    int taken = 0;
    auto take = [&](size_t x) {
        // the carve-out must follow `sizes` entry by entry
        if (taken >= (int)(sizeof(sizes) / sizeof(sizes[0])) || sizes[taken] != x) return (void*)nullptr;
        ++taken;
        void* r = p;
        p += round_up(x, 256);
        return p <= end ? r : (void*)nullptr;
    };
    b->Q64 = (double*)take((size_t)ldq * ldq * 8);
    b->Qhi = (__nv_bfloat16*)take((size_t)n * ldk * 2);
    b->Qlo = (__nv_bfloat16*)take((size_t)n * ldk * 2);
    b->bn2 = (double*)take((size_t)k * 8);
    b->X64 = (double*)take(d8);
    b->Y64 = (double*)take(d8);
    b->G64 = (double*)take(d8);
    BatchState& s = b->s;
    s.n = n;
    s.ldq = ldq;
    s.ldk = ldk;
    s.k = k;
    s.mtiles = b->mtiles;
    s.Y = (float*)take(f);
    s.G = (float*)take(f);
    s.GB = (float*)take(f);
    s.E = (float*)take(f);
    s.W = (float*)take(f);
    s.Vhi = (__nv_bfloat16*)take((size_t)k * ldk * 2);
    s.Vlo = (__nv_bfloat16*)take((size_t)k * ldk * 2);
    s.kpart = (double*)take((size_t)b->mtiles * k * 8);
    s.colst = (int*)take((size_t)k * 4);
    s.iters = (int*)take((size_t)k * 4);
    s.best_iter = (int*)take((size_t)k * 4);
    s.map_act = (int*)take((size_t)k * 4);
    s.map_clip = (int*)take((size_t)k * 4);
    b->rounds = (int*)take((size_t)k * 4);
    s.best = (double*)take((size_t)k * 8);
    s.eps = (double*)take((size_t)k * 8);
    s.gamma = (double*)take((size_t)k * 8);
    b->fin = (int*)take((size_t)k * 4);
    b->rel = (double*)take((size_t)k * 8);
    b->obj = (double*)take((size_t)k * 8);
    s.counters = (int*)take(64);
    s.rows = (unsigned long long*)take(64);
    s.limits = (int*)take(64);
    b->react = (int*)take(64);
    if (!b->react || taken != (int)(sizeof(sizes) / sizeof(sizes[0])))
        return ALN_ERR_CUDA;  // layout and size table disagree: never launch on it
    if (cudaMemsetAsync(b->pool, 0, b->pool_bytes, c->stream) != cudaSuccess) return ALN_ERR_CUDA;
    return ALN_OK;
}

static cudaError_t bw_iteration(aln_ctx* c, BatchWork* b) {
    BatchState& s = b->s;
    k_breset<<<1, 1, 0, c->stream>>>(s.counters);
    k_bmask<<<(unsigned)b->k, kBMThreads, 0, c->stream>>>(s);
    cudaError_t e = launch_bgemm_tc(0, b->Qhi, b->Qlo, b->n, b->ldk, s.Vhi, s.Vlo, b->k,
                                    s.counters, s.map_act, b->ldq, s.W, s.GB, s.kpart, nullptr,
                                    c->flags + 1, c->stream);
    if (e != cudaSuccess) return e;
    k_bupdate<<<(unsigned)b->k, kBMThreads, 0, c->stream>>>(s);
    return launch_bgemm_tc(1, b->Qhi, b->Qlo, b->n, b->ldk, s.Vhi, s.Vlo, b->k, s.counters + 1,
                           s.map_clip, b->ldq, nullptr, nullptr, nullptr, s.G, c->flags + 1,
                           c->stream);
}

__global__ void k_btail_records(GProb* __restrict__ gp, int64_t k, int64_t d, int64_t n,
                                int64_t ldq) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= k) return;
    GProb g = {};
    g.d = (int32_t)d;
    g.n = (int32_t)n;
    g.ldq = (int32_t)ldq;
    g.qoff = 0;
    g.voff = col * ldq;
    g.foff = col * ldq;
    gp[col] = g;
}

// Buffers of the tail and its problem records: column c is a problem of n
// unknowns over the shared Q (qoff 0), its q and y at c·ldq.
static aln_status bw_tail_alloc(aln_ctx* c, BatchWork* b) {
    const int64_t k = b->k;
    const size_t need = round_up(k * sizeof(GProb), 256) + round_up(k * sizeof(GStat), 256) +
                        round_up(k * 8, 256) + round_up(2 * k * 4, 256) + 256;
    if (b->tail_bytes < need) {
        if (b->tail) cudaFree(b->tail);
        b->tail = nullptr;
        b->tail_bytes = 0;
        if (cudaMalloc(&b->tail, need) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
        b->tail_bytes = need;
    }
    uint8_t* p = (uint8_t*)b->tail;
    b->tgp = (GProb*)p;
    p += round_up(k * sizeof(GProb), 256);
    b->tstat = (GStat*)p;
    p += round_up(k * sizeof(GStat), 256);
    b->ttgt = (double*)p;
    p += round_up(k * 8, 256);
    b->torder = (int*)p;
    p += round_up(2 * k * 4, 256);
    b->tcnt = (int*)p;
    k_btail_records<<<(unsigned)ceil_div(k, 256), 256, 0, c->stream>>>(b->tgp, k, c->d, b->n,
                                                                          b->ldq);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? ALN_OK : ALN_ERR_CUDA;
}

static aln_status bw_capture(aln_ctx* c, BatchWork* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return ALN_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->chunk && e == cudaSuccess; ++i) e = bw_iteration(c, b);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return ALN_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? ALN_OK : ALN_ERR_CUDA;
}

void batch_free(aln_ctx* c) {
    BatchWork* b = (BatchWork*)c->batch;
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->pool) cudaFree(b->pool);
    if (b->tail) cudaFree(b->tail);
    if (b->host) cudaFreeHost(b->host);
    delete b;
    c->batch = nullptr;
}

// The FP64 scaled matrix of the checks from FP32 A by exact digit products.
static cudaError_t oz_gram(aln_ctx* c, BatchWork* b) {
    const size_t need = oz_work_bytes(c->d, c->n, c->n);
    if (c->oz_work_bytes < need) {
        if (c->oz_work) cudaFree(c->oz_work);
        c->oz_work = nullptr;
        c->oz_work_bytes = 0;
        cudaError_t e = cudaMalloc(&c->oz_work, need);
        if (e != cudaSuccess) return e;
        c->oz_work_bytes = need;
    }
    c->launches += 4;
    return launch_oz_gram((const float*)c->A, c->lda, c->d, c->n, c->inv_s, b->Q64, c->ldq,
                          c->oz_work, c->oz_work_bytes, c->flags + 1, c->stream);
}

// Alg. 1 for a batch: s and q in FP64 (prepare kernels), Q64 in FP64 (kept for
// the checks), Q in FP32 and its BF16 split for the tensor-core iteration.
aln_status batch_prepare(aln_ctx* c) {
    BatchWork* b = (BatchWork*)c->batch;
    if (!b) {
        b = new (std::nothrow) BatchWork();
        if (!b) return ALN_ERR_OUT_OF_MEMORY;
        c->batch = b;
        if (cudaMallocHost(&b->host, 64) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
    }
    aln_status st = bw_alloc(c, b);
    if (st != ALN_OK) return st;
    st = bw_tail_alloc(c, b);
    if (st != ALN_OK) return st;
    const cudaError_t eg =
        c->dtype == ALN_DTYPE_F32
            ? oz_gram(c, b)
            : launch_gram64(c->A, c->dtype, c->d, c->n, c->lda, c->inv_s, b->Q64, c->ldq,
                            c->stream);
    if (eg != cudaSuccess) return ALN_ERR_CUDA;
    k_qsplit<<<(unsigned)c->n, kBThreads, 0, c->stream>>>(b->Q64, c->ldq, c->n, b->ldk,
                                                        (float*)c->Q, b->Qhi, b->Qlo);
    k_bnorm2<<<(unsigned)c->k, kBThreads, 0, c->stream>>>(c->B, c->dtype, c->d, c->ldb, b->bn2);
    c->launches += 3;
    if (cudaGetLastError() != cudaSuccess) return ALN_ERR_CUDA;
    b->small_vpl = c->n <= 32 ? 1 : c->n <= 64 ? 2 : c->n <= 128 ? 4 : 0;
    if (b->small_vpl) return ALN_OK;  // the warp-per-column kernel needs no graph
    return bw_capture(c, b);
}

// g = float(g64) for every column (start point given).
__global__ void k_bsetg(BatchState s, const double* __restrict__ G64) {
    const int64_t c = blockIdx.x;
    for (int64_t i = threadIdx.x; i < s.n; i += blockDim.x)
        s.G[c * s.ldq + i] = (float)G64[c * s.ldq + i];
}


// G64 = Q64·Y64 + q for every column, FP64-accurate (exact BF16 digit
// products on the tensor cores; the digits keep 49 bits below each row of
// Q64 and each y).
static aln_status bw_qy(aln_ctx* c, BatchWork* b) {
    const size_t need = oz_work_bytes(c->n, c->n, b->k);
    if (c->oz_work_bytes < need) {
        if (c->oz_work) cudaFree(c->oz_work);
        c->oz_work = nullptr;
        c->oz_work_bytes = 0;
        if (cudaMalloc(&c->oz_work, need) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
        c->oz_work_bytes = need;
    }
    if (launch_oz_product(1, ALN_DTYPE_F64, b->Q64, c->ldq, ALN_DTYPE_F64, b->Y64, c->ldq, c->n,
                          c->n, b->k, c->q64, b->G64, c->ldq, c->oz_work, c->oz_work_bytes,
                          c->flags + 1, c->stream) != cudaSuccess)
        return ALN_ERR_CUDA;
    c->launches += 3;
    return ALN_OK;
}

// FP64 check of every not-yet-final column; returns how many were restarted.
static aln_status bw_check(aln_ctx* c, BatchWork* b, double tol, int max_refine, int* restarted) {
    BatchState& s = b->s;
    const int64_t k = b->k;
    cudaEventRecord(c->ev[6], c->stream);
    k_bunscale<<<(unsigned)k, kBThreads, 0, c->stream>>>(s, c->s, b->X64, b->Y64,
                                                         b->small_vpl ? s.E : nullptr);
    // g = Q y + q in FP64 accuracy (exact digit products on the tensor cores)
    {
        aln_status gs = bw_qy(c, b);
        if (gs != ALN_OK) return gs;
    }
    cudaMemsetAsync(b->react, 0, sizeof(int), c->stream);
    k_bcheck<<<(unsigned)k, kBThreads, 0, c->stream>>>(s, b->G64, b->Y64, c->q64, b->bn2, c->den,
                                                       tol,
                                                       b->small_vpl ? kSmallRefineFactor
                                                                    : kBatchRefineFactor,
                                                       batch_gain(c), max_refine,
                                                       b->rounds, b->fin,
                                                       b->rel, b->obj, b->react);
    cudaEventRecord(c->ev[7], c->stream);
    c->launches += 3;
    if (cudaMemcpyAsync(b->host + 1, b->react, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return ALN_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]) == cudaSuccess) c->stats.kkt_ms += ms;
    *restarted = b->host[1];
    return ALN_OK;
}

static bool dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

aln_status batch_solve(aln_ctx* c, double tol, int max_iter, double* X, int64_t ldx,
                       const double* X0, aln_solve_info* info) {
    BatchWork* b = (BatchWork*)c->batch;
    BatchState& s = b->s;
    const int64_t k = b->k;
    // iterations per captured chunk: 8, or the autotuner's choice
    const int chunk = c->tune_chunk > 0 ? c->tune_chunk : 8;
    if (!b->small_vpl && chunk != b->chunk) {
        b->chunk = chunk;
        aln_status cs = bw_capture(c, b);
        if (cs != ALN_OK) return cs;
    }
    const double* X0dev = nullptr;
    if (X0) {  // stage the start points in X64 (ld = ldq) and check them
        if (cudaMemcpy2DAsync(b->X64, c->ldq * 8, X0, ldx * 8, c->n * 8, k,
                              dev_ptr(X0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream) != cudaSuccess)
            return ALN_ERR_CUDA;
        cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream);
        if (launch_check_finite(b->X64, ALN_DTYPE_F64, c->n, k, c->ldq, c->flags, c->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(c->flags_host, c->flags, sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return ALN_ERR_CUDA;
        if (c->flags_host[0]) return ALN_ERR_NONFINITE;
        X0dev = b->X64;
    }
    // per-solve limits live in device memory (the graph holds the state by value)
    int lim[2] = {max_iter, c->opt.stagnation};
    if (cudaMemcpyAsync(s.limits, lim, sizeof(lim), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
        return ALN_ERR_CUDA;
    k_binit<<<(unsigned)k, kBThreads, 0, c->stream>>>(
        s, c->q64, X0dev, c->ldq, c->s, c->den, inner_target(tol, 0.5, 1.0, batch_gain(c)),
        b->rounds);
    cudaMemsetAsync(b->fin, 0xff, (size_t)k * 4, c->stream);  // -1: not final yet
    cudaMemsetAsync(s.rows, 0, 24, c->stream);
    c->launches += 1;
    if (X0dev) {  // g = Q y0 + q, in FP64, for a start point
        k_bunscale<<<(unsigned)k, kBThreads, 0, c->stream>>>(s, c->s, b->X64, b->Y64,
                                                             b->small_vpl ? s.E : nullptr);
        aln_status gs = bw_qy(c, b);
        if (gs != ALN_OK) return gs;
        k_bsetg<<<(unsigned)k, kBThreads, 0, c->stream>>>(s, b->G64);
        c->launches += 3;
    }
    const int max_refine = c->opt.max_refine;
    // tail: at most tail_max running columns go to the grouped kernels
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    const bool tail_ok = !b->small_vpl && tail_smem_bytes(c->ldq, false) + 1024 <= (size_t)optin;
    const bool tail_cl = tail_ok && tail_smem_bytes(c->ldq, true) + 1024 <= (size_t)optin;
    const int64_t tail_max = c->tune_tail > 0 ? (int64_t)c->tune_tail : 2LL * c->num_sms;
    const int budget = c->tune_budget > 0 ? c->tune_budget : kTailBudget;
    auto run_tail = [&]() -> aln_status {
        int* cur = b->torder;
        int* nxt = b->torder + k;
        if (cudaMemsetAsync(b->tcnt, 0, 2 * sizeof(int), c->stream) != cudaSuccess)
            return ALN_ERR_CUDA;
        // (G64 is free until the FP64 check: it carries g between launches)
        k_btail_in<<<(unsigned)k, kBThreads, 0, c->stream>>>(s, c->den, b->Y64, b->G64,
                                                             b->tstat, b->ttgt, cur, b->tcnt);
        c->launches += 1;
        if (cudaMemcpyAsync(b->host + 2, b->tcnt, sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return ALN_ERR_CUDA;
        int count = b->host[2];
        while (count > 0) {
            // the largest cluster that still gives every column its own
            // CTAs; no budget once the cluster cannot grow any more
            int cs = 1;
            while (tail_cl && cs < 8 && (int64_t)count * cs * 2 <= c->num_sms) cs *= 2;
            const int bud = (cs < 8 && count > 1) ? budget : 0;
            aln_status ts = tail_launch(c, b->tgp, cur, count, b->tcnt + 2, (const float*)c->Q,
                                        c->ldq, c->q64, c->den, b->Y64, b->G64, b->tstat,
                                        b->ttgt, max_iter, bud, cs);
            if (ts != ALN_OK) return ts;
            if (cudaMemsetAsync(b->tcnt + 1, 0, sizeof(int), c->stream) != cudaSuccess)
                return ALN_ERR_CUDA;
            k_btail_out<<<(unsigned)count, kBThreads, 0, c->stream>>>(s, b->Y64, b->tstat, cur,
                                                                      nxt, b->tcnt + 1);
            c->launches += 1;
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(b->host + 2, b->tcnt + 1, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return ALN_ERR_CUDA;
            count = b->host[2];
            std::swap(cur, nxt);
        }
        return ALN_OK;
    };
    int64_t active = k;  // running columns at the start of a round
    for (int round = 0;; ++round) {
        // inner runs: the captured chunk until no column is running (small n:
        // one warp-per-column launch runs every column to its stop)
        const int64_t bound = b->small_vpl ? 1 : max_iter / b->chunk + 3;
        int64_t l = 0;
        cudaEventRecord(c->ev[8], c->stream);
        if (b->small_vpl) {
            const int vpl = b->small_vpl;
            const size_t smem = (size_t)(vpl * 32) * (vpl * 32) * 4 + 8 * 2 * (vpl * 32) * 4;
            // a resident grid (the column queue feeds it)
            auto fn = vpl == 1 ? k_bsmall<1> : vpl == 2 ? k_bsmall<2> : k_bsmall<4>;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return ALN_ERR_CUDA;
            int per_sm = 1;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem) !=
                    cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
            const unsigned grid = (unsigned)std::max<int64_t>(
                1, std::min<int64_t>((k + 7) / 8, (int64_t)per_sm * c->num_sms));
            if (cudaMemsetAsync(s.counters + 2, 0, sizeof(int), c->stream) != cudaSuccess)
                return ALN_ERR_CUDA;
            fn<<<grid, 256, smem, c->stream>>>(s, (const float*)c->Q);
            if (cudaGetLastError() != cudaSuccess) return ALN_ERR_CUDA;
            c->launches += 1;
            l = 1;
        }
        bool handed = false;
        if (tail_ok && active <= tail_max) {  // few columns: no batched chunk at all
            cudaEventRecord(c->ev[10], c->stream);
            aln_status ts = run_tail();
            if (ts != ALN_OK) return ts;
            handed = true;
            l = bound;
        }
        for (; l < bound; ++l) {
            if (cudaGraphLaunch(b->graph, c->stream) != cudaSuccess) return ALN_ERR_CUDA;
            c->launches += 5LL * b->chunk;
            if (cudaMemcpyAsync(b->host, s.counters, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return ALN_ERR_CUDA;
            if (b->host[0] == 0) break;
            if (tail_ok && b->host[0] <= tail_max) {  // the rest: the tail
                cudaEventRecord(c->ev[10], c->stream);
                aln_status ts = run_tail();
                if (ts != ALN_OK) return ts;
                handed = true;
                break;
            }
        }
        cudaEventRecord(c->ev[9], c->stream);
        cudaEventSynchronize(c->ev[9]);
        float ms = 0.f, tms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[8], c->ev[9]) == cudaSuccess)
            c->stats.iterate_ms += ms;
        if (handed && cudaEventElapsedTime(&tms, c->ev[10], c->ev[9]) == cudaSuccess)
            c->stats.phase_us[1] += 1e3 * tms;
        c->stats.phase_us[0] += 1e3 * (ms - (handed ? tms : 0.f));
        if (!b->small_vpl && !handed && l == bound) return ALN_ERR_TIMEOUT;
        int restarted = 0;
        aln_status st = bw_check(c, b, tol, max_refine, &restarted);
        if (st != ALN_OK) return st;
        if (restarted == 0) break;
        active = restarted;
    }
    // results: x (FP64) and per-column records
    const bool x_dev = [&] {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, X) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    }();
    if (cudaMemcpy2DAsync(X, ldx * 8, b->X64, c->ldq * 8, c->n * 8, k,
                          x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess)
        return ALN_ERR_CUDA;
    unsigned long long rows[3] = {0, 0, 0};
    cudaMemcpyAsync(rows, s.rows, sizeof(rows), cudaMemcpyDeviceToHost, c->stream);
    if (info) {
        int* tmp_i = new (std::nothrow) int[3 * k];
        double* tmp_d = new (std::nothrow) double[2 * k];
        if (!tmp_i || !tmp_d) {
            delete[] tmp_i;
            delete[] tmp_d;
            return ALN_ERR_OUT_OF_MEMORY;
        }
        cudaMemcpyAsync(tmp_i, s.iters, k * 4, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(tmp_i + k, b->fin, k * 4, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(tmp_i + 2 * k, b->rounds, k * 4, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(tmp_d, b->rel, k * 8, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(tmp_d + k, b->obj, k * 8, cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            delete[] tmp_i;
            delete[] tmp_d;
            return ALN_ERR_CUDA;
        }
        int64_t total = 0;
        for (int64_t j = 0; j < k; ++j) {
            info[j].iters = tmp_i[j];
            info[j].status = tmp_i[k + j];
            info[j].refine_rounds = tmp_i[2 * k + j];
            info[j].reserved = 0;
            info[j].rel_kkt = tmp_d[j];
            info[j].objective = tmp_d[k + j];
            total += tmp_i[j];
        }
        c->stats.iterations = total;
        delete[] tmp_i;
        delete[] tmp_d;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ALN_ERR_CUDA;
    c->stats.passive_rows = (int64_t)rows[0];
    c->stats.clipped_rows = (int64_t)rows[1];
    c->stats.product_bytes = 4.0 * (double)s.n * (rows[0] + rows[1]);
    c->stats.clipped_iterations = (int32_t)rows[2];
    return ALN_OK;
}

}  // namespace aln
