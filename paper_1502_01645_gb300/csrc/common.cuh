// Shared device helpers and the library context of libaln.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "aln.h"

namespace aln {

constexpr int kWarp = 32;

// Device-resident state of one Alg. 2 run on one right-hand side.  Written by
// the iteration kernels, read back by the host after each persistent launch.
struct IterState {
    double eps;       // stop threshold on ‖ḡ‖² (absolute)
    double gbar2;     // ‖ḡ‖² when the loop stopped
    double alpha;     // last step size
    int32_t iter;     // iterations done in this run
    int32_t max_iter; // iteration cap of this run
    int32_t done;     // 1 once the loop has stopped
    int32_t status;   // aln_rhs_status
    int32_t npassive; // |P| when the loop stopped
    int32_t window;   // stagnation window (iterations without a new best ‖ḡ‖²)
    double best_g2;   // smallest ‖ḡ‖² seen in this run
    int32_t best_iter;
    int32_t pad;
    int64_t sum_passive;  // Σ_k |P_k|: rows of Q read for w = Qḡ
    int64_t sum_clip;     // Σ_k |C_k|: rows read for the clipped correction
    uint64_t phase_ns[6]; // block 0's time per phase: product, barrier, update,
                          // clipped correction, mask, other
};

template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int N = 2;
};

__device__ __forceinline__ float vget(const float4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ double vget(const double2& v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4& v, int i, float x) {
    if (i == 0) v.x = x;
    else if (i == 1) v.y = x;
    else if (i == 2) v.z = x;
    else v.w = x;
}
__device__ __forceinline__ void vset(double2& v, int i, double x) {
    if (i == 0) v.x = x;
    else v.y = x;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed shuffle tree, then warp 0 over the warp sums).
// Result is valid in thread 0.  `scratch` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        r = lane < nw ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Sum of p[0..count) computed by one warp in a fixed order; valid in all lanes.
__device__ __forceinline__ double warp_sum_array(const double* __restrict__ p, int count) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < count; i += 32) v += p[i];
    return warp_sum(v);
}
__device__ __forceinline__ int warp_sum_array_i(const int* __restrict__ p, int count) {
    const int lane = threadIdx.x & 31;
    int v = 0;
    for (int i = lane; i < count; i += 32) v += p[i];
    return warp_sum_i(v);
}

// Four consecutive elements at a 16-byte aligned address, widened to FP64.
__device__ __forceinline__ void load4(const float* p, double* o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double* o) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

// Three-term BF16 split of an FP32 value: a = h + m + l exactly (8 + 8 + 8
// significant bits cover FP32's 24; each difference below is exact in FP32).
__device__ __forceinline__ void split3_bf16(float a, __nv_bfloat16& h, __nv_bfloat16& m,
                                            __nv_bfloat16& l) {
    h = __float2bfloat16_rn(a);
    const float r1 = a - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Rounded products that the compiler may not fuse into a following add: the
// error-free transformations below need fl(a·b) as a separate value.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Per-thread accumulator of a dot product.  FP32 inputs use Dot2 (Ogita,
// Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005):
// the exact product error from an FMA (TwoProduct) and the exact addition
// error (TwoSum) are carried in a second float, so the result is as accurate
// as if accumulated in twice the working precision — without the FP64 pipe,
// which is narrow on this GPU.  FP64 inputs accumulate in FP64.
template <typename TA> struct DotAcc;
template <> struct DotAcc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = mul_rn(a, b);
        const float ep = fmaf(a, b, -p);   // a·b = p + ep exactly
        const float t = s + p;
        const float z = t - s;
        const float es = (s - (t - z)) + (p - z);  // s + p = t + es exactly
        s = t;
        c += es + ep;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// Stop target (relative KKT residual) of one inner FP32 run of Alg. 2 under
// progressive refinement: `gain` decades below the FP64 residual measured
// before the run (1 before the first run, where ḡ(0) = min(q, 0)), but not
// below factor·tol; gain ≤ 0 aims at factor·tol directly.
__host__ __device__ inline double inner_target(double tol, double factor, double rel_prev,
                                               int gain) {
    const double floor_t = factor * tol;
    if (gain <= 0) return floor_t;
    double t = rel_prev;
    for (int i = 0; i < gain; ++i) t *= 0.1;
    return t > floor_t ? t : floor_t;
}

// True when base + k·ld is 16-byte aligned for every k (vector loads allowed).
inline bool aligned16(const void* base, int64_t ld, size_t esz) {
    return ((uintptr_t)base % 16 == 0) && ((ld * (int64_t)esz) % 16 == 0);
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

}  // namespace aln

// --------------------------------------------------------------------------
// Library context (opaque to callers; see include/aln.h)
// --------------------------------------------------------------------------
struct aln_ctx {
    aln_options opt;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // created when the caller passes no stream
    void* host_pool = nullptr;          // pinned: iteration state, KKT result, flags
    int device = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;

    // problem
    int prepared = 0;
    int64_t d = 0, n = 0, k = 0;
    int32_t dtype = ALN_DTYPE_F32;
    const void* A = nullptr;  // device pointer actually used (caller's or copy)
    int64_t lda = 0;
    const void* B = nullptr;
    int64_t ldb = 0;
    void* A_copy = nullptr;   // owned copies of host inputs
    size_t A_copy_bytes = 0;
    void* B_copy = nullptr;
    size_t B_copy_bytes = 0;

    // derived problem (Alg. 1)
    int64_t ldq = 0;          // padded row length of Q and of every n-vector
    void* Q = nullptr;        // ldq × ldq, float (SPLIT_BF16) or double (FP64)
    size_t Q_bytes = 0;
    int Q_elt = 0;            // element size Q was zeroed for
    int64_t Q_n = 0;          // n Q was zeroed for (padding must stay 0)
    void* prep_pool = nullptr;  // s, inv_s, q64, den, flags
    size_t prep_bytes = 0;
    int64_t den_host_cap = 0;
    double* s = nullptr;      // n scale factors s_i = ‖A_i‖ (1 for zero columns)
    double* inv_s = nullptr;  // 1/s_i
    double* q64 = nullptr;    // k × ldq, q_c = −D⁻¹Aᵀb_c in FP64
    double* den = nullptr;    // k denominators ‖min(q_c, 0)‖
    double* den_host = nullptr;
    int* flags = nullptr;     // [0] nonfinite input, [1] tensor-core timeout
    int* flags_host = nullptr;
    // split copies of A for the tensor-core Gram
    int64_t ldk = 0;
    __nv_bfloat16* A_hi = nullptr;
    __nv_bfloat16* A_lo = nullptr;
    size_t split_bytes = 0;  // also holds the packed boxes of a CSC prepare
    // CSC prepare: device copies of host CSC arrays, occupancy, box numbering
    void* csc_pool = nullptr;
    size_t csc_bytes = 0;
    // 1 when A lives only as CSC arrays + packed boxes (no dense copy): the
    // KKT pass then reads those (launch_csc_kkt)
    int csc_kkt = 0;
    const int64_t* csc_cp = nullptr;
    const int32_t* csc_ri = nullptr;
    const float* csc_v = nullptr;
    uint32_t* csc_occ = nullptr;
    int32_t* csc_wbase = nullptr;
    int64_t* csc_toff = nullptr;
    double* csc_fpart = nullptr;
    int csc_W = 0;
    size_t csc_box_bytes = 0;  // one split term's packed boxes in A_hi
    void* g64_work = nullptr;  // split-K partial tiles of the FP64 Gram (small n)
    size_t g64_work_bytes = 0;
    void* oz_work = nullptr;   // digits and exponents of the exact-product q (batched)
    size_t oz_work_bytes = 0;
    void* sp_part = nullptr;   // split-K partial tiles of the block-sparse Gram
    size_t sp_part_bytes = 0;
    // tiles of Q that may be non-zero (block-sparse Gram; null = all): bit rt
    // of q_tmask[ct·q_tw + rt/32] for row tile rt, column tile ct (128 wide)
    const uint32_t* q_tmask = nullptr;
    int q_tw = 0;

    // iteration workspace (element type follows the precision)
    void* qv = nullptr;       // q of the right-hand side being solved (iteration type)
    void* y = nullptr;
    void* g = nullptr;
    void* gb = nullptr;
    void* w = nullptr;
    void* e = nullptr;
    void* part = nullptr;     // R × ldq matvec partials
    int R = 0;
    double* gpart = nullptr;  // block partials of ‖ḡ‖²
    int* cpart = nullptr;     // block partials of |P|
    double* kpart = nullptr;  // block partials of ḡᵀw
    int nb = 0;               // number of vector blocks
    aln::IterState* st = nullptr;
    aln::IterState* st_host = nullptr;
    size_t iter_bytes = 0;
    void* iter_pool = nullptr;

    // KKT workspace
    double* x64 = nullptr;    // ldq
    double* r64 = nullptr;    // d
    double* rpart = nullptr;  // CG × d
    int CG = 0;
    double* g64 = nullptr;    // ldq
    double* kkt_part = nullptr;
    double* kkt_out = nullptr;     // [rel, F]
    double* kkt_out_host = nullptr;
    void* kkt_pool = nullptr;
    size_t kkt_bytes = 0;

    // persistent Alg. 2 kernel geometry and its per-tile partials
    int p_CT = 0, p_R = 0, p_G = 0;
    int p_repl = 0;  // 1: replicated-state kernel (vectors fit in shared memory)
    int p_small = 0; // 1: FP64 loop on one thread-block cluster (small n, small64.cu)
    double lipschitz = -1.0;  // Anti+Acc: L = λ_max(Q) estimate (< 0: not computed)
    int power_products = 0;   // products of the power iteration that gave it
    double* p_gpart = nullptr;
    int* p_cpart = nullptr;
    double* p_kpart = nullptr;
    int* p_clip = nullptr;
    unsigned int* p_ticket = nullptr;
    void* p_sync = nullptr;

    // many right-hand sides sharing A (batch.cu); null when not in batch mode
    void* batch = nullptr;
    int batched = 0;
    // many independent problems (grouped.cu); null unless aln_prepare_grouped
    void* group = nullptr;
    int grouped = 0;
    // learned start point (mlp.cu); null until created
    void* mlp = nullptr;
    void* nmf = nullptr;     // aln_nmf work buffers (nmf.cu)

    // statistics (aln_get_stats)
    cudaEvent_t ev[12] = {};
    // host-input prepare: A copied in column chunks on copy_stream, each
    // chunk's column statistics and Gram tile rows run as it lands
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[64] = {};
    aln_stats stats = {};
    int64_t launches = 0;

    // autotune (autotune.cu): the cache file, the options as the caller gave
    // them (restored for a shape with no cached choice), the shape whose
    // choice is in force, and the choices that have no public option
    std::string tune_path;
    aln_options user_opt;
    std::string tuned_key;
    int tune_pR = 0;     // row groups of the persistent Alg. 2 kernel (0 = derived)
    int tune_chunk = 0;  // batched solver: iterations per captured chunk (0 = 8)
    int tune_tail = 0;   // batched solver: running columns handed to the tail
                         // (0 = 2 per SM)
    int tune_budget = 0; // batched tail: iterations per launch (0 = 64)
};
