// aln_kkt_residual_noalloc: the FP64 KKT residual / objective of one solution
// with every piece of scratch in a fixed array compiled into the library, so
// the call allocates nothing.
//
// Who needs this: code that must not call cudaMalloc — a caller running with a
// fixed device-memory budget, a callback invoked while the caller's own memory
// pool is exhausted or locked, or a scheduler that forbids allocation on its
// hot path (cudaMalloc can synchronize the device and fail under pressure).
// The regular aln_kkt_residual needs a prepared context, whose workspace is
// allocated by aln_prepare.
//
// The scratch array below is part of the library image: every GPU on which the
// library's device code is loaded holds it until the process exits.  All calls
// share it and each call overwrites it (the flag word is cleared by the call's
// first kernel), so two calls whose kernels overlap on the GPU — different
// streams with no ordering between them — race and give wrong results.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace aln {
namespace {

// 2^21 doubles = 16 MiB of scratch.
constexpr int64_t kNoallocDoubles = ALN_NOALLOC_SCRATCH_DOUBLES;
static __device__ __align__(256) double g_noalloc_scratch[ALN_NOALLOC_SCRATCH_DOUBLES];

constexpr int kNaThreads = 256;
constexpr int kNaRows = 4 * kNaThreads;
constexpr int kNaFparts = 512;

// Layout of the scratch (offsets in doubles):
//   [0, 8)                 flag word (non-finite input) and padding
//   s      n               column norms ‖A_i‖ (1 for a zero column)
//   qm     n               min(q_i, 0)², q_i = −(Aᵀb)_i / s_i
//   gb2    n               ḡ_i² of the residual
//   fpart  512             block partials of ‖r‖²
//   r      d               r = A x − b
//   rpart  CG·d            column-group partials of A x
struct NaLayout {
    double* s;
    double* qm;
    double* gb2;
    double* fpart;
    double* r;
    double* rpart;
    int* flag;
    int CG;
};

__device__ __forceinline__ double na_block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

__global__ void k_na_clear(int* flag) { *flag = 0; }

// One block per column: s_i, and min(q_i, 0)² with q_i = −A_iᵀb / s_i.
template <typename TA>
__global__ void __launch_bounds__(kNaThreads) k_na_colstats(const TA* __restrict__ A, int64_t d,
                                                            int64_t lda, const TA* __restrict__ b,
                                                            NaLayout L) {
    __shared__ double sc[32];
    const int64_t i = blockIdx.x;
    const TA* col = A + i * lda;
    double s2 = 0.0, c = 0.0;
    bool bad = false;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        const double a = (double)col[t], bt = (double)b[t];
        s2 = fma(a, a, s2);
        c = fma(a, bt, c);
        bad |= !isfinite(a) || !isfinite(bt);
    }
    s2 = na_block_sum(s2, sc);
    c = na_block_sum(c, sc);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        const double si = s2 > 0.0 ? sqrt(s2) : 1.0;
        const double qi = -c / si;
        L.s[i] = si;
        L.qm[i] = qi < 0.0 ? qi * qi : 0.0;
        if (bad) atomicOr(L.flag, 1);
    }
}

// rpart[cg][t] = Σ_{i in group cg, x_i ≠ 0} A_ti x_i (four rows per thread).
template <typename TA>
__global__ void __launch_bounds__(kNaThreads) k_na_ax(const TA* __restrict__ A, int64_t d,
                                                      int64_t n, int64_t lda,
                                                      const double* __restrict__ x,
                                                      int64_t cols_per_group, NaLayout L) {
    const int64_t t0 = ((int64_t)blockIdx.x * kNaThreads + threadIdx.x) * 4;
    if (t0 >= d) return;
    const int64_t i0 = (int64_t)blockIdx.y * cols_per_group;
    const int64_t i1 = min(n, i0 + cols_per_group);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = i0; i < i1; ++i) {
        const double xi = x[i];
        if (xi == 0.0) continue;
        const TA* p = A + i * lda + t0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (t0 + u < d) acc[u] = fma((double)p[u], xi, acc[u]);
    }
    double* out = L.rpart + (int64_t)blockIdx.y * d + t0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (t0 + u < d) out[u] = acc[u];
}

// r = Σ_cg rpart − b, block partials of ‖r‖².
template <typename TA>
__global__ void __launch_bounds__(kNaThreads) k_na_r(int64_t d, const TA* __restrict__ b,
                                                     NaLayout L) {
    __shared__ double sc[32];
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < d;
         t += (int64_t)gridDim.x * blockDim.x) {
        double v = -(double)b[t];
        for (int cg = 0; cg < L.CG; ++cg) v += L.rpart[(int64_t)cg * d + t];
        L.r[t] = v;
        acc = fma(v, v, acc);
    }
    acc = na_block_sum(acc, sc);
    if (threadIdx.x == 0) L.fpart[blockIdx.x] = acc;
}

// One block per column: g_i = A_iᵀr / s_i, ḡ_i on P(s·x), store ḡ_i².
template <typename TA>
__global__ void __launch_bounds__(kNaThreads) k_na_grad(const TA* __restrict__ A, int64_t d,
                                                        int64_t lda,
                                                        const double* __restrict__ x,
                                                        NaLayout L) {
    __shared__ double sc[32];
    const int64_t i = blockIdx.x;
    const TA* col = A + i * lda;
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) acc = fma((double)col[t], L.r[t], acc);
    acc = na_block_sum(acc, sc);
    if (threadIdx.x == 0) {
        const double si = L.s[i];
        const double gi = acc / si;
        const bool P = x[i] * si > 0.0 || gi < 0.0;
        L.gb2[i] = P ? gi * gi : 0.0;
        if (!isfinite(x[i])) atomicOr(L.flag, 1);
    }
}

__global__ void k_na_final(int64_t n, int nf, NaLayout L, double* __restrict__ out) {
    __shared__ double sc[32];
    double g = 0.0, q = 0.0, f = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        g += L.gb2[i];
        q += L.qm[i];
    }
    for (int i = threadIdx.x; i < nf; i += blockDim.x) f += L.fpart[i];
    g = na_block_sum(g, sc);
    q = na_block_sum(q, sc);
    f = na_block_sum(f, sc);
    if (threadIdx.x == 0) {
        const double num = sqrt(g), den = sqrt(q);
        const bool bad = *(volatile int*)L.flag != 0;
        out[0] = bad ? (double)NAN : (den > 0.0 ? num / den : num);
        out[1] = bad ? (double)NAN : 0.5 * f;
    }
}

// True when p is device (or managed) memory.  A host pointer handed to the
// kernels below would be dereferenced on the GPU, so every argument is checked
// before anything is launched (cudaPointerGetAttributes allocates nothing).
bool na_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array, looked up once per device with that
// device current.
std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 64;
double* g_na_ptr[kNaMaxDevices] = {};

cudaError_t na_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

template <typename TA>
void na_launch(const TA* A, int64_t d, int64_t n, int64_t lda, const TA* b, const double* x,
               double* out, const NaLayout& L, cudaStream_t st) {
    const int64_t cpg = ceil_div(n, L.CG);
    const int nf = (int)std::min<int64_t>(ceil_div(d, kNaThreads), kNaFparts);
    k_na_clear<<<1, 1, 0, st>>>(L.flag);
    k_na_colstats<TA><<<(unsigned)n, kNaThreads, 0, st>>>(A, d, lda, b, L);
    k_na_ax<TA><<<dim3((unsigned)ceil_div(d, kNaRows), (unsigned)L.CG), kNaThreads, 0, st>>>(
        A, d, n, lda, x, cpg, L);
    k_na_r<TA><<<nf, kNaThreads, 0, st>>>(d, b, L);
    k_na_grad<TA><<<(unsigned)n, kNaThreads, 0, st>>>(A, d, lda, x, L);
    k_na_final<<<1, kNaThreads, 0, st>>>(n, nf, L, out);
}

}  // namespace
}  // namespace aln

extern "C" aln_status aln_kkt_residual_noalloc(const void* A, int64_t d, int64_t n, int64_t lda,
                                               int32_t dtype, const void* b, const double* x,
                                               double* out, void* stream) {
    using namespace aln;
    if (!A || !b || !x || !out) return ALN_ERR_INVALID_ARG;
    if (d < 1 || n < 1 || lda < d) return ALN_ERR_INVALID_ARG;
    if (dtype != ALN_DTYPE_F32 && dtype != ALN_DTYPE_F64) return ALN_ERR_INVALID_ARG;
    if (!na_device_ptr(A) || !na_device_ptr(b) || !na_device_ptr(x) || !na_device_ptr(out))
        return ALN_ERR_INVALID_ARG;  // host memory: the kernels cannot read it
    // fixed part: flag block (8) + s, qm, gb2 (3n) + fpart (512) + r (d) + rpart (CG·d)
    const int64_t fixed = 8 + 3 * n + kNaFparts + d;
    if (n > kNoallocDoubles || d > kNoallocDoubles || fixed + d > kNoallocDoubles)
        return ALN_ERR_INVALID_ARG;  // beyond the fixed scratch: use aln_kkt_residual
    double* base = nullptr;
    if (na_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return ALN_ERR_CUDA;
    }
    NaLayout L;
    L.flag = (int*)base;
    L.s = base + 8;
    L.qm = L.s + n;
    L.gb2 = L.qm + n;
    L.fpart = L.gb2 + n;
    L.r = L.fpart + kNaFparts;
    L.rpart = L.r + d;
    L.CG = (int)std::max<int64_t>(1, std::min<int64_t>(8, (kNoallocDoubles - fixed) / d));
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == ALN_DTYPE_F32)
        na_launch<float>((const float*)A, d, n, lda, (const float*)b, x, out, L, st);
    else
        na_launch<double>((const double*)A, d, n, lda, (const double*)b, x, out, L, st);
    return cudaGetLastError() == cudaSuccess ? ALN_OK : ALN_ERR_CUDA;
}
