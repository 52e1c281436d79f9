// Non-negative matrix factorisation V ≈ W·H by alternating NNLS (ANLS), the
// application the paper motivates its solver with (§1; §2.2 on reusing work
// across the many right-hand sides of such factorisations).  Each outer
// iteration is two calls of the library's own multi-RHS solve:
//
//   H-step: Alg. 1 + Alg. 2 with matrix W (m×r) and the n columns of V as
//           right-hand sides, started from the previous H;
//   W-step: the same with matrix Hᵀ (n×r) and the m rows of V (columns of
//           Vᵀ) as right-hand sides, started from the previous W.
//
// With n, m ≥ batch_min both steps take the batched tcgen05 solver.  The
// kernels here only move data: Vᵀ once, and after each step the solution
// (right-hand sides × r, row-major FP64) transposed into the next step's
// column-major FP32 matrix.
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace aln {
namespace {

constexpr int kTile = 32;

// dst[j + i·ldd] = src[i + j·lds] for i < rows, j < cols (FP32 transpose).
__global__ void k_transpose_f32(const float* __restrict__ src, int64_t rows, int64_t cols,
                                int64_t lds, float* __restrict__ dst, int64_t ldd) {
    __shared__ float t[kTile][kTile + 1];
    const int64_t i0 = (int64_t)blockIdx.x * kTile, j0 = (int64_t)blockIdx.y * kTile;
    for (int jj = threadIdx.y; jj < kTile; jj += blockDim.y) {
        const int64_t i = i0 + threadIdx.x, j = j0 + jj;
        t[jj][threadIdx.x] = (i < rows && j < cols) ? src[i + j * lds] : 0.0f;
    }
    __syncthreads();
    for (int ii = threadIdx.y; ii < kTile; ii += blockDim.y) {
        const int64_t j = j0 + threadIdx.x, i = i0 + ii;
        if (i < rows && j < cols) dst[j + i * ldd] = t[threadIdx.x][ii];
    }
}

// Row-major k×r FP64 (solution rows) → column-major k×r FP32 (next matrix):
// dst[c + i·k] = src[c·r + i].
__global__ void k_rows_to_cols_f32(const double* __restrict__ src, int64_t k, int64_t r,
                                   float* __restrict__ dst) {
    const int64_t total = k * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, c = e - i * k;  // consecutive threads: consecutive c
        dst[c + i * k] = (float)src[c * r + i];
    }
}

// Column-major rows×cols FP64 (ld) → row-major (ld cols) FP64, projected
// onto x ⪰ 0: dst[i·cols + j] = max(src[i + j·ld], 0).
__global__ void k_cols_to_rows_f64(const double* __restrict__ src, int64_t rows, int64_t cols,
                                   int64_t ld, double* __restrict__ dst) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e - i * cols;
        const double v = src[i + j * ld];
        dst[e] = v > 0.0 ? v : 0.0;
    }
}

// Row-major rows×cols FP64 → column-major (ld) FP64: dst[i + j·ld] = src[i·cols + j].
__global__ void k_rows_to_cols_f64(const double* __restrict__ src, int64_t rows, int64_t cols,
                                   double* __restrict__ dst, int64_t ld) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / rows, i = e - j * rows;  // consecutive threads: consecutive i
        dst[i + j * ld] = src[i * cols + j];
    }
}

// x := max(x, 0) over n entries.
__global__ void k_clip_nonneg(double* __restrict__ x, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        x[e] = x[e] > 0.0 ? x[e] : 0.0;
}

unsigned grid_of(int64_t work, int cap) {
    const int64_t b = (work + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct NmfWork {
    void* pool = nullptr;
    size_t bytes = 0;
    std::vector<aln_solve_info> info;
};

void nmf_free(aln_ctx* c) {
    NmfWork* w = (NmfWork*)c->nmf;
    if (!w) return;
    if (w->pool) cudaFree(w->pool);
    delete w;
    c->nmf = nullptr;
}

}  // namespace aln

using namespace aln;

#define NMF_TRY(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            cudaGetLastError();                             \
            return e_ == cudaErrorMemoryAllocation ? ALN_ERR_OUT_OF_MEMORY : ALN_ERR_CUDA; \
        }                                                   \
    } while (0)
#define NMF_CHECK(call)               \
    do {                              \
        aln_status s_ = (call);       \
        if (s_ != ALN_OK) return s_;  \
    } while (0)

extern "C" aln_status aln_nmf(aln_ctx* c, const float* V, int64_t m, int64_t n, int64_t ldv,
                              int64_t r, double* W, int64_t ldw, double* H, int64_t ldh,
                              int32_t outer, double tol, int32_t max_iter, double* objective) {
    if (!c || !V || !W || !H || m < 1 || n < 1 || r < 1 || ldv < m || ldw < m || ldh < r ||
        outer < 1 || !(tol > 0.0) || !std::isfinite(tol) || r > m || r > n ||
        m > ((int64_t)1 << 30) || n > ((int64_t)1 << 30) || r > 4096)
        return ALN_ERR_INVALID_ARG;
    NmfWork* w = (NmfWork*)c->nmf;
    if (!w) {
        w = new (std::nothrow) NmfWork();
        if (!w) return ALN_ERR_OUT_OF_MEMORY;
        c->nmf = w;
    }
    // device work: V (m×n), Vᵀ (n×m), A_H (m×r), A_W (n×r) in FP32; W rows
    // (m×r) ×2, H columns (n×r) ×2 in FP64; a staging block for W / H
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t fV = up((size_t)m * n * 4), fAH = up((size_t)m * r * 4),
                 fAW = up((size_t)n * r * 4), dW = up((size_t)m * r * 8),
                 dH = up((size_t)n * r * 8), stage = up((size_t)std::max(m * r, n * r) * 8);
    const size_t need = 2 * fV + fAH + fAW + 2 * dW + 2 * dH + stage;
    if (w->bytes < need) {
        if (w->pool) cudaFree(w->pool);
        w->pool = nullptr;
        w->bytes = 0;
        if (cudaMalloc(&w->pool, need) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
        w->bytes = need;
    }
    uint8_t* p = (uint8_t*)w->pool;
    auto take = [&](size_t b) {
        uint8_t* q = p;
        p += b;
        return q;
    };
    float* Vd = (float*)take(fV);
    float* Vt = (float*)take(fV);
    float* AH = (float*)take(fAH);
    float* AW = (float*)take(fAW);
    double* Wr[2] = {(double*)take(dW), (double*)take(dW)};
    double* Hc[2] = {(double*)take(dH), (double*)take(dH)};
    double* st = (double*)take(stage);
    cudaStream_t s = c->stream;
    if ((int64_t)w->info.size() < std::max(m, n)) w->info.resize((size_t)std::max(m, n));

    // V (column-major, ld m) and its transpose Vᵀ (n×m, ld n)
    NMF_TRY(cudaMemcpy2DAsync(Vd, (size_t)m * 4, V, (size_t)ldv * 4, (size_t)m * 4, (size_t)n,
                              on_device(V) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              s));
    {
        dim3 grid((unsigned)((m + kTile - 1) / kTile), (unsigned)((n + kTile - 1) / kTile));
        k_transpose_f32<<<grid, dim3(kTile, 8), 0, s>>>(Vd, m, n, m, Vt, n);
        NMF_TRY(cudaGetLastError());
        c->launches += 1;
    }
    // start: W (m×r, ld ldw) → rows (m×r row-major, ⪰ 0) and A_H;
    //        H (r×n, ld ldh) → columns (n×r row-major = H column-major, ⪰ 0)
    const unsigned gw = grid_of(m * r, 8 * c->num_sms), gh = grid_of(n * r, 8 * c->num_sms);
    NMF_TRY(cudaMemcpy2DAsync(st, (size_t)m * 8, W, (size_t)ldw * 8, (size_t)m * 8, (size_t)r,
                              on_device(W) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              s));
    k_cols_to_rows_f64<<<gw, 256, 0, s>>>(st, m, r, m, Wr[0]);
    k_rows_to_cols_f32<<<gw, 256, 0, s>>>(Wr[0], m, r, AH);
    NMF_TRY(cudaMemcpy2DAsync(Hc[0], (size_t)r * 8, H, (size_t)ldh * 8, (size_t)r * 8, (size_t)n,
                              on_device(H) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              s));
    k_clip_nonneg<<<gh, 256, 0, s>>>(Hc[0], n * r);
    NMF_TRY(cudaGetLastError());
    c->launches += 3;

    int cw = 0, ch = 0;  // which buffer holds the current W rows / H columns
    for (int32_t t = 0; t < outer; ++t) {
        // H-step: matrix W (m×r), right-hand sides the n columns of V
        NMF_CHECK(aln_prepare(c, AH, m, r, m, ALN_DTYPE_F32, Vd, n, m));
        NMF_CHECK(aln_solve(c, tol, max_iter, Hc[1 - ch], r, Hc[ch], w->info.data()));
        ch = 1 - ch;
        k_rows_to_cols_f32<<<gh, 256, 0, s>>>(Hc[ch], n, r, AW);  // A_W = Hᵀ (n×r)
        NMF_TRY(cudaGetLastError());
        c->launches += 1;
        // W-step: matrix Hᵀ (n×r), right-hand sides the m rows of V
        NMF_CHECK(aln_prepare(c, AW, n, r, n, ALN_DTYPE_F32, Vt, m, n));
        NMF_CHECK(aln_solve(c, tol, max_iter, Wr[1 - cw], r, Wr[cw], w->info.data()));
        cw = 1 - cw;
        if (objective) {
            double f = 0.0;
            for (int64_t i = 0; i < m; ++i) f += w->info[(size_t)i].objective;
            objective[t] = f;
        }
        k_rows_to_cols_f32<<<gw, 256, 0, s>>>(Wr[cw], m, r, AH);  // A_H = W (m×r)
        NMF_TRY(cudaGetLastError());
        c->launches += 1;
    }
    // results: W column-major (ld ldw), H column-major (ld ldh)
    k_rows_to_cols_f64<<<gw, 256, 0, s>>>(Wr[cw], m, r, st, m);
    NMF_TRY(cudaGetLastError());
    c->launches += 1;
    NMF_TRY(cudaMemcpy2DAsync(W, (size_t)ldw * 8, st, (size_t)m * 8, (size_t)m * 8, (size_t)r,
                              on_device(W) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              s));
    NMF_TRY(cudaMemcpy2DAsync(H, (size_t)ldh * 8, Hc[ch], (size_t)r * 8, (size_t)r * 8,
                              (size_t)n,
                              on_device(H) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              s));
    NMF_TRY(cudaStreamSynchronize(s));
    return ALN_OK;
}
