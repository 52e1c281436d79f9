// Set-up kernels of Alg. 2 (§3) on one right-hand side: the start point,
// the initial gradient (g = q at y = 0, or g = Qy0 + q with a start point), the
// gradient refresh from the FP64 KKT pass, and the final x = y/s (Alg. 1).
// The iteration itself runs in the persistent kernel (persist.cu).
//
// Q is symmetric, so Qv = Σ_j v_j Q[j, :]: k_rowmv walks the rows j with
// v_j ≠ 0, each a contiguous, coalesced run of ldq elements, and writes one
// partial per row group that k_finish sums in a fixed order.
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

constexpr int kVecThreads = 256;
constexpr int kMvWarps = 8;

// qv = q, y = x0·s (the start point mapped by Eq. Rescaling; 0 without one), e = 0.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_vec_init(int n, int64_t ldq,
                                                          const double* __restrict__ q64,
                                                          const double* __restrict__ x0,
                                                          const double* __restrict__ s,
                                                          T* __restrict__ qv, T* __restrict__ y,
                                                          T* __restrict__ e) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ldq;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool in = i < n;
        qv[i] = in ? (T)q64[i] : T(0);
        y[i] = (in && x0) ? (T)(x0[i] * s[i]) : T(0);
        e[i] = T(0);
    }
}

__global__ void k_state_reset(IterState* st, double eps, int max_iter, int window) {
    st->eps = eps;
    st->window = window;
    st->best_g2 = 1.0 / 0.0;
    st->best_iter = 0;
    st->gbar2 = 0.0;
    st->alpha = 0.0;
    st->iter = 0;
    st->max_iter = max_iter;
    st->done = 0;
    st->status = ALN_RHS_MAXITER;
    st->npassive = 0;
}

// part[r][cols] = Σ_{j ∈ group r, v_j ≠ 0} v_j Q[j][cols].  Block = 8 warps on
// one tile of 32·VN columns; warps interleave over the group's rows and U rows
// per warp are in flight at once.  With check_conv, the block first applies
// Alg. 2's stop rule to the partial sums of the previous k_finish.
template <typename T, int U>
__global__ void __launch_bounds__(kMvWarps * 32) k_rowmv(
    const T* __restrict__ Q, int64_t ldq, int n, const T* __restrict__ v, int rows_per_group,
    T* __restrict__ part, IterState* __restrict__ st, int check_conv,
    const double* __restrict__ gpart, const int* __restrict__ cpart, int nb) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int TILE = 32 * VN;
    __shared__ int s_stop;
    __shared__ T red[kMvWarps][TILE];
    if (st->done) return;
    if (check_conv) {
        if (threadIdx.x < 32) {
            const double gam = warp_sum_array(gpart, nb);
            const int cnt = warp_sum_array_i(cpart, nb);
            if (threadIdx.x == 0) {
                int stop = 1, status = ALN_RHS_CONVERGED;
                if (!isfinite(gam)) status = ALN_RHS_NONFINITE;
                else if (cnt == 0) status = ALN_RHS_EMPTY_PASSIVE;
                else if (gam < st->eps || gam == 0.0) status = ALN_RHS_CONVERGED;
                else if (st->iter >= st->max_iter) status = ALN_RHS_MAXITER;
                else if (st->iter - st->best_iter > st->window) status = ALN_RHS_STAGNATED;
                else stop = 0;
                s_stop = stop;
                if (stop && blockIdx.x == 0 && blockIdx.y == 0) {
                    st->done = 1;
                    st->status = status;
                    st->gbar2 = gam;
                    st->npassive = cnt;
                }
            }
        }
        __syncthreads();
        if (s_stop) return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = (int64_t)blockIdx.x * TILE + lane * VN;
    const int j0 = blockIdx.y * rows_per_group;
    const int j1 = min(n, j0 + rows_per_group);
    T acc[VN];
#pragma unroll
    for (int c = 0; c < VN; ++c) acc[c] = T(0);
    for (int jb = j0 + warp; jb < j1; jb += kMvWarps * U) {
        T vv[U];
        V qq[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jb + kMvWarps * u;
            vv[u] = j < j1 ? v[j] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jb + kMvWarps * u;
            if (vv[u] != T(0))
                qq[u] = *reinterpret_cast<const V*>(Q + (int64_t)j * ldq + col);
            else
                qq[u] = V{};
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < VN; ++c) acc[c] = fma(vv[u], vget(qq[u], c), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < VN; ++c) red[warp][lane * VN + c] = acc[c];
    __syncthreads();
    if (threadIdx.x < TILE) {
        T s = T(0);
#pragma unroll
        for (int w2 = 0; w2 < kMvWarps; ++w2) s += red[w2][threadIdx.x];
        part[(int64_t)blockIdx.y * ldq + (int64_t)blockIdx.x * TILE + threadIdx.x] = s;
    }
}

// g_i = base_i + Σ_r part[r][i], where base is q (init), the FP64 gradient from
// the KKT pass (refinement), or g itself; then ḡ = g on P(y), and the block
// partials of ‖ḡ‖² and |P| for the next stop test.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_finish(
    int n, int64_t ldq, const T* __restrict__ part, int R, const T* __restrict__ qv,
    const double* __restrict__ g64, int base_mode, const T* __restrict__ y, T* __restrict__ g,
    T* __restrict__ gb, double* __restrict__ gpart, int* __restrict__ cpart,
    const IterState* __restrict__ st, int check_done) {
    __shared__ double scratch[32];
    __shared__ int iscratch[32];
    if (check_done && st->done) return;
    double acc = 0.0;
    int cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T gi = base_mode == 0 ? g[i] : base_mode == 1 ? qv[i] : (T)g64[i];
        for (int r = 0; r < R; ++r) gi += part[(int64_t)r * ldq + i];
        g[i] = gi;
        const bool P = y[i] > T(0) || gi < T(0);
        const T gbi = P ? gi : T(0);
        gb[i] = gbi;
        acc += (double)gbi * (double)gbi;
        cnt += P ? 1 : 0;
    }
    acc = block_sum(acc, scratch);
    // integer block sum
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int v = warp_sum_i(cnt);
        if (lane == 0) iscratch[wid] = v;
        __syncthreads();
        if (wid == 0) {
            v = lane < (int)(blockDim.x >> 5) ? iscratch[lane] : 0;
            v = warp_sum_i(v);
            if (lane == 0) cpart[blockIdx.x] = v;
        }
    }
    if (threadIdx.x == 0) gpart[blockIdx.x] = acc;
}

// x = (y + ylo)/s (Eq. Rescaling); ylo: the low part of a float-pair
// iterate, or null.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_unscale(int n, const T* __restrict__ y,
                                                         const T* __restrict__ ylo,
                                                         const double* __restrict__ s,
                                                         double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = ((double)y[i] + (ylo ? (double)ylo[i] : 0.0)) / s[i];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <typename T>
static void rowmv_launch(aln_ctx* c, const T* v, int check_conv) {
    constexpr int TILE = 32 * Vec16<T>::N;
    const int rows_per_group = (int)ceil_div(c->n, c->R);
    const dim3 grid((unsigned)(c->ldq / TILE), (unsigned)c->R);
    k_rowmv<T, 4><<<grid, kMvWarps * 32, 0, c->stream>>>(
        (const T*)c->Q, c->ldq, (int)c->n, v, rows_per_group, (T*)c->part, c->st, check_conv,
        c->gpart, c->cpart, c->nb);
}

cudaError_t launch_state_reset(aln_ctx* c, double eps, int max_iter) {
    k_state_reset<<<1, 1, 0, c->stream>>>(c->st, eps, max_iter, c->opt.stagnation);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_iter_setup(aln_ctx* c, const double* q64, const double* x0, double eps,
                              int max_iter) {
    const int n = (int)c->n;
    k_state_reset<<<1, 1, 0, c->stream>>>(c->st, eps, max_iter, c->opt.stagnation);
    k_vec_init<T><<<(unsigned)std::min<int64_t>(ceil_div(c->ldq, kVecThreads), 1024), kVecThreads,
                    0, c->stream>>>(n, c->ldq, q64, x0, c->s, (T*)c->qv, (T*)c->y, (T*)c->e);
    if (x0) {
        // g = Q y0 + q (Alg. 2 with a start point other than 0)
        rowmv_launch<T>(c, (const T*)c->y, 0);
        k_finish<T><<<c->nb, kVecThreads, 0, c->stream>>>(
            n, c->ldq, (const T*)c->part, c->R, (const T*)c->qv, nullptr, 1, (const T*)c->y,
            (T*)c->g, (T*)c->gb, c->gpart, c->cpart, c->st, 0);
    } else {
        // Alg. 2: x⁰ = 0, ∇f = q
        k_finish<T><<<c->nb, kVecThreads, 0, c->stream>>>(
            n, c->ldq, (const T*)c->part, 0, (const T*)c->qv, nullptr, 1, (const T*)c->y,
            (T*)c->g, (T*)c->gb, c->gpart, c->cpart, c->st, 0);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_iter_refresh_from_g64(aln_ctx* c, double eps, int max_iter) {
    k_state_reset<<<1, 1, 0, c->stream>>>(c->st, eps, max_iter, c->opt.stagnation);
    k_finish<T><<<c->nb, kVecThreads, 0, c->stream>>>(
        (int)c->n, c->ldq, (const T*)c->part, 0, (const T*)c->qv, c->g64, 2, (const T*)c->y,
        (T*)c->g, (T*)c->gb, c->gpart, c->cpart, c->st, 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unscale(aln_ctx* c, double* x64) {
    // the replicated FP32 kernel keeps the low part of y in e (zero from the
    // set-up, and never written by Anti+Acc); the tiled kernel uses e for
    // its clipped corrections
    const T* ylo = (c->p_repl && sizeof(T) == 4) ? (const T*)c->e : nullptr;
    k_unscale<T><<<(unsigned)std::min<int64_t>(ceil_div(c->n, kVecThreads), 1024), kVecThreads, 0,
                   c->stream>>>((int)c->n, (const T*)c->y, ylo, c->s, x64);
    return cudaGetLastError();
}

template cudaError_t launch_iter_setup<float>(aln_ctx*, const double*, const double*, double, int);
template cudaError_t launch_iter_setup<double>(aln_ctx*, const double*, const double*, double,
                                               int);
template cudaError_t launch_iter_refresh_from_g64<float>(aln_ctx*, double, int);
template cudaError_t launch_iter_refresh_from_g64<double>(aln_ctx*, double, int);
template cudaError_t launch_unscale<float>(aln_ctx*, double*);
template cudaError_t launch_unscale<double>(aln_ctx*, double*);

}  // namespace aln
