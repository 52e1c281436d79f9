// Alg. 2 (§3) on one right-hand side as ONE persistent cooperative kernel.
//
// The vector state (y, g, ḡ, w, e) is owned by column tiles of TILE = 32·VN
// elements (128 FP32 / 64 FP64); the symmetric product Qv = Σ_j v_j Q[j, :] is
// split into work items (column tile ct, row group rg).  One iteration:
//
//   (a) γ = ‖ḡ‖², |P| from the per-tile partials (every block sums the same
//       array in the same order, so every block takes the same decision);
//       stop if P = ∅, γ < ε, the iteration cap, or the stagnation window.
//   (b) w = Qḡ: every item sums the passive rows of its group into a partial;
//       the last item of a column tile to finish (atomic ticket) adds the R
//       partials in fixed order, writes w for the tile and κ_ct = ḡᵀw there.
//   --- grid barrier ---
//   (c) κ = Σ κ_ct, α = γ/κ; each tile: y⁺ = [y − αḡ]₊, e = clipped part,
//       g ← g − αw, and the mask of the next iterate assuming no clipping
//       (ḡ, γ_ct, |P|_ct); clip_ct = number of clipped entries.
//   --- grid barrier ---
//   (d) only if Σ clip_ct > 0: u = Qe over the clipped rows (same item
//       scheme); the last item of a tile adds u to g and recomputes the mask.
//       --- grid barrier ---
//
// So an iteration costs two grid barriers, three when some variable hits the
// bound.  All sums are in a fixed order: results are bitwise reproducible.
// The grid barrier spins with a time limit; on expiry the kernel records
// ALN_RHS timeout in the state and every block leaves the loop.
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

constexpr int kPThreads = 1024;
constexpr int kPWarps = kPThreads / 32;
constexpr int kPU = 4;                        // rows in flight per warp
constexpr uint64_t kBarrierNs = 2000000000ull; // 2 s per barrier wait
constexpr int kStatusTimeout = -1;             // state status after a barrier timeout

__device__ __forceinline__ uint64_t p_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sums over the per-tile partial arrays through L2 (written by other blocks).
__device__ __forceinline__ double warp_sum_cg(const double* p, int count) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < count; i += 32) v += __ldcg(p + i);
    return warp_sum(v);
}
__device__ __forceinline__ int warp_sum_cg_i(const int* p, int count) {
    const int lane = threadIdx.x & 31;
    int v = 0;
    for (int i = lane; i < count; i += 32) v += __ldcg(p + i);
    return warp_sum_i(v);
}

struct PersistSync {
    unsigned int arrive;
    unsigned int gen;
    unsigned int timeout;
    unsigned int pad;
};

// Sense-free generation barrier over the co-resident grid (cooperative launch).
__device__ __forceinline__ bool grid_barrier(PersistSync* s, unsigned int nblocks) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = &s->gen;
        const unsigned int gen = *vgen;
        __threadfence();
        const unsigned int prev = atomicAdd(&s->arrive, 1u);
        if (prev == nblocks - 1) {
            atomicExch(&s->arrive, 0u);
            __threadfence();
            atomicAdd(&s->gen, 1u);
        } else {
            const uint64_t t0 = p_globaltimer();
            unsigned int spins = 0;
            while (*vgen == gen) {
                if ((++spins & 255u) == 0 && p_globaltimer() - t0 > kBarrierNs) {
                    ok = 0;
                    atomicExch(&s->timeout, 1u);
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile unsigned int*)&s->timeout) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
struct PersistArgs {
    const T* Q;
    int64_t ldq;
    int n;
    int CT;          // column tiles
    int R;           // row groups
    int rows_per_group;
    T* y;
    T* g;
    T* gb;
    T* w;
    T* e;
    T* part;         // R × ldq
    double* gpart;   // CT
    int* cpart;      // CT
    double* kpart;   // CT
    int* clip;       // CT
    unsigned int* ticket;  // CT
    PersistSync* sync;
    IterState* st;
};

// Partial of Σ_{j ∈ group rg, v_j ≠ 0} v_j Q[j, tile ct] into part[rg][tile].
template <typename T>
__device__ __forceinline__ void mv_item(const PersistArgs<T>& a, const T* __restrict__ v, int ct,
                                        int rg, T* red) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int TILE = 32 * VN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = (int64_t)ct * TILE + lane * VN;
    const int j0 = rg * a.rows_per_group;
    const int j1 = min(a.n, j0 + a.rows_per_group);
    T acc[VN];
#pragma unroll
    for (int c = 0; c < VN; ++c) acc[c] = T(0);
    for (int jb = j0 + warp; jb < j1; jb += kPWarps * kPU) {
        T vv[kPU];
        V qq[kPU];
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const int j = jb + kPWarps * u;
            vv[u] = j < j1 ? __ldcg(v + j) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const int j = jb + kPWarps * u;
            if (vv[u] != T(0))
                qq[u] = __ldg(reinterpret_cast<const V*>(a.Q + (int64_t)j * a.ldq + col));
            else
                qq[u] = V{};
        }
#pragma unroll
        for (int u = 0; u < kPU; ++u)
#pragma unroll
            for (int c = 0; c < VN; ++c) acc[c] = fma(vv[u], vget(qq[u], c), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < VN; ++c) red[warp * TILE + lane * VN + c] = acc[c];
    __syncthreads();
    if (threadIdx.x < TILE) {
        T s = T(0);
#pragma unroll 8
        for (int w2 = 0; w2 < kPWarps; ++w2) s += red[w2 * TILE + threadIdx.x];
        __stcg(a.part + (int64_t)rg * a.ldq + (int64_t)ct * TILE + threadIdx.x, s);
    }
}

// After an item: take a ticket for its tile; returns true in the block that
// completes the tile (it then sees every partial of the tile).
__device__ __forceinline__ bool last_of_tile(unsigned int* ticket, int ct, int R) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(ticket + ct, 1u);
        s_last = (t == (unsigned int)(R - 1));
        if (s_last) ticket[ct] = 0u;  // reset for the next product
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Mask of one tile: ḡ = g on P(y), partial γ and |P| (threads < TILE).
template <typename T>
__device__ __forceinline__ void tile_mask(const PersistArgs<T>& a, int ct, double* sd, int* si) {
    constexpr int TILE = 32 * Vec16<T>::N;
    double v = 0.0;
    int c = 0;
    if (threadIdx.x < TILE) {
        const int64_t i = (int64_t)ct * TILE + threadIdx.x;
        if (i < a.n) {
            const T yi = __ldcg(a.y + i), gi = __ldcg(a.g + i);
            const bool P = yi > T(0) || gi < T(0);
            const T gbi = P ? gi : T(0);
            __stcg(a.gb + i, gbi);
            v = (double)gbi * (double)gbi;
            c = P ? 1 : 0;
        }
    }
    // TILE ≤ 128 threads = warps 0..3
    v = warp_sum(v);
    c = warp_sum_i(c);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0 && wid < TILE / 32) {
        sd[wid] = v;
        si[wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        int k = 0;
        for (int w2 = 0; w2 < TILE / 32; ++w2) {
            s += sd[w2];
            k += si[w2];
        }
        __stcg(a.gpart + ct, s);
        __stcg(a.cpart + ct, k);
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_alg2_persist(PersistArgs<T> a) {
    constexpr int TILE = 32 * Vec16<T>::N;
    __shared__ T red[kPWarps * TILE];
    __shared__ double sd[32];
    __shared__ int si[32];
    __shared__ double s_scal[4];
    __shared__ int s_flag[4];
    const unsigned int G = gridDim.x;
    const int items = a.CT * a.R;

    // prologue: mask of the start point
    for (int ct = blockIdx.x; ct < a.CT; ct += G) tile_mask(a, ct, sd, si);
    if (!grid_barrier(a.sync, G)) return;

    IterState* st = a.st;
    const double eps = st->eps;
    const int max_iter = st->max_iter, window = st->window;
    double best = 1.0 / 0.0;
    int best_iter = 0;
    int iter = 0;
    long long sum_passive = 0, sum_clip = 0;
    int status = ALN_RHS_MAXITER;
    double gam = 0.0;
    int cnt = 0;
    bool timed_out = false;

    for (;;) {
        // (a) stop test, identical in every block
        if (threadIdx.x < 32) {
            const double g2 = warp_sum_cg(a.gpart, a.CT);
            const int c2 = warp_sum_cg_i(a.cpart, a.CT);
            if (threadIdx.x == 0) {
                s_scal[0] = g2;
                s_flag[0] = c2;
            }
        }
        __syncthreads();
        gam = s_scal[0];
        cnt = s_flag[0];
        int stop = 1;
        if (!isfinite(gam)) status = ALN_RHS_NONFINITE;
        else if (cnt == 0) status = ALN_RHS_EMPTY_PASSIVE;
        else if (gam < eps || gam == 0.0) status = ALN_RHS_CONVERGED;
        else if (iter >= max_iter) status = ALN_RHS_MAXITER;
        else if (iter - best_iter > window) status = ALN_RHS_STAGNATED;
        else stop = 0;
        if (stop) break;
        if (gam < best) {
            best = gam;
            best_iter = iter;
        }

        // (b) w = Qḡ with per-tile completion
        for (int it = blockIdx.x; it < items; it += G) {
            const int ct = it % a.CT, rg = it / a.CT;
            mv_item(a, a.gb, ct, rg, red);
            if (last_of_tile(a.ticket, ct, a.R)) {
                double kap = 0.0;
                if (threadIdx.x < TILE) {
                    const int64_t i = (int64_t)ct * TILE + threadIdx.x;
                    T wi = T(0);
                    for (int r = 0; r < a.R; ++r) wi += __ldcg(a.part + (int64_t)r * a.ldq + i);
                    __stcg(a.w + i, wi);
                    if (i < a.n) kap = (double)__ldcg(a.gb + i) * (double)wi;
                }
                kap = warp_sum(kap);
                if ((threadIdx.x & 31) == 0 && (threadIdx.x >> 5) < TILE / 32)
                    sd[threadIdx.x >> 5] = kap;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double s = 0.0;
                    for (int w2 = 0; w2 < TILE / 32; ++w2) s += sd[w2];
                    __stcg(a.kpart + ct, s);
                }
                __syncthreads();
            }
        }
        if (!grid_barrier(a.sync, G)) {
            timed_out = true;
            break;
        }

        // (c) step size, projected update, gradient update, provisional mask
        if (threadIdx.x < 32) {
            const double k2 = warp_sum_cg(a.kpart, a.CT);
            if (threadIdx.x == 0) s_scal[1] = k2;
        }
        __syncthreads();
        const double kap = s_scal[1];
        if (!isfinite(kap)) {
            status = ALN_RHS_NONFINITE;
            break;
        }
        if (kap <= 0.0) {
            status = ALN_RHS_CURVATURE;
            break;
        }
        const double alpha = gam / kap;
        sum_passive += cnt;
        const T aT = (T)alpha;
        for (int ct = blockIdx.x; ct < a.CT; ct += G) {
            int clipped = 0;
            if (threadIdx.x < TILE) {
                const int64_t i = (int64_t)ct * TILE + threadIdx.x;
                if (i < a.n) {
                    const T yi = __ldcg(a.y + i);
                    const T step = aT * __ldcg(a.gb + i);
                    T yn = yi - step;
                    T ei = T(0);
                    if (yn < T(0)) {
                        ei = step - yi;
                        yn = T(0);
                        clipped = 1;
                    }
                    __stcg(a.y + i, yn);
                    __stcg(a.e + i, ei);
                    __stcg(a.g + i, __ldcg(a.g + i) - aT * __ldcg(a.w + i));
                }
            }
            clipped = __syncthreads_count(clipped);
            if (threadIdx.x == 0) __stcg(a.clip + ct, clipped);
            tile_mask(a, ct, sd, si);
        }
        ++iter;
        if (!grid_barrier(a.sync, G)) {
            timed_out = true;
            break;
        }

        // (d) clipped correction g += Q e (only when something was clipped)
        if (threadIdx.x < 32) {
            int c3 = 0;
            for (int i = threadIdx.x; i < a.CT; i += 32) c3 += __ldcg(a.clip + i);
            c3 = warp_sum_i(c3);
            if (threadIdx.x == 0) s_flag[1] = c3;
        }
        __syncthreads();
        sum_clip += s_flag[1];
        if (s_flag[1] > 0) {
            for (int it = blockIdx.x; it < items; it += G) {
                const int ct = it % a.CT, rg = it / a.CT;
                mv_item(a, a.e, ct, rg, red);
                if (last_of_tile(a.ticket, ct, a.R)) {
                    if (threadIdx.x < TILE) {
                        const int64_t i = (int64_t)ct * TILE + threadIdx.x;
                        T ui = T(0);
                        for (int r = 0; r < a.R; ++r)
                            ui += __ldcg(a.part + (int64_t)r * a.ldq + i);
                        if (i < a.n) __stcg(a.g + i, __ldcg(a.g + i) + ui);
                    }
                    __syncthreads();
                    tile_mask(a, ct, sd, si);
                }
            }
            if (!grid_barrier(a.sync, G)) {
                timed_out = true;
                break;
            }
        }
    }

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = iter;
        st->done = 1;
        st->status = timed_out ? kStatusTimeout : status;
        st->gbar2 = gam;
        st->npassive = cnt;
        st->best_g2 = best;
        st->best_iter = best_iter;
        st->sum_passive = sum_passive;
        st->sum_clip = sum_clip;
    }
}

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_alg2_persist(aln_ctx* c) {
    PersistArgs<T> a;
    a.Q = (const T*)c->Q;
    a.ldq = c->ldq;
    a.n = (int)c->n;
    a.CT = c->p_CT;
    a.R = c->p_R;
    a.rows_per_group = (int)ceil_div(c->n, c->p_R);
    a.y = (T*)c->y;
    a.g = (T*)c->g;
    a.gb = (T*)c->gb;
    a.w = (T*)c->w;
    a.e = (T*)c->e;
    a.part = (T*)c->part;
    a.gpart = c->p_gpart;
    a.cpart = c->p_cpart;
    a.kpart = c->p_kpart;
    a.clip = c->p_clip;
    a.ticket = c->p_ticket;
    a.sync = (PersistSync*)c->p_sync;
    a.st = c->st;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_alg2_persist<T>, dim3(c->p_G),
                                       dim3(kPThreads), args, 0, c->stream);
}

template <typename T>
int persist_max_blocks(int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_alg2_persist<T>, kPThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * num_sms;
}

template cudaError_t launch_alg2_persist<float>(aln_ctx*);
template cudaError_t launch_alg2_persist<double>(aln_ctx*);
template int persist_max_blocks<float>(int);
template int persist_max_blocks<double>(int);

size_t persist_sync_bytes() { return sizeof(PersistSync); }

}  // namespace aln
