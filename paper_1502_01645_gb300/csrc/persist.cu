// Alg. 2 (§3) on one right-hand side as ONE persistent cooperative kernel.
//
// The vector state (y, g, ḡ, w, e) is owned by column tiles of TILE = 32·VN
// elements (128 FP32 / 64 FP64).  Q is symmetric, so Qv = Σ_j v_j Q[j, :]; the
// product is split into work items (column tile ct, row group rg), each the
// sum over the rows j of its group with v_j ≠ 0 (each row a contiguous
// 16-byte-aligned run).  One iteration:
//
//   (a) γ = ‖ḡ‖², |P| from per-tile partials (every block sums the same array
//       in the same order and takes the same decision); stop if P = ∅,
//       γ < ε, the iteration cap, or the stagnation window (§5's rule).
//   (b) w-partials: item (ct, rg) writes part[rg][tile] and its share of the
//       curvature, κ_item = Σ_{i ∈ tile} ḡ_i part[rg][i]  (κ = ḡᵀQḡ = Σ κ_item).
//   --- grid barrier ---
//   (c) κ = Σ κ_item, α = γ/κ (exact line search).  Each tile: w = Σ_rg part,
//       y⁺ = [y − αḡ]₊, e = the clipped part (e_i = αḡ_i − y_i where
//       y_i − αḡ_i < 0), g ← g − αw, and the mask of the new iterate as if
//       nothing was clipped (ḡ, γ_ct, |P|_ct); clip_ct = number clipped.
//   --- grid barrier ---
//   (d) only if Σ clip_ct > 0: u = Qe over the clipped rows with the same
//       items; the last item of a tile to finish (atomic ticket) adds u to g
//       and recomputes that tile's mask.  --- grid barrier ---
//
// Since y⁺ − y = −αḡ + e, g + Q(y⁺ − y) = g − αw + Qe: the product Qḡ of the
// step size is reused and only clipped rows are read a second time (exact
// algebra; the paper counts a second O(n·S(n)) product, §4.2).
//
// Two grid barriers per iteration (three when something is clipped).  Every
// sum has a fixed order, so results are bitwise reproducible.  Each barrier
// wait is bounded (2 s on %globaltimer); on expiry the kernel flags a timeout
// and every block leaves the loop.
#include "common.cuh"
#include "dfloat.cuh"
#include "gridsync.cuh"
#include "kernels.cuh"

namespace aln {

constexpr int kPThreads = 1024;
constexpr int kPWarps = kPThreads / 32;
constexpr int kPU = 4;                          // Q rows in flight per warp (64 KB per SM)
constexpr int kMaxItems = 64 * 1024;

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
    double* kitem;   // CT·R
    int* clip;       // CT
    unsigned int* ticket;  // CT
    PersistSync* sync;
    IterState* st;
    uint64_t wait_ns;      // limit of one grid-barrier wait
    unsigned int skew;     // extra arrivals every barrier waits for (tests: 0 normally)
};

// Partial of Σ_{j ∈ group rg, v_j ≠ 0} v_j Q[j, tile ct] into part[rg][tile].
// Each warp takes a contiguous chunk of the group's rows, loads 64 entries of
// v at once, compacts the non-zero ones with a ballot and keeps kPU row loads
// of Q in flight.  Returns (in threads < TILE) the partial of its column.
template <typename T>
__device__ __forceinline__ T mv_item(const PersistArgs<T>& a, const T* __restrict__ v, int ct,
                                     int rg, T* red) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int TILE = 32 * VN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = (int64_t)ct * TILE + lane * VN;
    const int g0 = rg * a.rows_per_group;
    const int g1 = min(a.n, g0 + a.rows_per_group);
    const int chunk = (g1 - g0 + kPWarps - 1) / kPWarps;
    const int r0 = g0 + warp * chunk;
    const int r1 = min(g1, r0 + chunk);
    T acc[VN];
#pragma unroll
    for (int c = 0; c < VN; ++c) acc[c] = T(0);
    for (int base = r0; base < r1; base += 64) {
        const int ja = base + lane, jb = base + 32 + lane;
        const T va = ja < r1 ? __ldcg(v + ja) : T(0);
        const T vb = jb < r1 ? __ldcg(v + jb) : T(0);
        unsigned int ma = __ballot_sync(0xffffffffu, va != T(0));
        unsigned int mb = __ballot_sync(0xffffffffu, vb != T(0));
        while (ma | mb) {  // warp-uniform
            T vv[kPU];
            V qq[kPU];
#pragma unroll
            for (int u = 0; u < kPU; ++u) {
                int j = -1;
                T vj = T(0);
                if (ma) {
                    const int src = __ffs(ma) - 1;
                    ma &= ma - 1;
                    j = base + src;
                    vj = __shfl_sync(0xffffffffu, va, src);
                } else if (mb) {
                    const int src = __ffs(mb) - 1;
                    mb &= mb - 1;
                    j = base + 32 + src;
                    vj = __shfl_sync(0xffffffffu, vb, src);
                }
                vv[u] = vj;
                qq[u] = j >= 0 ? __ldg(reinterpret_cast<const V*>(a.Q + (int64_t)j * a.ldq + col))
                               : V{};
            }
#pragma unroll
            for (int u = 0; u < kPU; ++u)
#pragma unroll
                for (int c = 0; c < VN; ++c) acc[c] = fma(vv[u], vget(qq[u], c), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < VN; ++c) red[warp * TILE + lane * VN + c] = acc[c];
    __syncthreads();
    T s = T(0);
    if (threadIdx.x < TILE) {
#pragma unroll 8
        for (int w2 = 0; w2 < kPWarps; ++w2) s += red[w2 * TILE + threadIdx.x];
        __stcg(a.part + (int64_t)rg * a.ldq + (int64_t)ct * TILE + threadIdx.x, s);
    }
    __syncthreads();
    return s;
}

// Block sum over the first TILE threads (warps 0..TILE/32-1) in fixed order;
// result in thread 0.
template <int TILE>
__device__ __forceinline__ double tile_sum(double v, double* sd) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0 && wid < TILE / 32) sd[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w2 = 0; w2 < TILE / 32; ++w2) s += sd[w2];
    __syncthreads();
    return s;
}
template <int TILE>
__device__ __forceinline__ int tile_sum_i(int v, int* si) {
    v = warp_sum_i(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0 && wid < TILE / 32) si[wid] = v;
    __syncthreads();
    int s = 0;
    if (threadIdx.x == 0)
        for (int w2 = 0; w2 < TILE / 32; ++w2) s += si[w2];
    __syncthreads();
    return s;
}

// Mask of one tile from (y, g) held in registers by threads < TILE: writes ḡ
// and the tile's ‖ḡ‖² and |P| partials.
template <typename T>
__device__ __forceinline__ void tile_mask(const PersistArgs<T>& a, int ct, bool in, T yi, T gi,
                                          double* sd, int* si) {
    constexpr int TILE = 32 * Vec16<T>::N;
    double v = 0.0;
    int c = 0;
    if (threadIdx.x < TILE && in) {
        const int64_t i = (int64_t)ct * TILE + threadIdx.x;
        const bool P = yi > T(0) || gi < T(0);
        const T gbi = P ? gi : T(0);
        __stcg(a.gb + i, gbi);
        v = (double)gbi * (double)gbi;
        c = P ? 1 : 0;
    }
    v = tile_sum<TILE>(v, sd);
    c = tile_sum_i<TILE>(c, si);
    if (threadIdx.x == 0) {
        __stcg(a.gpart + ct, v);
        __stcg(a.cpart + ct, c);
    }
}

template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_alg2_persist(PersistArgs<T> a) {
    constexpr int TILE = 32 * Vec16<T>::N;
    __shared__ T red[kPWarps * TILE];
    __shared__ double sd[32];
    __shared__ int si[32];
    __shared__ double s_scal[2];
    __shared__ int s_flag[2];
    const unsigned int G = gridDim.x;
    const int items = a.CT * a.R;
    unsigned int bar = 0;  // completion count of the next barrier, minus G

    // prologue: mask of the start point
    for (int ct = blockIdx.x; ct < a.CT; ct += G) {
        const int64_t i = (int64_t)ct * TILE + threadIdx.x;
        const bool in = threadIdx.x < TILE && i < a.n;
        const T yi = in ? __ldcg(a.y + i) : T(0), gi = in ? __ldcg(a.g + i) : T(0);
        tile_mask(a, ct, in, yi, gi, sd, si);
    }
    bool ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns);

    IterState* st = a.st;
    const double eps = st->eps;
    const int max_iter = st->max_iter, window = st->window;
    double best = 1.0 / 0.0;
    int best_iter = 0, iter = 0, status = ALN_RHS_MAXITER, cnt = 0;
    double gam = 0.0;
    long long sum_passive = 0, sum_clip = 0;

    while (ok) {
        // (a) stop test, identical in every block
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double g2 = 0.0;
            int c2 = 0;
            for (int i = lane; i < a.CT; i += 32) {
                g2 += __ldcg(a.gpart + i);
                c2 += __ldcg(a.cpart + i);
            }
            g2 = warp_sum(g2);
            c2 = warp_sum_i(c2);
            if (lane == 0) {
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

        // (b) w-partials and curvature shares
        for (int it = blockIdx.x; it < items; it += G) {
            const int ct = it % a.CT, rg = it / a.CT;
            const int64_t i = (int64_t)ct * TILE + threadIdx.x;
            const T gbi = (threadIdx.x < TILE && i < a.n) ? __ldcg(a.gb + i) : T(0);
            const T pw = mv_item(a, a.gb, ct, rg, red);
            const double k = tile_sum<TILE>((double)gbi * (double)pw, sd);
            if (threadIdx.x == 0) __stcg(a.kitem + it, k);
        }
        if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;

        // (c) step, projection, gradient update, provisional mask
        if (threadIdx.x < 32) {
            double k2 = 0.0;
            for (int i = threadIdx.x; i < items; i += 32) k2 += __ldcg(a.kitem + i);
            k2 = warp_sum(k2);
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
        const T aT = (T)(gam / kap);
        sum_passive += cnt;
        for (int ct = blockIdx.x; ct < a.CT; ct += G) {
            const int64_t i = (int64_t)ct * TILE + threadIdx.x;
            const bool in = threadIdx.x < TILE && i < a.n;
            T yn = T(0), gn = T(0);
            int clipped = 0;
            if (in) {
                T wi = T(0);
                for (int r = 0; r < a.R; ++r) wi += __ldcg(a.part + (int64_t)r * a.ldq + i);
                const T yi = __ldcg(a.y + i);
                const T step = aT * __ldcg(a.gb + i);
                yn = yi - step;
                T ei = T(0);
                if (yn < T(0)) {
                    ei = step - yi;
                    yn = T(0);
                    clipped = 1;
                }
                gn = __ldcg(a.g + i) - aT * wi;
                __stcg(a.y + i, yn);
                __stcg(a.e + i, ei);
                __stcg(a.g + i, gn);
            }
            clipped = __syncthreads_count(clipped);
            if (threadIdx.x == 0) __stcg(a.clip + ct, clipped);
            tile_mask(a, ct, in, yn, gn, sd, si);
        }
        ++iter;
        if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;

        // (d) clipped correction g += Q e (only when something was clipped)
        if (threadIdx.x < 32) {
            int c3 = 0;
            for (int i = threadIdx.x; i < a.CT; i += 32) c3 += __ldcg(a.clip + i);
            c3 = warp_sum_i(c3);
            if (threadIdx.x == 0) s_flag[1] = c3;
        }
        __syncthreads();
        const int nclip = s_flag[1];
        sum_clip += nclip;
        if (nclip > 0) {
            __shared__ int s_last;
            for (int it = blockIdx.x; it < items; it += G) {
                const int ct = it % a.CT, rg = it / a.CT;
                (void)mv_item(a, a.e, ct, rg, red);
                if (threadIdx.x == 0) {
                    unsigned int t;
                    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                                 : "=r"(t)
                                 : "l"(a.ticket + ct), "r"(1u)
                                 : "memory");
                    s_last = t == (unsigned int)(a.R - 1);
                    if (s_last) a.ticket[ct] = 0u;  // reset for the next correction
                }
                __syncthreads();
                if (s_last) {
                    const int64_t i = (int64_t)ct * TILE + threadIdx.x;
                    const bool in = threadIdx.x < TILE && i < a.n;
                    T yi = T(0), gi = T(0);
                    if (in) {
                        T ui = T(0);
                        for (int r = 0; r < a.R; ++r)
                            ui += __ldcg(a.part + (int64_t)r * a.ldq + i);
                        yi = __ldcg(a.y + i);
                        gi = __ldcg(a.g + i) + ui;
                        __stcg(a.g + i, gi);
                    }
                    tile_mask(a, ct, in, yi, gi, sd, si);
                }
                __syncthreads();
            }
            if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;
        }
    }

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = iter;
        st->done = 1;
        st->status = ok ? status : kStatusTimeout;
        st->gbar2 = gam;
        st->npassive = cnt;
        st->best_g2 = best;
        st->best_iter = best_iter;
        st->sum_passive = sum_passive;
        st->sum_clip = sum_clip;
    }
}

// ===========================================================================
// Replicated-state variant (n up to a few thousand): every block keeps the
// whole of y, g, ḡ and w in shared memory and repeats the O(n) elementwise
// work of (c) and the mask itself, in the same order, so every block holds
// bitwise-identical vectors.  Only the products cross blocks: each work item
// writes its partial of Qḡ and its curvature share, one grid barrier later
// every block reads all partials (R·n values) and continues on its own.  An
// iteration therefore costs ONE grid barrier (two when something is clipped:
// Qe crosses blocks too).  The partial and curvature buffers alternate with
// the iteration parity, because a block may start the next product while a
// slower block still reads this one's partials; no block can run two
// iterations ahead, since every iteration passes a barrier.
// ===========================================================================
template <typename T>
struct ReplArgs {
    const T* Q;
    int64_t ldq;
    int n;
    int CT;
    int R;
    int rows_per_group;
    T* y;            // in/out (global), ldq
    T* ylo;          // in/out (global), ldq: low part of the float-pair y (FP32 only)
    T* g;            // in/out (global), ldq
    T* part;         // 2 × R × ldq  (w partials, by iteration parity)
    T* part2;        // R × ldq      (Qe partials)
    double* kitem;   // 2 × CT·R     (curvature shares, by parity)
    PersistSync* sync;
    IterState* st;
    // nullable: bit rt of tmask[ct·tw + rt/32] set when the 128×128 tile
    // (row tile rt, column tile ct) of Q may be non-zero (tiles of Q known to
    // be zero, from a block-sparse Gram, are skipped by the products)
    const uint32_t* tmask;
    int tw;
    uint64_t wait_ns;      // limit of one grid-barrier wait
    unsigned int skew;     // extra arrivals every barrier waits for (tests: 0 normally)
};

// Warp sum in the iteration type (xor tree: every lane gets the sum).
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Is the 128×128 tile of Q holding row j, column tile ct possibly non-zero?
__device__ __forceinline__ bool tile_nz(const uint32_t* __restrict__ tm_ct, int j) {
    const int rt = j >> 7;
    return (__ldg(tm_ct + (rt >> 5)) >> (rt & 31)) & 1u;
}

// Partial Σ_{j ∈ group rg, v_j ≠ 0} v_j Q[j, tile ct] with v in shared memory;
// written to dst[rg][tile]; returns the partial in threads < TILE.  With
// tmask, rows whose tile of Q in column tile ct is zero are skipped (their
// terms are exact zeros), FP32 tiles of 128 columns only.
//
// With ksc (a 33-double scratch), the item's curvature share
// κ_item = Σ_{i ∈ tile} v_i·partial_i is formed in the same block-barrier
// steps: warp sums over the TILE threads, then thread 0 adds the warp sums in
// FP64 (the xor tree of those sums, the zero ones of other warps left out)
// into *kappa (thread 0 only).
template <typename T, bool DIFF = false, typename S = double>
__device__ __forceinline__ T mv_item_rep(const T* __restrict__ Q, int64_t ldq, int n,
                                         int rows_per_group, const T* v, int ct, int rg,
                                         T* __restrict__ dst, T* red,
                                         const double* __restrict__ add = nullptr,
                                         const T* vsub = nullptr,
                                         const uint32_t* __restrict__ tmask = nullptr,
                                         int tw = 0, double* ksc = nullptr,
                                         S* kappa = nullptr) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int TILE = 32 * VN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = (int64_t)ct * TILE + lane * VN;
    const int g0 = rg * rows_per_group;
    const int g1 = min(n, g0 + rows_per_group);
    const int chunk = (g1 - g0 + kPWarps - 1) / kPWarps;
    const int r0 = g0 + warp * chunk;
    const int r1 = min(g1, r0 + chunk);
    T acc[VN];
#pragma unroll
    for (int c = 0; c < VN; ++c) acc[c] = T(0);
    const uint32_t* tm = tmask ? tmask + (int64_t)ct * tw : nullptr;
    for (int base = r0; base < r1; base += 32) {
        const int jl = base + lane;
        // the multiplied vector is v, or v − vsub (DIFF)
        T vl = jl < r1 ? (DIFF ? v[jl] - vsub[jl] : v[jl]) : T(0);
        if (tm && vl != T(0) && !tile_nz(tm, jl)) vl = T(0);
        unsigned int m = __ballot_sync(0xffffffffu, vl != T(0));
        while (m) {  // warp-uniform
            T vv[kPU];
            V qq[kPU];
#pragma unroll
            for (int u = 0; u < kPU; ++u) {
                if (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    vv[u] = DIFF ? __shfl_sync(0xffffffffu, vl, src) : v[base + src];
                    qq[u] = __ldg(reinterpret_cast<const V*>(Q + (int64_t)(base + src) * ldq + col));
                } else {
                    vv[u] = T(0);
                    qq[u] = V{};
                }
            }
#pragma unroll
            for (int u = 0; u < kPU; ++u)
#pragma unroll
                for (int c = 0; c < VN; ++c) acc[c] = fma(vv[u], vget(qq[u], c), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < VN; ++c) red[warp * TILE + lane * VN + c] = acc[c];
    __syncthreads();
    T s = T(0);
    constexpr int NW = TILE / 32;
    T* sv = reinterpret_cast<T*>(ksc);
    if (threadIdx.x < TILE) {
#pragma unroll 8
        for (int w2 = 0; w2 < kPWarps; ++w2) s += red[w2 * TILE + threadIdx.x];
        // `add` (a vector of n entries) joins the partial of row group 0
        const int64_t i = (int64_t)ct * TILE + threadIdx.x;
        if (add && rg == 0 && i < n) s += (T)add[i];
        __stcg(dst + (int64_t)rg * ldq + i, s);
        if (ksc) {
            const T pk = warp_sum_t(i < n ? v[i] * s : T(0));
            if (lane == 0) sv[warp] = pk;
        }
    }
    __syncthreads();
    if (ksc && threadIdx.x == 0) {
        S pw[NW];
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) sc_set(pw[w2], sv[w2]);
#pragma unroll
        for (int o = NW / 2; o >= 1; o >>= 1)
#pragma unroll
            for (int i2 = 0; i2 < o; ++i2) pw[i2] = sc_add(pw[i2], pw[i2 + o]);
        *kappa = pw[0];
    }
    return s;
}

// Block sums whose result every thread receives (fixed tree: warp shuffles,
// then the warp sums in warp order).
__device__ __forceinline__ double block_sum_bcast(double v, double* sc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sc[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += sc[w2];
    return s;
}

// GB300's FP64 pipe is narrow: an FP64 instruction costs a warp about 16
// cycles of its SM's FP64 unit even with one active lane, and instructions
// of different warps queue there.  The per-iteration reductions therefore
// run in the iteration type T across lanes and warps (warp_sum_t), and only
// the final sum over the warp partials is done wider, by one warp, then
// broadcast through shared memory: the warp partials are widened by that
// warp alone — to FP64 here (block_sum_td), or to the scalar type of the
// replicated kernel (block_sum3: FP32 pairs in the FP32 kernel).  The
// scalars of the step (γ = ‖ḡ‖², κ = ḡᵀQḡ, α = γ/κ) need more than FP32 —
// with FP32 scalars the FP32 iteration drifted from the true gradient by
// about 10⁻⁴ (relative) and needed several times more iterations.
template <typename T>
__device__ __forceinline__ double block_sum_td(T v, double* sc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T* sv = reinterpret_cast<T*>(sc);  // the warp partials in T, widened by warp 0
    v = warp_sum_t(v);
    __syncthreads();
    if (lane == 0) sv[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double x = lane < (int)(blockDim.x >> 5) ? (double)sv[lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) sc[32] = x;
    }
    __syncthreads();
    return sc[32];
}

// One block reduction for the update step: the value v (partials in T
// within warps, the 32 warp partials added in the scalar type S by warp 0,
// the same tree as block_sum_td) and two counts.  The counts travel packed in one int
// (a + 2^16·b: both stay below 2^15 here, since the replicated-state kernels
// hold n < 2^14 entries).  The warp partials of v are stored in T and
// widened by warp 0 alone (exact, and one FP64 instruction instead of one per
// warp on the narrow FP64 pipe).  With v_if_b_zero, the wide sum is formed
// only when the total b is 0 (*v_out is 0 otherwise).  sd holds 33 doubles,
// si 66 ints.
template <typename T, typename S = double>
__device__ __forceinline__ void block_sum3(T v, int a, int b, double* sd, int* si, S* v_out,
                                           int* a_out, int* b_out, bool v_if_b_zero = false) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T* sv = reinterpret_cast<T*>(sd);  // the warp partials, in T
    v = warp_sum_t(v);
    int ab = (int)__reduce_add_sync(0xffffffffu, (unsigned)(a + (b << 16)));  // one redux
    __syncthreads();  // earlier readers of sd / si are done
    if (lane == 0) {
        sv[wid] = v;
        si[wid] = ab;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (int)(blockDim.x >> 5);
        ab = (int)__reduce_add_sync(0xffffffffu, (unsigned)(lane < nw ? si[lane] : 0));
        const int xb = ab >> 16;
        S x;
        sc_set(x, T(0));
        if (!v_if_b_zero || xb == 0) {
            S lv;
            sc_set(lv, lane < nw ? sv[lane] : T(0));
            x = sc_warp_sum(lv);
        }
        if (lane == 0) {
            *reinterpret_cast<S*>(sd + 32) = x;
            si[64] = ab & 0xffff;
            si[65] = xb;
        }
    }
    __syncthreads();
    *v_out = *reinterpret_cast<const S*>(sd + 32);
    *a_out = si[64];
    *b_out = si[65];
}

// Mask of the whole replicated state: ḡ = g on P(y); returns ‖ḡ‖² and |P|
// (fixed reduction tree, identical in every block; si holds 66 ints).
template <typename T, typename S = double>
__device__ __forceinline__ void mask_all(int n, const T* sy, const T* sg, T* sgb, double* st,
                                         int* si, S* g2_out, int* cnt_out) {
    T v = T(0);
    int c = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const T yi = sy[j], gi = sg[j];
        const bool P = yi > T(0) || gi < T(0);
        const T gb = P ? gi : T(0);
        sgb[j] = gb;
        v = fma(gb, gb, v);
        c += P ? 1 : 0;
    }
    int unused;
    block_sum3<T, S>(v, c, 0, st, si, g2_out, cnt_out, &unused);
}

constexpr int kLocalClip = 8;  // clipped rows a block multiplies by itself

// The step α = γ/κ in the iteration type.  FP64: the quotient itself.  FP32:
// formed on the FP32 pipe (GB300's FP64 divide is a long dependent sequence
// on a narrow pipe): the quotient of the leading FP32 parts of γ and κ,
// corrected once with the residual of their FP32-pair splits (one Newton
// step of the division), within an FP32 ulp or so of (float)(γ/κ).
template <typename T>
__device__ __forceinline__ T step_quotient(double gam, double kap) {
    if (sizeof(T) == 8) return (T)(gam / kap);
    const float gh = (float)gam, kh = (float)kap;
    const float gl = (float)(gam - (double)gh), kl = (float)(kap - (double)kh);
    const float q = __fdiv_rn(gh, kh);
    const float r = fmaf(-q, kh, gh) + fmaf(-q, kl, gl);
    return (T)(q + __fdiv_rn(r, kh));
}
// The same from FP32-pair scalars (no FP64 at all).
template <typename T>
__device__ __forceinline__ T step_quotient(DF gam, DF kap) {
    return (T)df_quotient(gam, kap);
}

// dst[j] (+)= Σ_r part[r][j] for j < n, r in order.  16-byte loads, two
// vectors per thread per pass, so that for n up to 8·blockDim.x (FP32) one
// pass issues all of a thread's loads at once (the partials were written by
// other SMs: each round trip is a full L2 latency).  Rows of part are ldq
// long (a multiple of the vector width) and fully written, so the vector
// loads stay in bounds.
template <typename T>
__device__ __forceinline__ void sum_partials(const T* __restrict__ part, int R, int64_t ldq,
                                             int n, T* dst, bool accumulate, int t0 = 0) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    const int nv = (n + VN - 1) / VN;
    const int tid = (int)threadIdx.x - t0, nt = (int)blockDim.x - t0;  // threads t0.. take part
    if (tid < 0) return;
    for (int v0 = tid; v0 < nv; v0 += 2 * nt) {
        const int v1 = v0 + nt;
        T a0[VN], a1[VN];
#pragma unroll
        for (int c = 0; c < VN; ++c) a0[c] = a1[c] = T(0);
#pragma unroll 2
        for (int r = 0; r < R; ++r) {
            const V* row = reinterpret_cast<const V*>(part + (int64_t)r * ldq);
            const V x0 = __ldcg(row + v0);
            const V x1 = v1 < nv ? __ldcg(row + v1) : V{};
#pragma unroll
            for (int c = 0; c < VN; ++c) {
                a0[c] += vget(x0, c);
                a1[c] += vget(x1, c);
            }
        }
#pragma unroll
        for (int c = 0; c < VN; ++c) {
            const int j0 = v0 * VN + c, j1 = v1 * VN + c;
            if (j0 < n) dst[j0] = accumulate ? dst[j0] + a0[c] : a0[c];
            if (v1 < nv && j1 < n) dst[j1] = accumulate ? dst[j1] + a1[c] : a1[c];
        }
    }
}

// Indices j < n with e_j ≠ 0 in increasing order into list[0..kLocalClip):
// each warp scans a contiguous range, warp counts are prefix-summed.
template <typename T>
__device__ __forceinline__ void clipped_list(int n, const T* e, int* list, int* si) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (n + nw - 1) / nw;
    const int j0 = wid * per, j1 = min(n, j0 + per);
    int count = 0;
    for (int b = j0; b < j1; b += 32) {
        const int j = b + lane;
        count += __popc(__ballot_sync(0xffffffffu, j < j1 && e[j] != T(0)));
    }
    __syncthreads();
    if (lane == 0) si[wid] = count;
    __syncthreads();
    int base = 0;
    for (int w2 = 0; w2 < wid; ++w2) base += si[w2];
    for (int b = j0; b < j1; b += 32) {
        const int j = b + lane;
        const bool nz = j < j1 && e[j] != T(0);
        const unsigned int m = __ballot_sync(0xffffffffu, nz);
        const int idx = base + __popc(m & ((1u << lane) - 1u));
        if (nz && idx < kLocalClip) list[idx] = j;
        base += __popc(m);
    }
    __syncthreads();
}

// One vector (entries j = v·VN + c, 16 bytes) of the update of (c):
// y⁺ = [y − αḡ]₊ (a float pair in FP32: TwoSum, then renormalise), e = the
// clipped part (e_j = y⁺_j − (y_j − αḡ_j) where y_j − αḡ_j < 0), g ← g − αw,
// and the mask of the new point as if nothing was clipped (ḡ, and the
// partials of ‖ḡ‖², |P| and the clipped count).  Entries j ≥ n stay zero.
template <typename T, bool TAIL>
__device__ __forceinline__ void update_vec_(int v, int n, T aT, const T (&w)[Vec16<T>::N], T* sy,
                                            T* syl, T* sg, T* sgb, T* se, T& v2, int& cP,
                                            int& clipped) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr bool DF = sizeof(T) == 4;
    V* py = reinterpret_cast<V*>(sy) + v;
    V* pyl = reinterpret_cast<V*>(syl) + v;
    V* pg = reinterpret_cast<V*>(sg) + v;
    V* pgb = reinterpret_cast<V*>(sgb) + v;
    const V y4 = *py, g4 = *pg, gb4 = *pgb;
    V yl4 = {};
    if (DF) yl4 = *pyl;
    V yo, ylo, go, gbo, eo;
#pragma unroll
    for (int c = 0; c < VN; ++c) {
        const bool in = !TAIL || v * VN + c < n;
        const T yi = vget(y4, c);
        T yn, nl = T(0), ej = T(0);
        if (DF) {
            const T step = __fmul_rn((float)aT, (float)vget(gb4, c));
            const T s1 = yi - step;
            const T bb = s1 - yi;
            const T er = (yi - (s1 - bb)) + (-step - bb);
            const T t = vget(yl4, c) + er;
            yn = s1 + t;
            nl = t - (yn - s1);
            if (yn < T(0)) {  // clipped: y⁺ = 0, e = y⁺ − (y − αḡ)
                ej = -(yn + nl);
                yn = T(0);
                nl = T(0);
                clipped += in ? 1 : 0;
            }
        } else {
            const T step = aT * vget(gb4, c);
            yn = yi - step;
            if (yn < T(0)) {
                ej = step - yi;
                yn = T(0);
                clipped += in ? 1 : 0;
            }
        }
        const T gn = vget(g4, c) - aT * w[c];
        const bool P = in && (yn > T(0) || gn < T(0));
        const T gb = P ? gn : T(0);
        v2 = fma(gb, gb, v2);
        cP += P ? 1 : 0;
        vset(yo, c, in ? yn : T(0));
        vset(ylo, c, in ? nl : T(0));
        vset(go, c, in ? gn : T(0));
        vset(gbo, c, gb);
        vset(eo, c, in ? ej : T(0));
    }
    *py = yo;
    if (DF) *pyl = ylo;
    *pg = go;
    *pgb = gbo;
    reinterpret_cast<V*>(se)[v] = eo;
}
// The vectors wholly below n skip the per-entry bounds selects.
template <typename T>
__device__ __forceinline__ void update_vec(int v, int n, T aT, const T (&w)[Vec16<T>::N], T* sy,
                                           T* syl, T* sg, T* sgb, T* se, T& v2, int& cP,
                                           int& clipped) {
    if ((v + 1) * Vec16<T>::N <= n)
        update_vec_<T, false>(v, n, aT, w, sy, syl, sg, sgb, se, v2, cP, clipped);
    else
        update_vec_<T, true>(v, n, aT, w, sy, syl, sg, sgb, se, v2, cP, clipped);
}

// g ← g + acc for one vector, then its mask (ḡ, and the partials of ‖ḡ‖²
// and |P|).  Entries j ≥ n stay zero.
template <typename T, bool TAIL>
__device__ __forceinline__ void add_mask_vec_(int v, int n, const T (&acc)[Vec16<T>::N],
                                              const T* sy, T* sg, T* sgb, T& v2, int& cP) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    V* pg = reinterpret_cast<V*>(sg) + v;
    const V y4 = reinterpret_cast<const V*>(sy)[v], g4 = *pg;
    V go, gbo;
#pragma unroll
    for (int c = 0; c < VN; ++c) {
        const bool in = !TAIL || v * VN + c < n;
        const T gi = vget(g4, c) + acc[c];
        const bool P = in && (vget(y4, c) > T(0) || gi < T(0));
        const T gb = P ? gi : T(0);
        v2 = fma(gb, gb, v2);
        cP += P ? 1 : 0;
        vset(go, c, in ? gi : T(0));
        vset(gbo, c, gb);
    }
    *pg = go;
    reinterpret_cast<V*>(sgb)[v] = gbo;
}
template <typename T>
__device__ __forceinline__ void add_mask_vec(int v, int n, const T (&acc)[Vec16<T>::N],
                                             const T* sy, T* sg, T* sgb, T& v2, int& cP) {
    if ((v + 1) * Vec16<T>::N <= n)
        add_mask_vec_<T, false>(v, n, acc, sy, sg, sgb, v2, cP);
    else
        add_mask_vec_<T, true>(v, n, acc, sy, sg, sgb, v2, cP);
}

// The clipped correction from the grid's partials, in the same pass as the
// mask: g ← g + Σ_r part[r] (r in order), ḡ, and the partials of ‖ḡ‖², |P|.
// Two vectors per thread per pass keep 2R loads in flight.
template <typename T>
__device__ __forceinline__ void add_partials_mask(const T* __restrict__ part, int R, int64_t ldq,
                                                  int n, const T* sy, T* sg, T* sgb, T& v2,
                                                  int& cP) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    const int nv = (n + VN - 1) / VN, nt = (int)blockDim.x;
    for (int v0 = threadIdx.x; v0 < nv; v0 += 2 * nt) {
        const int v1 = v0 + nt;
        T a0[VN], a1[VN];
#pragma unroll
        for (int c = 0; c < VN; ++c) a0[c] = a1[c] = T(0);
#pragma unroll 2
        for (int r = 0; r < R; ++r) {
            const V* row = reinterpret_cast<const V*>(part + (int64_t)r * ldq);
            const V x0 = __ldcg(row + v0);
            const V x1 = v1 < nv ? __ldcg(row + v1) : V{};
#pragma unroll
            for (int c = 0; c < VN; ++c) {
                a0[c] += vget(x0, c);
                a1[c] += vget(x1, c);
            }
        }
        add_mask_vec<T>(v0, n, a0, sy, sg, sgb, v2, cP);
        if (v1 < nv) add_mask_vec<T>(v1, n, a1, sy, sg, sgb, v2, cP);
    }
}

// The clipped correction from the few clipped rows of Q (list order), in
// the same pass as the mask; with tmask, tiles of Q known to be zero are not
// read (FP32 only).
template <typename T>
__device__ __forceinline__ void add_rows_mask(const T* __restrict__ Q, int64_t ldq, int n,
                                              const int* list, int count, const T* e,
                                              const T* sy, T* sg, T* sgb,
                                              const uint32_t* __restrict__ tmask, int tw, T& v2,
                                              int& cP) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    const int nv = (n + VN - 1) / VN;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const int64_t i = (int64_t)v * VN;
        T acc[VN];
#pragma unroll
        for (int c = 0; c < VN; ++c) acc[c] = T(0);
        const uint32_t* tm = tmask ? tmask + (i >> 7) * tw : nullptr;
#pragma unroll
        for (int k = 0; k < kLocalClip; ++k) {
            if (k < count && (!tm || tile_nz(tm, list[k]))) {
                const int j = list[k];
                const V q = __ldg(reinterpret_cast<const V*>(Q + (int64_t)j * ldq + i));
                const T ej = e[j];
#pragma unroll
                for (int c = 0; c < VN; ++c) acc[c] = fma(ej, vget(q, c), acc[c]);
            }
        }
        add_mask_vec<T>(v, n, acc, sy, sg, sgb, v2, cP);
    }
}

template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_alg2_repl(ReplArgs<T> a) {
    constexpr int TILE = 32 * Vec16<T>::N;
    extern __shared__ __align__(16) uint8_t smraw[];
    T* sy = reinterpret_cast<T*>(smraw);
    T* sg = sy + a.ldq;
    T* sgb = sg + a.ldq;
    T* sw = sgb + a.ldq;     // w, then e
    T* red = sw + a.ldq;     // kPWarps × TILE
    // FP32: the iterate is a pair y = sy + syl (|syl| ≤ ulp(sy)/2), so the
    // FP64 refinement converges below the FP32 rounding of y (the steps αḡ
    // near the optimum are far below ulp(y)); FP64 needs no low part.
    constexpr bool DF = sizeof(T) == 4;
    T* syl = red + kPWarps * TILE;
    __shared__ int si[32];
    __shared__ double s_t[33];
    __shared__ int s_i3[66];
    __shared__ T s_alpha;
    __shared__ int s_flag;   // 0 continue, 1 stop
    __shared__ int s_clip[kLocalClip];
    const unsigned int G = gridDim.x;
    const int items = a.CT * a.R;
    const int n = a.n;
    unsigned int bar = 0;

    // entries n..ldq stay zero throughout (the vector passes read them)
    for (int j = threadIdx.x; j < a.ldq; j += blockDim.x) {
        sy[j] = j < n ? __ldcg(a.y + j) : T(0);
        if (DF) syl[j] = j < n ? __ldcg(a.ylo + j) : T(0);
        sg[j] = j < n ? __ldcg(a.g + j) : T(0);
        sgb[j] = T(0);
        sw[j] = T(0);
    }
    __syncthreads();
    using S = Sc<T>;  // step scalars: FP32 pairs (FP32 kernel) or FP64
    S gam;
    int cnt;
    mask_all<T, S>(n, sy, sg, sgb, s_t, s_i3, &gam, &cnt);

    // Scalar control state lives in thread 0 (FP64 compares and the division
    // are issued once, not by every thread).
    IterState* st = a.st;
    const S eps = sc_of_double<S>(st->eps);
    const int max_iter = st->max_iter, window = st->window;
    // thread 0's bookkeeping lives in shared memory, not in registers of
    // every thread (the kernel runs at the 64-register limit of 1024 threads)
    __shared__ S s_best;
    __shared__ int s_best_iter, s_nclip_iters;
    __shared__ long long s_sum_passive, s_sum_clip;
    __shared__ uint64_t s_prof[5], s_tprev;  // block 0's phase times (ns)
    if (threadIdx.x == 0) {
        s_best = sc_inf<S>();
        s_best_iter = s_nclip_iters = 0;
        s_sum_passive = s_sum_clip = 0;
        for (int k = 0; k < 5; ++k) s_prof[k] = 0;
    }
    int iter = 0, status = ALN_RHS_MAXITER;
    bool ok = true;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    constexpr int VN = Vec16<T>::N;
    const int nv = (n + VN - 1) / VN;             // 16-byte vectors of the state
    const int tid = (int)threadIdx.x - 32;        // gather / update threads: warps 1..
    const int nt = (int)blockDim.x - 32;

    for (;;) {
        if (threadIdx.x == 0) {
            int stop = 1;
            if (!sc_finite(gam)) status = ALN_RHS_NONFINITE;
            else if (cnt == 0) status = ALN_RHS_EMPTY_PASSIVE;
            else if (sc_lt(gam, eps) || sc_zero(gam)) status = ALN_RHS_CONVERGED;
            else if (iter >= max_iter) status = ALN_RHS_MAXITER;
            else if (iter - s_best_iter > window) status = ALN_RHS_STAGNATED;
            else stop = 0;
            if (!stop && sc_lt(gam, s_best)) {
                s_best = gam;
                s_best_iter = iter;
            }
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) break;
        const int par = iter & 1;
        T* part = a.part + (int64_t)par * a.R * a.ldq;
        double* kitem = a.kitem + (int64_t)par * items;
        if (timer) s_tprev = p_globaltimer();
        auto lap = [&](int k) {
            if (timer) {
                const uint64_t t = p_globaltimer();
                s_prof[k] += t - s_tprev;
                s_tprev = t;
            }
        };

        // w-partials and curvature shares of this block's items
        for (int it = blockIdx.x; it < items; it += G) {
            const int ct = it % a.CT, rg = it / a.CT;
            S k;
            sc_set(k, T(0));
            (void)mv_item_rep<T, false, S>(a.Q, a.ldq, n, a.rows_per_group, sgb, ct, rg, part,
                                           red, nullptr, nullptr, a.tmask, a.tw, s_t, &k);
            if (threadIdx.x == 0) sc_stcg(kitem + it, k);
        }
        lap(0);
        if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;
        lap(1);

        // every block: κ (warp 0) while warps 1.. gather their vectors of
        // w = Σ_r partials (r in order) into registers — two per thread,
        // any further ones through sw — then α, the projected update, the
        // gradient update and the new mask, vector by vector
        T w0[VN], w1[VN];
#pragma unroll
        for (int c = 0; c < VN; ++c) w0[c] = w1[c] = T(0);
        const int v0 = tid, v1 = tid + nt;
        if (threadIdx.x < 32) {
            // four independent accumulators per lane, then a pairwise and
            // a shuffle tree: the FP64 adds form a short dependent chain
            S kv[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) sc_set(kv[m], T(0));
#pragma unroll 4
            for (int i = threadIdx.x, m = 0; i < items; i += 32, m = (m + 1) & 3)
                kv[m] = sc_add(kv[m], sc_ldcg<S>(kitem + i));
            const S k2 = sc_warp_sum(sc_add(sc_add(kv[0], kv[1]), sc_add(kv[2], kv[3])));
            if (threadIdx.x == 0) {
                int stop = 0;
                if (!sc_finite(k2)) {
                    status = ALN_RHS_NONFINITE;
                    stop = 1;
                } else if (sc_nonpos(k2)) {
                    status = ALN_RHS_CURVATURE;
                    stop = 1;
                }
                s_alpha = stop ? T(0) : step_quotient<T>(gam, k2);
                s_flag = stop;
            }
        } else {
            using V = typename Vec16<T>::type;
            if (v0 < nv) {
#pragma unroll 2
                for (int r = 0; r < a.R; ++r) {
                    const V* row = reinterpret_cast<const V*>(part + (int64_t)r * a.ldq);
                    const V x0 = __ldcg(row + v0);
                    const V x1 = v1 < nv ? __ldcg(row + v1) : V{};
#pragma unroll
                    for (int c = 0; c < VN; ++c) {
                        w0[c] += vget(x0, c);
                        w1[c] += vget(x1, c);
                    }
                }
            }
            for (int v = tid + 2 * nt; v < nv; v += nt) {
                T acc[VN];
#pragma unroll
                for (int c = 0; c < VN; ++c) acc[c] = T(0);
                for (int r = 0; r < a.R; ++r) {
                    const V x = __ldcg(reinterpret_cast<const V*>(part + (int64_t)r * a.ldq) + v);
#pragma unroll
                    for (int c = 0; c < VN; ++c) acc[c] += vget(x, c);
                }
                V o;
#pragma unroll
                for (int c = 0; c < VN; ++c) vset(o, c, acc[c]);
                reinterpret_cast<V*>(sw)[v] = o;
            }
        }
        __syncthreads();
        if (s_flag) break;
        const T aT = s_alpha;
        if (threadIdx.x == 0) s_sum_passive += cnt;
        // The mask of the new point is formed in the same pass; it is final
        // when nothing was clipped (then g needs no correction).  sw takes e.
        int clipped = 0, cP = 0;
        T v2 = T(0);
        if (tid >= 0) {
            if (v0 < nv) update_vec<T>(v0, n, aT, w0, sy, syl, sg, sgb, sw, v2, cP, clipped);
            if (v1 < nv) update_vec<T>(v1, n, aT, w1, sy, syl, sg, sgb, sw, v2, cP, clipped);
            for (int v = tid + 2 * nt; v < nv; v += nt) {
                T wv[VN];
#pragma unroll
                for (int c = 0; c < VN; ++c) wv[c] = sw[(int64_t)v * VN + c];
                update_vec<T>(v, n, aT, wv, sy, syl, sg, sgb, sw, v2, cP, clipped);
            }
        }
        S gam2;
        int cnt2, nclip;
        // identical in every block; ‖ḡ‖² is formed only when nothing was
        // clipped (else the clipped correction's mask replaces it)
        block_sum3<T, S>(v2, cP, clipped, s_t, s_i3, &gam2, &cnt2, &nclip, true);
        ++iter;
        if (threadIdx.x == 0) s_sum_clip += nclip;
        lap(2);

        if (nclip > 0) {
            // g ← g + Qe and the mask of the new point, in one pass
            T v3 = T(0);
            int cP3 = 0, unused;
            if (nclip <= kLocalClip) {
                // Few clipped rows: every block forms Qe itself from those
                // rows of Q (listed in index order, so all blocks add in the
                // same order) — no product pass over the grid and no barrier.
                clipped_list(n, sw, s_clip, si);
                add_rows_mask<T>(a.Q, a.ldq, n, s_clip, nclip, sw, sy, sg, sgb, a.tmask, a.tw,
                                 v3, cP3);
            } else {
                // Q e crosses blocks: partials, barrier, every block sums them
                for (int it = blockIdx.x; it < items; it += G) {
                    const int ct = it % a.CT, rg = it / a.CT;
                    (void)mv_item_rep<T>(a.Q, a.ldq, n, a.rows_per_group, sw, ct, rg, a.part2,
                                         red, nullptr, nullptr, a.tmask, a.tw);
                }
                if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;
                add_partials_mask<T>(a.part2, a.R, a.ldq, n, sy, sg, sgb, v3, cP3);
            }
            block_sum3<T, S>(v3, cP3, 0, s_t, s_i3, &gam, &cnt, &unused);
            if (threadIdx.x == 0) ++s_nclip_iters;
        } else {
            gam = gam2;
            cnt = cnt2;
        }
        lap(3);
    }

    if (blockIdx.x == 0) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            a.y[j] = sy[j];
            if (DF) a.ylo[j] = syl[j];
            a.g[j] = sg[j];
        }
        if (threadIdx.x == 0) {
            st->iter = iter;
            st->done = 1;
            st->status = ok ? status : kStatusTimeout;
            st->gbar2 = sc_double(gam);
            st->npassive = cnt;
            st->best_g2 = sc_double(s_best);
            st->best_iter = s_best_iter;
            st->sum_passive = s_sum_passive;
            st->sum_clip = s_sum_clip;
            for (int k = 0; k < 5; ++k) st->phase_ns[k] = s_prof[k];
            st->phase_ns[5] = (uint64_t)s_nclip_iters;  // iterations that took the clipped path
        }
    }
}

template <typename T>
size_t repl_smem_bytes(int64_t ldq) {  // FP32 adds the low part of y
    return (size_t)((sizeof(T) == 4 ? 5 : 4) * ldq + kPWarps * 32 * Vec16<T>::N) * sizeof(T);
}

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_alg2_persist(aln_ctx* c) {
    if (c->p_repl) {
        ReplArgs<T> r;
        r.Q = (const T*)c->Q;
        r.ldq = c->ldq;
        r.n = (int)c->n;
        r.CT = c->p_CT;
        r.R = c->p_R;
        r.rows_per_group = (int)ceil_div(c->n, c->p_R);
        r.y = (T*)c->y;
        r.ylo = (T*)c->e;  // the tiled kernel's e buffer, unused by this one
        r.g = (T*)c->g;
        r.part = (T*)c->part;
        r.part2 = (T*)c->part + (int64_t)2 * c->p_R * c->ldq;
        r.kitem = c->p_kpart;
        r.sync = (PersistSync*)c->p_sync;
        r.wait_ns = barrier_wait_ns(c);
        r.skew = (unsigned int)c->opt.test_barrier_skew;
        r.st = c->st;
        // zero tiles of Q from the block-sparse Gram (FP32, 128-wide tiles)
        r.tmask = sizeof(T) == 4 ? c->q_tmask : nullptr;
        r.tw = c->q_tw;
        const size_t smem = repl_smem_bytes<T>(c->ldq);
        cudaError_t e = cudaFuncSetAttribute(k_alg2_repl<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        void* args[] = {&r};
        return cudaLaunchCooperativeKernel((const void*)k_alg2_repl<T>, dim3(c->p_G),
                                           dim3(kPThreads), args, smem, c->stream);
    }
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
    a.kitem = c->p_kpart;
    a.clip = c->p_clip;
    a.ticket = c->p_ticket;
    a.sync = (PersistSync*)c->p_sync;
    a.wait_ns = barrier_wait_ns(c);
    a.skew = (unsigned int)c->opt.test_barrier_skew;
    a.st = c->st;
    if ((int64_t)a.CT * a.R > kMaxItems) return cudaErrorInvalidValue;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_alg2_persist<T>, dim3(c->p_G),
                                       dim3(kPThreads), args, 0, c->stream);
}

// Co-resident blocks of the persistent kernel for row length ldq.  With
// `repl`, the replicated-state kernel and its shared-memory footprint are
// tried first; *repl is cleared when its state does not fit on an SM.
template <typename T>
int persist_max_blocks(int num_sms, int64_t ldq, int* repl) {
    int per_sm = 0;
    if (*repl) {
        const size_t smem = repl_smem_bytes<T>(ldq);
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (smem + 4096 <= (size_t)optin &&
            cudaFuncSetAttribute(k_alg2_repl<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_alg2_repl<T>, kPThreads,
                                                          smem) == cudaSuccess &&
            per_sm > 0)
            return per_sm * num_sms;
        cudaGetLastError();
        *repl = 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_alg2_persist<T>, kPThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * num_sms;
}

// ===========================================================================
// Anti+Acc (§5): the scaling of Alg. 1 followed by Nesterov's accelerated
// projected gradient with the constant step 1/L (the optimal gradient method
// the paper cites for its accelerated baselines), in the replicated-state
// layout of k_alg2_repl: every block keeps x_k, x_{k−1}, ∇f(x_k), ∇f(x_{k−1})
// in shared memory and repeats the elementwise work; only the product
// ∇f(x_k) = Qx_k + q crosses blocks (partials, one grid barrier, gather).
//
//   Y_k     = x_{k−1} + β (x_{k−1} − x_{k−2}),  β = (α_{k−1} − 1)/α_k
//   ∇f(Y_k) = ∇f(x_{k−1}) + β (∇f(x_{k−1}) − ∇f(x_{k−2}))   (f is quadratic)
//   x_k     = [Y_k − ∇f(Y_k)/L]₊,  α_{k+1} = (1 + √(4α_k² + 1))/2
//
// with x_{−1} = x_{−2} = y⁰ and α_0 = 1 (so the first two steps carry no
// momentum).  The stop rule is Alg. 2's at x_k: ‖ḡ(x_k)‖² < ε or P = ∅.  The
// momentum scalars are FP64 in thread 0.  The gradient is carried the way
// Alg. 2 carries it, ∇f(x_k) = ∇f(x_{k−1}) + Q(x_k − x_{k−1}): in FP32 a
// fresh Qx_k + q would put a floor of about 10⁻⁷·‖Q‖‖x‖ under ‖ḡ‖ that the
// FP64 refinement could not lower, whereas the increments shrink with the
// steps, so each refinement round (restarting from the exact FP64 gradient)
// gains accuracy.
// ===========================================================================
template <typename T>
struct AccArgs {
    const T* Q;
    int64_t ldq;
    int n;
    int CT;
    int R;
    int rows_per_group;
    T* y;             // in/out (global): start point, then x at the stop
    T* g;             // in/out (global): ∇f there
    T* part;          // 2 × R × ldq (partials of Qx + q, by iteration parity)
    double inv_L;     // 1/L
    int window;       // stagnation window (iterations without a new best ‖ḡ‖²)
    PersistSync* sync;
    IterState* st;
    uint64_t wait_ns;      // limit of one grid-barrier wait
    unsigned int skew;     // extra arrivals every barrier waits for (tests: 0 normally)
};

// ḡ over the replicated vectors: ‖ḡ‖², |P| and the number of non-zero
// entries of the last step d (the rows of Q its product read).
template <typename T>
__device__ __forceinline__ void acc_mask(int n, const T* sx, const T* sg, const T* sd_or_x,
                                         const T* sxp, double* sd, int* si, double* g2, int* cnt,
                                         int* nnz) {
    T v = T(0);
    int cp = 0, cz = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const T xj = sx[j], gj = sg[j];
        const bool P = xj > T(0) || gj < T(0);
        const T gb = P ? gj : T(0);
        v = fma(gb, gb, v);
        cp += P ? 1 : 0;
        const T dj = sxp ? sd_or_x[j] - sxp[j] : sd_or_x[j];
        cz += dj != T(0) ? 1 : 0;
    }
    block_sum3<T>(v, cp, cz, sd, si, g2, cnt, nnz);
}

// FP32: the iterate is a pair x = xh + xl (|xl| ≤ ulp(xh)/2), as in the
// grouped Alg. 2 kernel: the steps ∇f/L of the accelerated method are far
// below ulp(x) near the optimum and would be lost in an FP32 x.  The step
// d = x_k − x_{k−1} is kept in its own vector for the gradient product.
// FP64: plain x; the product takes x_k − x_{k−1} on the fly.
template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_acc_repl(AccArgs<T> a) {
    constexpr bool DF = sizeof(T) == 4;
    extern __shared__ __align__(16) uint8_t smraw[];
    T* sx = reinterpret_cast<T*>(smraw);  // x_{k−1} (high part)
    T* sxp = sx + a.ldq;                  // x_{k−2} (high part)
    T* sg = sxp + a.ldq;                  // ∇f(x_{k−1})
    T* sgp = sg + a.ldq;                  // ∇f(x_{k−2})
    T* red = sgp + a.ldq;                 // kPWarps × TILE
    T* sxl = red + kPWarps * 32 * Vec16<T>::N;  // DF: low parts of x_{k−1}, x_{k−2}; step d
    T* sxpl = sxl + a.ldq;
    T* sdd = sxpl + a.ldq;
    __shared__ double s_t[33];
    __shared__ int s_i3[66];
    __shared__ T s_beta;
    __shared__ int s_flag;
    const unsigned int G = gridDim.x;
    const int items = a.CT * a.R;
    const int n = a.n;
    unsigned int bar = 0;

    for (int j = threadIdx.x; j < a.ldq; j += blockDim.x) {
        const T x = j < n ? __ldcg(a.y + j) : T(0);
        const T g = j < n ? __ldcg(a.g + j) : T(0);
        sx[j] = x;
        sxp[j] = x;
        sg[j] = g;
        sgp[j] = g;
        if (DF) {
            sxl[j] = T(0);
            sxpl[j] = T(0);
            sdd[j] = T(0);
        }
    }
    __syncthreads();
    double gam;
    int cnt, nnz;
    acc_mask(n, sx, sg, DF ? sdd : sx, DF ? nullptr : sxp, s_t, s_i3, &gam, &cnt, &nnz);

    IterState* st = a.st;
    const double eps = st->eps;
    const int max_iter = st->max_iter, window = a.window;
    double best = 1.0 / 0.0;
    int best_iter = 0, iter = 0, status = ALN_RHS_MAXITER;
    double a_prev = 1.0, a_cur = 1.0;  // α_{k−1}, α_k (thread 0)
    long long sum_rows = 0;
    uint64_t prof[5] = {0, 0, 0, 0, 0};
    bool ok = true;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    const T invL = (T)a.inv_L;

    for (;;) {
        if (threadIdx.x == 0) {
            int stop = 1;
            if (!isfinite(gam)) status = ALN_RHS_NONFINITE;
            else if (cnt == 0) status = ALN_RHS_EMPTY_PASSIVE;
            else if (gam < eps || gam == 0.0) status = ALN_RHS_CONVERGED;
            else if (iter >= max_iter) status = ALN_RHS_MAXITER;
            else if (iter - best_iter > window) status = ALN_RHS_STAGNATED;
            else stop = 0;
            if (!stop && gam < best) {
                best = gam;
                best_iter = iter;
            }
            if (!stop) {
                s_beta = (T)((a_prev - 1.0) / a_cur);
                a_prev = a_cur;
                a_cur = 0.5 * (1.0 + sqrt(4.0 * a_cur * a_cur + 1.0));
            }
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) break;
        uint64_t t_prev = timer ? p_globaltimer() : 0;
        auto lap = [&](int k) {
            if (timer) {
                const uint64_t t = p_globaltimer();
                prof[k] += t - t_prev;
                t_prev = t;
            }
        };
        const T beta = s_beta;
        // x_k = [Y − ∇f(Y)/L]₊ = [x + β(x − x_p) − (g + β(g − g_p))/L]₊; the
        // history shifts by one
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T xh = sx[j], xph = sxp[j], g = sg[j], gp = sgp[j];
            const T gY = g + beta * (g - gp);
            if (DF) {
                const T xl = sxl[j], xpl = sxpl[j];
                const T d = (xh - xph) + (xl - xpl);
                const T u = beta * d - gY * invL;  // Y − ∇f(Y)/L − x
                // (xh, xl) + u: TwoSum, then renormalise
                const T s = xh + u;
                const T bb = s - xh;
                const T er = (xh - (s - bb)) + (u - bb);
                const T t = xl + er;
                T nh = s + t;
                T nl = t - (nh - s);
                if (nh < T(0) || (nh == T(0) && nl < T(0))) {
                    nh = T(0);
                    nl = T(0);
                }
                sxp[j] = xh;
                sxpl[j] = xl;
                sx[j] = nh;
                sxl[j] = nl;
                sdd[j] = (nh - xh) + (nl - xl);  // x_k − x_{k−1}
            } else {
                const T Y = xh + beta * (xh - xph);
                const T xn = Y - gY * invL;
                sxp[j] = xh;
                sx[j] = xn > T(0) ? xn : T(0);
            }
            sgp[j] = g;
        }
        __syncthreads();
        lap(0);
        // ∇f(x_k) = ∇f(x_{k−1}) + Q(x_k − x_{k−1}): partials, barrier, gather
        T* part = a.part + (int64_t)(iter & 1) * a.R * a.ldq;
        for (int it = blockIdx.x; it < items; it += G) {
            const int ct = it % a.CT, rg = it / a.CT;
            if (DF)
                (void)mv_item_rep(a.Q, a.ldq, n, a.rows_per_group, sdd, ct, rg, part, red);
            else
                (void)mv_item_rep<T, true>(a.Q, a.ldq, n, a.rows_per_group, sx, ct, rg, part,
                                           red, nullptr, sxp);
        }
        ++iter;
        lap(1);
        if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;
        lap(2);
        sum_partials(part, a.R, a.ldq, n, sg, true);  // sg still holds ∇f(x_{k−1})
        __syncthreads();
        acc_mask(n, sx, sg, DF ? sdd : sx, DF ? nullptr : sxp, s_t, s_i3, &gam, &cnt, &nnz);
        sum_rows += nnz;  // rows of Q this product read: nnz(x_k − x_{k−1})
        lap(3);
    }
    if (blockIdx.x == 0) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            a.y[j] = DF ? sx[j] + sxl[j] : sx[j];
            a.g[j] = sg[j];
        }
        if (threadIdx.x == 0) {
            st->iter = iter;
            st->done = 1;
            st->status = ok ? status : kStatusTimeout;
            st->gbar2 = gam;
            st->npassive = cnt;
            st->best_g2 = best;
            st->best_iter = best_iter;
            st->sum_passive = sum_rows;
            st->sum_clip = 0;
            for (int k = 0; k < 5; ++k) st->phase_ns[k] = prof[k];
            st->phase_ns[5] = 0;
        }
    }
}

// Power iteration for L = λ_max(Q) (the Anti+Acc step 1/L): v⁰_i = 1 + (i mod
// 5)/8 normalised; u = Qv, ρ = vᵀu, v ← u/‖u‖; stops when two successive ρ
// agree to `tol` (relative) or after max_steps products.  Same replicated
// layout: one grid barrier per product.  out[0] = ρ, out[1] = products.
template <typename T>
struct PowerArgs {
    const T* Q;
    int64_t ldq;
    int n;
    int CT;
    int R;
    int rows_per_group;
    T* part;  // 2 × R × ldq
    double tol;
    int max_steps;
    PersistSync* sync;
    double* out;
    uint64_t wait_ns;      // limit of one grid-barrier wait
    unsigned int skew;     // extra arrivals every barrier waits for (tests: 0 normally)
};

template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_power_repl(PowerArgs<T> a) {
    extern __shared__ __align__(16) uint8_t smraw[];
    T* sv = reinterpret_cast<T*>(smraw);
    T* su = sv + a.ldq;
    T* red = su + a.ldq;
    __shared__ double s_t[33];
    __shared__ double s_scale;
    __shared__ int s_flag;
    const unsigned int G = gridDim.x;
    const int items = a.CT * a.R;
    const int n = a.n;
    unsigned int bar = 0;
    double part2 = 0.0;
    for (int j = threadIdx.x; j < a.ldq; j += blockDim.x) {
        const double v = j < n ? 1.0 + (double)(j % 5) / 8.0 : 0.0;
        part2 += v * v;
    }
    const double nv2 = block_sum_bcast(part2, s_t);
    const double inv0 = 1.0 / sqrt(nv2);
    for (int j = threadIdx.x; j < a.ldq; j += blockDim.x)
        sv[j] = j < n ? (T)((1.0 + (double)(j % 5) / 8.0) * inv0) : T(0);
    __syncthreads();
    double rho = 0.0, rho_prev = 0.0;
    int t = 0;
    bool ok = true;
    for (;;) {
        T* part = a.part + (int64_t)(t & 1) * a.R * a.ldq;
        for (int it = blockIdx.x; it < items; it += G) {
            const int ct = it % a.CT, rg = it / a.CT;
            (void)mv_item_rep(a.Q, a.ldq, n, a.rows_per_group, sv, ct, rg, part, red);
        }
        ++t;
        if (!(ok = grid_barrier(a.sync, (bar += G) + a.skew, a.wait_ns))) break;
        sum_partials(part, a.R, a.ldq, n, su, false);
        __syncthreads();
        T pr = T(0), pu = T(0);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            pr = fma(sv[j], su[j], pr);
            pu = fma(su[j], su[j], pu);
        }
        rho = block_sum_td<T>(pr, s_t);
        const double nu2 = block_sum_td<T>(pu, s_t);
        if (threadIdx.x == 0) {
            int stop = 0;
            if (t > 1 && fabs(rho - rho_prev) <= a.tol * fabs(rho)) stop = 1;
            else if (!(nu2 > 0.0) || !isfinite(nu2) || t >= a.max_steps) stop = 1;
            rho_prev = rho;
            s_scale = stop ? 0.0 : 1.0 / sqrt(nu2);
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) break;
        const T sc = (T)s_scale;
        for (int j = threadIdx.x; j < n; j += blockDim.x) sv[j] = su[j] * sc;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] = ok ? rho : -1.0;
        a.out[1] = ok ? (double)t : -1.0;
    }
}

template <typename T>
size_t acc_smem_bytes(int64_t ldq) {  // FP32 adds the low parts and the step vector
    return (size_t)((sizeof(T) == 4 ? 7 : 4) * ldq + kPWarps * 32 * Vec16<T>::N) * sizeof(T);
}
template <typename T>
size_t power_smem_bytes(int64_t ldq) {
    return (size_t)(2 * ldq + kPWarps * 32 * Vec16<T>::N) * sizeof(T);
}

// Anti+Acc iteration for the state set up by launch_iter_setup (y, g = ∇f(y),
// eps, max_iter).  Needs the replicated layout (the vectors in shared
// memory); otherwise cudaErrorInvalidValue.
template <typename T>
cudaError_t launch_acc_persist(aln_ctx* c) {
    const size_t smem = acc_smem_bytes<T>(c->ldq);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (!c->p_repl || smem + 4096 > (size_t)optin || !(c->lipschitz > 0.0))
        return cudaErrorInvalidValue;
    AccArgs<T> r;
    r.Q = (const T*)c->Q;
    r.ldq = c->ldq;
    r.n = (int)c->n;
    r.CT = c->p_CT;
    r.R = c->p_R;
    r.rows_per_group = (int)ceil_div(c->n, c->p_R);
    r.y = (T*)c->y;
    r.g = (T*)c->g;
    r.part = (T*)c->part;
    r.inv_L = 1.0 / c->lipschitz;
    // The accelerated method's ‖ḡ‖ is not monotone: an FP32 run ends after
    // 10× the stagnation window without a new best (the FP64 refinement then
    // restarts it from the exact gradient, with fresh momentum); the FP64
    // iteration has no such stop.
    r.window = sizeof(T) == 8 ? (1 << 30) : 10 * c->opt.stagnation;
    r.sync = (PersistSync*)c->p_sync;
    r.wait_ns = barrier_wait_ns(c);
    r.skew = (unsigned int)c->opt.test_barrier_skew;
    r.st = c->st;
    cudaError_t e = cudaFuncSetAttribute(k_acc_repl<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_acc_repl<T>, kPThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm * c->num_sms < c->p_G) return cudaErrorInvalidValue;
    void* args[] = {&r};
    return cudaLaunchCooperativeKernel((const void*)k_acc_repl<T>, dim3(c->p_G), dim3(kPThreads),
                                       args, smem, c->stream);
}

// Power iteration on the prepared Q; out (device) receives ρ and the number
// of products.  Same layout requirements as launch_acc_persist.
template <typename T>
cudaError_t launch_power(aln_ctx* c, double tol, int max_steps, double* out) {
    const size_t smem = power_smem_bytes<T>(c->ldq);
    if (!c->p_repl) return cudaErrorInvalidValue;
    PowerArgs<T> r;
    r.Q = (const T*)c->Q;
    r.ldq = c->ldq;
    r.n = (int)c->n;
    r.CT = c->p_CT;
    r.R = c->p_R;
    r.rows_per_group = (int)ceil_div(c->n, c->p_R);
    r.part = (T*)c->part;
    r.tol = tol;
    r.max_steps = max_steps;
    r.sync = (PersistSync*)c->p_sync;
    r.wait_ns = barrier_wait_ns(c);
    r.skew = (unsigned int)c->opt.test_barrier_skew;
    r.out = out;
    cudaError_t e = cudaFuncSetAttribute(k_power_repl<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_power_repl<T>, kPThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm * c->num_sms < c->p_G) return cudaErrorInvalidValue;
    void* args[] = {&r};
    return cudaLaunchCooperativeKernel((const void*)k_power_repl<T>, dim3(c->p_G),
                                       dim3(kPThreads), args, smem, c->stream);
}

size_t acc_smem_need(bool f64, int64_t ldq) {
    return f64 ? acc_smem_bytes<double>(ldq) : acc_smem_bytes<float>(ldq);
}

template cudaError_t launch_acc_persist<float>(aln_ctx*);
template cudaError_t launch_acc_persist<double>(aln_ctx*);
template cudaError_t launch_power<float>(aln_ctx*, double, int, double*);
template cudaError_t launch_power<double>(aln_ctx*, double, int, double*);

template cudaError_t launch_alg2_persist<float>(aln_ctx*);
template cudaError_t launch_alg2_persist<double>(aln_ctx*);
template int persist_max_blocks<float>(int, int64_t, int*);
template int persist_max_blocks<double>(int, int64_t, int*);

size_t persist_sync_bytes() { return sizeof(PersistSync); }

}  // namespace aln
