// Alg. 1 and Alg. 2 (§3) on many independent NNLS problems of different sizes
// in a few launches (the uneven-batch workload: hundreds of problems with n
// from tens to a thousand).
//
//   k_gcolstats    one block per column slot of every problem: s_j = ‖A_j‖,
//                  q_j = −A_jᵀb/s_j (Dot2, FP64-accurate), and the hi/lo BF16
//                  split written straight into pre-swizzled 16 KiB operand
//                  tiles (pack_index); slots past n_p zero their tile rows.
//   k_ggram_tc     (gemm_tc.cu) every problem's lower-triangle Gram tiles in
//                  one tcgen05 launch, tiles fed by 1-D bulk copies.
//   k_galg2<T>     persistent: each 1024-thread block takes the next problem
//                  from a longest-first queue and runs Alg. 2 on it alone —
//                  iteration vectors in shared memory, Q_p staged in shared
//                  memory when it fits (else read from L2), products over the
//                  compacted passive / clipped index lists, no grid barrier.
//   k_gkkt_*       FP64 KKT residual from A for every unfinished problem,
//                  then the refinement decision (restart from the exact
//                  gradient) in k_gkkt_final.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "blockops.cuh"
#include "cluster.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace aln {
namespace {

constexpr int kGMaxN = 4096;      // largest n of a grouped problem
constexpr int kKeySlot = 0, kKeyV = 1, kKeyR = 2;
// Problems with n ≥ kGClusterMinN whose Q_p does not fit in one block's
// shared memory are solved by a cluster of blocks (k_galg2c; kGCluster unless
// the options say otherwise): each iteration of such a problem is bound by one
// SM's read rate of Q_p from L2, and the largest of them sets the length of
// the whole run.
constexpr int kGCluster = 4;
constexpr int kGClusterMinN = 512;
// A refinement run stops at this fraction of tol.  Measured on the 512-problem
// uneven batch: 0.25 → 44.6 ms, 0.5 → 40.2 ms, 0.75 → 36.8 ms per solve; 0.75
// left the ill-conditioned 1100×1030 test problem at ‖Δx‖/‖x*‖ ≈ 1.1e-5 at
// tol 1e-9 (above the 1e-5 solution gate), 0.5 keeps it below.
constexpr double kGRefineFactor = 0.5;

template <int KEY>
__device__ __forceinline__ int64_t gkey(const GProb& g) {
    return KEY == kKeySlot ? g.slot : (KEY == kKeyV ? g.voff : g.roff);
}
// Largest p with key(p) ≤ x (keys strictly increase with p).
template <int KEY>
__device__ __forceinline__ int find_prob(const GProb* __restrict__ gp, int count, int64_t x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gkey<KEY>(gp[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Prepare (Alg. 1): scale factors, q, split operand tiles
// ---------------------------------------------------------------------------
template <typename TA>
__global__ void __launch_bounds__(128) k_gcolstats(const GProb* __restrict__ gp, int count,
                                                   int split, double* __restrict__ s,
                                                   double* __restrict__ inv_s,
                                                   double* __restrict__ q64, int* __restrict__ flags,
                                                   __nv_bfloat16* __restrict__ hi,
                                                   __nv_bfloat16* __restrict__ mid,
                                                   __nv_bfloat16* __restrict__ lo) {
    __shared__ double scratch[32];
    const int p = find_prob<kKeySlot>(gp, count, blockIdx.x);
    const GProb P = gp[p];
    const int j = (int)((int64_t)blockIdx.x - P.slot);
    const int kpad = P.KB * 64;
    const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
    if (j >= P.n) {  // rows of the last operand tile past n_p: zero
        if (split)
            for (int t = threadIdx.x; t < kpad; t += blockDim.x) {
                const int64_t e = pack_index(P.pack, P.KB, j, t);
                hi[e] = z;
                mid[e] = z;
                lo[e] = z;
            }
        return;
    }
    const TA* col = (const TA*)P.A + (int64_t)j * P.lda;
    const TA* b = (const TA*)P.b;
    DotAcc<TA> sq, dot;
    bool bad = false;
    for (int t0 = threadIdx.x; t0 < P.d; t0 += 4 * blockDim.x) {
        TA av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * blockDim.x;
            av[u] = t < P.d ? col[t] : TA(0);
            bv[u] = t < P.d ? b[t] : TA(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            sq.add(av[u], av[u]);
            dot.add(av[u], bv[u]);
            bad |= !isfinite(av[u]) || !isfinite(bv[u]);
            const int t = t0 + u * blockDim.x;
            if (split && t < P.d) {
                __nv_bfloat16 h, m, l;
                split3_bf16((float)av[u], h, m, l);
                const int64_t e = pack_index(P.pack, P.KB, j, t);
                hi[e] = h;
                mid[e] = m;
                lo[e] = l;
            }
        }
    }
    if (split)
        for (int t = P.d + threadIdx.x; t < kpad; t += blockDim.x) {
            const int64_t e = pack_index(P.pack, P.KB, j, t);
            hi[e] = z;
            mid[e] = z;
            lo[e] = z;
        }
    const double s2 = block_sum(sq.value(), scratch);
    const double ab = block_sum(dot.value(), scratch);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        // Eq. Rescaling: s_j = √H_jj, and s_j := 1 for a zero column
        const double sj = s2 > 0.0 ? sqrt(s2) : 1.0;
        s[P.voff + j] = sj;
        inv_s[P.voff + j] = 1.0 / sj;
        q64[P.voff + j] = -ab / sj;  // q = −D⁻¹Aᵀb (Eq. NQPQ)
        if (bad) atomicOr(flags, 1);
    }
}

// ‖min(q_p, 0)‖ per problem (the projected gradient at y = 0) and ‖b_p‖².
template <typename TA>
__global__ void __launch_bounds__(256) k_gden(const GProb* __restrict__ gp,
                                              const double* __restrict__ q64,
                                              double* __restrict__ den, double* __restrict__ bn2) {
    __shared__ double scratch[32];
    const GProb P = gp[blockIdx.x];
    double v = 0.0, w = 0.0;
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
        const double qi = q64[P.voff + i];
        const double m = qi < 0.0 ? qi : 0.0;
        v = fma(m, m, v);
    }
    const TA* b = (const TA*)P.b;
    for (int t = threadIdx.x; t < P.d; t += blockDim.x) {
        const double bt = (double)b[t];
        w = fma(bt, bt, w);
    }
    v = block_sum(v, scratch);
    w = block_sum(w, scratch);
    if (threadIdx.x == 0) {
        den[blockIdx.x] = sqrt(v);
        bn2[blockIdx.x] = w;
    }
}

// Q_p (FP32, split-BF16 Gram) → FP64 packed row-major n_p×n_p blocks.
template <typename T>
__global__ void k_gexport_q(const GProb* __restrict__ gp, const T* __restrict__ Q,
                            const int64_t* __restrict__ qout_off, double* __restrict__ out) {
    const GProb P = gp[blockIdx.x];
    const int64_t nn = (int64_t)P.n * P.n;
    double* dst = out + qout_off[blockIdx.x];
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int64_t i = e / P.n, j = e - i * P.n;
        dst[e] = (double)Q[P.qoff + i * P.ldq + j];
    }
}

// ---------------------------------------------------------------------------
// Alg. 2, one problem per block
// ---------------------------------------------------------------------------
template <typename T>
struct GSolveArgs {
    const GProb* gp;
    const int* order;      // problems of this run, largest first
    int nactive;
    int* queue;            // next index into order (zeroed before the launch)
    const T* Q;            // pool
    const double* q64;     // packed (voff)
    const double* g64;     // packed (voff): exact gradient for a restart (gmode 1)
    const double* den;     // per problem ‖min(q,0)‖
    double* y;             // packed (foff), in/out
    GStat* stat;
    const double* tgt;     // per problem: inner stop ‖ḡ‖ < tgt_p·den_p (relative KKT)
    int gmode;             // 0: g = Q y + q here; 1: g = g64
    int max_iter;
    int window;
    int smem_bytes;
    const int* run;        // nullable: problems p with run[p] = 0 are passed over
                           // (the graph-captured refinement rounds)
    int budget;            // > 0: a problem stops with kRhsPaused after this many
                           // iterations of this launch (the batched solver's tail)
    double* gout;          // nullable, packed (voff): g at the end of the run, so
                           // that a paused problem resumes with it (gmode 1)
};

// --- thread-block clusters (large problems, several CTAs per problem): cluster.cuh

// w (+)= Q·v over the listed columns for every row.  With CL, CTA `rank` of
// the cluster computes rows [rank·S, rank·S + S) into its exchange buffer xb,
// and after a cluster barrier every CTA gathers all slices (distributed
// shared memory), so all CTAs hold the same w.
template <typename T, bool CL>
__device__ __forceinline__ void product(const T* Q, int ldq, int n, const int* list, int cnt,
                                        const T* v, T* out, bool accumulate, T* red, T* xb,
                                        int rank, int S) {
    if (!CL) {
        gmv(Q, ldq, 0, n, list, cnt, v, out, accumulate, red);
        return;
    }
    const int lo = min(n, rank * S), hi = min(n, lo + S);
    gmv(Q, ldq, lo, hi, list, cnt, v, xb, false, red);
    cluster_sync();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = i / S;
        const T val = r == rank ? xb[i] : ld_cluster(cluster_addr(xb + i, r), T(0));
        out[i] = accumulate ? out[i] + val : val;
    }
    __syncthreads();
}

// Alg. 2 on problem p by one CTA (CL = false) or by the CTAs of a cluster (CL).
template <typename T, bool CL>
__device__ void solve_one(const GSolveArgs<T>& a, int p, uint8_t* sm, int rank, int C) {
    constexpr int VN = Vec16<T>::N;
    constexpr int TILE = 32 * VN;
    __shared__ GRed<T> rs;
    __shared__ T s_alpha;
    __shared__ int s_flag;
    const GProb P = a.gp[p];
    const int n = P.n, ldq = P.ldq;
    // The iterate is a pair y = sy + syl (|syl| ≤ ulp(sy)/2), about 48 bits in
    // the FP32 case: the FP64 refinement rounds then converge to FP64-level
    // KKT residuals instead of stalling at the rounding of y to FP32.
    T* sy = reinterpret_cast<T*>(sm);
    T* syl = sy + ldq;
    T* sg = syl + ldq;
    T* sgb = sg + ldq;
    T* sw = sgb + ldq;  // w = Qḡ, then e (the clipped part of the step)
    int* lp = reinterpret_cast<int*>(sw + ldq);
    int* lc = lp + ldq;
    T* red = reinterpret_cast<T*>(lc + ldq);
    T* xb0 = red + kGWarps * TILE;  // cluster exchange buffers (two, used in turn)
    T* xb1 = xb0 + ldq;
    T* sQ = CL ? xb1 + ldq : xb0;
    const int64_t used = (int64_t)((uint8_t*)sQ - sm);
    const bool qin =
        !CL && (int64_t)n * ldq * (int64_t)sizeof(T) <= (int64_t)a.smem_bytes - used;
    const int S = CL ? ((n + C - 1) / C + TILE - 1) / TILE * TILE : n;
    int pc = 0;  // products so far: selects the exchange buffer
    auto xb = [&]() { return (pc++ & 1) ? xb1 : xb0; };
    const T* Qg = a.Q + P.qoff;
    if (qin) {  // stage Q_p in shared memory for all iterations
        using V = typename Vec16<T>::type;
        const int64_t nv = (int64_t)n * ldq / VN;
        const V* src = reinterpret_cast<const V*>(Qg);
        V* dst = reinterpret_cast<V*>(sQ);
        for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) dst[e] = __ldg(src + e);
    }
    const T* Qp = qin ? sQ : Qg;
    const double* q = a.q64 + P.voff;
    GStat st = a.stat[p];
    const double sf = a.tgt[p] * (a.den[p] > 0.0 ? a.den[p] : 1.0);
    for (int i = threadIdx.x; i < ldq; i += blockDim.x) {
        const double yv = i < n ? a.y[P.foff + i] : 0.0;
        const T yh = (T)yv;
        sy[i] = yh;
        syl[i] = (T)(yv - (double)yh);
        sw[i] = T(0);
        if (a.gmode == 1) sg[i] = i < n ? (T)a.g64[P.voff + i] : T(0);
    }
    __syncthreads();
    // With a cluster, rank 0 alone writes y and the statistics back: no CTA
    // may still be reading them then, or the replicas would start apart.
    if (CL) cluster_sync();
    if (a.gmode == 0) {
        // g = Q y + q (Alg. 2 start; y = 0 gives g = q)
        const int cy = glist(n, sy, lp, &rs);
        product<T, CL>(Qp, ldq, n, lp, cy, sy, sg, false, red, xb(), rank, S);
        for (int i = threadIdx.x; i < n; i += blockDim.x) sg[i] += (T)q[i];
        __syncthreads();
    }

    // step scalars: normalised FP32 pairs in the FP32 kernel (the SM's FP64
    // unit is narrow and up to two 1024-thread blocks share it), FP64 in the
    // FP64 kernel
    using SC = Sc<T>;
    const SC eps = sc_of_double<SC>(sf * sf);
    const int max_iter = a.max_iter, window = a.window;
    const int iter0 = st.iters;
    int iter = st.iters, best_iter = st.iters, status = ALN_RHS_MAXITER;
    SC best = sc_inf<SC>();
    int64_t sum_passive = 0, sum_clip = 0;
    int clip_iters = 0;
    SC gam;
    int cntP, cntL;
    gmask<T, SC>(n, sy, sg, sgb, lp, &rs, &gam, &cntP, &cntL);
    for (;;) {
        if (threadIdx.x == 0) {
            int stop = 1;
            if (!sc_finite(gam)) status = ALN_RHS_NONFINITE;
            else if (cntP == 0) status = ALN_RHS_EMPTY_PASSIVE;
            else if (sc_lt(gam, eps) || sc_zero(gam)) status = ALN_RHS_CONVERGED;
            else if (iter >= max_iter) status = ALN_RHS_MAXITER;
            else if (iter - best_iter > window) status = ALN_RHS_STAGNATED;
            else if (a.budget > 0 && iter - iter0 >= a.budget) status = kRhsPaused;
            else stop = 0;
            if (!stop && sc_lt(gam, best)) {
                best = gam;
                best_iter = iter;
            }
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) break;
        // w = Qḡ over the passive columns, κ = ḡᵀw, α = ‖ḡ‖²/κ (exact line search)
        product<T, CL>(Qp, ldq, n, lp, cntL, sgb, sw, false, red, xb(), rank, S);
        T kp = T(0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) kp = fma(sgb[i], sw[i], kp);
        SC kap;
        int unused_c, unused_l;
        (void)block_totals<T, SC>(&rs, kp, 0, 0, &kap, &unused_c, &unused_l);
        if (threadIdx.x == 0) {
            int stop = 0;
            if (!sc_finite(kap)) {
                status = ALN_RHS_NONFINITE;
                stop = 1;
            } else if (sc_nonpos(kap)) {
                status = ALN_RHS_CURVATURE;
                stop = 1;
            }
            s_alpha = stop ? T(0) : (T)sc_quot(gam, kap);
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) break;
        const T alpha = s_alpha;
        sum_passive += cntP;
        // y⁺ = [y − αḡ]₊, g ← g − αw, e = y⁺ − (y − αḡ) on the clipped set;
        // then g ← g + Q e, so that g = Q y⁺ + q (Q(y⁺ − y) = −αw + Qe)
        int nclip = 0;
        {
            const int lane = threadIdx.x & 31;
            int c0, c1;
            warp_chunks(n, c0, c1);
            int cl = 0;
            for (int c = c0; c < c1; ++c) {
                const int i = c * 32 + lane;
                T ei = T(0);
                if (i < n) {
                    // (yh, yl) − step, exactly: TwoSum, then renormalise
                    const T yh = sy[i], yl = syl[i];
                    const T step = mul_rn(alpha, sgb[i]);
                    const T s1 = yh - step;
                    const T bb = s1 - yh;
                    const T er = (yh - (s1 - bb)) + (-step - bb);
                    const T t = yl + er;
                    T nh = s1 + t;
                    T nl = t - (nh - s1);
                    if (nh < T(0)) {  // clipped: y⁺ = 0, e = y⁺ − (y − αḡ)
                        ei = -(nh + nl);
                        nh = T(0);
                        nl = T(0);
                    }
                    sy[i] = nh;
                    syl[i] = nl;
                    sg[i] = sg[i] - alpha * sw[i];
                    sw[i] = ei;
                }
                cl += __popc(__ballot_sync(0xffffffffu, ei != T(0)));
            }
            double vt;
            int ct;
            int base = block_totals(&rs, T(0), 0, cl, &vt, &ct, &nclip, false);
            for (int c = c0; c < c1; ++c) {
                const int i = c * 32 + lane;
                const bool nz = i < n && sw[i] != T(0);
                const unsigned int m = __ballot_sync(0xffffffffu, nz);
                if (nz) lc[base + __popc(m & ((1u << lane) - 1u))] = i;
                base += __popc(m);
            }
            __syncthreads();
        }
        ++iter;
        sum_clip += nclip;
        if (nclip > 0) {
            if (CL && nclip <= 8)  // a few rows: every CTA forms Qe itself, no exchange
                gmv(Qp, ldq, 0, n, lc, nclip, sw, sg, true, red);
            else
                product<T, CL>(Qp, ldq, n, lc, nclip, sw, sg, true, red, xb(), rank, S);
            ++clip_iters;
        }
        gmask<T, SC>(n, sy, sg, sgb, lp, &rs, &gam, &cntP, &cntL);
    }
    if (!CL || rank == 0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            a.y[P.foff + i] = (double)sy[i] + (double)syl[i];
            if (a.gout) a.gout[P.voff + i] = (double)sg[i];
        }
    if (threadIdx.x == 0 && (!CL || rank == 0)) {
        st.iters = iter;
        st.status = status;
        st.clip_iters += clip_iters;
        st.npassive = cntP;
        st.sum_passive += sum_passive;
        st.sum_clip += sum_clip;
        st.gbar2 = sc_double(gam);
        a.stat[p] = st;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kGThreads, 1) k_galg2(GSolveArgs<T> a) {
    extern __shared__ __align__(16) uint8_t gsm[];
    __shared__ int s_p;
    for (;;) {
        if (threadIdx.x == 0) {
            int p;
            do {
                const int k = atomicAdd(a.queue, 1);
                p = k < a.nactive ? a.order[k] : -1;
            } while (p >= 0 && a.run && a.run[p] == 0);
            s_p = p;
        }
        __syncthreads();
        const int p = s_p;
        __syncthreads();
        if (p < 0) break;
        solve_one<T, false>(a, p, gsm, 0, 1);
    }
}

// Large problems: one problem per thread-block cluster (launched with a
// cluster dimension); rank 0 takes the next problem and writes its index
// into every CTA of the cluster.
template <typename T>
__global__ void __launch_bounds__(kGThreads, 1) k_galg2c(GSolveArgs<T> a) {
    extern __shared__ __align__(16) uint8_t gsm[];
    __shared__ int s_p;
    const int rank = cluster_rank(), C = cluster_ctas();
    cluster_sync();  // every CTA of the cluster has started
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            int p;
            do {
                const int k = atomicAdd(a.queue, 1);
                p = k < a.nactive ? a.order[k] : -1;
            } while (p >= 0 && a.run && a.run[p] == 0);
            for (int r = 0; r < C; ++r) st_cluster(cluster_addr(&s_p, r), p);
        }
        cluster_sync();
        const int p = s_p;
        if (p < 0) break;
        solve_one<T, true>(a, p, gsm, rank, C);
        // every CTA is done with s_p and with the exchange buffers before
        // rank 0 writes the next index and the next problem reuses them
        cluster_sync();
    }
}

// Shared memory of solve_one besides Q_p (the cluster variant adds its two
// exchange buffers).
template <typename T>
size_t gsolve_static_bytes(int ldq, bool cluster) {
    constexpr int TILE = 32 * Vec16<T>::N;
    return (size_t)ldq * ((cluster ? 7 : 5) * sizeof(T) + 2 * sizeof(int)) +
           (size_t)kGWarps * TILE * sizeof(T);
}

// y = x0·s (or 0), per problem.
__global__ void k_ginit(const GProb* __restrict__ gp, int count, int64_t total,
                        const double* __restrict__ x0, const double* __restrict__ s,
                        double* __restrict__ y, GStat* __restrict__ stat, int* __restrict__ fin,
                        int* __restrict__ rounds, double* __restrict__ tgt, double t0) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_prob<kKeyV>(gp, count, e);
        const GProb& P = gp[p];
        const int j = (int)(e - P.voff);
        y[P.foff + j] = x0 ? x0[e] * s[e] : 0.0;
        if (j == 0) {
            GStat z = {};
            stat[p] = z;
            fin[p] = -1;
            rounds[p] = 0;
            tgt[p] = t0;
        }
    }
}

// x = y/s (Eq. Rescaling), FP64.
__global__ void k_gunscale(const GProb* __restrict__ gp, int count, int64_t total,
                           const double* __restrict__ y, const double* __restrict__ s,
                           double* __restrict__ x) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_prob<kKeyV>(gp, count, e);
        const GProb& P = gp[p];
        x[e] = y[P.foff + (e - P.voff)] / s[e];
    }
}

// ---------------------------------------------------------------------------
// FP64 KKT from A for the problems still open (fin < 0)
// ---------------------------------------------------------------------------
// r = A x − b, one thread per row of every open problem.
template <typename TA>
__global__ void __launch_bounds__(256) k_gkkt_r(const GProb* __restrict__ gp, int count,
                                                int64_t total, const double* __restrict__ x,
                                                const int* __restrict__ fin,
                                                double* __restrict__ r) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_prob<kKeyR>(gp, count, e);
        if (fin[p] >= 0) continue;
        const GProb& P = gp[p];
        const int i = (int)(e - P.roff);
        const TA* A = (const TA*)P.A;
        const double* xp = x + P.voff;
        double acc = -(double)((const TA*)P.b)[i];
        for (int j = 0; j < P.n; ++j) {
            const double xj = xp[j];
            if (xj != 0.0) acc = fma((double)A[(int64_t)j * P.lda + i], xj, acc);
        }
        r[e] = acc;
    }
}

// ∇F_j = A_jᵀr, g_j = ∇F_j/s_j, ḡ_j² on P(y = s·x): one warp per column.
template <typename TA>
__global__ void __launch_bounds__(256) k_gkkt_g(const GProb* __restrict__ gp, int count,
                                                int64_t total, const double* __restrict__ x,
                                                const double* __restrict__ s,
                                                const double* __restrict__ r,
                                                const int* __restrict__ fin,
                                                double* __restrict__ g64,
                                                double* __restrict__ gpart) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total;
         e += warps) {
        const int p = find_prob<kKeyV>(gp, count, e);
        if (fin[p] >= 0) continue;
        const GProb& P = gp[p];
        const int j = (int)(e - P.voff);
        const TA* col = (const TA*)P.A + (int64_t)j * P.lda;
        const double* rp = r + P.roff;
        double acc = 0.0;
        for (int i = lane; i < P.d; i += 32) acc = fma((double)col[i], rp[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
            const double gj = acc / s[e];
            const double yj = x[e] * s[e];
            const bool Pj = yj > 0.0 || gj < 0.0;
            g64[e] = gj;
            gpart[e] = Pj ? gj * gj : 0.0;
        }
    }
}

// FP32 inputs: the same two passes on the FP32 pipe with FP64-level accuracy
// (Dot2: x and r as FP32 pairs hi + lo, exact products by FMA, TwoSum), since
// FP64 FMAs on this GPU made them compute-bound.
__global__ void k_gsplit(const double* __restrict__ v, int64_t m, float* __restrict__ hi,
                         float* __restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)v[i];
        hi[i] = h;
        lo[i] = (float)(v[i] - (double)h);
    }
}

struct GPair {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a, float h, float l) {  // += a·(h + l)
        const float p = mul_rn(a, h);
        const float ep = fmaf(a, h, -p);
        const float t = s + p;
        const float z = t - s;
        c += ((s - (t - z)) + (p - z)) + fmaf(a, l, ep);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__global__ void __launch_bounds__(256) k_gkkt_r32(const GProb* __restrict__ gp, int count,
                                                  int64_t total, const float* __restrict__ xh,
                                                  const float* __restrict__ xl,
                                                  const int* __restrict__ fin,
                                                  double* __restrict__ r) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_prob<kKeyR>(gp, count, e);
        if (fin[p] >= 0) continue;
        const GProb& P = gp[p];
        const int i = (int)(e - P.roff);
        const float* A = (const float*)P.A;
        const float* h = xh + P.voff;
        const float* l = xl + P.voff;
        GPair acc;
        for (int j = 0; j < P.n; ++j) {
            const float hj = h[j], lj = l[j];
            if (hj != 0.0f || lj != 0.0f) acc.add(A[(int64_t)j * P.lda + i], hj, lj);
        }
        r[e] = acc.value() - (double)((const float*)P.b)[i];
    }
}

__global__ void __launch_bounds__(256) k_gkkt_g32(const GProb* __restrict__ gp, int count,
                                                  int64_t total, const double* __restrict__ x,
                                                  const double* __restrict__ s,
                                                  const float* __restrict__ rh,
                                                  const float* __restrict__ rl,
                                                  const int* __restrict__ fin,
                                                  double* __restrict__ g64,
                                                  double* __restrict__ gpart) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total;
         e += warps) {
        const int p = find_prob<kKeyV>(gp, count, e);
        if (fin[p] >= 0) continue;
        const GProb& P = gp[p];
        const int j = (int)(e - P.voff);
        const float* col = (const float*)P.A + (int64_t)j * P.lda;
        GPair acc;
        for (int i = lane; i < P.d; i += 32) acc.add(col[i], rh[P.roff + i], rl[P.roff + i]);
        const double v = warp_sum(acc.value());
        if (lane == 0) {
            const double gj = v / s[e];
            const double yj = x[e] * s[e];
            const bool Pj = yj > 0.0 || gj < 0.0;
            g64[e] = gj;
            gpart[e] = Pj ? gj * gj : 0.0;
        }
    }
}

// Per open problem: rel_kkt = ‖ḡ‖/‖min(q,0)‖, F = ½‖r‖², and the decision:
// converged, terminal, or one more round from the exact gradient.
__global__ void __launch_bounds__(256) k_gkkt_final(const GProb* __restrict__ gp,
                                                    const double* __restrict__ gpart,
                                                    const double* __restrict__ r,
                                                    const double* __restrict__ den,
                                                    const GStat* __restrict__ stat, double tol,
                                                    int max_iter, int max_refine, int gain,
                                                    int refining, int* __restrict__ fin,
                                                    int* __restrict__ rounds,
                                                    double* __restrict__ tgt,
                                                    int* __restrict__ again,
                                                    double* __restrict__ rel_out,
                                                    double* __restrict__ obj_out) {
    __shared__ double scratch[32];
    const int p = blockIdx.x;
    if (fin[p] >= 0) return;
    const GProb P = gp[p];
    double g2 = 0.0, r2 = 0.0;
    for (int j = threadIdx.x; j < P.n; j += blockDim.x) g2 += gpart[P.voff + j];
    for (int i = threadIdx.x; i < P.d; i += blockDim.x) {
        const double ri = r[P.roff + i];
        r2 = fma(ri, ri, r2);
    }
    g2 = block_sum(g2, scratch);
    r2 = block_sum(r2, scratch);
    if (threadIdx.x == 0) {
        const double num = sqrt(g2);
        const double rel = den[p] > 0.0 ? num / den[p] : num;
        rel_out[p] = rel;
        obj_out[p] = 0.5 * r2;
        const int inner = stat[p].status;
        int f = -1;
        if (!refining) {
            f = ALN_RHS_CONVERGED;  // evaluation only (aln_kkt_residual)
        } else if (rel <= tol) {
            f = inner == ALN_RHS_EMPTY_PASSIVE ? ALN_RHS_EMPTY_PASSIVE : ALN_RHS_CONVERGED;
        } else if (inner == ALN_RHS_NONFINITE || inner == ALN_RHS_MAXITER ||
                   stat[p].iters >= max_iter) {
            f = inner == ALN_RHS_NONFINITE ? ALN_RHS_NONFINITE : ALN_RHS_MAXITER;
        } else if (rounds[p] >= max_refine) {
            f = inner == ALN_RHS_STAGNATED ? ALN_RHS_STAGNATED : ALN_RHS_MAXITER;
        } else {
            rounds[p] += 1;
            tgt[p] = inner_target(tol, kGRefineFactor, rel, gain);  // next run: from the exact gradient
        }
        if (f >= 0) fin[p] = f;
        again[p] = f < 0 ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct GroupWork {
    int count = 0;
    int32_t dtype = ALN_DTYPE_F32;
    int64_t sum_n = 0, sum_d = 0, sum_f = 0, sum_nn = 0;
    int max_ldq = 0;
    std::vector<GProb> hp;        // host copy of the records
    std::vector<int> order_all;   // problems, largest n first
    std::vector<int> run_order;   // host copy of order for the current run
    std::vector<int64_t> qexp;    // offsets of the exported packed Q blocks

    void* pool = nullptr;         // device: everything below
    size_t pool_bytes = 0;
    GProb* gp = nullptr;
    GTile* tiles = nullptr;
    int64_t ntiles = 0;
    int* order = nullptr;
    int* queue = nullptr;
    int* fin = nullptr;
    int* rounds = nullptr;
    int* again = nullptr;
    int* flags = nullptr;         // [0] nonfinite input, [1] tensor-core timeout
    int64_t* qexp_dev = nullptr;
    GStat* stat = nullptr;
    double *s = nullptr, *inv_s = nullptr, *q64 = nullptr, *g64 = nullptr, *x64 = nullptr,
           *gpart = nullptr, *r64 = nullptr, *den = nullptr, *bn2 = nullptr, *rel = nullptr,
           *obj = nullptr, *tgt = nullptr;
    float *xh = nullptr, *xl = nullptr, *rh = nullptr, *rl = nullptr;  // FP32 pairs
    void* y = nullptr;            // packed (foff), iteration type
    void* Q = nullptr;            // pool, iteration type
    __nv_bfloat16 *hi = nullptr, *mid = nullptr, *lo = nullptr;

    void* copies = nullptr;       // device copies of host inputs
    size_t copies_bytes = 0;
    void* host = nullptr;         // pinned: again/fin/rounds, rel, obj, stat
    size_t host_bytes = 0;
    int smem_bytes = 0;
    int grid = 0;
    int nbig = 0;                   // leading entries of order solved by clusters
    int max_clusters = -1;          // co-resident clusters of k_galg2c (-1: not asked yet)
    int cluster_size = 0;           // blocks per cluster that max_clusters is for
    cudaStream_t side = nullptr;    // second stream: k_galg2 beside k_galg2c
    cudaEvent_t fork = nullptr, join = nullptr;
    int64_t slots = 0;              // column slots of the prepare grid
    std::vector<aln_problem> last;  // records of the last layout
    int last_prec = -1;
    bool reuse_ok = false;          // last layout used device inputs only
    // graph of the whole solve (aln_options.group_graph): the rounds as one
    // captured launch sequence, valid for the key it was captured with
    cudaGraphExec_t graph = nullptr;
    double graph_tol = -1.0;
    int graph_max_iter = -1, graph_x0 = -1, graph_cs = -1;
};

bool is_dev(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

aln_status cuda_err(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return ALN_ERR_OUT_OF_MEMORY;
    }
    return ALN_ERR_CUDA;
}
#define G_TRY(call)                                    \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_err(e_);    \
    } while (0)
#define G_CHECK(call)                 \
    do {                              \
        aln_status s_ = (call);       \
        if (s_ != ALN_OK) return s_;  \
    } while (0)

aln_status grow(void** p, size_t* cap, size_t bytes) {
    if (*p && *cap >= bytes) return ALN_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ALN_ERR_OUT_OF_MEMORY;
    }
    *cap = bytes;
    return ALN_OK;
}

unsigned grid_for(int64_t work, int threads, int cap) {
    const int64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// Host-side state of the solver launches, made once before any of them (and
// before a stream capture): the side stream with its events, and the number
// of co-resident clusters of k_galg2c for the current cluster size.
template <typename T>
aln_status launch_state(aln_ctx* c, GroupWork* g) {
    if (!g->side) {
        G_TRY(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
        G_TRY(cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
        G_TRY(cudaEventCreateWithFlags(&g->join, cudaEventDisableTiming));
    }
    G_TRY(cudaFuncSetAttribute(k_galg2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               g->smem_bytes));
    G_TRY(cudaFuncSetAttribute(k_galg2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               g->smem_bytes));
    if (g->max_clusters < 0 && g->cluster_size > 1) {
        const int CS = g->cluster_size;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(kGThreads);
        cfg.dynamicSmemBytes = g->smem_bytes;
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(CS * (c->num_sms / CS));
        int m = 0;
        if (cudaOccupancyMaxActiveClusters(&m, k_galg2c<T>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            m = 0;
        }
        g->max_clusters = m;
    }
    return ALN_OK;
}

template <typename T>
aln_status run_solver(aln_ctx* c, GroupWork* g, int nactive, int gmode, int max_iter,
                      const int* run = nullptr) {
    GSolveArgs<T> a;
    a.run = run;
    a.budget = 0;
    a.gout = nullptr;
    a.gp = g->gp;
    a.order = g->order;
    a.nactive = nactive;
    a.queue = g->queue;
    a.Q = (const T*)g->Q;
    a.q64 = g->q64;
    a.g64 = g->g64;
    a.den = g->den;
    a.y = (double*)g->y;
    a.stat = g->stat;
    a.tgt = g->tgt;
    a.gmode = gmode;
    a.max_iter = max_iter;
    a.window = c->opt.stagnation;
    a.smem_bytes = g->smem_bytes;
    G_TRY(cudaFuncSetAttribute(k_galg2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               g->smem_bytes));
    G_TRY(cudaMemsetAsync(g->queue, 0, 2 * sizeof(int), c->stream));
    const int nbig = std::min(g->nbig, nactive), nsmall = nactive - nbig;
    const int CS = g->cluster_size;
    int ncl = 0;
    if (nbig > 0) {
        G_TRY(cudaFuncSetAttribute(k_galg2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   g->smem_bytes));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(kGThreads);
        cfg.dynamicSmemBytes = g->smem_bytes;
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (g->max_clusters < 0) {
            cfg.gridDim = dim3(CS * (c->num_sms / CS));
            int m = 0;
            if (cudaOccupancyMaxActiveClusters(&m, k_galg2c<T>, &cfg) != cudaSuccess) {
                cudaGetLastError();
                m = 0;
            }
            g->max_clusters = m;
        }
        // clusters for the large problems in proportion to their share of
        // the work (Σ n² per iteration), the other SMs for the rest
        double wb = 0.0, wt = 0.0;
        for (int k = 0; k < nactive; ++k) {
            const double n = (double)g->hp[g->run_order[k]].n;
            wt += n * n;
            if (k < nbig) wb += n * n;
        }
        ncl = (int)std::lround(wb / std::max(wt, 1.0) * c->num_sms / CS);
        ncl = std::max(1, std::min({ncl, nbig, g->max_clusters}));
        if (nsmall == 0) ncl = std::min(nbig, g->max_clusters);
        if (g->max_clusters <= 0) ncl = 0;  // no cluster fits: one kernel for all
    }
    if (ncl > 0) {
        if (!g->side) {
            G_TRY(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
            G_TRY(cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming));
            G_TRY(cudaEventCreateWithFlags(&g->join, cudaEventDisableTiming));
        }
        G_TRY(cudaEventRecord(g->fork, c->stream));
        GSolveArgs<T> b = a;
        b.nactive = nbig;
        b.queue = g->queue + 1;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(CS * ncl);
        cfg.blockDim = dim3(kGThreads);
        cfg.dynamicSmemBytes = g->smem_bytes;
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        G_TRY(cudaLaunchKernelEx(&cfg, k_galg2c<T>, b));
        c->launches += 1;
        if (nsmall > 0) {
            G_TRY(cudaStreamWaitEvent(g->side, g->fork, 0));
            a.order = g->order + nbig;
            a.nactive = nsmall;
            const int grid = std::max(1, std::min(nsmall, g->grid - CS * ncl));
            k_galg2<T><<<grid, kGThreads, g->smem_bytes, g->side>>>(a);
            G_TRY(cudaGetLastError());
            c->launches += 1;
            G_TRY(cudaEventRecord(g->join, g->side));
            G_TRY(cudaStreamWaitEvent(c->stream, g->join, 0));
        }
        return ALN_OK;
    }
    const int grid = std::min(nactive, g->grid);
    k_galg2<T><<<grid, kGThreads, g->smem_bytes, c->stream>>>(a);
    G_TRY(cudaGetLastError());
    c->launches += 1;
    return ALN_OK;
}

// Upload the order of the next run: the problems that clusters solve
// (largest first) ahead of the rest (largest first); sets g->nbig.
aln_status upload_order(aln_ctx* c, GroupWork* g, const std::vector<int>& list) {
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    g->run_order.clear();
    g->nbig = 0;
    const int cs = c->opt.group_cluster ? c->opt.group_cluster : kGCluster;
    if (cs != g->cluster_size) {
        g->cluster_size = cs;
        g->max_clusters = -1;
    }
    for (int pass = 0; pass < 2; ++pass)
        for (int p : list) {
            const GProb& P = g->hp[p];
            const size_t T = f64 ? 8 : 4;
            const size_t st = f64 ? gsolve_static_bytes<double>(P.ldq, true)
                                  : gsolve_static_bytes<float>(P.ldq, true);
            const size_t st1 = f64 ? gsolve_static_bytes<double>(P.ldq, false)
                                   : gsolve_static_bytes<float>(P.ldq, false);
            const bool fits = (size_t)P.n * P.ldq * T + st1 <= (size_t)g->smem_bytes;
            const bool big = cs > 1 && P.n >= kGClusterMinN && !fits &&
                             st <= (size_t)g->smem_bytes && g->max_clusters != 0;
            if (big == (pass == 0)) g->run_order.push_back(p);
            if (pass == 0 && big) g->nbig = (int)g->run_order.size();
        }
    if (g->run_order.empty()) return ALN_OK;
    G_TRY(cudaMemcpyAsync(g->order, g->run_order.data(), g->run_order.size() * sizeof(int),
                          cudaMemcpyHostToDevice, c->stream));
    return ALN_OK;
}

aln_status kkt_pass(aln_ctx* c, GroupWork* g, double tol, int max_iter, int max_refine,
                    int refining) {
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    const unsigned gr = grid_for(g->sum_d, 256, 8 * c->num_sms);
    const unsigned gg = grid_for(g->sum_n * 32, 256, 16 * c->num_sms);
    if (g->dtype == ALN_DTYPE_F32) {
        const unsigned gs = grid_for(std::max(g->sum_n, g->sum_d), 256, 8 * c->num_sms);
        k_gsplit<<<gs, 256, 0, c->stream>>>(g->x64, g->sum_n, g->xh, g->xl);
        k_gkkt_r32<<<gr, 256, 0, c->stream>>>(g->gp, g->count, g->sum_d, g->xh, g->xl, g->fin,
                                              g->r64);
        k_gsplit<<<gs, 256, 0, c->stream>>>(g->r64, g->sum_d, g->rh, g->rl);
        k_gkkt_g32<<<gg, 256, 0, c->stream>>>(g->gp, g->count, g->sum_n, g->x64, g->s, g->rh,
                                              g->rl, g->fin, g->g64, g->gpart);
        c->launches += 2;
    } else {
        k_gkkt_r<double><<<gr, 256, 0, c->stream>>>(g->gp, g->count, g->sum_d, g->x64, g->fin,
                                                    g->r64);
        k_gkkt_g<double><<<gg, 256, 0, c->stream>>>(g->gp, g->count, g->sum_n, g->x64, g->s,
                                                    g->r64, g->fin, g->g64, g->gpart);
    }
    k_gkkt_final<<<g->count, 256, 0, c->stream>>>(g->gp, g->gpart, g->r64, g->den, g->stat, tol,
                                                  max_iter, max_refine,
                                                  (f64 || c->opt.refine_gain == 0)
                                                      ? -1
                                                      : c->opt.refine_gain,
                                                  refining, g->fin, g->rounds, g->tgt, g->again,
                                                  g->rel, g->obj);
    G_TRY(cudaGetLastError());
    c->launches += 3;
    return ALN_OK;
}

}  // namespace

size_t tail_smem_bytes(int64_t ldq, bool cluster) {
    return (size_t)round_up(gsolve_static_bytes<float>((int)ldq, cluster), 128);
}

// Alg. 2 on `count` columns that share one FP32 Q (the batched solver's
// tail): column order[i] is problem order[i] of the grouped kernels (gp holds
// one record per column: qoff 0, voff = foff = column·ldq), solved by one CTA
// (cs = 1) or by a cluster of cs CTAs, from y (FP64, in/out) and the
// gradient g (FP64, in/out: the batched phase's FP32 gradient carried on, not
// re-formed from y, whose FP32 product would cost the accuracy the refinement
// rounds buy); budget > 0 pauses a column after that many iterations of this
// launch (status kRhsPaused).
aln_status tail_launch(aln_ctx* c, const GProb* gp, const int* order, int count, int* queue,
                       const float* Q, int64_t ldq, const double* q64, const double* den,
                       double* y, double* g, GStat* stat, const double* tgt, int max_iter,
                       int budget, int cs) {
    if (count <= 0) return ALN_OK;
    if (cs != 1 && cs != 2 && cs != 4 && cs != 8) return ALN_ERR_INVALID_ARG;
    GSolveArgs<float> a;
    a.gp = gp;
    a.order = order;
    a.nactive = count;
    a.queue = queue;
    a.Q = Q;
    a.q64 = q64;
    a.g64 = g;
    a.gout = g;
    a.den = den;
    a.y = y;
    a.stat = stat;
    a.tgt = tgt;
    a.gmode = 1;
    a.max_iter = max_iter;
    a.window = c->opt.stagnation;
    a.run = nullptr;
    a.budget = budget;
    a.smem_bytes = (int)tail_smem_bytes(ldq, cs > 1);
    G_TRY(cudaMemsetAsync(queue, 0, sizeof(int), c->stream));
    if (cs == 1) {
        G_TRY(cudaFuncSetAttribute(k_galg2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   a.smem_bytes));
        const unsigned grid = (unsigned)std::min(count, c->num_sms);
        k_galg2<float><<<grid, kGThreads, a.smem_bytes, c->stream>>>(a);
        G_TRY(cudaGetLastError());
        c->launches += 1;
        return ALN_OK;
    }
    G_TRY(cudaFuncSetAttribute(k_galg2c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               a.smem_bytes));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kGThreads);
    cfg.dynamicSmemBytes = a.smem_bytes;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(cs * (c->num_sms / cs));
    int m = 0;
    if (cudaOccupancyMaxActiveClusters(&m, k_galg2c<float>, &cfg) != cudaSuccess || m <= 0) {
        cudaGetLastError();
        return ALN_ERR_UNSUPPORTED;
    }
    cfg.gridDim = dim3(cs * std::min(count, m));
    G_TRY(cudaLaunchKernelEx(&cfg, k_galg2c<float>, a));
    c->launches += 1;
    return ALN_OK;
}

void group_shape(const aln_ctx* c, int* count, int64_t* sum_n, int64_t* max_n) {
    const GroupWork* g = (const GroupWork*)c->group;
    *count = g->count;
    *sum_n = g->sum_n;
    int64_t m = 0;
    for (int p = 0; p < g->count; ++p) m = std::max<int64_t>(m, g->hp[p].n);
    *max_n = m;
}

void group_free(aln_ctx* c) {
    GroupWork* g = (GroupWork*)c->group;
    if (!g) return;
    if (g->pool) cudaFree(g->pool);
    if (g->copies) cudaFree(g->copies);
    if (g->host) cudaFreeHost(g->host);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->join) cudaEventDestroy(g->join);
    if (g->side) cudaStreamDestroy(g->side);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    delete g;
    c->group = nullptr;
    c->grouped = 0;
}

// Layout, device pool and records of a new group (host inputs are copied).
static aln_status group_layout(aln_ctx* c, GroupWork* g, int32_t count, const aln_problem* probs,
                        int32_t dtype) {
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    const size_t esz = dtype == ALN_DTYPE_F64 ? 8 : 4;
    const size_t T = f64 ? 8 : 4;
    g->count = count;
    g->dtype = dtype;
    g->hp.assign(count, GProb{});

    // host inputs → one device block of copies
    size_t copy_bytes = 0;
    std::vector<char> a_dev(count), b_dev(count);
    for (int p = 0; p < count; ++p) {
        const aln_problem& q = probs[p];
        a_dev[p] = is_dev(q.A);
        b_dev[p] = is_dev(q.b);
        if (!a_dev[p]) copy_bytes += round_up((size_t)((q.n - 1) * q.lda + q.d) * esz, 256);
        if (!b_dev[p]) copy_bytes += round_up((size_t)q.d * esz, 256);
    }
    if (copy_bytes) G_CHECK(grow(&g->copies, &g->copies_bytes, copy_bytes));
    uint8_t* cp = (uint8_t*)g->copies;

    // layout of every problem
    int64_t slot = 0, pack = 0, qoff = 0, voff = 0, foff = 0, roff = 0, nn = 0;
    g->qexp.assign(count, 0);
    g->max_ldq = 0;
    std::vector<GTile> tiles;
    for (int p = 0; p < count; ++p) {
        const aln_problem& q = probs[p];
        GProb& P = g->hp[p];
        P.lda = q.lda;
        P.d = (int32_t)q.d;
        P.n = (int32_t)q.n;
        P.T = (int32_t)ceil_div(q.n, 128);
        P.KB = (int32_t)ceil_div(q.d, 64);
        P.ldq = (int32_t)round_up(q.n, 4);
        P.slot = slot;
        P.pack = pack;
        P.qoff = qoff;
        P.voff = voff;
        P.foff = foff;
        P.roff = roff;
        g->qexp[p] = nn;
        slot += 128 * (int64_t)P.T;
        pack += (int64_t)P.T * P.KB;
        qoff += (int64_t)P.n * P.ldq;
        voff += P.n;
        foff += P.ldq;
        roff += P.d;
        nn += (int64_t)P.n * P.n;
        g->max_ldq = std::max(g->max_ldq, P.ldq);
        if (a_dev[p]) {
            P.A = q.A;
        } else {
            const size_t bytes = (size_t)((q.n - 1) * q.lda + q.d) * esz;
            G_TRY(cudaMemcpyAsync(cp, q.A, bytes, cudaMemcpyHostToDevice, c->stream));
            P.A = cp;
            cp += round_up(bytes, 256);
        }
        if (b_dev[p]) {
            P.b = q.b;
        } else {
            const size_t bytes = (size_t)q.d * esz;
            G_TRY(cudaMemcpyAsync(cp, q.b, bytes, cudaMemcpyHostToDevice, c->stream));
            P.b = cp;
            cp += round_up(bytes, 256);
        }
        for (int tm = 0; tm < P.T; ++tm)
            for (int tn = 0; tn <= tm; ++tn) tiles.push_back(GTile{p, tm, tn, 0});
    }
    g->sum_n = voff;
    g->sum_d = roff;
    g->sum_f = foff;
    g->sum_nn = nn;
    // longest K first, so the long tiles do not end up in the last wave
    std::stable_sort(tiles.begin(), tiles.end(), [&](const GTile& x, const GTile& y) {
        return g->hp[x.p].KB > g->hp[y.p].KB;
    });
    g->ntiles = f64 ? 0 : (int64_t)tiles.size();
    g->order_all.resize(count);
    std::iota(g->order_all.begin(), g->order_all.end(), 0);
    std::stable_sort(g->order_all.begin(), g->order_all.end(), [&](int x, int y) {
        return g->hp[x].n > g->hp[y].n;
    });

    // device pool
    const size_t pack_elems = f64 ? 0 : (size_t)pack * kPackTile;
    size_t sizes[] = {
        (size_t)count * sizeof(GProb),                 // gp
        (size_t)std::max<int64_t>(g->ntiles, 1) * sizeof(GTile),  // tiles
        (size_t)count * sizeof(int),                   // order
        sizeof(int) * 4,                               // queue
        (size_t)count * sizeof(int),                   // fin
        (size_t)count * sizeof(int),                   // rounds
        (size_t)count * sizeof(int),                   // again
        sizeof(int) * 4,                               // flags
        (size_t)count * sizeof(int64_t),               // qexp
        (size_t)count * sizeof(GStat),                 // stat
        (size_t)voff * 8, (size_t)voff * 8, (size_t)voff * 8, (size_t)voff * 8,
        (size_t)voff * 8, (size_t)voff * 8,            // s, inv_s, q64, g64, x64, gpart
        (size_t)roff * 8,                              // r64
        (size_t)count * 8, (size_t)count * 8, (size_t)count * 8, (size_t)count * 8,  // den bn2 rel obj
        (size_t)count * 8,                             // tgt
        (size_t)voff * 4, (size_t)voff * 4, (size_t)roff * 4, (size_t)roff * 4,  // pairs
        (size_t)foff * 8,                              // y (FP64)
        (size_t)qoff * T,                              // Q
        pack_elems * 2, pack_elems * 2, pack_elems * 2,  // hi, mid, lo
    };
    const int nsz = (int)(sizeof(sizes) / sizeof(sizes[0]));
    size_t total = 0;
    for (int i = 0; i < nsz; ++i) total += round_up(sizes[i], 256);
    G_CHECK(grow(&g->pool, &g->pool_bytes, total));
    {
        uint8_t* p = (uint8_t*)g->pool;
        int k = 0;
        auto take = [&]() {
            void* r = p;
            p += round_up(sizes[k++], 256);
            return r;
        };
        g->gp = (GProb*)take();
        g->tiles = (GTile*)take();
        g->order = (int*)take();
        g->queue = (int*)take();
        g->fin = (int*)take();
        g->rounds = (int*)take();
        g->again = (int*)take();
        g->flags = (int*)take();
        g->qexp_dev = (int64_t*)take();
        g->stat = (GStat*)take();
        g->s = (double*)take();
        g->inv_s = (double*)take();
        g->q64 = (double*)take();
        g->g64 = (double*)take();
        g->x64 = (double*)take();
        g->gpart = (double*)take();
        g->r64 = (double*)take();
        g->den = (double*)take();
        g->bn2 = (double*)take();
        g->rel = (double*)take();
        g->obj = (double*)take();
        g->tgt = (double*)take();
        g->xh = (float*)take();
        g->xl = (float*)take();
        g->rh = (float*)take();
        g->rl = (float*)take();
        g->y = take();
        g->Q = take();
        g->hi = (__nv_bfloat16*)take();
        g->mid = (__nv_bfloat16*)take();
        g->lo = (__nv_bfloat16*)take();
        if (k != nsz || (size_t)(p - (uint8_t*)g->pool) != total) return ALN_ERR_CUDA;
    }
    // pinned host mirror: again, fin, rounds (ints), rel, obj (doubles), stat
    const size_t hb = round_up((size_t)count * 12, 64) + (size_t)count * 16 +
                      (size_t)count * sizeof(GStat) + 64;
    if (g->host_bytes < hb) {
        if (g->host) cudaFreeHost(g->host);
        g->host = nullptr;
        g->host_bytes = 0;
        if (cudaMallocHost(&g->host, hb) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
        g->host_bytes = hb;
    }

    // solver geometry: one block per SM, shared memory as large as allowed
    int optin = 0;
    G_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    g->smem_bytes = optin - 1024;  // static shared memory of the kernel
    const size_t need = f64 ? gsolve_static_bytes<double>(g->max_ldq, false)
                            : gsolve_static_bytes<float>(g->max_ldq, false);
    if ((size_t)g->smem_bytes < need) return ALN_ERR_UNSUPPORTED;
    g->grid = c->num_sms;
    g->slots = slot;

    G_TRY(cudaMemcpyAsync(g->gp, g->hp.data(), (size_t)count * sizeof(GProb),
                          cudaMemcpyHostToDevice, c->stream));
    if (g->ntiles)
        G_TRY(cudaMemcpyAsync(g->tiles, tiles.data(), (size_t)g->ntiles * sizeof(GTile),
                              cudaMemcpyHostToDevice, c->stream));
    G_TRY(cudaMemcpyAsync(g->qexp_dev, g->qexp.data(), (size_t)count * sizeof(int64_t),
                          cudaMemcpyHostToDevice, c->stream));
    G_TRY(cudaMemsetAsync(g->Q, 0, (size_t)qoff * T, c->stream));
    // remember the records: a later prepare of the same device buffers (new
    // contents, same shapes and addresses) reuses this layout as it is
    bool all_dev = true;
    for (int p = 0; p < count; ++p) all_dev = all_dev && a_dev[p] && b_dev[p];
    g->reuse_ok = all_dev;
    g->last.assign(probs, probs + count);
    g->last_prec = c->opt.precision;
    return ALN_OK;
}

aln_status group_prepare(aln_ctx* c, int32_t count, const aln_problem* probs, int32_t dtype) {
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    for (int p = 0; p < count; ++p)
        if (probs[p].n > kGMaxN) return ALN_ERR_INVALID_ARG;
    GroupWork* g = (GroupWork*)c->group;
    if (!g) {
        g = new (std::nothrow) GroupWork();
        if (!g) return ALN_ERR_OUT_OF_MEMORY;
        c->group = g;
    }
    const bool same = g->reuse_ok && g->pool && g->count == count && g->dtype == dtype &&
                      g->last_prec == c->opt.precision && g->last.size() == (size_t)count &&
                      std::memcmp(g->last.data(), probs, sizeof(aln_problem) * count) == 0;
    G_TRY(cudaEventRecord(c->ev[0], c->stream));
    if (!same) {
        g->reuse_ok = false;
        if (g->graph) cudaGraphExecDestroy(g->graph);  // its pointers are the old layout's
        g->graph = nullptr;
        G_CHECK(group_layout(c, g, count, probs, dtype));
    }
    G_TRY(cudaMemsetAsync(g->flags, 0, 4 * sizeof(int), c->stream));
    const unsigned slots = (unsigned)g->slots;
    if (dtype == ALN_DTYPE_F32)
        k_gcolstats<float><<<slots, 128, 0, c->stream>>>(g->gp, count, f64 ? 0 : 1, g->s,
                                                         g->inv_s, g->q64, g->flags, g->hi,
                                                         g->mid, g->lo);
    else
        k_gcolstats<double><<<slots, 128, 0, c->stream>>>(g->gp, count, f64 ? 0 : 1, g->s,
                                                          g->inv_s, g->q64, g->flags, g->hi,
                                                          g->mid, g->lo);
    if (dtype == ALN_DTYPE_F32)
        k_gden<float><<<count, 256, 0, c->stream>>>(g->gp, g->q64, g->den, g->bn2);
    else
        k_gden<double><<<count, 256, 0, c->stream>>>(g->gp, g->q64, g->den, g->bn2);
    G_TRY(cudaGetLastError());
    c->launches += 2;
    G_TRY(cudaEventRecord(c->ev[1], c->stream));
    if (f64) {
        // the plain method: FP64 Gram per problem
        for (int p = 0; p < count; ++p) {
            const GProb& P = g->hp[p];
            G_TRY(launch_gram64(P.A, dtype, P.d, P.n, P.lda, g->inv_s + P.voff,
                                (double*)g->Q + P.qoff, P.ldq, c->stream));
        }
        c->launches += count;
    } else {
        G_TRY(launch_ggram_tc(c->opt.gram_split, g->gp, g->tiles, g->ntiles, g->hi, g->mid, g->lo,
                              g->inv_s,
                              (float*)g->Q, g->flags + 1, c->stream));
        c->launches += 1;
    }
    G_TRY(cudaEventRecord(c->ev[2], c->stream));
    int* hflags = (int*)g->host;
    G_TRY(cudaMemcpyAsync(hflags, g->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    G_TRY(cudaEventRecord(c->ev[3], c->stream));
    G_TRY(cudaStreamSynchronize(c->stream));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, c->ev[0], c->ev[3]);
    cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
    c->stats.prepare_ms = a;
    c->stats.gram_ms = b;
    if (hflags[1]) return ALN_ERR_TIMEOUT;
    if (hflags[0]) return ALN_ERR_NONFINITE;
    c->grouped = 1;
    return ALN_OK;
}

namespace {
struct HostView {
    int* again;
    int* fin;
    int* rounds;
    double* rel;
    double* obj;
    GStat* stat;
};
HostView host_view(GroupWork* g) {
    HostView h;
    uint8_t* p = (uint8_t*)g->host;
    h.again = (int*)p;
    h.fin = h.again + g->count;
    h.rounds = h.fin + g->count;
    p += round_up((size_t)g->count * 12, 64);
    h.rel = (double*)p;
    h.obj = h.rel + g->count;
    p += (size_t)g->count * 16;
    h.stat = (GStat*)p;
    return h;
}
}  // namespace

aln_status group_solve(aln_ctx* c, double tol, int max_iter, double* X, const double* X0,
                       aln_solve_info* info) {
    GroupWork* g = (GroupWork*)c->group;
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    const int count = g->count;
    const int64_t N = g->sum_n;
    const bool x_dev = is_dev(X);
    const double* x0 = nullptr;
    if (X0) {
        // stage x0 in x64, check it on the host side of the copy
        G_TRY(cudaMemcpyAsync(g->x64, X0, (size_t)N * 8,
                              is_dev(X0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
        G_TRY(cudaMemsetAsync(g->flags, 0, sizeof(int), c->stream));
        G_TRY(launch_check_finite(g->x64, ALN_DTYPE_F64, N, 1, N, g->flags, c->stream));
        int* hf = (int*)g->host;
        G_TRY(cudaMemcpyAsync(hf, g->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        G_TRY(cudaStreamSynchronize(c->stream));
        if (hf[0]) return ALN_ERR_NONFINITE;
        x0 = g->x64;
    }
    const unsigned gv = grid_for(N, 256, 8 * c->num_sms);
    if (!c->opt.group_graph) {
        k_ginit<<<gv, 256, 0, c->stream>>>(g->gp, count, N, x0, g->s, (double*)g->y, g->stat,
                                           g->fin, g->rounds, g->tgt,
                                           inner_target(tol, 0.5, 1.0,
                                                        (f64 || c->opt.refine_gain == 0)
                                                            ? -1
                                                            : c->opt.refine_gain));
        G_TRY(cudaGetLastError());
        c->launches += 1;
    }
    G_CHECK(upload_order(c, g, g->order_all));
    HostView h = host_view(g);
    std::vector<int> next;
    next.reserve(count);
    int nactive = count;
    // Each inner run stops at its problem's target (progressive refinement:
    // a few decades below the last FP64 residual, at least tol/2 or tol/4);
    // later runs restart from the exact FP64 gradient.
    int gmode = 0;
    double iter_ms = 0.0, kkt_ms = 0.0;
    if (c->opt.group_graph) {
        G_CHECK(f64 ? launch_state<double>(c, g) : launch_state<float>(c, g));
        const bool same = g->graph && g->graph_tol == tol && g->graph_max_iter == max_iter &&
                          g->graph_x0 == (x0 ? 1 : 0) && g->graph_cs == g->cluster_size;
        if (!same) {
            if (g->graph) cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
            // the launch sequence of a whole solve: the start, round 0 over
            // every problem, then max_refine rounds over every problem that
            // pass over those the last FP64 check finished (again[p] = 0);
            // a problem is final after at most max_refine refinements, so
            // the result equals the host-driven loop's, problem by problem
            cudaGraph_t gr = nullptr;
            G_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            aln_status st = ALN_OK;
            k_ginit<<<gv, 256, 0, c->stream>>>(g->gp, count, N, x0, g->s, (double*)g->y, g->stat,
                                               g->fin, g->rounds, g->tgt,
                                               inner_target(tol, 0.5, 1.0,
                                                            (f64 || c->opt.refine_gain == 0)
                                                                ? -1
                                                                : c->opt.refine_gain));
            for (int round = 0; st == ALN_OK && round <= c->opt.max_refine; ++round) {
                st = f64 ? run_solver<double>(c, g, count, round ? 1 : 0, max_iter,
                                              round ? g->again : nullptr)
                         : run_solver<float>(c, g, count, round ? 1 : 0, max_iter,
                                             round ? g->again : nullptr);
                if (st != ALN_OK) break;
                k_gunscale<<<gv, 256, 0, c->stream>>>(g->gp, count, N, (const double*)g->y, g->s,
                                                      g->x64);
                st = kkt_pass(c, g, tol, max_iter, c->opt.max_refine, 1);
            }
            const cudaError_t ec = cudaStreamEndCapture(c->stream, &gr);
            if (st == ALN_OK && ec == cudaSuccess)
                st = cudaGraphInstantiate(&g->graph, gr, 0) == cudaSuccess ? ALN_OK : ALN_ERR_CUDA;
            else if (st == ALN_OK)
                st = ALN_ERR_CUDA;
            if (gr) cudaGraphDestroy(gr);
            if (st != ALN_OK) {
                cudaGetLastError();
                g->graph = nullptr;
                return st;
            }
            g->graph_tol = tol;
            g->graph_max_iter = max_iter;
            g->graph_x0 = x0 ? 1 : 0;
            g->graph_cs = g->cluster_size;
        }
        G_TRY(cudaEventRecord(c->ev[6], c->stream));
        G_TRY(cudaGraphLaunch(g->graph, c->stream));
        G_TRY(cudaEventRecord(c->ev[7], c->stream));
        G_TRY(cudaStreamSynchronize(c->stream));
        float a = 0.f;
        if (cudaEventElapsedTime(&a, c->ev[6], c->ev[7]) == cudaSuccess) iter_ms = a;
        c->launches += 1;
    }
    for (int round = 0; !c->opt.group_graph; ++round) {
        G_TRY(cudaEventRecord(c->ev[6], c->stream));
        G_CHECK(f64 ? run_solver<double>(c, g, nactive, gmode, max_iter)
                    : run_solver<float>(c, g, nactive, gmode, max_iter));
        G_TRY(cudaEventRecord(c->ev[7], c->stream));
        k_gunscale<<<gv, 256, 0, c->stream>>>(g->gp, count, N, (const double*)g->y, g->s,
                                              g->x64);
        G_TRY(cudaGetLastError());
        c->launches += 1;
        G_CHECK(kkt_pass(c, g, tol, max_iter, c->opt.max_refine, 1));
        G_TRY(cudaEventRecord(c->ev[8], c->stream));
        G_TRY(cudaMemcpyAsync(h.again, g->again, (size_t)count * sizeof(int),
                              cudaMemcpyDeviceToHost, c->stream));
        G_TRY(cudaStreamSynchronize(c->stream));
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, c->ev[6], c->ev[7]) == cudaSuccess) iter_ms += a;
        if (cudaEventElapsedTime(&b, c->ev[7], c->ev[8]) == cudaSuccess) kkt_ms += b;
        next.clear();
        for (int p : g->order_all)
            if (h.again[p]) next.push_back(p);
        if (next.empty()) break;
        nactive = (int)next.size();
        G_CHECK(upload_order(c, g, next));
        gmode = 1;
    }
    // results
    G_TRY(cudaMemcpyAsync(X, g->x64, (size_t)N * 8,
                          x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    G_TRY(cudaMemcpyAsync(h.fin, g->fin, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost,
                          c->stream));
    G_TRY(cudaMemcpyAsync(h.rounds, g->rounds, (size_t)count * sizeof(int),
                          cudaMemcpyDeviceToHost, c->stream));
    G_TRY(cudaMemcpyAsync(h.rel, g->rel, (size_t)count * 8, cudaMemcpyDeviceToHost, c->stream));
    G_TRY(cudaMemcpyAsync(h.obj, g->obj, (size_t)count * 8, cudaMemcpyDeviceToHost, c->stream));
    G_TRY(cudaMemcpyAsync(h.stat, g->stat, (size_t)count * sizeof(GStat),
                          cudaMemcpyDeviceToHost, c->stream));
    G_TRY(cudaStreamSynchronize(c->stream));
    int64_t iters = 0, sp = 0, sc = 0;
    int ci = 0;
    double qbytes = 0.0;
    const double tsz = f64 ? 8.0 : 4.0;
    for (int p = 0; p < count; ++p) {
        iters += h.stat[p].iters;
        sp += h.stat[p].sum_passive;
        sc += h.stat[p].sum_clip;
        ci += h.stat[p].clip_iters;
        qbytes += tsz * g->hp[p].n * (double)(h.stat[p].sum_passive + h.stat[p].sum_clip);
        if (info) {
            info[p].iters = h.stat[p].iters;
            info[p].status = h.fin[p];
            info[p].refine_rounds = h.rounds[p];
            info[p].reserved = 0;
            info[p].rel_kkt = h.rel[p];
            info[p].objective = h.obj[p];
        }
    }
    c->stats.iterations = iters;
    c->stats.passive_rows = sp;
    c->stats.clipped_rows = sc;
    c->stats.clipped_iterations = ci;
    c->stats.product_bytes = qbytes;
    c->stats.iterate_ms = iter_ms;
    c->stats.kkt_ms = kkt_ms;
    c->p_G = std::min(count, g->grid);
    return ALN_OK;
}

aln_status group_kkt(aln_ctx* c, const double* X, double* rel_kkt, double* objective) {
    GroupWork* g = (GroupWork*)c->group;
    const int count = g->count;
    G_TRY(cudaMemcpyAsync(g->x64, X, (size_t)g->sum_n * 8,
                          is_dev(X) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          c->stream));
    G_TRY(cudaMemsetAsync(g->fin, 0xff, (size_t)count * sizeof(int), c->stream));  // all open
    G_CHECK(kkt_pass(c, g, 0.0, 0, 0, 0));
    G_TRY(cudaMemcpyAsync(rel_kkt, g->rel, (size_t)count * 8,
                          is_dev(rel_kkt) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream));
    if (objective)
        G_TRY(cudaMemcpyAsync(objective, g->obj, (size_t)count * 8,
                              is_dev(objective) ? cudaMemcpyDeviceToDevice
                                                : cudaMemcpyDeviceToHost,
                              c->stream));
    G_TRY(cudaStreamSynchronize(c->stream));
    return ALN_OK;
}

aln_status group_export(aln_ctx* c, double* Q, double* q, double* s) {
    GroupWork* g = (GroupWork*)c->group;
    const bool f64 = c->opt.precision == ALN_PREC_FP64;
    if (Q) {
        const bool dev = is_dev(Q);
        double* dst = Q;
        double* tmp = nullptr;
        if (!dev) {
            G_TRY(cudaMalloc(&tmp, (size_t)g->sum_nn * 8));
            dst = tmp;
        }
        const unsigned grid = (unsigned)g->count;
        if (f64)
            k_gexport_q<double><<<grid, 256, 0, c->stream>>>(g->gp, (const double*)g->Q,
                                                             g->qexp_dev, dst);
        else
            k_gexport_q<float><<<grid, 256, 0, c->stream>>>(g->gp, (const float*)g->Q,
                                                            g->qexp_dev, dst);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && !dev)
            e = cudaMemcpyAsync(Q, tmp, (size_t)g->sum_nn * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (tmp) cudaFree(tmp);
        if (e != cudaSuccess) return cuda_err(e);
    }
    if (q)
        G_TRY(cudaMemcpyAsync(q, g->q64, (size_t)g->sum_n * 8,
                              is_dev(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->stream));
    if (s)
        G_TRY(cudaMemcpyAsync(s, g->s, (size_t)g->sum_n * 8,
                              is_dev(s) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->stream));
    G_TRY(cudaStreamSynchronize(c->stream));
    return ALN_OK;
}

}  // namespace aln
