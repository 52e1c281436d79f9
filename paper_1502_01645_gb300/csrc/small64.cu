// Alg. 2 (§3) in FP64 for one small problem (n up to about 460, where the
// slices of Q fit in shared memory) on ONE thread-block cluster: no grid
// barrier, Q held in the cluster's shared memory.
//
// The plain FP64 method on a small problem is latency-bound: the grid-wide
// kernel pays a grid barrier and several FP64 reductions of the whole vector
// per iteration, while the work is a few tens of thousands of FMAs.  Here the
// C CTAs of one cluster (8, or 16 when n ≤ 256 and 16-CTA clusters fit)
// split the rows of Q: CTA r keeps the columns
// [r·S, r·S + S) of Q (rows, since Q is symmetric) for every j, i.e.
// Qs[j][i] = Q[j][r·S + i], the slice of every state vector (y, g, w, e), and
// a full copy of ḡ (and of e when rows were clipped) gathered through
// distributed shared memory.  One iteration:
//
//   (1) w_i = Σ_j Q_ij ḡ_j for the slice: lane ↔ row i, warp ↔ a range of j
//       (skipping ḡ_j = 0, warp-uniform), warp partials added in warp order;
//       the slice's share of κ = ḡᵀw.
//   (2) cluster exchange of the κ shares (rank order), α = ‖ḡ‖²/κ.
//   (3) y⁺ = [y − αḡ]₊, e = the clipped part, g ← g − αw, the mask of y⁺
//       as if nothing was clipped; exchange of ‖ḡ‖², |P|, |C| and all-gather
//       of ḡ (and e).
//   (4) with rows clipped: g ← g + Qe on the slice (since y⁺ − y = −αḡ + e),
//       the mask of y⁺, a second exchange and all-gather of ḡ.
//
// Every sum has a fixed order, so the iterates are reproducible; every CTA
// takes the same decisions from the same exchanged totals.  The loop needs no
// bounded wait: the cluster barrier is a hardware barrier over one cluster.
#include <stdio.h>

#include "cluster.cuh"
#include "common.cuh"
#include "kernels.cuh"

// Phase tracing for tuning (off unless built with -DALN_S64_TRACE): CTA 0
// thread 0 accumulates %globaltimer laps and prints the per-iteration means.
#ifdef ALN_S64_TRACE
#define S64_TRACE(k)                                                        \
    do {                                                                    \
        if (tracer) {                                                       \
            uint64_t t_;                                                    \
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));          \
            trc[k] += t_ - t_last;                                          \
            t_last = t_;                                                    \
        }                                                                   \
    } while (0)
#else
#define S64_TRACE(k) \
    do {             \
    } while (0)
#endif

namespace aln {
namespace {

constexpr int kSC = 8;            // CTAs of the cluster (the portable size)
constexpr int kSC16 = 16;         // the non-portable size, for n ≤ 16·16
constexpr int kSThreads = 256;    // 8 warps
constexpr int kSWarps = kSThreads / 32;
constexpr int kSMaxS = 64;        // slice rows per CTA (two per lane)

struct S64Args {
    const double* Q;
    int64_t ldq;
    int n;
    int S;        // slice length, ⌈n/C⌉ (≤ 64: the first ⌈S/32⌉ warps hold it)
    double* y;    // in/out (global)
    double* g;    // in/out (global)
    IterState* st;
};

struct SRec {
    double v;    // the CTA's share of the exchanged sum (κ or ‖ḡ‖²)
    int cnt;     // its |P|
    int clip;    // its |C|
};

// Publish this CTA's record, cluster barrier, warp 0 adds the C records in
// rank order; lanes < C each load one record.  Totals land in *tot.
template <int C>
__device__ __forceinline__ void s_exchange(SRec* slot, const SRec& mine, SRec* tot) {
    if (threadIdx.x == 0) *slot = mine;
    cluster_sync();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double v = 0.0;
        int cnt = 0, clip = 0;
        if (lane < C) {
            const uint32_t b = cluster_addr(slot, lane);
            v = ld_cluster(b + (uint32_t)offsetof(SRec, v), 0.0);
            cnt = ld_cluster(b + (uint32_t)offsetof(SRec, cnt), 0);
            clip = ld_cluster(b + (uint32_t)offsetof(SRec, clip), 0);
        }
        // pairwise tree over the C ranks (fixed order)
#pragma unroll
        for (int o = 1; o < C; o <<= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, v, o);
            const int oc = __shfl_down_sync(0xffffffffu, cnt, o);
            const int ol = __shfl_down_sync(0xffffffffu, clip, o);
            if ((lane & (2 * o - 1)) == 0) {
                v += ov;
                cnt += oc;
                clip += ol;
            }
        }
        if (lane == 0) {
            tot->v = v;
            tot->cnt = cnt;
            tot->clip = clip;
        }
    }
    __syncthreads();
}

// All-gather: full[j] for every j < n from the owning CTA's slice (own copy
// for this CTA's slice).  Called after a cluster barrier that published the
// slices; the caller synchronises afterwards.
__device__ __forceinline__ void s_allgather(const double* slice, double* full, int n, int S,
                                            int rank) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int r = j / S, i = j - r * S;
        full[j] = r == rank ? slice[i] : ld_cluster(cluster_addr(slice + i, r), 0.0);
    }
}

// Sums over the slice (held by the first nsw warps; the others hold zeros):
// warp sums in those warps, then thread 0 adds them in warp order.  The
// totals are valid in thread 0 only (the caller publishes them from there).
// GB300's FP64 unit is narrow (about 16 cycles per warp instruction even
// with few active lanes), so no warp outside the slice issues FP64 work.
__device__ __forceinline__ void s_sum0(double v, int c, int nsw, double* sd, int* si, double* v_out,
                                       int* c_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < nsw) {
        v = warp_sum(v);
        c = (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
        if (lane == 0) {
            sd[warp] = v;
            si[warp] = c;
        }
    }
    __syncthreads();
    double t = 0.0;
    int tc = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < nsw; ++w) {
            t += sd[w];
            tc += si[w];
        }
    }
    *v_out = t;
    *c_out = tc;
}

// out_i = Σ_{j: v_j ≠ 0} Qs[j][i] v_j for the slice rows (lane ↔ row, two
// rows per lane; warp ↔ a contiguous range of j), warp partials added in
// warp order.  The non-zero j of a 32-wide chunk are compacted with a ballot
// (an integer test of the bits: ±0 have no other bits set) and taken two at a
// time, one per accumulator (the k-th non-zero j of the range goes to
// accumulator k mod 2), so the FP64 unit — narrow on this GPU and the bound
// of this loop — sees only the FMAs themselves, with two independent chains.
template <int C>
__device__ __forceinline__ void s_product(const double* Qs, int S, int n, const double* v,
                                          double* red, double* out);

// The 16-CTA form (S ≤ 16 rows per CTA): a half-warp per j, so one FMA
// instruction serves two j of the compacted list (lane = 16·h + row, half h
// takes the j of its parity).  Each step takes up to four j: the first pair
// into accumulator 0, the second into accumulator 1 (two independent FMA
// chains); the halves are added at the end (half 0 + half 1).
__device__ __forceinline__ void s_product_packed(const double* Qs, int S, int n, const double* v,
                                                 double* red, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (n + kSWarps - 1) / kSWarps;
    const int j0 = warp * per, j1 = min(n, j0 + per);
    const int h = lane >> 4, i = lane & 15;
    const bool in = i < S;
    double a0 = 0.0, a1 = 0.0;
    for (int base = j0; base < j1; base += 32) {
        const int jl = base + lane;
        const bool nz = jl < j1 && (__double_as_longlong(v[jl]) << 1) != 0;
        unsigned int m = __ballot_sync(0xffffffffu, nz);
        while (m) {  // warp-uniform
            int q[4];  // the next four j of the list (−1 past its end)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                q[t] = m ? base + __ffs(m) - 1 : -1;
                m &= m - 1;  // no-op once m is 0
            }
            const int ja = h == 0 ? q[0] : q[1], jb = h == 0 ? q[2] : q[3];
            if (in && ja >= 0) a0 = fma(Qs[(int64_t)ja * S + i], v[ja], a0);
            if (in && jb >= 0) a1 = fma(Qs[(int64_t)jb * S + i], v[jb], a1);
        }
    }
    double acc = a0 + a1;
    acc += __shfl_down_sync(0xffffffffu, acc, 16);  // half 0 + half 1
    if (lane < 16) red[warp * kSMaxS + lane] = acc;
    __syncthreads();
    for (int r = threadIdx.x; r < S; r += blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kSWarps; ++w) s += red[w * kSMaxS + r];
        out[r] = s;
    }
    __syncthreads();
}

template <>
__device__ __forceinline__ void s_product<kSC16>(const double* Qs, int S, int n, const double* v,
                                                 double* red, double* out) {
    s_product_packed(Qs, S, n, v, red, out);
}

template <>
__device__ __forceinline__ void s_product<kSC>(const double* Qs, int S, int n, const double* v,
                                               double* red, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (n + kSWarps - 1) / kSWarps;
    const int j0 = warp * per, j1 = min(n, j0 + per);
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    const int i0 = lane, i1 = lane + 32;
    const bool in0 = i0 < S, in1 = S > 32 && i1 < S;
    bool odd = false;  // the next non-zero j goes to accumulator 1
    for (int base = j0; base < j1; base += 32) {
        const int jl = base + lane;
        const bool nz = jl < j1 && (__double_as_longlong(v[jl]) << 1) != 0;
        unsigned int m = __ballot_sync(0xffffffffu, nz);
        if (odd && m) {  // one j to accumulator 1 first (warp-uniform)
            const int j = base + __ffs(m) - 1;
            m &= m - 1;
            const double vj = v[j];
            const double* col = Qs + (int64_t)j * S;
            if (in0) a1 = fma(col[i0], vj, a1);
            if (in1) b1 = fma(col[i1], vj, b1);
            odd = false;
        }
        while (m) {
            const int ja = base + __ffs(m) - 1;
            m &= m - 1;
            const double va = v[ja];
            const double* ca = Qs + (int64_t)ja * S;
            if (m) {
                const int jb = base + __ffs(m) - 1;
                m &= m - 1;
                const double vb = v[jb];
                const double* cb = Qs + (int64_t)jb * S;
                if (in0) {
                    a0 = fma(ca[i0], va, a0);
                    a1 = fma(cb[i0], vb, a1);
                }
                if (in1) {
                    b0 = fma(ca[i1], va, b0);
                    b1 = fma(cb[i1], vb, b1);
                }
            } else {
                if (in0) a0 = fma(ca[i0], va, a0);
                if (in1) b0 = fma(ca[i1], va, b0);
                odd = true;
            }
        }
    }
    red[warp * kSMaxS + i0] = a0 + a1;
    if (in1) red[warp * kSMaxS + i1] = b0 + b1;  // rows ≥ S are never read
    __syncthreads();
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kSWarps; ++w) s += red[w * kSMaxS + i];
        out[i] = s;
    }
    __syncthreads();
}

// Mask of the slice: ḡ = g on P(y); returns (in thread 0) ‖ḡ‖² and |P| of
// the slice (S ≤ 64 entries: the first nsw warps, one entry per thread).
__device__ __forceinline__ void s_mask(const double* y, const double* g, double* gb, int len,
                                       int S, int nsw, double* sd, int* si, double* g2,
                                       int* cnt) {
    double v = 0.0;
    int c = 0;
    const int i = threadIdx.x;
    if (i < S) {
        if (i < len) {
            const bool P = y[i] > 0.0 || g[i] < 0.0;
            const double b = P ? g[i] : 0.0;
            gb[i] = b;
            v = fma(b, b, v);
            c += P ? 1 : 0;
        } else {
            gb[i] = 0.0;
        }
    }
    s_sum0(v, c, nsw, sd, si, g2, cnt);
    __syncthreads();
}

template <int C>
__global__ void __launch_bounds__(kSThreads, 1) k_alg2_small64(S64Args a) {
    extern __shared__ __align__(16) double smd[];
    const int S = a.S, n = a.n;
    const int nsw = (S + 31) / 32;  // warps holding the slice
    const int rank = cluster_rank();
    const int s0 = min(n, rank * S), len = min(n, s0 + S) - s0;
    double* Qs = smd;                      // n × S: Qs[j][i] = Q[j][s0 + i]
    double* gfull = Qs + (int64_t)n * S;   // ḡ, all n entries
    double* efull = gfull + n;             // e, all n entries
    double* sy = efull + n;                // slice vectors
    double* sg = sy + S;
    double* sgb = sg + S;
    double* sw = sgb + S;                  // w, then e (published for the gather)
    double* su = sw + S;                   // Qe on the slice
    double* red = su + S;                  // kSWarps × kSMaxS
    __shared__ SRec slot[3];
    __shared__ SRec tot;
    __shared__ double sd[kSWarps];
    __shared__ int si[kSWarps];
    __shared__ double s_alpha;
    __shared__ int s_flag;
#ifdef ALN_S64_TRACE
    const bool tracer = rank == 0 && threadIdx.x == 0;
    uint64_t trc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t t_last = 0;
    if (tracer) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_last));
#endif

    for (int64_t e = threadIdx.x; e < (int64_t)n * S; e += blockDim.x) {
        const int j = (int)(e / S), i = (int)(e - (int64_t)j * S);
        Qs[e] = i < len ? a.Q[(int64_t)j * a.ldq + s0 + i] : 0.0;
    }
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
        sy[i] = i < len ? a.y[s0 + i] : 0.0;
        sg[i] = i < len ? a.g[s0 + i] : 0.0;
        sw[i] = 0.0;
    }
    __syncthreads();

    IterState* st = a.st;
    const double eps = st->eps;
    const int max_iter = st->max_iter, window = st->window;
    double best = 1.0 / 0.0, gam = 0.0;
    int best_iter = 0, iter = 0, status = ALN_RHS_MAXITER, cnt = 0;
    long long sum_passive = 0, sum_clip = 0;
    int nclip_iters = 0;

    // mask of the start point, exchange, gather of ḡ
    {
        double g2;
        int c;
        s_mask(sy, sg, sgb, len, S, nsw, sd, si, &g2, &c);
        SRec m{g2, c, 0};
        s_exchange<C>(&slot[2], m, &tot);  // its cluster barrier also publishes sgb
        s_allgather(sgb, gfull, n, S, rank);
        __syncthreads();
        gam = tot.v;
        cnt = tot.cnt;
    }

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
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) break;
        S64_TRACE(0);

        // (1) w on the slice, κ share
        s_product<C>(Qs, S, n, gfull, red, sw);
        S64_TRACE(1);
        double kp = 0.0;
        if ((int)threadIdx.x < len) kp = sgb[threadIdx.x] * sw[threadIdx.x];
        {
            int unused;
            s_sum0(kp, 0, nsw, sd, si, &kp, &unused);
        }
        S64_TRACE(2);
        // (2) κ over the cluster, α
        s_exchange<C>(&slot[0], SRec{kp, 0, 0}, &tot);
        S64_TRACE(3);
        if (threadIdx.x == 0) {
            const double k2 = tot.v;
            int stop = 0;
            if (!isfinite(k2)) stop = ALN_RHS_NONFINITE;
            else if (k2 <= 0.0) stop = ALN_RHS_CURVATURE;
            s_alpha = stop ? 0.0 : gam / k2;
            s_flag = stop;
        }
        __syncthreads();
        if (s_flag) {
            status = s_flag;
            break;
        }
        const double al = s_alpha;
        sum_passive += cnt;
        S64_TRACE(4);
        // (3) projected update, gradient update, mask as if nothing clipped
        double v2 = 0.0;
        int cP = 0, clipped = 0;
        for (int i = threadIdx.x; i < S; i += blockDim.x) {
            if (i < len) {
                const double yi = sy[i];
                double yn = yi - al * sgb[i];
                double ej = 0.0;
                if (yn < 0.0) {
                    ej = -yn;
                    yn = 0.0;
                    ++clipped;
                }
                const double gn = sg[i] - al * sw[i];
                sy[i] = yn;
                sg[i] = gn;
                sw[i] = ej;  // w is consumed; the buffer now holds e
                const bool P = yn > 0.0 || gn < 0.0;
                const double b = P ? gn : 0.0;
                sgb[i] = b;
                v2 = fma(b, b, v2);
                cP += P ? 1 : 0;
            } else {
                sgb[i] = 0.0;
                sw[i] = 0.0;
            }
        }
        {
            int packed;  // |P| and |C| of the slice, packed (each ≤ 64)
            s_sum0(v2, cP | (clipped << 16), nsw, sd, si, &v2, &packed);
            cP = packed & 0xffff;
            clipped = packed >> 16;
        }
        ++iter;
        S64_TRACE(5);
        s_exchange<C>(&slot[1], SRec{v2, cP, clipped}, &tot);  // publishes sgb and e too
        S64_TRACE(6);
        const int nclip = tot.clip;
        sum_clip += nclip;
        if (nclip == 0) {
            s_allgather(sgb, gfull, n, S, rank);
            __syncthreads();
            gam = tot.v;
            cnt = tot.cnt;
            S64_TRACE(7);
            continue;
        }
        ++nclip_iters;
        // (4) g += Qe on the slice from the gathered e
        s_allgather(sw, efull, n, S, rank);
        __syncthreads();
        // (into su: peers may still be reading this CTA's e in sw)
        s_product<C>(Qs, S, n, efull, red, su);
        for (int i = threadIdx.x; i < len; i += blockDim.x) sg[i] += su[i];
        __syncthreads();
        double g2;
        int c;
        s_mask(sy, sg, sgb, len, S, nsw, sd, si, &g2, &c);
        s_exchange<C>(&slot[2], SRec{g2, c, 0}, &tot);
        s_allgather(sgb, gfull, n, S, rank);
        __syncthreads();
        gam = tot.v;
        cnt = tot.cnt;
        S64_TRACE(8);
    }

    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        a.y[s0 + i] = sy[i];
        a.g[s0 + i] = sg[i];
    }
    if (rank == 0 && threadIdx.x == 0) {
        st->iter = iter;
        st->done = 1;
        st->status = status;
        st->gbar2 = gam;
        st->npassive = cnt;
        st->best_g2 = best;
        st->best_iter = best_iter;
        st->sum_passive = sum_passive;
        st->sum_clip = sum_clip;
        for (int k = 0; k < 5; ++k) st->phase_ns[k] = 0;
        st->phase_ns[5] = (uint64_t)nclip_iters;
#ifdef ALN_S64_TRACE
        const double it = iter > 0 ? (double)iter : 1.0;
        printf("s64_trace iters=%d clipped=%d | top %.0f product %.0f kred %.0f kexch %.0f "
               "alpha %.0f update %.0f exch %.0f gather %.0f clip %.0f ns\n",
               iter, nclip_iters, trc[0] / it, trc[1] / it, trc[2] / it, trc[3] / it,
               trc[4] / it, trc[5] / it, trc[6] / it, trc[7] / it, trc[8] / it);
#endif
    }
    // no CTA leaves while a peer may still read its shared memory
    cluster_sync();
}

size_t s64_smem_bytes(int n, int S) {
    return (size_t)((int64_t)n * S + 2 * n + 5 * S + kSWarps * kSMaxS) * sizeof(double);
}

}  // namespace

// The single-cluster FP64 loop applies when the slices of Q fit in shared
// memory (S ≤ kSMaxS rows per CTA and n·S doubles within the opt-in limit).
bool small64_fits(const aln_ctx* c, int optin_smem) {
    const int64_t n = c->n;
    if (n < 1) return false;
    const int S = (int)ceil_div(n, (int64_t)kSC);
    if (S > kSMaxS) return false;
    return s64_smem_bytes((int)n, S) + 4096 <= (size_t)optin_smem;
}

namespace {
template <int C>
cudaError_t launch_small64_c(const S64Args& a, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kSThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_alg2_small64<C>, a);
}

// Can a 16-CTA cluster of the kernel with this shared memory be resident?
// (Non-portable size: asked once per device and size class.)
bool cluster16_fits(size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    static int known[64] = {};      // 0 unknown, 1 yes, 2 no
    static size_t known_smem[64] = {};
    if (known[dev] != 0 && known_smem[dev] >= smem) return known[dev] == 1;
    bool ok = cudaFuncSetAttribute(k_alg2_small64<kSC16>,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(k_alg2_small64<kSC16>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem) == cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3(kSC16);
        cfg.blockDim = dim3(kSThreads);
        cfg.dynamicSmemBytes = smem;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kSC16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        ok = cudaOccupancyMaxActiveClusters(&nc, k_alg2_small64<kSC16>, &cfg) == cudaSuccess &&
             nc >= 1;
    }
    cudaGetLastError();  // a refused size leaves no error behind
    known[dev] = ok ? 1 : 2;
    known_smem[dev] = smem;
    return ok;
}
}  // namespace

// 16 CTAs when every CTA holds at most 16 rows (n ≤ 256) and such a cluster
// fits on the GPU (each FP64 FMA instruction then serves two j); else 8.
cudaError_t launch_alg2_small64(aln_ctx* c) {
    S64Args a;
    a.Q = (const double*)c->Q;
    a.ldq = c->ldq;
    a.n = (int)c->n;
    a.y = (double*)c->y;
    a.g = (double*)c->g;
    a.st = c->st;
    const int S16 = (int)ceil_div(c->n, (int64_t)kSC16);
    if (S16 <= 16) {
        a.S = S16;
        const size_t smem = s64_smem_bytes(a.n, a.S);
        if (cluster16_fits(smem)) return launch_small64_c<kSC16>(a, smem, c->stream);
    }
    a.S = (int)ceil_div(c->n, (int64_t)kSC);
    const size_t smem = s64_smem_bytes(a.n, a.S);
    cudaError_t e = cudaFuncSetAttribute(k_alg2_small64<kSC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_small64_c<kSC>(a, smem, c->stream);
}

}  // namespace aln
