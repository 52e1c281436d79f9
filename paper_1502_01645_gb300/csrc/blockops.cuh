// Block-level building blocks of Alg. 2 (§3) for one problem held by one
// 1024-thread block: per-warp and block reductions (FP64 over the warp
// partials), the passive mask with its compacted row list, and the product
// over listed rows of a symmetric Q.  Used by the grouped solver (one block
// or cluster per problem) and by the batched solver's per-column tail.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace aln {

constexpr int kGThreads = 1024;
constexpr int kGWarps = kGThreads / 32;
constexpr int kGU = 8;  // rows of Q in flight per lane in the product

template <typename T>
__device__ __forceinline__ T gwarp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int gwarp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Exclusive prefix over lanes of v; *total receives the sum of all lanes.
__device__ __forceinline__ int gwarp_scan_excl(int v, int* total) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Shared scratch of the block-wide reductions and list builders.
template <typename T>
struct GRed {
    T wsum[kGWarps];  // warp partials in the iteration type (widened by warp 0)
    int wcnt[kGWarps];
    int wlist[kGWarps];
    int base[kGWarps];
    double tsum;  // the total, in the caller's scalar type (8 bytes either way)
    int tcnt, tlist;
};

// Contiguous range of 32-element chunks scanned by this warp.
__device__ __forceinline__ void warp_chunks(int n, int& c0, int& c1) {
    const int nchunk = (n + 31) >> 5;
    const int per = (nchunk + kGWarps - 1) / kGWarps;
    c0 = (threadIdx.x >> 5) * per;
    c1 = min(nchunk, c0 + per);
}

// Reduce per-warp (value, count, list count) and give each warp its list
// base; every thread receives the totals.  The value's warp partials are
// widened and added by warp 0 alone, in the scalar type S (FP64, or
// normalised FP32 pairs in the FP32 kernels): the step scalars (γ = ‖ḡ‖²,
// κ = ḡᵀQḡ) need more than FP32 — with FP32 scalars the FP32 iteration
// drifts from the true gradient and needs several times more iterations —
// while an FP64 instruction costs a warp about 16 cycles of its SM's narrow
// FP64 unit even with one active lane.  With need_v false (a count only) the
// wide sum is skipped and *vt is 0.
template <typename T, typename S = double>
__device__ __forceinline__ int block_totals(GRed<T>* r, T v, int cnt, int lcnt, S* vt, int* ct,
                                            int* lt, bool need_v = true) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (need_v) v = gwarp_sum(v);
    __syncthreads();  // earlier readers of r are done
    if (lane == 0) {
        r->wsum[wid] = v;
        r->wcnt[wid] = cnt;
        r->wlist[wid] = lcnt;
    }
    __syncthreads();
    if (wid == 0) {
        S x;
        sc_set(x, T(0));
        if (need_v) {
            S lv;
            sc_set(lv, r->wsum[lane]);
            x = sc_warp_sum(lv);
        }
        const int c = gwarp_sum_i(r->wcnt[lane]);
        int total;
        r->base[lane] = gwarp_scan_excl(r->wlist[lane], &total);
        if (lane == 0) {
            *reinterpret_cast<S*>(&r->tsum) = x;
            r->tcnt = c;
            r->tlist = total;
        }
    }
    __syncthreads();
    *vt = *reinterpret_cast<const S*>(&r->tsum);
    *ct = r->tcnt;
    *lt = r->tlist;
    return r->base[wid];
}

// Passive set of Alg. 2 (strict: y_i > 0 or g_i < 0), ḡ = g on P, ‖ḡ‖²,
// |P|, and the ascending list of i with ḡ_i ≠ 0 (the columns of Q the
// product needs).
template <typename T, typename S = double>
__device__ __forceinline__ void gmask(int n, const T* sy, const T* sg, T* sgb, int* list,
                                      GRed<T>* r, S* gam, int* cntP, int* cntL) {
    const int lane = threadIdx.x & 31;
    int c0, c1;
    warp_chunks(n, c0, c1);
    T v = T(0);
    int cp = 0, cl = 0;
    for (int c = c0; c < c1; ++c) {
        const int i = c * 32 + lane;
        T gb = T(0);
        bool P = false;
        if (i < n) {
            const T yi = sy[i], gi = sg[i];
            P = yi > T(0) || gi < T(0);
            gb = P ? gi : T(0);
            sgb[i] = gb;
        }
        v = fma(gb, gb, v);
        cp += __popc(__ballot_sync(0xffffffffu, P));
        cl += __popc(__ballot_sync(0xffffffffu, gb != T(0)));
    }
    int base = block_totals<T, S>(r, v, cp, cl, gam, cntP, cntL);
    for (int c = c0; c < c1; ++c) {
        const int i = c * 32 + lane;
        const bool nz = i < n && sgb[i] != T(0);
        const unsigned int m = __ballot_sync(0xffffffffu, nz);
        if (nz) list[base + __popc(m & ((1u << lane) - 1u))] = i;
        base += __popc(m);
    }
    __syncthreads();
}

// Ascending list of i < n with v_i ≠ 0; returns its length (all threads).
template <typename T>
__device__ __forceinline__ int glist(int n, const T* v, int* list, GRed<T>* r) {
    const int lane = threadIdx.x & 31;
    int c0, c1;
    warp_chunks(n, c0, c1);
    int cl = 0;
    for (int c = c0; c < c1; ++c) {
        const int i = c * 32 + lane;
        cl += __popc(__ballot_sync(0xffffffffu, i < n && v[i] != T(0)));
    }
    double vt;
    int ct, lt;
    int base = block_totals(r, T(0), 0, cl, &vt, &ct, &lt, false);
    for (int c = c0; c < c1; ++c) {
        const int i = c * 32 + lane;
        const bool nz = i < n && v[i] != T(0);
        const unsigned int m = __ballot_sync(0xffffffffu, nz);
        if (nz) list[base + __popc(m & ((1u << lane) - 1u))] = i;
        base += __popc(m);
    }
    __syncthreads();
    return lt;
}

// out[i] (+)= Σ_k Q[list[k]][i] · v[list[k]] for lo ≤ i < hi — the product of
// Alg. 2 restricted to the listed columns (Q is symmetric; row list[k] is
// read) and to a range of rows (lo a multiple of 32·VN).  Warps split the
// range into 32·VN-wide tiles and the list into S strided subsets; the S
// partials are added in subset order (deterministic).
template <typename T>
__device__ __forceinline__ void gmv(const T* Q, int ldq, int lo, int hi, const int* list, int cnt,
                                    const T* v, T* out, bool accumulate, T* red) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::N;
    constexpr int TILE = 32 * VN;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int CT = hi > lo ? (hi - lo + TILE - 1) / TILE : 0;
    if (CT == 0) {  // uniform: nothing in range
        __syncthreads();
        return;
    }
    const int CTw = CT < kGWarps ? CT : kGWarps;
    const int S = kGWarps / CTw;
    const int sub = wid / CTw;
    if (sub < S) {
        for (int ct = wid % CTw; ct < CT; ct += CTw) {
            const int col = lo + ct * TILE + lane * VN;
            const bool cv = col < hi;  // then col + VN ≤ ldq (ldq is a multiple of 4)
            T acc[VN];
#pragma unroll
            for (int c = 0; c < VN; ++c) acc[c] = T(0);
            int k = sub;
            for (; k + (kGU - 1) * S < cnt; k += kGU * S) {
                V qq[kGU];
                T vv[kGU];
#pragma unroll
                for (int u = 0; u < kGU; ++u) {
                    const int j = list[k + u * S];
                    qq[u] = cv ? *reinterpret_cast<const V*>(Q + (int64_t)j * ldq + col) : V{};
                    vv[u] = v[j];
                }
#pragma unroll
                for (int u = 0; u < kGU; ++u)
#pragma unroll
                    for (int c = 0; c < VN; ++c) acc[c] = fma(vv[u], vget(qq[u], c), acc[c]);
            }
            for (; k < cnt; k += S) {
                const int j = list[k];
                const V q = cv ? *reinterpret_cast<const V*>(Q + (int64_t)j * ldq + col) : V{};
                const T vj = v[j];
#pragma unroll
                for (int c = 0; c < VN; ++c) acc[c] = fma(vj, vget(q, c), acc[c]);
            }
            if (S == 1) {
                if (cv)
#pragma unroll
                    for (int c = 0; c < VN; ++c)
                        if (col + c < hi) out[col + c] = accumulate ? out[col + c] + acc[c] : acc[c];
            } else {
#pragma unroll
                for (int c = 0; c < VN; ++c) red[(sub * CT + ct) * TILE + lane * VN + c] = acc[c];
            }
        }
    }
    if (S > 1) {
        __syncthreads();
        for (int ii = threadIdx.x; ii < hi - lo; ii += blockDim.x) {
            const int ct = ii / TILE, rr = ii - ct * TILE;
            T s = T(0);
            for (int s2 = 0; s2 < S; ++s2) s += red[(s2 * CT + ct) * TILE + rr];
            const int i = lo + ii;
            out[i] = accumulate ? out[i] + s : s;
        }
    }
    __syncthreads();
}

}  // namespace aln
