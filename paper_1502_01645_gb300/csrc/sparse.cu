// Alg. 1 (§3) for a sparse, possibly tall A given in compressed sparse
// column (CSC) form: column j holds the entries vals[t], rows row_idx[t] for
// col_ptr[j] ≤ t < col_ptr[j+1], rows strictly increasing.
//
// Every step reads only the stored entries:
//   k_csc_check     the structure (bounds, order) and finiteness;
//   k_csc_colstats  s_j² = Σ a_tj², (Aᵀb_c)_j for up to four right-hand
//                   sides, the occupancy bitmap of the Gram's operand boxes
//                   (64 rows × 128 columns), and where a path still needs it
//                   the scatter into a dense column-major copy of A;
//   k_csc_tiles / k_csc_offsets  number the occupied boxes, column tile by
//                   column tile (a popcount prefix per bitmap word);
//   k_csc_pack      the exact three-term BF16 split of every entry, written
//                   into its box in the pre-swizzled layout the tensor-core
//                   Gram copies verbatim (pack_index);
//   k_csc_pairs / k_csc_items  the Gram's work list: the common blocks of
//                   every tile pair, and chunks of them for the CTAs;
//   k_csc_kkt_ax / k_csc_kkt_grad  the FP64 KKT pass without a dense copy of
//                   A (r = Ax − b from the packed boxes, Aᵀr from the entries).
// The Gram (launch_sgram_tc, gemm_tc.cu) multiplies, for each tile pair, only
// the K blocks occupied in both column tiles: a block that is zero in either
// operand adds exactly zero to H = AᵀA, so Q is that of the dense A up to how
// its FP32 sums are grouped (pairs with many common blocks are split over
// several CTAs, from a work list built by k_csc_pairs / k_csc_items).
#include "common.cuh"
#include "kernels.cuh"

namespace aln {

namespace {

constexpr int kCscThreads = 256;
constexpr int kCscWarps = kCscThreads / 32;

// Exclusive prefix sum over a 256-thread block; *total gets the block sum.
__device__ __forceinline__ int64_t block_scan_excl(int64_t v, int64_t* s_w, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    int64_t before = 0, all = 0;
    for (int w = 0; w < kCscWarps; ++w) {
        if (w < wid) before += s_w[w];
        all += s_w[w];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

// One warp per column.  flags[2] |= 1 for a malformed structure (col_ptr not
// non-decreasing within [0, nnz], col_ptr[0] ≠ 0, col_ptr[n] ≠ nnz, a row out
// of [0, d), rows not strictly increasing); flags[0] |= 1 for a NaN/Inf value.
// A column whose bounds are malformed is not read further.
template <typename T>
__global__ void __launch_bounds__(kCscThreads) k_csc_check(const int64_t* __restrict__ cp,
                                                           const int32_t* __restrict__ ri,
                                                           const T* __restrict__ v, int64_t d,
                                                           int64_t n, int64_t nnz,
                                                           int* __restrict__ flags) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kCscWarps + (threadIdx.x >> 5);
    if (j >= n) return;
    const int64_t p0 = cp[j], p1 = cp[j + 1];
    bool bad = p0 < 0 || p1 < p0 || p1 > nnz || (j == 0 && p0 != 0) || (j == n - 1 && p1 != nnz);
    if (bad) {
        if (lane == 0) atomicOr(&flags[2], 1);
        return;
    }
    bool nonfinite = false;
    for (int64_t t = p0 + lane; t < p1; t += 32) {
        const int32_t r = ri[t];
        bad |= r < 0 || (int64_t)r >= d || (t > p0 && ri[t - 1] >= r);
        nonfinite |= !isfinite(v[t]);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&flags[2], 1);
    if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicOr(&flags[0], 1);
}

// One warp per column j: the column statistics of Alg. 1 from the stored
// entries (same definitions as the dense k_colstats: s_j = √Σa², or 1 for an
// empty column; q_cj = −(Aᵀb_c)_j / s_j for c < kc ≤ 4), the scatter
// A[j·lda + row] = a (A zeroed beforehand), and with OCC the occupancy bit of
// box (column tile j/128, K block row/64) in occ[tile·W + kb/32].
template <typename T, bool OCC>
__global__ void __launch_bounds__(kCscThreads)
    k_csc_colstats(const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                   const T* __restrict__ v, int64_t n, const T* __restrict__ B, int kc,
                   int64_t ldb, T* __restrict__ A, int64_t lda, double* __restrict__ s,
                   double* __restrict__ inv_s, double* __restrict__ q64, int64_t ldq,
                   uint32_t* __restrict__ occ, int W) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kCscWarps + (threadIdx.x >> 5);
    if (j >= n) return;
    const int64_t p0 = cp[j], p1 = cp[j + 1];
    DotAcc<T> sq, dot[4];
    T* col = A ? A + j * lda : nullptr;  // no dense copy when A is null
    uint32_t* occ_t = OCC ? occ + (j >> 7) * (int64_t)W : nullptr;
    for (int64_t t = p0 + lane; t < p1; t += 32) {
        const int32_t r = ri[t];
        const T a = v[t];
        sq.add(a, a);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < kc) dot[c].add(a, B[(int64_t)c * ldb + r]);
        if (col) col[r] = a;
        if (OCC) {
            const int kb = r >> 6;
            // rows are increasing: only the first entry of a K block sets its bit
            if (t == p0 || (ri[t - 1] >> 6) != kb) atomicOr(&occ_t[kb >> 5], 1u << (kb & 31));
        }
    }
    const double s2 = warp_sum(sq.value());
    double ds[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) ds[c] = c < kc ? warp_sum(dot[c].value()) : 0.0;
    if (lane == 0) {
        const double sj = s2 > 0.0 ? sqrt(s2) : 1.0;
        s[j] = sj;
        inv_s[j] = 1.0 / sj;
        for (int c = 0; c < kc; ++c) q64[(int64_t)c * ldq + j] = -ds[c] / sj;
    }
}

// One block per column tile: wbase[tile·W + w] = occupied boxes of the tile
// in words before w; cnt[tile] = occupied boxes of the tile.
__global__ void __launch_bounds__(kCscThreads) k_csc_tiles(const uint32_t* __restrict__ occ, int W,
                                                           int32_t* __restrict__ wbase,
                                                           int64_t* __restrict__ cnt) {
    __shared__ int64_t s_w[kCscWarps];
    const int64_t base = (int64_t)blockIdx.x * W;
    int64_t run = 0;
    for (int w0 = 0; w0 < W; w0 += kCscThreads) {
        const int w = w0 + threadIdx.x;
        const int64_t c = w < W ? __popc(occ[base + w]) : 0;
        int64_t tot;
        const int64_t ex = block_scan_excl(c, s_w, &tot);
        if (w < W) wbase[base + w] = (int32_t)(run + ex);
        run += tot;
    }
    if (threadIdx.x == 0) cnt[blockIdx.x] = run;
}

// One block: toff[I] = Σ_{J<I} cnt[J] for I ≤ T (toff[T] = all boxes).
__global__ void __launch_bounds__(kCscThreads) k_csc_offsets(const int64_t* __restrict__ cnt,
                                                             int64_t T,
                                                             int64_t* __restrict__ toff) {
    __shared__ int64_t s_w[kCscWarps];
    int64_t run = 0;
    for (int64_t i0 = 0; i0 < T; i0 += kCscThreads) {
        const int64_t i = i0 + threadIdx.x;
        const int64_t c = i < T ? cnt[i] : 0;
        int64_t tot;
        const int64_t ex = block_scan_excl(c, s_w, &tot);
        if (i < T) toff[i] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) toff[T] = run;
}

// One warp per column: every entry's three BF16 terms into its box (boxes
// zeroed beforehand; rows ≥ d and columns ≥ n stay zero).
template <typename T>
__global__ void __launch_bounds__(kCscThreads)
    k_csc_pack(const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
               const T* __restrict__ v, int64_t n, const uint32_t* __restrict__ occ, int W,
               const int32_t* __restrict__ wbase, const int64_t* __restrict__ toff,
               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ mid,
               __nv_bfloat16* __restrict__ lo) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kCscWarps + (threadIdx.x >> 5);
    if (j >= n) return;
    const int64_t p0 = cp[j], p1 = cp[j + 1];
    const int64_t tw = (j >> 7) * (int64_t)W;
    const int64_t t0 = toff[j >> 7];
    for (int64_t t = p0 + lane; t < p1; t += 32) {
        const int32_t r = ri[t];
        const int kb = r >> 6, w = kb >> 5;
        const uint32_t below = (1u << (kb & 31)) - 1u;
        const int64_t box = t0 + wbase[tw + w] + __popc(occ[tw + w] & below);
        const int64_t at = pack_index(box, 0, (int)(j & 127), r & 63);
        __nv_bfloat16 h, m, l;
        split3_bf16((float)v[t], h, m, l);
        hi[at] = h;
        mid[at] = m;
        lo[at] = l;
    }
}

// ---------------------------------------------------------------------------
// FP64 KKT residual of Def. 1 from the CSC form (FP32 values), the same
// quantities as the dense pass (kkt.cu) without a dense copy of A:
//   k_csc_kkt_ax   one block per 64-row block kb: r = A x − b over the occupied
//                  boxes of the packed operand — their three BF16 terms add up
//                  exactly to the FP32 entry (h + (m + l) = a) — visiting the
//                  column tiles in increasing order (a fixed summation order),
//                  and fpart[kb] = Σ r² over the block;
//   k_csc_kkt_grad one warp per column: ∇F_j = A_jᵀ r from the stored entries,
//                  g_j = ∇F_j / s_j (kept for the refinement), ḡ_j² on P(s·x).
// ---------------------------------------------------------------------------
// Lower-triangle pair index t → (I, J), J ≤ I, t = I(I+1)/2 + J.
__device__ __forceinline__ void tri_pair(int64_t t, int& I, int& J) {
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    I = (int)r;
    J = (int)(t - r * (r + 1) / 2);
}

// One warp per tile pair: the K blocks occupied in both tiles.
__global__ void __launch_bounds__(kCscThreads) k_csc_pairs(const uint32_t* __restrict__ occ, int W,
                                                           int64_t P, int32_t* __restrict__ Lp) {
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kCscWarps + (threadIdx.x >> 5);
    if (p >= P) return;
    int I, J;
    tri_pair(p, I, J);
    const uint32_t* oa = occ + (int64_t)I * W;
    const uint32_t* ob = occ + (int64_t)J * W;
    int c = 0;
    for (int w = lane; w < W; w += 32) c += __popc(oa[w] & ob[w]);
    c = warp_sum_i(c);
    if (lane == 0) Lp[p] = c;
}

// One block: the chunk size KC from the total work, then every non-empty
// pair's chunks (even split of its Lp blocks) and partial slots for the pairs
// split in more than one chunk, in pair order.
__global__ void __launch_bounds__(kCscThreads) k_csc_items(const int32_t* __restrict__ Lp, int64_t P,
                                                           int num_sms, SItem* __restrict__ items,
                                                           int64_t* __restrict__ meta) {
    __shared__ int64_t s_w[kCscWarps];
    int64_t tot = 0;
    for (int64_t p0 = 0; p0 < P; p0 += kCscThreads) {
        const int64_t p = p0 + threadIdx.x;
        int64_t t;
        block_scan_excl(p < P ? Lp[p] : 0, s_w, &t);
        tot += t;
    }
    const int64_t kc0 = (tot + num_sms - 1) / num_sms;
    const int64_t KC = kc0 > 16 ? kc0 : 16;
    int64_t run_i = 0, run_s = 0;
    for (int64_t p0 = 0; p0 < P; p0 += kCscThreads) {
        const int64_t p = p0 + threadIdx.x;
        const int64_t L = p < P ? Lp[p] : 0;
        const int64_t S = L > 0 ? (L + KC - 1) / KC : 0;
        int64_t ti, ts;
        const int64_t ei = block_scan_excl(S, s_w, &ti);
        const int64_t es = block_scan_excl(S > 1 ? S : 0, s_w, &ts);
        if (S > 0) {
            int I, J;
            tri_pair(p, I, J);
            for (int64_t c = 0; c < S; ++c) {
                const int64_t k0 = c * L / S, k1 = (c + 1) * L / S;
                SItem it;
                it.I = I;
                it.J = J;
                it.k0 = (int32_t)k0;
                it.nk = (int32_t)(k1 - k0);
                it.S = (int32_t)S;
                it.c = (int32_t)c;
                it.slot = S > 1 ? (int32_t)(run_s + es + c) : -1;
                it.pair = (int32_t)p;
                items[run_i + ei + c] = it;
            }
        }
        run_i += ti;
        run_s += ts;
    }
    if (threadIdx.x == 0) {
        meta[0] = run_i;
        meta[1] = run_s;
    }
}

// Non-zero tiles of Q: every pair with a common block marks its tile and
// the mirror, bit rt of mask[ct·tw + rt/32] (mask zeroed beforehand).
__global__ void __launch_bounds__(kCscThreads) k_csc_qmask(const int32_t* __restrict__ Lp,
                                                           int64_t P, int tw,
                                                           uint32_t* __restrict__ mask) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || Lp[p] == 0) return;
    int I, J;
    tri_pair(p, I, J);
    atomicOr(&mask[(int64_t)J * tw + (I >> 5)], 1u << (I & 31));
    atomicOr(&mask[(int64_t)I * tw + (J >> 5)], 1u << (J & 31));
}

// Float-pair accumulator on the FP32 pipe (this GPU's FP64 pipe is narrow):
// += a·(h + l) with the product's rounding error from an FMA (TwoProduct) and
// the addition's from TwoSum kept in c (Ogita, Rump & Oishi 2005).
struct FPair {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a, float h, float l) {
        const float p = __fmul_rn(a, h);
        const float ep = fmaf(a, h, -p);
        const float t = s + p;
        const float z = t - s;
        c += ((s - (t - z)) + (p - z)) + fmaf(a, l, ep);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Thread t owns rows 8·(t mod 8) … +7 of the block (one 16-byte chunk of
// eight BF16 per split term and column) for the four columns 4·(t / 8) … +3 of
// every tile; x_j enters as the FP32 pair (hi, lo) and each row sums in a
// float pair, flushed to FP64 every 16 tiles; the 32 column groups' partial
// rows are then added in a fixed order.  Writes r in FP64 and as FP32 pairs.
__global__ void __launch_bounds__(kCscThreads)
    k_csc_kkt_ax(const uint32_t* __restrict__ occ, int W, const int32_t* __restrict__ wbase,
                 const int64_t* __restrict__ toff, int64_t T, const __nv_bfloat16* __restrict__ hi,
                 const __nv_bfloat16* __restrict__ mid, const __nv_bfloat16* __restrict__ lo,
                 const double* __restrict__ x, int64_t n, const float* __restrict__ b, int64_t d,
                 double* __restrict__ r, float* __restrict__ rh, float* __restrict__ rl,
                 double* __restrict__ fpart) {
    __shared__ float2 s_x[128];
    __shared__ double s_part[32][65];
    __shared__ int s_list[kCscThreads];
    __shared__ int s_wc[kCscWarps];
    __shared__ double s_red[kCscWarps];
    const int kb = blockIdx.x, wq = kb >> 5;
    const uint32_t bit = 1u << (kb & 31);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ch = threadIdx.x & 7, cg = threadIdx.x >> 3;  // row chunk, column group
    double accd[8];
    FPair acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) accd[e] = 0.0;
    int since = 0;  // tiles added into the pairs since their last flush
    for (int64_t I0 = 0; I0 < T; I0 += kCscThreads) {
        // the tiles of this chunk that hold block kb, in increasing order
        const int64_t I = I0 + threadIdx.x;
        const bool has = I < T && (occ[I * W + wq] & bit);
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        if (lane == 0) s_wc[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kCscWarps; ++w) {
            before += w < wid ? s_wc[w] : 0;
            total += s_wc[w];
        }
        if (has) s_list[before + __popc(bal & ((1u << lane) - 1u))] = (int)(I - I0);
        __syncthreads();
        for (int u = 0; u < total; ++u) {
            const int64_t tI = I0 + s_list[u];
            const int64_t ow = tI * W + wq;
            const int64_t box = toff[tI] + wbase[ow] + __popc(occ[ow] & (bit - 1u));
            if (threadIdx.x < 128) {
                const int64_t j = tI * 128 + threadIdx.x;
                const double xv = j < n ? x[j] : 0.0;
                const float xh = (float)xv;
                s_x[threadIdx.x] = make_float2(xh, (float)(xv - (double)xh));
            }
            __syncthreads();
            const int64_t base = box * kPackTile;
            uint4 vh[4], vm[4], vl[4];
            float2 xq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = cg * 4 + q;
                xq[q] = s_x[c];
                // 16-byte chunk ch of column c sits at chunk position ch ^ (c mod 8)
                const int64_t at = base + c * 64 + ((ch ^ (c & 7)) << 3);
                if (xq[q].x != 0.0f) {  // x is sparse at the optimum
                    vh[q] = __ldg(reinterpret_cast<const uint4*>(hi + at));
                    vm[q] = __ldg(reinterpret_cast<const uint4*>(mid + at));
                    vl[q] = __ldg(reinterpret_cast<const uint4*>(lo + at));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (xq[q].x == 0.0f) continue;
                const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&vh[q]);
                const __nv_bfloat16* m8 = reinterpret_cast<const __nv_bfloat16*>(&vm[q]);
                const __nv_bfloat16* l8 = reinterpret_cast<const __nv_bfloat16*>(&vl[q]);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float a = __bfloat162float(h8[e]) +
                                    (__bfloat162float(m8[e]) + __bfloat162float(l8[e]));
                    acc[e].add(a, xq[q].x, xq[q].y);
                }
            }
            if (++since == 16) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    accd[e] += acc[e].value();
                    acc[e] = FPair();
                }
                since = 0;
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) s_part[cg][ch * 8 + e] = accd[e] + acc[e].value();
    __syncthreads();
    double v2 = 0.0;
    if (threadIdx.x < 64) {
        const int64_t row = (int64_t)kb * 64 + threadIdx.x;
        double v = 0.0;
        for (int g = 0; g < 32; ++g) v += s_part[g][threadIdx.x];
        if (row < d) {
            v -= (double)b[row];
            r[row] = v;
            const float h = (float)v;
            rh[row] = h;
            rl[row] = (float)(v - (double)h);
            v2 = v * v;
        }
    }
    v2 = warp_sum(v2);
    if (lane == 0) s_red[wid] = v2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kCscWarps; ++w) t += s_red[w];
        fpart[kb] = t;
    }
}

// One warp per column: ∇F_j = A_jᵀ r from the stored entries, in float pairs
// (r as FP32 pairs) per lane, lanes added in FP64.
__global__ void __launch_bounds__(kCscThreads)
    k_csc_kkt_grad(const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                   const float* __restrict__ v, int64_t n, const float* __restrict__ rh,
                   const float* __restrict__ rl, const double* __restrict__ s,
                   const double* __restrict__ x, double* __restrict__ g64,
                   double* __restrict__ gpart) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kCscWarps + (threadIdx.x >> 5);
    if (j >= n) return;
    FPair acc;
    for (int64_t t = cp[j] + lane; t < cp[j + 1]; t += 32) {
        const int32_t row = ri[t];
        acc.add(v[t], rh[row], rl[row]);
    }
    const double grad = warp_sum(acc.value());
    if (lane == 0) {
        const double gj = grad / s[j];
        const double yj = x[j] * s[j];
        g64[j] = gj;
        gpart[j] = (yj > 0.0 || gj < 0.0) ? gj * gj : 0.0;
    }
}

}  // namespace

cudaError_t launch_csc_kkt(const int64_t* cp, const int32_t* ri, const float* v, int64_t d,
                           int64_t n, const uint32_t* occ, int W, const int32_t* wbase,
                           const int64_t* toff, const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                           const __nv_bfloat16* lo, const double* x, const float* b,
                           const double* s, double* r, float* rh, float* rl, double* fpart,
                           double* g64, double* gpart, cudaStream_t st) {
    const int64_t T = ceil_div(n, 128), KB = ceil_div(d, 64);
    k_csc_kkt_ax<<<(unsigned)KB, kCscThreads, 0, st>>>(occ, W, wbase, toff, T, hi, mid, lo, x, n, b,
                                                       d, r, rh, rl, fpart);
    k_csc_kkt_grad<<<(unsigned)ceil_div(n, kCscWarps), kCscThreads, 0, st>>>(cp, ri, v, n, rh, rl, s,
                                                                            x, g64, gpart);
    return cudaGetLastError();
}

cudaError_t launch_csc_check(const int64_t* cp, const int32_t* ri, const void* v, int32_t dtype,
                             int64_t d, int64_t n, int64_t nnz, int* flags, cudaStream_t st) {
    const unsigned grid = (unsigned)ceil_div(n, kCscWarps);
    if (dtype == ALN_DTYPE_F64)
        k_csc_check<double><<<grid, kCscThreads, 0, st>>>(cp, ri, (const double*)v, d, n, nnz, flags);
    else
        k_csc_check<float><<<grid, kCscThreads, 0, st>>>(cp, ri, (const float*)v, d, n, nnz, flags);
    return cudaGetLastError();
}

cudaError_t launch_csc_colstats(const int64_t* cp, const int32_t* ri, const void* v,
                                int32_t dtype, int64_t n, const void* B, int kc, int64_t ldb,
                                void* A, int64_t lda, double* s, double* inv_s, double* q64,
                                int64_t ldq, uint32_t* occ, int W, cudaStream_t st) {
    const unsigned grid = (unsigned)ceil_div(n, kCscWarps);
#define ALN_CSC_STATS(T, OCC)                                                                    \
    k_csc_colstats<T, OCC><<<grid, kCscThreads, 0, st>>>(cp, ri, (const T*)v, n, (const T*)B, kc, \
                                                         ldb, (T*)A, lda, s, inv_s, q64, ldq,    \
                                                         occ, W)
    if (dtype == ALN_DTYPE_F64) {
        if (occ)
            ALN_CSC_STATS(double, true);
        else
            ALN_CSC_STATS(double, false);
    } else {
        if (occ)
            ALN_CSC_STATS(float, true);
        else
            ALN_CSC_STATS(float, false);
    }
#undef ALN_CSC_STATS
    return cudaGetLastError();
}

cudaError_t launch_csc_number(const uint32_t* occ, int W, int64_t T, int32_t* wbase, int64_t* cnt,
                              int64_t* toff, cudaStream_t st) {
    k_csc_tiles<<<(unsigned)T, kCscThreads, 0, st>>>(occ, W, wbase, cnt);
    k_csc_offsets<<<1, kCscThreads, 0, st>>>(cnt, T, toff);
    return cudaGetLastError();
}

cudaError_t launch_csc_worklist(const uint32_t* occ, int W, int64_t T, int num_sms, int32_t* Lp,
                                SItem* items, int64_t* meta, cudaStream_t st) {
    const int64_t P = T * (T + 1) / 2;
    k_csc_pairs<<<(unsigned)ceil_div(P, kCscWarps), kCscThreads, 0, st>>>(occ, W, P, Lp);
    k_csc_items<<<1, kCscThreads, 0, st>>>(Lp, P, num_sms, items, meta);
    return cudaGetLastError();
}

cudaError_t launch_csc_qmask(const int32_t* Lp, int64_t T, uint32_t* mask, cudaStream_t st) {
    const int64_t P = T * (T + 1) / 2;
    const int tw = (int)ceil_div(T, 32);
    cudaError_t e = cudaMemsetAsync(mask, 0, (size_t)T * tw * 4, st);
    if (e != cudaSuccess) return e;
    k_csc_qmask<<<(unsigned)ceil_div(P, kCscThreads), kCscThreads, 0, st>>>(Lp, P, tw, mask);
    return cudaGetLastError();
}

cudaError_t launch_csc_pack(const int64_t* cp, const int32_t* ri, const void* v, int32_t dtype,
                            int64_t n, const uint32_t* occ, int W, const int32_t* wbase,
                            const int64_t* toff, __nv_bfloat16* hi, __nv_bfloat16* mid,
                            __nv_bfloat16* lo, cudaStream_t st) {
    const unsigned grid = (unsigned)ceil_div(n, kCscWarps);
    if (dtype == ALN_DTYPE_F64)
        k_csc_pack<double><<<grid, kCscThreads, 0, st>>>(cp, ri, (const double*)v, n, occ, W, wbase,
                                                         toff, hi, mid, lo);
    else
        k_csc_pack<float><<<grid, kCscThreads, 0, st>>>(cp, ri, (const float*)v, n, occ, W, wbase,
                                                        toff, hi, mid, lo);
    return cudaGetLastError();
}

}  // namespace aln
