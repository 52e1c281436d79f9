// Split-BF16 Gram on the 5th-generation tensor cores (tcgen05 + TMA, sm_103a).
//
// Alg. 1 (§3) forms H = AᵀA and Q = D⁻¹HD⁻¹ with D = diag(√H_ii) (Eq. NQPQ).
// Here every FP32 element of A is split exactly into three BF16 terms,
// a = h + m + l (|m| ≤ 2⁻⁸|a|, |l| ≤ 2⁻¹⁶|a|), and
//     H ≈ hᵀh + hᵀm + mᵀh + mᵀm + hᵀl + lᵀh
// (the dropped m·l, l·m, l·l terms are ≤ 2·2⁻²⁴|a_i a_j|) is accumulated in
// FP32 in tensor memory.  A two-term split (error 2⁻¹⁸ per product) perturbs
// Q by about n·10⁻⁵ in norm — as large as λ_min(Q) at n = 5000 — and made
// Alg. 2 several times slower to converge; the third term costs twice the
// tensor work and removes that.  The epilogue multiplies by the FP64 scale
// factors 1/s_i, 1/s_j (rounded to FP32), sets Q_ii to 1 (0 for a zero
// column, Eq. Rescaling) and writes each lower-triangle tile and its mirror.
//
// Kernel structure: one 128×128 output tile per CTA (see gram_tile below for
// the loader, MMA and promotion roles).  Every wait is bounded (1 s on
// %globaltimer); on expiry the CTA sets *timeout_flag, waits (bounded) for its
// own copies and MMAs, frees its tensor memory and exits without storing.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace aln {
namespace tc {

struct GramArgs {
    int64_t n;
    int64_t t0;  // first lower-triangle tile of this launch (a range of tile rows)
    int num_kb;
    int S;                 // chunks of the K range per tile pair (split K; 1 = none)
    float* part;           // S partial tiles per pair (S > 1)
    unsigned int* ticket;  // one counter per pair of the launch (S > 1)
    const double* inv_s;
    float* Q;
    int64_t ldq;
    int* timeout_flag;
};

__device__ __forceinline__ void tri_decode(int64_t t, int& I, int& J) {
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    I = (int)r;
    J = (int)(t - r * (r + 1) / 2);
}

// ---------------------------------------------------------------------------
// Three-term split Gram with promoted accumulation.
//
// The tensor core adds each MMA's products into its FP32 accumulator with
// truncation: measured on this GPU, the Gram of FP32 data carries a negative
// bias growing linearly with the number of accumulation steps (about
// −4.7·10⁻⁹·d relative), so a Gram over d = 20000 rows is off by ~10⁻⁴ in every
// entry — a near rank-one perturbation of norm ~n·10⁻⁴, larger than λ_min(Q).
// Here every 64-wide K block is summed into a fresh TMEM accumulator (the
// five small cross terms first, then the four h·h steps, so only four large
// truncating steps per block) and four promotion warps add it into FP32
// registers with round-to-nearest while the MMA thread fills the other of two
// TMEM accumulators.
//
// Roles (192 threads): warp 0, one lane: loads (TMA tiles or bulk copies of
// pre-swizzled tiles) into a 2-stage ring of 6 boxes (A: h, m, l; B: h, m, l);
// warp 1, one lane: the MMAs; warps 2–5: promotion, then scale and store (warp
// w owns TMEM lanes and tile rows 32·(w mod 4) … +31).  Every wait is bounded.
// ---------------------------------------------------------------------------
// NS = number of split terms (3: h, m, l; 2: h, m).  Stages of 2·NS boxes;
// K blocks per promoted accumulator (CHUNK): 1 with six products per K step,
// 2 with three (the MMA would otherwise outrun the promotion).
template <int NS>
struct GramCfg {
    static constexpr int STAGES = NS == 3 ? 2 : 3;
    static constexpr int STAGE_BYTES = 2 * NS * TILE_BYTES;
    static constexpr int CHUNK = NS == 3 ? 1 : 2;
};
constexpr int G3_SMEM_BYTES = 2 * 6 * TILE_BYTES + 1024 + 256;  // = 3·4·TILE_BYTES + …
constexpr int G3_THREADS = 192;
constexpr uint32_t G3_TMEM_COLS = 2 * BM;  // two 128-column accumulators

// One K block of the split products, the small cross terms first and the
// four h·h steps last (`fresh` starts a new accumulator).  NS = 3: hm, mh,
// mm, hl, lh, then hh; NS = 2: hm, mh, then hh.  a/b: shared addresses of the
// h boxes (m, l follow at TILE_BYTES, 2·TILE_BYTES).
template <int NS>
__device__ __forceinline__ void gram_chunk(uint32_t tmem, uint32_t a, uint32_t b, bool fresh) {
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BM);
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;  // 16 BF16 along K
        const uint64_t ah = sdesc_sw128(a + off), am = sdesc_sw128(a + TILE_BYTES + off);
        const uint64_t bh = sdesc_sw128(b + off), bm = sdesc_sw128(b + TILE_BYTES + off);
        umma_bf16(tmem, ah, bm, idesc, (fresh && kk == 0) ? 0u : 1u);
        umma_bf16(tmem, am, bh, idesc, 1u);
        if (NS == 3) {
            const uint64_t al = sdesc_sw128(a + 2 * TILE_BYTES + off),
                           bl = sdesc_sw128(b + 2 * TILE_BYTES + off);
            umma_bf16(tmem, am, bm, idesc, 1u);
            umma_bf16(tmem, ah, bl, idesc, 1u);
            umma_bf16(tmem, al, bh, idesc, 1u);
        }
    }
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;
        umma_bf16(tmem, sdesc_sw128(a + off), sdesc_sw128(b + off), idesc, 1u);
    }
}

// acc[c] += the accumulator row this thread's lane reads (128 columns).
__device__ __forceinline__ void gram_promote(float (&acc)[BM], uint32_t tb) {
#pragma unroll
    for (int c0 = 0; c0 < BM; c0 += 16) {
        float v[16];
        tmem_ld16(tb + c0, v);
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[c0 + t] += v[t];
    }
}

// Scale and store one promoted tile row: Q_ij = H_ij·(1/s_i)·(1/s_j) (FP32
// factors), Q_ii = 1 (0 for a zero column, Eq. Rescaling); diagonal tiles keep
// the lower triangle and mirror it, so Q is exactly symmetric.
__device__ __forceinline__ void gram_store(const float (&acc)[BM], int64_t row, int64_t n0,
                                            bool diag, int64_t n, const double* __restrict__ inv_s,
                                            const float* s_cs, float* __restrict__ Q,
                                            int64_t ldq) {
    const bool rv = row < n;
    if (!rv) return;
    const float rs = (float)inv_s[row];
    const int cols = (int)(n - n0 < (int64_t)BM ? n - n0 : (int64_t)BM);
#pragma unroll
    for (int c0 = 0; c0 < BM; c0 += 16) {
        if (c0 >= cols) continue;
        float o[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            o[t] = acc[c0 + t] * rs * s_cs[c0 + t];
            if (diag && row == n0 + c0 + t) o[t] = acc[c0 + t] != 0.0f ? 1.0f : 0.0f;
        }
        const int64_t j0 = n0 + c0;
        if (diag) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int64_t j = j0 + t;
                if (c0 + t < cols && j <= row) {
                    Q[row * ldq + j] = o[t];
                    Q[j * ldq + row] = o[t];
                }
            }
        } else {
            float* dst = Q + row * ldq + j0;
            if (c0 + 16 <= cols) {
#pragma unroll
                for (int t = 0; t < 16; t += 4)
                    *reinterpret_cast<float4*>(dst + t) =
                        make_float4(o[t], o[t + 1], o[t + 2], o[t + 3]);
            } else {
                for (int t = 0; t < cols - c0; ++t) dst[t] = o[t];
            }
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (c0 + t < cols) Q[(j0 + t) * ldq + row] = o[t];
        }
    }
}

// One 128×128 output tile of a split product, accumulated in FP32 registers:
// acc[c] of the promotion warps (warp w ≥ 2 holds tile row 32·(w mod 4) +
// lane) = Σ_K A[row]·B[c] over the num_kb K blocks the loader copies (A and B
// boxes of NS terms each; diag: B = A, one set of boxes).  Sets up its
// barriers; returns false (uniformly) when a bounded wait expired — nothing is
// then in flight and acc is incomplete.  Tensor memory (G3_TMEM_COLS columns):
// `tmem_given` when the caller holds it (a CTA that runs several tiles
// allocates once — no allocation may follow the relinquish of the permit),
// else allocated and freed here.
constexpr uint32_t kNoTmem = 0xffffffffu;

template <int NS, class Loader>
__device__ __forceinline__ bool promoted_tile(Loader& ld, int num_kb, bool diag,
                                              float (&acc)[BM], uint32_t tmem_given = kNoTmem) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    using C = GramCfg<NS>;
    uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);  // one arrival per promotion warp
        }
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bool own = tmem_given == kNoTmem;
    if (own && warp == 1) {
        tmem_alloc(tmem_slot, G3_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = own ? *tmem_slot : tmem_given;
#pragma unroll
    for (int c = 0; c < BM; ++c) acc[c] = 0.0f;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int kb = 0; kb < num_kb; ++kb) {
            const int s = kb % C::STAGES;
            if (kb >= C::STAGES && !mbar_wait(&empty[s], ((kb / C::STAGES) & 1) ^ 1)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            uint8_t* sb = smem + s * C::STAGE_BYTES;
            mbar_expect_tx(&full[s], (diag ? NS : 2 * NS) * TILE_BYTES);
            ld.load(sb, kb, diag, &full[s]);
            ++issued;
        }
        // our own copies in flight: the last ≤ STAGES loads (bounded wait)
        for (int kb = max(0, issued - C::STAGES); kb < issued; ++kb)
            if (!mbar_wait(&full[kb % C::STAGES], (kb / C::STAGES) & 1)) s_abort = 1;
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < num_kb; ++kb) {
            const int s = kb % C::STAGES, ch = kb / C::CHUNK, b = ch & 1;
            const bool fresh = kb % C::CHUNK == 0;
            const bool last = kb % C::CHUNK == C::CHUNK - 1 || kb == num_kb - 1;
            if (!mbar_wait(&full[s], (kb / C::STAGES) & 1) ||
                (fresh && ch >= 2 && !mbar_wait(&tempty[b], ((ch >> 1) & 1) ^ 1))) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + s * C::STAGE_BYTES);
            const uint32_t b0 = diag ? a0 : a0 + NS * TILE_BYTES;
            gram_chunk<NS>(tmem + (uint32_t)(b * BM), a0, b0, fresh);
            umma_commit(&empty[s]);
            if (last) umma_commit(&tfull[b]);
        }
        // always commit (but for an empty K range): `done` then also covers
        // MMAs issued before an abort
        if (num_kb > 0) umma_commit(done);
    } else if (warp >= 2) {
        const uint32_t tb = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        const int nch = (num_kb + C::CHUNK - 1) / C::CHUNK;
        for (int kb = 0; kb < nch; ++kb) {  // kb: chunk index
            const int b = kb & 1;
            if (!mbar_wait(&tfull[b], (kb >> 1) & 1)) {
                s_abort = 1;
                break;
            }
            tc_fence_after();
            gram_promote(acc, tb + (uint32_t)(b * BM));
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
            if (*(volatile int*)&s_abort) break;
        }
    }
    __syncwarp();
    if (warp == 1 && num_kb > 0) {
        const bool ok = mbar_wait(done, 0);  // no MMA in flight past this point
        if (!ok) s_abort = 1;
    }
    tc_fence_after();
    __syncthreads();
    const bool ok = !s_abort;
    tc_fence_before();
    __syncthreads();
    if (own && warp == 1) tmem_dealloc(tmem, G3_TMEM_COLS);
    return ok;
}

// One lower-triangle output tile of Q = D⁻¹HD⁻¹ (rows m0.., columns n0..).
// The loader is taken by value: a loader may keep a cursor over the K blocks
// it copies (k_sgram_tc); load() is called for the blocks in order.
//
// Split K (part ≠ null): this CTA is chunk c of S of its tile pair; it writes
// its unscaled partial tile to part + c·128² (part points at the pair's first
// slot), and the pair's last chunk to arrive on *ticket adds the S partials
// in slot order — a fixed order, whichever CTA is last — and stores the tile.
//
// Returns false (uniformly) after a timeout.  Ends with a block barrier, so a
// CTA may run several tiles in turn (tmem: as for promoted_tile).
template <int NS, class Loader>
__device__ __forceinline__ bool gram_tile(Loader ld, int num_kb, bool diag, int64_t m0,
                                           int64_t n0, int64_t n, const double* __restrict__ inv_s,
                                           float* __restrict__ Q, int64_t ldq,
                                           int* timeout_flag, float* part = nullptr, int S = 1,
                                           int c = 0, unsigned int* ticket = nullptr,
                                           uint32_t tmem = kNoTmem) {
    __shared__ float s_cs[BM];
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < BM) {  // visible after promoted_tile's first barrier
        const int64_t j = n0 + threadIdx.x;
        s_cs[threadIdx.x] = j < n ? (float)inv_s[j] : 0.0f;
    }
    float acc[BM];
    const bool ok = promoted_tile<NS>(ld, num_kb, diag, acc, tmem);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(timeout_flag, 1);
        return false;
    }
    if (part == nullptr) {
        if (warp >= 2)
            gram_store(acc, m0 + 32 * (warp & 3) + lane, n0, diag, n, inv_s, s_cs, Q, ldq);
        __syncthreads();  // s_cs is rewritten by the next tile of this CTA
        return true;
    }
    const int row = 32 * (warp & 3) + lane;
    if (warp >= 2) {
        float4* dst = reinterpret_cast<float4*>(part + ((int64_t)c * BM + row) * BM);
#pragma unroll
        for (int t = 0; t < BM / 4; ++t)
            __stcg(dst + t, make_float4(acc[4 * t], acc[4 * t + 1], acc[4 * t + 2],
                                        acc[4 * t + 3]));
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == (unsigned int)(S - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (warp >= 2) {
#pragma unroll
            for (int t = 0; t < BM; ++t) acc[t] = 0.0f;
            for (int q = 0; q < S; ++q) {
                const float4* src =
                    reinterpret_cast<const float4*>(part + ((int64_t)q * BM + row) * BM);
#pragma unroll
                for (int t = 0; t < BM / 4; ++t) {
                    const float4 v = __ldcg(src + t);
                    acc[4 * t] += v.x;
                    acc[4 * t + 1] += v.y;
                    acc[4 * t + 2] += v.z;
                    acc[4 * t + 3] += v.w;
                }
            }
            gram_store(acc, m0 + row, n0, diag, n, inv_s, s_cs, Q, ldq);
        }
        if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch
    }
    __syncthreads();  // s_cs and s_last are rewritten by the next tile of this CTA
    return true;
}

template <int NS>
struct TmaLoader {
    const CUtensorMap* mh;
    const CUtensorMap* mm;
    const CUtensorMap* ml;
    int m0, n0;
    int k0;  // first K block of this CTA's chunk
    __device__ __forceinline__ void load(uint8_t* sb, int kb, bool diag, uint64_t* bar) const {
        const int x = (kb + k0) * BK;
        tma_load_2d(sb, mh, bar, x, m0);
        tma_load_2d(sb + TILE_BYTES, mm, bar, x, m0);
        if (NS == 3) tma_load_2d(sb + 2 * TILE_BYTES, ml, bar, x, m0);
        if (!diag) {
            tma_load_2d(sb + NS * TILE_BYTES, mh, bar, x, n0);
            tma_load_2d(sb + (NS + 1) * TILE_BYTES, mm, bar, x, n0);
            if (NS == 3) tma_load_2d(sb + 5 * TILE_BYTES, ml, bar, x, n0);
        }
    }
};

// Stream-K pass over the pairs [t0, t0 + R) (the last partial wave): CTA b of
// G takes the K blocks [⌊bW/G⌋, ⌊(b+1)W/G⌋) of the W = R·num_kb blocks laid
// out pair after pair, one pair segment at a time.  A pair whose blocks span
// several CTAs is summed from their partial tiles in CTA order (a fixed
// order) by the last of them to finish.
struct GramSK {
    int64_t R;
    int G;
    int maxseg;
    float* part;            // R × maxseg partial tiles
    unsigned int* ticket;   // R
};

__device__ __forceinline__ int64_t sk_owner(int64_t x, int64_t W, int G) {
    // the CTA b with ⌊bW/G⌋ ≤ x < ⌊(b+1)W/G⌋
    int64_t b = x * G / W;
    while (b + 1 < G && (b + 1) * W / G <= x) ++b;
    while (b > 0 && b * W / G > x) --b;
    return b;
}

template <int NS>
__global__ void __launch_bounds__(G3_THREADS, 1)
    k_gram_sk(const __grid_constant__ CUtensorMap m_hi, const __grid_constant__ CUtensorMap m_mid,
              const __grid_constant__ CUtensorMap m_lo, GramArgs p, GramSK sk) {
    const int64_t nkb = p.num_kb, W = sk.R * nkb;
    const int64_t b = blockIdx.x;
    const int64_t g0 = b * W / sk.G, g1 = (b + 1) * W / sk.G;
    if (g0 >= g1) return;  // uniform: no work, no tensor memory
    // tensor memory for every segment of this CTA, allocated once
    __shared__ uint32_t s_tmem;
    if (threadIdx.x >> 5 == 1) {
        tmem_alloc(&s_tmem, G3_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    for (int64_t g = g0; g < g1;) {
        const int64_t tl = g / nkb;  // pair of the tail
        const int64_t kb0 = g - tl * nkb;
        const int64_t kb1 = min(nkb, g1 - tl * nkb);
        const int64_t first = sk_owner(tl * nkb, W, sk.G);
        const int64_t last = sk_owner((tl + 1) * nkb - 1, W, sk.G);
        const int nseg = (int)(last - first + 1), seg = (int)(b - first);
        int tm, tn;
        tri_decode(p.t0 + tl, tm, tn);
        const TmaLoader<NS> ld{&m_hi, &m_mid, &m_lo, tm * BM, tn * BM, (int)kb0};
        float* part = nseg > 1 ? sk.part + tl * sk.maxseg * (int64_t)(BM * BM) : nullptr;
        if (!gram_tile<NS>(ld, (int)(kb1 - kb0), tm == tn, (int64_t)tm * BM, (int64_t)tn * BM,
                           p.n, p.inv_s, p.Q, p.ldq, p.timeout_flag, part, nseg, seg,
                           sk.ticket + tl, tmem))
            break;  // timed out: nothing in flight (the flag is set)
        g = tl * nkb + kb1;
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x >> 5 == 1) tmem_dealloc(tmem, G3_TMEM_COLS);
}

template <int NS>
__global__ void __launch_bounds__(G3_THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap m_hi, const __grid_constant__ CUtensorMap m_mid,
              const __grid_constant__ CUtensorMap m_lo, GramArgs p) {
    // CTA = (tile pair, chunk c of S): K blocks [c·num_kb/S, (c+1)·num_kb/S)
    const int64_t pi = blockIdx.x / p.S;
    const int c = (int)(blockIdx.x - pi * p.S);
    int tm, tn;
    tri_decode(pi + p.t0, tm, tn);
    const int k0 = (int)((int64_t)c * p.num_kb / p.S);
    const int k1 = (int)((int64_t)(c + 1) * p.num_kb / p.S);
    const TmaLoader<NS> ld{&m_hi, &m_mid, &m_lo, tm * BM, tn * BM, k0};
    float* part = p.S > 1 ? p.part + pi * p.S * (int64_t)(BM * BM) : nullptr;
    gram_tile<NS>(ld, k1 - k0, tm == tn, (int64_t)tm * BM, (int64_t)tn * BM, p.n, p.inv_s, p.Q,
                  p.ldq, p.timeout_flag, part, p.S, c, p.ticket + pi);
}

// ---------------------------------------------------------------------------
// Grouped Gram: the lower-triangle tiles of many problems' Q_p in one launch.
// The operands come pre-tiled (pack_index): every 128×64 BF16 box is 16 KiB
// contiguous in global memory, already in the 128-byte-swizzled order, so the
// loader moves it with a 1-D bulk copy (cp.async.bulk) — no tensor map per
// problem.  The tile table is sorted by K length (longest first) on the host.
// ---------------------------------------------------------------------------
struct GGramArgs {
    const GProb* gp;
    const GTile* tiles;
    const __nv_bfloat16* hi;
    const __nv_bfloat16* mid;
    const __nv_bfloat16* lo;
    const double* inv_s;  // packed by GProb::voff
    float* Q;             // pool; problem p at GProb::qoff, row length GProb::ldq
    int* timeout_flag;
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    uint64_t gaddr;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(gaddr) : "l"(reinterpret_cast<uint64_t>(src)));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(gaddr), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <int NS>
struct BulkLoader {
    const __nv_bfloat16* hi;
    const __nv_bfloat16* mid;
    const __nv_bfloat16* lo;
    int64_t ta, tb;  // first element of the row tile / column tile (kb = 0)
    __device__ __forceinline__ void load(uint8_t* sb, int kb, bool diag, uint64_t* bar) const {
        const int64_t off = (int64_t)kb * kPackTile;
        bulk_load(sb, hi + ta + off, TILE_BYTES, bar);
        bulk_load(sb + TILE_BYTES, mid + ta + off, TILE_BYTES, bar);
        if (NS == 3) bulk_load(sb + 2 * TILE_BYTES, lo + ta + off, TILE_BYTES, bar);
        if (!diag) {
            bulk_load(sb + NS * TILE_BYTES, hi + tb + off, TILE_BYTES, bar);
            bulk_load(sb + (NS + 1) * TILE_BYTES, mid + tb + off, TILE_BYTES, bar);
            if (NS == 3) bulk_load(sb + 5 * TILE_BYTES, lo + tb + off, TILE_BYTES, bar);
        }
    }
};

template <int NS>
__global__ void __launch_bounds__(G3_THREADS, 1) k_ggram_tc(GGramArgs a) {
    const GTile tl = a.tiles[blockIdx.x];
    const GProb P = a.gp[tl.p];
    const BulkLoader<NS> ld{a.hi, a.mid, a.lo, (P.pack + (int64_t)tl.tm * P.KB) * kPackTile,
                            (P.pack + (int64_t)tl.tn * P.KB) * kPackTile};
    gram_tile<NS>(ld, P.KB, tl.tm == tl.tn, (int64_t)tl.tm * BM, (int64_t)tl.tn * BM, P.n,
                  a.inv_s + P.voff, a.Q + P.qoff, P.ldq, a.timeout_flag);
}

// ---------------------------------------------------------------------------
// Block-sparse Gram (sparse.cu builds the operands): the occupied 128×64 boxes
// of each column tile are packed in K order (pack_index layout) from box
// toff[tile]; occupancy bit kb of word occ[tile·W + kb/32] marks K block kb,
// and wbase[tile·W + w] counts the tile's boxes in the words before w.  A CTA
// takes one work item (SItem): a chunk of the K blocks occupied in both tiles
// of its pair (I, J ≤ I), in increasing K order; pairs with no common block
// have no item (their tiles of Q are zeroed beforehand), and a pair with more
// blocks than the chunk size is split over several CTAs (split K).
// ---------------------------------------------------------------------------
struct SGramArgs {
    int64_t n;
    const SItem* items;
    float* part;
    unsigned int* ticket;
    int W;
    const uint32_t* occ;
    const int32_t* wbase;
    const int64_t* toff;
    const __nv_bfloat16* hi;
    const __nv_bfloat16* mid;
    const __nv_bfloat16* lo;
    const double* inv_s;
    float* Q;
    int64_t ldq;
    int* timeout_flag;
};

template <int NS>
struct SparseLoader {
    const __nv_bfloat16* hi;
    const __nv_bfloat16* mid;
    const __nv_bfloat16* lo;
    const uint32_t* oa;  // occupancy words of the row tile I / column tile J
    const uint32_t* ob;
    const int32_t* wa;
    const int32_t* wb;
    int64_t ta, tb;      // first box of tile I / J
    int W;
    int skip;            // common blocks before this chunk (< 0: cursor placed)
    int w;               // cursor: current word, and its common bits not yet copied
    uint32_t m;
    __device__ __forceinline__ void load(uint8_t* sb, int, bool diag, uint64_t* bar) {
        if (skip >= 0) {  // first call: move past the chunk's first `skip` common blocks
            int k = skip;
            skip = -1;
            w = 0;
            m = oa[0] & ob[0];
            for (;;) {
                const int pc = __popc(m);
                if (k < pc) break;
                k -= pc;
                if (w + 1 >= W) {
                    m = 0u;
                    break;
                }
                ++w;
                m = oa[w] & ob[w];
            }
            for (; k > 0 && m != 0u; --k) m &= m - 1u;
        }
        while (m == 0u && w + 1 < W) {
            ++w;
            m = oa[w] & ob[w];
        }
        if (m == 0u) return;  // cannot happen (load() runs once per common bit); the
                              // consumer's bounded wait on the stage then ends the tile
        const int bit = __ffs(m) - 1;
        m &= m - 1u;
        const uint32_t below = (1u << bit) - 1u;
        const int64_t xa = (ta + wa[w] + __popc(oa[w] & below)) * kPackTile;
        bulk_load(sb, hi + xa, TILE_BYTES, bar);
        bulk_load(sb + TILE_BYTES, mid + xa, TILE_BYTES, bar);
        if (NS == 3) bulk_load(sb + 2 * TILE_BYTES, lo + xa, TILE_BYTES, bar);
        if (!diag) {
            const int64_t xb = (tb + wb[w] + __popc(ob[w] & below)) * kPackTile;
            bulk_load(sb + NS * TILE_BYTES, hi + xb, TILE_BYTES, bar);
            bulk_load(sb + (NS + 1) * TILE_BYTES, mid + xb, TILE_BYTES, bar);
            if (NS == 3) bulk_load(sb + 5 * TILE_BYTES, lo + xb, TILE_BYTES, bar);
        }
    }
};

template <int NS>
__global__ void __launch_bounds__(G3_THREADS, 1) k_sgram_tc(SGramArgs a) {
    const SItem it = a.items[blockIdx.x];
    const int tm = it.I, tn = it.J;
    const uint32_t* oa = a.occ + (int64_t)tm * a.W;
    const uint32_t* ob = a.occ + (int64_t)tn * a.W;
    const SparseLoader<NS> ld{a.hi,       a.mid, a.lo, oa, ob, a.wbase + (int64_t)tm * a.W,
                              a.wbase + (int64_t)tn * a.W, a.toff[tm], a.toff[tn], a.W, it.k0,
                              0,          0u};
    float* part = it.S > 1 ? a.part + (int64_t)(it.slot - it.c) * BM * BM : nullptr;
    gram_tile<NS>(ld, it.nk, tm == tn, (int64_t)tm * BM, (int64_t)tn * BM, a.n, a.inv_s, a.Q,
                  a.ldq, a.timeout_flag, part, it.S, it.c, a.ticket + it.pair);
}

// ---------------------------------------------------------------------------
// Batched product for many right-hand sides sharing Q (Alg. 2 on k columns):
//   D[i][p] = Σ_j Q[i][j] V[p][j],   V = the split of ḡ (or of e) for the
//   compacted set of columns p < *ncols (map[p] = original column).
// Same pipeline as the Gram (3-stage TMA ring, one MMA thread, 3 split
// products, FP32 accumulation in TMEM); the CTA grid covers the maximum column
// count and CTAs past *ncols exit at once.  Epilogues:
//   BMODE_W: W[p][i] = D, and the curvature partial of the row tile,
//            kpart[mtile][p] = Σ_{i ∈ tile} ḡ[map[p]][i] · D[i][p];
//   BMODE_U: g[map[p]][i] += D  (the clipped correction Q e).
// ---------------------------------------------------------------------------
constexpr int BMODE_W = 0;
constexpr int BMODE_U = 1;

struct BatchArgs {
    int64_t n;            // rows of Q (= M)
    int num_kb;
    const int* ncols;     // device: number of compacted columns
    const int* map;       // compact index → column
    int64_t ldq;          // row length of every per-column vector
    float* W;             // [kmax][ldq]   (BMODE_W)
    const float* gb;      // [k][ldq]      (BMODE_W)
    double* kpart;        // [mtiles][kmax](BMODE_W)
    int64_t kmax;
    float* g;             // [k][ldq]      (BMODE_U)
    int* timeout_flag;
};

template <int MODE>
__global__ void __launch_bounds__(128, 1)
    k_bgemm_tc(const __grid_constant__ CUtensorMap a_hi, const __grid_constant__ CUtensorMap a_lo,
               const __grid_constant__ CUtensorMap b_hi, const __grid_constant__ CUtensorMap b_lo,
               BatchArgs p) {
    const int ncols = *p.ncols;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BM;
    if (n0 >= ncols) return;  // uniform: before any barrier or TMEM use

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    __shared__ int s_map[BM];
    __shared__ float s_red[4][BM];
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const int64_t pp = n0 + threadIdx.x;
        s_map[threadIdx.x] = pp < ncols ? p.map[pp] : -1;
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        int issued = 0;
        for (int kb = 0; kb < p.num_kb; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            uint8_t* sb = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], 4 * TILE_BYTES);
            tma_load_2d(sb, &a_hi, &full[s], kb * BK, (int)m0);
            tma_load_2d(sb + TILE_BYTES, &a_lo, &full[s], kb * BK, (int)m0);
            tma_load_2d(sb + 2 * TILE_BYTES, &b_hi, &full[s], kb * BK, (int)n0);
            tma_load_2d(sb + 3 * TILE_BYTES, &b_lo, &full[s], kb * BK, (int)n0);
            ++issued;
        }
        for (int kb = max(0, issued - STAGES); kb < issued; ++kb)
            if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1)) s_abort = 1;
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16_f32(BM, BM);
        for (int kb = 0; kb < p.num_kb; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
                s_abort = 1;
                break;
            }
            if (*(volatile int*)&s_abort) break;
            tc_fence_after();
            const uint32_t a_h = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t a_l = a_h + TILE_BYTES;
            const uint32_t b_h = a_h + 2 * TILE_BYTES;
            const uint32_t b_l = a_h + 3 * TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t off = kk * 32;
                const uint64_t dah = sdesc_sw128(a_h + off), dal = sdesc_sw128(a_l + off);
                const uint64_t dbh = sdesc_sw128(b_h + off), dbl = sdesc_sw128(b_l + off);
                umma_bf16(tmem, dah, dbh, idesc, (kb | kk) != 0 ? 1u : 0u);
                umma_bf16(tmem, dah, dbl, idesc, 1u);
                umma_bf16(tmem, dal, dbh, idesc, 1u);
            }
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    __syncwarp();

    const bool ok = mbar_wait(done, 0);
    tc_fence_after();
    if (!ok) s_abort = 1;
    __syncthreads();
    const bool good = !s_abort;
    const int64_t row = m0 + warp * 32 + lane;
    const bool rv = row < p.n;
    const int cols = (int)(ncols - n0 < (int64_t)BM ? ncols - n0 : (int64_t)BM);
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
    if (good) {
        for (int c0 = 0; c0 < cols; c0 += 16) {
            float v[16];
            tmem_ld16(tbase + c0, v);
            // the 16 columns' global operands are loaded before any is used,
            // so their latencies overlap (one dependent load per column put a
            // full L2 round trip on the critical path of every column)
            int colv[16];
            float xv[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int cc = c0 + t;
                colv[t] = cc < cols ? s_map[cc] : -1;
                const bool in = colv[t] >= 0 && rv;
                const int64_t off = (int64_t)(in ? colv[t] : 0) * p.ldq + (in ? row : 0);
                xv[t] = in ? (MODE == BMODE_W ? __ldg(p.gb + off) : p.g[off]) : 0.0f;
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int cc = c0 + t;
                const bool in = colv[t] >= 0 && rv;
                if (MODE == BMODE_W) {
                    // curvature partial in FP32 (the FP64 pipe is narrow on
                    // this GPU); the row-tile partials are summed in FP64
                    if (in) p.W[(n0 + cc) * p.ldq + row] = v[t];
                    float kp = in ? xv[t] * v[t] : 0.0f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) kp += __shfl_xor_sync(0xffffffffu, kp, o);
                    if (lane == 0) s_red[warp][cc] = kp;
                } else {
                    if (in) p.g[(int64_t)colv[t] * p.ldq + row] = xv[t] + v[t];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(p.timeout_flag, 1);
    }
    if (MODE == BMODE_W) {
        __syncthreads();
        if (good && threadIdx.x < cols) {
            const float s = (s_red[0][threadIdx.x] + s_red[1][threadIdx.x]) +
                            (s_red[2][threadIdx.x] + s_red[3][threadIdx.x]);
            p.kpart[(int64_t)blockIdx.x * p.kmax + n0 + threadIdx.x] = (double)s;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace tc

bool tc_supported(int cc_major, int cc_minor) { return cc_major == 10 && cc_minor == 3; }

cudaError_t launch_gram_tc(int nsplit, const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                           const __nv_bfloat16* lo, int64_t d, int64_t n, int64_t ldk,
                           const double* inv_s, float* Q, int64_t ldq, int* timeout_flag,
                           cudaStream_t st, int64_t row0, int64_t row1, float* part,
                           unsigned int* ticket, int split, float* sk_part,
                           unsigned int* sk_ticket, int num_sms) {
    const int64_t tiles = ceil_div(n, tc::BM);
    if (row1 < 0 || row1 > tiles) row1 = tiles;
    if (row0 < 0 || row0 >= row1) return cudaSuccess;
    // tiles (I, J ≤ I) with row0 ≤ I < row1 are the contiguous range
    // [row0(row0+1)/2, row1(row1+1)/2) of the triangle order
    return launch_gram_tc_pairs(nsplit, hi, mid, lo, d, n, ldk, inv_s, Q, ldq, timeout_flag, st,
                                row0 * (row0 + 1) / 2, row1 * (row1 + 1) / 2, part, ticket,
                                split, sk_part, sk_ticket, num_sms);
}

cudaError_t launch_gram_tc_pairs(int nsplit, const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                                 const __nv_bfloat16* lo, int64_t d, int64_t n, int64_t ldk,
                                 const double* inv_s, float* Q, int64_t ldq, int* timeout_flag,
                                 cudaStream_t st, int64_t p0, int64_t p1, float* part,
                                 unsigned int* ticket, int split, float* sk_part,
                                 unsigned int* sk_ticket, int num_sms) {
    using namespace tc;
    // TMA rules: 16-byte aligned base and row stride; x coordinates are
    // multiples of 64 BF16 (128 bytes) by construction.
    if (nsplit != 2 && nsplit != 3) return cudaErrorInvalidValue;
    if (nsplit == 2) lo = mid;  // unused: any valid map
    if (((uintptr_t)hi & 15) || ((uintptr_t)mid & 15) || ((uintptr_t)lo & 15) ||
        (ldk * 2) % 16 != 0 || ldq % 4 != 0)
        return cudaErrorInvalidValue;
    CUtensorMap mh, mm, ml;
    if (!make_map(&mh, hi, ldk, n, ldk) || !make_map(&mm, mid, ldk, n, ldk) ||
        !make_map(&ml, lo, ldk, n, ldk))
        return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    if (!attr[nsplit - 2]) {
        cudaError_t e = cudaFuncSetAttribute(nsplit == 3 ? k_gram_tc<3> : k_gram_tc<2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G3_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr[nsplit - 2] = true;
    }
    GramArgs a;
    a.n = n;
    a.num_kb = (int)ceil_div(ldk, BK);
    a.inv_s = inv_s;
    a.Q = Q;
    a.ldq = ldq;
    a.timeout_flag = timeout_flag;
    const int64_t tiles = ceil_div(n, BM), total = tiles * (tiles + 1) / 2;
    if (p1 < 0 || p1 > total) p1 = total;
    if (p0 < 0 || p0 >= p1) return cudaSuccess;
    a.t0 = p0;
    const int64_t pairs = p1 - p0;
    a.S = (part && ticket && split > 1) ? split : 1;
    a.part = part;
    a.ticket = ticket;
    const unsigned grid = (unsigned)(pairs * a.S);
    // stream-K for the last partial wave of the whole matrix, in the launch
    // that ends the triangle (when all of that wave's pairs are in it): the
    // same split whether the matrix came in one launch or in row chunks
    int64_t R = 0;
    if (a.S == 1 && p1 == total && sk_part && sk_ticket) {
        R = gram_sk_tail(total, num_sms);
        if (R > pairs) R = 0;
    }
    const unsigned full = R > 0 ? (unsigned)(pairs - R) : grid;  // R > 0 only with S = 1
    if (full > 0) {  // a launch may hold the stream-K tail alone
        if (nsplit == 3)
            k_gram_tc<3><<<full, G3_THREADS, G3_SMEM_BYTES, st>>>(mh, mm, ml, a);
        else
            k_gram_tc<2><<<full, G3_THREADS, G3_SMEM_BYTES, st>>>(mh, mm, ml, a);
    }
    if (R > 0) {
        static bool sk_attr[2] = {false, false};
        if (!sk_attr[nsplit - 2]) {
            cudaError_t e = cudaFuncSetAttribute(nsplit == 3 ? k_gram_sk<3> : k_gram_sk<2>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 G3_SMEM_BYTES);
            if (e != cudaSuccess) return e;
            sk_attr[nsplit - 2] = true;
        }
        GramArgs t = a;
        t.t0 = a.t0 + (int64_t)full;  // = tiles·(tiles+1)/2 − R
        GramSK sk{R, num_sms, gram_sk_maxseg(R, num_sms), sk_part, sk_ticket};
        if (nsplit == 3)
            k_gram_sk<3><<<(unsigned)num_sms, G3_THREADS, G3_SMEM_BYTES, st>>>(mh, mm, ml, t, sk);
        else
            k_gram_sk<2><<<(unsigned)num_sms, G3_THREADS, G3_SMEM_BYTES, st>>>(mh, mm, ml, t, sk);
    }
    return cudaGetLastError();
}

cudaError_t launch_ggram_tc(int nsplit, const GProb* gp, const GTile* tiles, int64_t ntiles,
                            const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                            const __nv_bfloat16* lo, const double* inv_s, float* Q,
                            int* timeout_flag, cudaStream_t st) {
    using namespace tc;
    if (ntiles <= 0) return cudaSuccess;
    if (nsplit != 2 && nsplit != 3) return cudaErrorInvalidValue;
    if (nsplit == 2) lo = mid;
    if (((uintptr_t)hi & 15) || ((uintptr_t)mid & 15) || ((uintptr_t)lo & 15) ||
        ((uintptr_t)Q & 15))
        return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    if (!attr[nsplit - 2]) {
        cudaError_t e = cudaFuncSetAttribute(nsplit == 3 ? k_ggram_tc<3> : k_ggram_tc<2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G3_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr[nsplit - 2] = true;
    }
    GGramArgs a;
    a.gp = gp;
    a.tiles = tiles;
    a.hi = hi;
    a.mid = mid;
    a.lo = lo;
    a.inv_s = inv_s;
    a.Q = Q;
    a.timeout_flag = timeout_flag;
    if (nsplit == 3)
        k_ggram_tc<3><<<(unsigned)ntiles, G3_THREADS, G3_SMEM_BYTES, st>>>(a);
    else
        k_ggram_tc<2><<<(unsigned)ntiles, G3_THREADS, G3_SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sgram_tc(int nsplit, const SItem* items, int64_t nitems, const uint32_t* occ,
                            int W, const int32_t* wbase, const int64_t* toff,
                            const __nv_bfloat16* hi, const __nv_bfloat16* mid,
                            const __nv_bfloat16* lo, int64_t n, const double* inv_s, float* Q,
                            int64_t ldq, float* part, unsigned int* ticket, int* timeout_flag,
                            cudaStream_t st) {
    using namespace tc;
    if (nitems <= 0) return cudaSuccess;
    if (nsplit != 2 && nsplit != 3) return cudaErrorInvalidValue;
    if (nsplit == 2) lo = mid;
    if (((uintptr_t)hi & 15) || ((uintptr_t)mid & 15) || ((uintptr_t)lo & 15) || W < 1)
        return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    if (!attr[nsplit - 2]) {
        cudaError_t e = cudaFuncSetAttribute(nsplit == 3 ? k_sgram_tc<3> : k_sgram_tc<2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             G3_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr[nsplit - 2] = true;
    }
    SGramArgs a;
    a.n = n;
    a.items = items;
    a.part = part;
    a.ticket = ticket;
    a.W = W;
    a.occ = occ;
    a.wbase = wbase;
    a.toff = toff;
    a.hi = hi;
    a.mid = mid;
    a.lo = lo;
    a.inv_s = inv_s;
    a.Q = Q;
    a.ldq = ldq;
    a.timeout_flag = timeout_flag;
    const unsigned grid = (unsigned)nitems;
    if (nsplit == 3)
        k_sgram_tc<3><<<grid, G3_THREADS, G3_SMEM_BYTES, st>>>(a);
    else
        k_sgram_tc<2><<<grid, G3_THREADS, G3_SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bgemm_tc(int mode, const __nv_bfloat16* q_hi, const __nv_bfloat16* q_lo,
                            int64_t n, int64_t ldk, const __nv_bfloat16* v_hi,
                            const __nv_bfloat16* v_lo, int64_t kmax, const int* ncols,
                            const int* map, int64_t ldq, float* W, const float* gb, double* kpart,
                            float* g, int* timeout_flag, cudaStream_t st) {
    using namespace tc;
    if (((uintptr_t)q_hi & 15) || ((uintptr_t)q_lo & 15) || ((uintptr_t)v_hi & 15) ||
        ((uintptr_t)v_lo & 15) || (ldk * 2) % 16 != 0)
        return cudaErrorInvalidValue;
    CUtensorMap ah, al, bh, bl;
    if (!make_map(&ah, q_hi, ldk, n, ldk) || !make_map(&al, q_lo, ldk, n, ldk) ||
        !make_map(&bh, v_hi, ldk, kmax, ldk) || !make_map(&bl, v_lo, ldk, kmax, ldk))
        return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    if (!attr[mode]) {
        cudaError_t e = cudaFuncSetAttribute(mode == BMODE_W ? k_bgemm_tc<BMODE_W> : k_bgemm_tc<BMODE_U>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr[mode] = true;
    }
    BatchArgs a;
    a.n = n;
    a.num_kb = (int)ceil_div(ldk, BK);
    a.ncols = ncols;
    a.map = map;
    a.ldq = ldq;
    a.W = W;
    a.gb = gb;
    a.kpart = kpart;
    a.kmax = kmax;
    a.g = g;
    a.timeout_flag = timeout_flag;
    const dim3 grid((unsigned)ceil_div(n, BM), (unsigned)ceil_div(kmax, BM));
    if (mode == BMODE_W)
        k_bgemm_tc<BMODE_W><<<grid, 128, SMEM_BYTES, st>>>(ah, al, bh, bl, a);
    else
        k_bgemm_tc<BMODE_U><<<grid, 128, SMEM_BYTES, st>>>(ah, al, bh, bl, a);
    return cudaGetLastError();
}

}  // namespace aln
