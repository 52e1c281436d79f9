// Grid-wide barrier of the persistent (cooperatively launched) solver
// kernels, with a bounded wait: arrivals spread over several counters, a
// per-launch wait limit on %globaltimer, and a timeout word that the first
// block whose wait expired sets so that every other block gives up too.
#pragma once

#include "common.cuh"

namespace aln {

constexpr uint64_t kBarrierNs = 2000000000ull;  // default limit of one barrier wait: 2 s
constexpr int kStatusTimeout = -1;              // state status after a barrier timeout

// Limit of one grid-barrier wait for this context's launches.
inline uint64_t barrier_wait_ns(const aln_ctx* c) {
    return c->opt.wait_limit_us > 0 ? (uint64_t)c->opt.wait_limit_us * 1000ull : kBarrierNs;
}

__device__ __forceinline__ uint64_t p_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int kSyncLanes = 8;  // arrival counters, one 128-byte line each

struct PersistSync {
    // monotonic arrivals spread over kSyncLanes counters (block b adds to
    // counter b mod kSyncLanes, so the arrivals do not queue on one L2 line);
    // barrier k completes when their sum reaches k·G
    unsigned int count[kSyncLanes][32];
    unsigned int timeout;  // set by the first block whose wait expired
    unsigned int pad[31];
};

// Grid barrier over the co-resident grid (cooperative launch).  Arrival is a
// release reduction on the block's counter; warp 0 then polls all counters
// (relaxed loads, one per lane), and once their sum reaches `target` (this
// barrier's completion count, tracked identically by every block) each
// polling lane re-reads its counter with an acquire load before the block
// continues.
__device__ __forceinline__ bool grid_barrier(PersistSync* s, unsigned int target,
                                             uint64_t wait_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0)
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(
                             &s->count[blockIdx.x % kSyncLanes][0]),
                         "r"(1u)
                         : "memory");
        int ok = 1;
        unsigned int spins = 0;
        uint64_t t0 = 0;
        for (;;) {
            unsigned int v = 0;
            if (lane < kSyncLanes)
                asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v)
                             : "l"(&s->count[lane][0])
                             : "memory");
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            v = __shfl_sync(0xffffffffu, v, 0);
            if ((int)(v - target) >= 0) {
                // acquire: re-read each counter with an acquire load (it reads
                // from the release sequence of every arrival added to it), a
                // lighter order than a full fence; the block barrier below
                // carries it to the other threads
                if (lane < kSyncLanes) {
                    unsigned int u;
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(u)
                                 : "l"(&s->count[lane][0])
                                 : "memory");
                    asm volatile("" ::"r"(u));  // the value itself is not needed
                }
                break;
            }
            __nanosleep(8);
            int stop = 0;
            if (lane == 0 && (++spins & 1023u) == 0) {
                const uint64_t t = p_globaltimer();
                if (t0 == 0) {
                    t0 = t;
                } else if (t - t0 > wait_ns) {
                    atomicExch(&s->timeout, 1u);
                    stop = 1;
                }
                if (*(volatile unsigned int*)&s->timeout) stop = 1;
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) {
                ok = 0;
                break;
            }
        }
        __syncwarp();
        if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace aln
