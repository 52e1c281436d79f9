// C ABI of libaln (include/aln.h): context, workspace, Alg. 1 prepare, the
// Alg. 2 solve loop with FP64 KKT checks and refinement, and inspection calls.
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"
#include "kernels.cuh"

using namespace aln;

namespace {

#define ALN_TRY(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_status(e_);  \
    } while (0)
#define ALN_CHECK(st)                          \
    do {                                       \
        aln_status s_ = (st);                  \
        if (s_ != ALN_OK) return s_;           \
    } while (0)

aln_status cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return ALN_ERR_OUT_OF_MEMORY;
    }
    return ALN_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// (Re)allocate a device buffer so that it holds at least `bytes`.
aln_status ensure(void** p, size_t* cap, size_t bytes) {
    if (*cap >= bytes && *p) return ALN_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (bytes == 0) return ALN_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ALN_ERR_OUT_OF_MEMORY;
    }
    *cap = bytes;
    return ALN_OK;
}

size_t elt(int32_t dtype) { return dtype == ALN_DTYPE_F64 ? 8 : 4; }
bool fp64(const aln_ctx* c) { return c->opt.precision == ALN_PREC_FP64; }

// Host buffers → device: owned copy; device buffers are used in place.
aln_status resolve_input(aln_ctx* c, const void* src, int64_t rows, int64_t cols, int64_t ld,
                         size_t esz, void** copy, size_t* cap, const void** out) {
    if (is_device_ptr(src)) {
        *out = src;
        return ALN_OK;
    }
    const size_t bytes = (size_t)((cols - 1) * ld + rows) * esz;
    ALN_CHECK(ensure(copy, cap, bytes));
    ALN_TRY(cudaMemcpyAsync(*copy, src, bytes, cudaMemcpyHostToDevice, c->stream));
    *out = *copy;
    return ALN_OK;
}

}  // namespace

namespace aln {

// Iteration and KKT workspace for the current (n, d, precision).
aln_status alloc_workspace(aln_ctx* c) {
    const size_t T = fp64(c) ? 8 : 4;
    const int64_t ldq = c->ldq, n = c->n, d = c->d;
    // matvec geometry: tile of 32·VN columns, R row groups
    const int64_t col_tiles = ldq / (fp64(c) ? 64 : 128);
    int R = c->opt.row_groups;
    if (R <= 0) {
        const int64_t want = 2 * (int64_t)c->num_sms;  // ≈ 2 blocks per SM
        R = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(want, col_tiles), ceil_div(n, 16)));
        R = std::min(R, 64);
    }
    c->R = R;
    c->nb = (int)std::min<int64_t>(ceil_div(n, 256), 1024);

    // Persistent kernel: column tiles × row groups, about one work item per
    // block (one block per SM, or the option), at least 32 rows per group.
    c->p_CT = (int)col_tiles;
    const int64_t blocks_wanted = c->opt.persist_blocks > 0 ? c->opt.persist_blocks : c->num_sms;
    int pR = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_wanted / col_tiles,
                                                         ceil_div(n, 32)));
    if (c->tune_pR > 0) pR = c->tune_pR;  // the autotuner's choice
    c->p_R = std::min(pR, 64);
    // The replicated-state kernel is used whenever its vectors fit in shared
    // memory, unless the options ask for the tiled one.
    c->p_repl = c->opt.iter_kernel == 1 ? 0 : 1;
    const int maxG = fp64(c) ? persist_max_blocks<double>(c->num_sms, ldq, &c->p_repl)
                             : persist_max_blocks<float>(c->num_sms, ldq, &c->p_repl);
    if (maxG <= 0) return ALN_ERR_CUDA;
    int G = c->opt.persist_blocks > 0 ? c->opt.persist_blocks : c->num_sms;
    G = (int)std::min<int64_t>({(int64_t)G, (int64_t)maxG, (int64_t)c->p_CT * c->p_R});
    c->p_G = std::max(G, 1);
    // partials: R (chain set-up) / R_p (tiled kernel) / 3·R_p (replicated: two
    // parity buffers for Qḡ and one for Qe)
    const int64_t RP = std::max<int64_t>(R, 3 * (int64_t)c->p_R);

    const size_t vec = (size_t)ldq * T;
    const size_t ct = (size_t)c->p_CT;
    size_t bytes = 6 * vec + (size_t)RP * vec + 2 * (size_t)c->nb * 8 + (size_t)c->nb * 4 + 256 +
                   4 * round_up(ct * 8, 256) + round_up(2 * ct * c->p_R * 8, 256) + 256 + 256;
    bytes = round_up(bytes, 256) + 16 * 256;
    ALN_CHECK(ensure(&c->iter_pool, &c->iter_bytes, bytes + 1024));
    uint8_t* p = (uint8_t*)c->iter_pool;
    auto take = [&](size_t b) {
        uint8_t* r = p;
        p += round_up(b, 256);
        return (void*)r;
    };
    c->qv = take(vec);
    c->y = take(vec);
    c->g = take(vec);
    c->gb = take(vec);
    c->w = take(vec);
    c->e = take(vec);
    c->part = take((size_t)RP * vec);
    c->gpart = (double*)take((size_t)c->nb * 8);
    c->kpart = (double*)take((size_t)c->nb * 8);
    c->cpart = (int*)take((size_t)c->nb * 4);
    c->st = (IterState*)take(sizeof(IterState));
    c->p_gpart = (double*)take(ct * 8);
    c->p_kpart = (double*)take(2 * ct * c->p_R * 8);  // curvature share per work item (×2 parity)
    c->p_cpart = (int*)take(ct * 8);
    c->p_clip = (int*)take(ct * 8);
    c->p_ticket = (unsigned int*)take(ct * 8);
    c->p_sync = take(persist_sync_bytes());
    ALN_TRY(cudaMemsetAsync(c->iter_pool, 0, c->iter_bytes, c->stream));
    // A small FP64 problem runs its loop on one thread-block cluster
    // (iter_kernel 0 = auto or 3).
    c->p_small = 0;
    if (fp64(c) && c->opt.algorithm == ALN_ALG_ANTILOP &&
        (c->opt.iter_kernel == 0 || c->opt.iter_kernel == 3)) {
        int optin = 0;
        ALN_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                       c->device));
        c->p_small = small64_fits(c, optin) ? 1 : 0;
    }

    // KKT: x64 (ldq), g64 (ldq), r64 (d), rpart (CG·d), parts, out
    const int64_t row_blocks = ceil_div(d, 1024);  // k_kkt_ax: 4 rows × 256 threads
    int CG = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(4 * (int64_t)c->num_sms, row_blocks),
                                                         ceil_div(n, 32)));
    CG = std::min(CG, 64);
    c->CG = CG;
    const int64_t ng = n;  // one ḡ² partial per column
    // rpart also holds the FP32 pairs of x and r (2·ldq + 2·d floats)
    const size_t pairs = round_up((int64_t)(2 * ldq + 2 * d) * 4, 256) + 256;
    size_t kb = 2 * (size_t)ldq * 8 + (size_t)d * 8 + (size_t)CG * d * 8 + pairs + (512 + ng) * 8 +
                64;
    kb = round_up(kb, 256) + 2048;
    ALN_CHECK(ensure(&c->kkt_pool, &c->kkt_bytes, kb));
    p = (uint8_t*)c->kkt_pool;
    c->x64 = (double*)take((size_t)ldq * 8);
    c->g64 = (double*)take((size_t)ldq * 8);
    c->r64 = (double*)take((size_t)d * 8);
    c->rpart = (double*)take((size_t)CG * d * 8 + pairs);
    c->kkt_part = (double*)take((512 + ng) * 8);
    c->kkt_out = (double*)take(64);
    ALN_TRY(cudaMemsetAsync(c->kkt_pool, 0, c->kkt_bytes, c->stream));
    return ALN_OK;
}

// One launch of the persistent Alg. 2 (or Anti+Acc) kernel: it loops on the
// device until a stop rule fires (the state's eps, max_iter and stagnation
// window were set by the set-up kernels) and leaves the outcome in the
// iteration state.  The barrier words and tile tickets are cleared first, so
// a previous timeout cannot leak into this run.
aln_status run_until_done(aln_ctx* c) {
    ALN_TRY(cudaMemsetAsync(c->p_sync, 0, persist_sync_bytes(), c->stream));
    ALN_TRY(cudaMemsetAsync(c->p_ticket, 0, (size_t)c->p_CT * sizeof(unsigned int), c->stream));
    ALN_TRY(cudaEventRecord(c->ev[6], c->stream));
    if (c->opt.algorithm == ALN_ALG_ANTI_ACC)
        ALN_TRY(fp64(c) ? launch_acc_persist<double>(c) : launch_acc_persist<float>(c));
    else if (c->p_small && c->opt.test_barrier_skew == 0)  // (the knob tests grid barriers)
        ALN_TRY(launch_alg2_small64(c));
    else
        ALN_TRY(fp64(c) ? launch_alg2_persist<double>(c) : launch_alg2_persist<float>(c));
    ALN_TRY(cudaEventRecord(c->ev[7], c->stream));
    c->launches += 1;
    ALN_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(IterState), cudaMemcpyDeviceToHost,
                            c->stream));
    ALN_TRY(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]) == cudaSuccess) c->stats.iterate_ms += ms;
    if (c->st_host->status < 0 || !c->st_host->done) return ALN_ERR_TIMEOUT;
    c->stats.passive_rows += c->st_host->sum_passive;
    c->stats.clipped_rows += c->st_host->sum_clip;
    c->stats.product_bytes += (double)(fp64(c) ? 8 : 4) * (double)c->n *
                              (double)(c->st_host->sum_passive + c->st_host->sum_clip);
    if (c->p_repl || c->p_small) {
        for (int k = 0; k < 5; ++k) c->stats.phase_us[k] += 1e-3 * (double)c->st_host->phase_ns[k];
        c->stats.clipped_iterations += (int32_t)c->st_host->phase_ns[5];
    }
    return ALN_OK;
}

}  // namespace aln

namespace {

// Anti+Acc: L = λ_max(Q) of the prepared Q by the power iteration, once per
// prepare.  Needs the replicated layout (else ALN_ERR_UNSUPPORTED).
aln_status ensure_lipschitz(aln_ctx* c) {
    if (c->lipschitz > 0.0) return ALN_OK;
    const bool f64 = fp64(c);
    const size_t need = acc_smem_need(f64, c->ldq) + 4096;
    int optin = 0;
    ALN_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (!c->p_repl || need > (size_t)optin) return ALN_ERR_UNSUPPORTED;
    ALN_TRY(cudaMemsetAsync(c->p_sync, 0, persist_sync_bytes(), c->stream));
    const double tol = f64 ? 1e-7 : 1e-6;  // FP32 quotients carry ~1e-7 noise
    ALN_TRY(f64 ? launch_power<double>(c, tol, 500, c->kkt_out)
                : launch_power<float>(c, tol, 500, c->kkt_out));
    c->launches += 1;
    ALN_TRY(cudaMemcpyAsync(c->kkt_out_host, c->kkt_out, 2 * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    ALN_TRY(cudaStreamSynchronize(c->stream));
    const double rho = c->kkt_out_host[0], steps = c->kkt_out_host[1];
    if (steps < 0.0) return ALN_ERR_TIMEOUT;
    if (!std::isfinite(rho)) return ALN_ERR_NONFINITE;
    c->lipschitz = rho > 0.0 ? rho : 1.0;  // Q = 0: any step (the gradient is q)
    c->power_products = (int)steps;
    c->stats.lipschitz = c->lipschitz;
    c->stats.power_products = c->power_products;
    return ALN_OK;
}

aln_status kkt_eval(aln_ctx* c, int64_t rhs, const double* x64dev, double* rel, double* F) {
    const void* b = (const uint8_t*)c->B + (size_t)rhs * c->ldb * elt(c->dtype);
    ALN_TRY(cudaEventRecord(c->ev[6], c->stream));
    ALN_TRY(launch_kkt(c, x64dev, b, c->den_host[rhs], c->kkt_out));
    c->launches += 4;
    ALN_TRY(cudaEventRecord(c->ev[7], c->stream));
    ALN_TRY(cudaMemcpyAsync(c->kkt_out_host, c->kkt_out, 2 * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    ALN_TRY(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]) == cudaSuccess) c->stats.kkt_ms += ms;
    *rel = c->kkt_out_host[0];
    *F = c->kkt_out_host[1];
    return ALN_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// Kernels local to the ABI layer (export / conversions)
// ----------------------------------------------------------------------------
template <typename TS>
__global__ void k_copy_to_f64(const TS* __restrict__ src, int64_t lds, double* __restrict__ dst,
                              int64_t ldd, int64_t rows, int64_t cols) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols, c = e - r * cols;
        dst[r * ldd + c] = (double)src[r * lds + c];
    }
}

// Shared by aln_prepare and aln_prepare_csc (c->d, c->dtype set): Q (zeroed
// when its shape changes), s, inv_s, q64, den, flags, the pinned copy of den,
// and the choice of the many-right-hand-side solver.
// q = −D⁻¹AᵀB for FP32 A and B to FP64 accuracy (the batched FP64 checks
// need it): exact BF16 digit products on the tensor cores.
static aln_status qvec32(aln_ctx* c, int64_t d, int64_t n, int64_t lda, int64_t k, int64_t ldb) {
    ALN_CHECK(ensure(&c->oz_work, &c->oz_work_bytes, oz_work_bytes(d, n, k)));
    ALN_TRY(launch_oz_atb((const float*)c->A, lda, (const float*)c->B, ldb, d, n, k, c->inv_s,
                          c->q64, c->ldq, c->oz_work, c->oz_work_bytes, c->flags + 1, c->stream));
    c->launches += 3;
    return ALN_OK;
}

static aln_status prep_buffers(aln_ctx* c, int64_t n, int64_t k) {
    const bool f64 = fp64(c);
    const int64_t ldq = round_up(n, 128);
    const size_t qbytes = (size_t)ldq * ldq * (f64 ? 8 : 4);
    const bool fresh_q = c->Q == nullptr || c->ldq != ldq || c->Q_elt != (f64 ? 8 : 4);
    ALN_CHECK(ensure(&c->Q, &c->Q_bytes, qbytes));
    c->ldq = ldq;
    c->Q_elt = f64 ? 8 : 4;
    if (fresh_q || c->Q_n != n) ALN_TRY(cudaMemsetAsync(c->Q, 0, c->Q_bytes, c->stream));
    c->Q_n = n;

    // s, inv_s, q64 (k·ldq), den (k), flags
    const size_t pb = round_up((size_t)2 * ldq * 8, 256) + round_up((size_t)k * ldq * 8, 256) +
                      round_up((size_t)k * 8, 256) + 256;
    ALN_CHECK(ensure(&c->prep_pool, &c->prep_bytes, pb));
    uint8_t* p = (uint8_t*)c->prep_pool;
    c->s = (double*)p;
    c->inv_s = c->s + ldq;
    p += round_up((size_t)2 * ldq * 8, 256);
    c->q64 = (double*)p;
    p += round_up((size_t)k * ldq * 8, 256);
    c->den = (double*)p;
    p += round_up((size_t)k * 8, 256);
    c->flags = (int*)p;
    ALN_TRY(cudaMemsetAsync(c->prep_pool, 0, c->prep_bytes, c->stream));
    if (c->den_host_cap < k) {
        if (c->den_host) cudaFreeHost(c->den_host);
        c->den_host = nullptr;
        c->den_host_cap = 0;
        if (cudaMallocHost(&c->den_host, (size_t)k * 8) != cudaSuccess) {
            cudaGetLastError();
            return ALN_ERR_OUT_OF_MEMORY;
        }
        c->den_host_cap = k;
    }

    // Many right-hand sides in mixed precision: the batched solver (batch.cu)
    // forms Q in FP64 once (it also serves the FP64 checks) and iterates all
    // columns together with tensor-core products.
    c->batched = (!f64 && k >= c->opt.batch_min && c->opt.algorithm == ALN_ALG_ANTILOP) ? 1 : 0;
    c->lipschitz = -1.0;  // Q changes: the Anti+Acc step is estimated again
    c->power_products = 0;
    c->stats.lipschitz = 0.0;
    c->stats.power_products = 0;

    return ALN_OK;
}

// Shared tail of the prepare calls: workspace, flags and denominators to the
// host, timings (ev[0]..ev[3] recorded by the caller), input status.
static aln_status prep_finish(aln_ctx* c, int64_t k) {
    ALN_CHECK(alloc_workspace(c));
    ALN_TRY(cudaMemcpyAsync(c->flags_host, c->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream));
    ALN_TRY(cudaMemcpyAsync(c->den_host, c->den, (size_t)k * 8, cudaMemcpyDeviceToHost,
                            c->stream));
    ALN_TRY(cudaEventRecord(c->ev[3], c->stream));
    ALN_TRY(cudaStreamSynchronize(c->stream));
    {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, c->ev[0], c->ev[3]);
        cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
        c->stats.prepare_ms = a;
        c->stats.gram_ms = b;
    }
    if (c->flags_host[1]) return ALN_ERR_TIMEOUT;
    if (c->flags_host[0]) return ALN_ERR_NONFINITE;

    return ALN_OK;
}

extern "C" {

void aln_default_options(aln_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = ALN_PREC_SPLIT_BF16;
    opt->max_refine = 8;
    opt->persist_blocks = 0;
    opt->row_groups = 0;
    opt->stagnation = 100;
    opt->iter_kernel = 0;
    opt->batch_min = 8;
    opt->refine_gain = 0;
    opt->gram_split = 3;
    opt->group_cluster = 4;
    opt->algorithm = ALN_ALG_ANTILOP;
}

int32_t aln_version(void) { return ALN_VERSION; }

const char* aln_status_string(aln_status s) {
    switch (s) {
        case ALN_OK: return "ALN_OK";
        case ALN_ERR_INVALID_ARG: return "ALN_ERR_INVALID_ARG";
        case ALN_ERR_NOT_PREPARED: return "ALN_ERR_NOT_PREPARED";
        case ALN_ERR_NONFINITE: return "ALN_ERR_NONFINITE";
        case ALN_ERR_OUT_OF_MEMORY: return "ALN_ERR_OUT_OF_MEMORY";
        case ALN_ERR_CUDA: return "ALN_ERR_CUDA";
        case ALN_ERR_TIMEOUT: return "ALN_ERR_TIMEOUT";
        case ALN_ERR_UNSUPPORTED: return "ALN_ERR_UNSUPPORTED";
    }
    return "ALN_ERR_UNKNOWN";
}

aln_status aln_create(aln_ctx** out, const aln_options* opt, void* stream) {
    if (!out) return ALN_ERR_INVALID_ARG;
    *out = nullptr;
    aln_options o;
    aln_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != ALN_PREC_FP64 && o.precision != ALN_PREC_SPLIT_BF16)
        return ALN_ERR_INVALID_ARG;
    if (o.max_refine < 0 || o.persist_blocks < 0 || o.row_groups < 0 || o.stagnation < 0 ||
        o.iter_kernel < 0 || o.iter_kernel > 3 || o.batch_min < 0)
        return ALN_ERR_INVALID_ARG;
    if (o.stagnation == 0) o.stagnation = 100;
    if (o.batch_min == 0) o.batch_min = 8;
    if (o.refine_gain > 16) return ALN_ERR_INVALID_ARG;
    if (o.gram_split == 0) o.gram_split = 3;
    if (o.gram_split != 2 && o.gram_split != 3) return ALN_ERR_INVALID_ARG;
    if (o.algorithm != ALN_ALG_ANTILOP && o.algorithm != ALN_ALG_ANTI_ACC)
        return ALN_ERR_INVALID_ARG;
    if (o.wait_limit_us < 0 || o.test_barrier_skew < 0 || o.test_barrier_skew > 1024 ||
        o.group_graph < 0 || o.group_graph > 1 || o.autotune < 0 || o.autotune > 2)
        return ALN_ERR_INVALID_ARG;
    if (o.autotune > 0 && (!o.autotune_cache || !o.autotune_cache[0]))
        return ALN_ERR_INVALID_ARG;
    if (o.group_cluster == 0) o.group_cluster = 4;
    if (o.group_cluster != 1 && o.group_cluster != 2 && o.group_cluster != 4 &&
        o.group_cluster != 8)
        return ALN_ERR_INVALID_ARG;
    aln_ctx* c = new (std::nothrow) aln_ctx();
    if (!c) return ALN_ERR_OUT_OF_MEMORY;
    if (o.autotune_cache) c->tune_path = o.autotune_cache;  // a copy: the caller's may go
    o.autotune_cache = nullptr;
    c->opt = o;
    c->user_opt = o;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, c->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return ALN_ERR_CUDA;
    }
    if (o.precision == ALN_PREC_SPLIT_BF16 && !tc_supported(c->cc_major, c->cc_minor)) {
        delete c;
        return ALN_ERR_UNSUPPORTED;
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        // A private blocking stream: ordered after legacy-stream work and, unlike
        // the legacy stream itself, usable for stream capture by callers.
        if (cudaStreamCreate(&c->own_stream) != cudaSuccess) {
            delete c;
            return ALN_ERR_CUDA;
        }
        c->stream = c->own_stream;
    }
    if (cudaMallocHost(&c->host_pool, 4096) != cudaSuccess) {
        cudaGetLastError();
        if (c->own_stream) cudaStreamDestroy(c->own_stream);
        delete c;
        return ALN_ERR_OUT_OF_MEMORY;
    }
    for (auto& ev : c->ev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            cudaGetLastError();
            aln_destroy(c);
            return ALN_ERR_CUDA;
        }
    }
    uint8_t* h = (uint8_t*)c->host_pool;
    c->st_host = (IterState*)h;
    c->kkt_out_host = (double*)(h + 256);
    c->flags_host = (int*)(h + 512);
    *out = c;
    return ALN_OK;
}

void aln_destroy(aln_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    batch_free(c);
    group_free(c);
    mlp_free(c);
    nmf_free(c);
    void* bufs[] = {c->A_copy, c->B_copy,    c->Q,        c->prep_pool, c->A_hi,
                    c->iter_pool, c->kkt_pool, c->csc_pool, c->sp_part, c->g64_work,
                    c->oz_work};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (c->den_host) cudaFreeHost(c->den_host);
    if (c->host_pool) cudaFreeHost(c->host_pool);
    for (auto ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : c->copy_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

aln_status aln_prepare(aln_ctx* c, const void* A, int64_t d, int64_t n, int64_t lda, int32_t dtype,
                       const void* B, int64_t k, int64_t ldb) {
    if (!c || !A || !B) return ALN_ERR_INVALID_ARG;
    if (d < 1 || n < 1 || k < 1 || lda < d || ldb < d) return ALN_ERR_INVALID_ARG;
    if (dtype != ALN_DTYPE_F32 && dtype != ALN_DTYPE_F64) return ALN_ERR_INVALID_ARG;
    if (n > (int64_t)1 << 20 || d > ((int64_t)1 << 31) - 64) return ALN_ERR_INVALID_ARG;
    c->prepared = 0;
    c->grouped = 0;
    c->csc_kkt = 0;
    c->q_tmask = nullptr;
    c->stats.prepare_ms = c->stats.gram_ms = 0.0;
    const size_t esz = elt(dtype);
    // A on the host, single-problem split path with q fused in the column
    // statistics: copy A in column chunks and overlap the copy with the
    // statistics and Gram tile rows of the chunks already on the device
    const bool pipelined = !is_device_ptr(A) && c->opt.precision == ALN_PREC_SPLIT_BF16 &&
                           k <= 4 && k < c->opt.batch_min && n > 256;
    if (pipelined) {
        const size_t bytes = (size_t)((n - 1) * lda + d) * esz;
        ALN_CHECK(ensure(&c->A_copy, &c->A_copy_bytes, bytes));
        c->A = c->A_copy;
    } else {
        ALN_CHECK(resolve_input(c, A, d, n, lda, esz, &c->A_copy, &c->A_copy_bytes, &c->A));
    }
    ALN_CHECK(resolve_input(c, B, d, k, ldb, esz, &c->B_copy, &c->B_copy_bytes, &c->B));
    c->d = d;
    c->n = n;
    c->k = k;
    c->lda = lda;
    c->ldb = ldb;
    c->dtype = dtype;
    ALN_CHECK(prep_buffers(c, n, k));
    const bool f64 = fp64(c);
    const int64_t ldq = c->ldq;

    // split copies for the tensor-core Gram
    __nv_bfloat16 *hi = nullptr, *mid = nullptr, *lo = nullptr;
    if (!f64 && !c->batched) {
        c->ldk = round_up(d, 64);
        const size_t sb = (size_t)n * c->ldk * 2;
        ALN_CHECK(ensure((void**)&c->A_hi, &c->split_bytes, 3 * round_up(sb, 1024)));
        hi = c->A_hi;
        mid = (__nv_bfloat16*)((uint8_t*)c->A_hi + round_up(sb, 1024));
        lo = (__nv_bfloat16*)((uint8_t*)c->A_hi + 2 * round_up(sb, 1024));
        c->A_lo = lo;
    }

    // split K in the tensor-core Gram: with fewer tile pairs than SMs (tall,
    // narrow A) each pair's K range runs over several CTAs.  The split is fixed
    // by the whole matrix, so host input (launched chunk by chunk below) and
    // device input (one launch) give the same Q
    const int64_t chunk_cols = std::max<int64_t>(512, round_up(ceil_div(n, 63), 128));
    float* gpart = nullptr;
    unsigned int* gticket = nullptr;
    int gsplit = 1;
    if (!f64 && !c->batched) {
        const int64_t tiles = ceil_div(n, 128);
        const int64_t pairs = tiles * (tiles + 1) / 2;
        gsplit = gram_split_k(pairs, ceil_div(c->ldk, 64), c->num_sms);
        if (gsplit > 1) {  // a chunked launch covers at most all pairs
            const size_t pb = (size_t)pairs * gsplit * 128 * 128 * 4;
            ALN_CHECK(ensure(&c->sp_part, &c->sp_part_bytes, pb + round_up((size_t)pairs * 4, 256)));
            gpart = (float*)c->sp_part;
            gticket = (unsigned int*)((uint8_t*)c->sp_part + pb);
            ALN_TRY(cudaMemsetAsync(gticket, 0, (size_t)pairs * 4, c->stream));
        }
    }
    // without split K, the pairs past the last full wave of the Gram run as
    // stream-K (equal K shares per SM) in the launch that ends the triangle
    float* skp = nullptr;
    unsigned int* skt = nullptr;
    if (!f64 && !c->batched && gsplit == 1) {
        const int64_t tiles = ceil_div(n, 128), pairs = tiles * (tiles + 1) / 2;
        const int64_t tail = gram_sk_tail(pairs, c->num_sms);
        // host input launches the Gram in whole waves as the chunks arrive,
        // so the launch that ends the triangle always holds the whole tail:
        // both inputs give the same Q bits
        if (tail > 0) {
            ALN_CHECK(ensure(&c->sp_part, &c->sp_part_bytes, gram_sk_bytes(pairs, c->num_sms)));
            skp = (float*)c->sp_part;
            skt = (unsigned int*)((uint8_t*)c->sp_part + gram_sk_part_bytes(pairs, c->num_sms));
            ALN_TRY(cudaMemsetAsync(skt, 0, (size_t)tail * 4, c->stream));
        }
    }

    // Alg. 1: scale factors, q, (split), Gram
    ALN_TRY(cudaEventRecord(c->ev[0], c->stream));
    ALN_TRY(launch_check_finite(c->B, dtype, d, k, ldb, c->flags, c->stream));
    const int kc = k <= 4 ? (int)k : 0;
    if (pipelined) {
        if (!c->copy_stream) {
            ALN_TRY(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
            for (auto& ev : c->copy_ev)
                ALN_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
        // the copy stream starts after the main stream's earlier work (the
        // previous users of the A buffer)
        ALN_TRY(cudaEventRecord(c->copy_ev[0], c->stream));
        ALN_TRY(cudaStreamWaitEvent(c->copy_stream, c->copy_ev[0], 0));
        // A Gram launch lasts at least one tile pair's full K loop (about
        // 0.4 ms at d = 20000) whatever its size, so the pairs that a chunk
        // completes wait until they fill whole waves (the SM count, one CTA
        // per SM); the chunk that ends the matrix launches the rest, with
        // the stream-K tail.  Each pair is computed alike in any launch.
        const int64_t per = chunk_cols;
        const int64_t tiles = ceil_div(n, 128);
        int64_t launched = 0;  // tile pairs launched (triangle order)
        int e = 1;
        for (int64_t c0 = 0; c0 < n; c0 += per, ++e) {
            const int64_t c1 = std::min(n, c0 + per);
            const uint8_t* src = (const uint8_t*)A + (size_t)c0 * lda * esz;
            uint8_t* dst = (uint8_t*)c->A_copy + (size_t)c0 * lda * esz;
            ALN_TRY(cudaMemcpy2DAsync(dst, (size_t)lda * esz, src, (size_t)lda * esz, (size_t)d * esz,
                                      (size_t)(c1 - c0), cudaMemcpyHostToDevice, c->copy_stream));
            ALN_TRY(cudaEventRecord(c->copy_ev[e], c->copy_stream));
            ALN_TRY(cudaStreamWaitEvent(c->stream, c->copy_ev[e], 0));
            ALN_TRY(launch_colstats(dst, dtype, d, c1 - c0, lda, c->B, kc, ldb, c->s + c0,
                                    c->inv_s + c0, c->q64 + c0, ldq, c->flags, hi + c0 * c->ldk,
                                    mid + c0 * c->ldk, lo + c0 * c->ldk, c->ldk, c->stream));
            if (c0 == 0) ALN_TRY(cudaEventRecord(c->ev[1], c->stream));
            const int64_t r1 = c1 == n ? tiles : c1 / 128;  // tile rows complete
            int64_t upto = r1 * (r1 + 1) / 2;                // pairs ready
            if (c1 < n && gsplit == 1)
                upto = launched + (upto - launched) / c->num_sms * c->num_sms;
            if (upto > launched) {
                ALN_TRY(launch_gram_tc_pairs(c->opt.gram_split, hi, mid, lo, d, n, c->ldk,
                                             c->inv_s, (float*)c->Q, ldq, c->flags + 1,
                                             c->stream, launched, upto, gpart, gticket, gsplit,
                                             skp, skt, c->num_sms));
                launched = upto;
                ++c->launches;
            }
            ++c->launches;
        }
    } else {
        ALN_TRY(launch_colstats(c->A, dtype, d, n, lda, c->B, kc, ldb, c->s, c->inv_s, c->q64,
                                ldq, c->flags, hi, mid, lo, c->ldk, c->stream));
    }
    if (kc == 0) {
        if (c->batched && dtype == ALN_DTYPE_F32)  // FP64-accurate, exact digit products
            ALN_CHECK(qvec32(c, d, n, lda, k, ldb));
        else
            ALN_TRY(launch_qvec64(c->A, dtype, d, n, lda, c->B, k, ldb, c->inv_s, c->q64, ldq,
                                  c->stream));
    }
    ALN_TRY(launch_denominators(c->q64, n, ldq, k, c->den, c->stream));
    if (!pipelined) ALN_TRY(cudaEventRecord(c->ev[1], c->stream));
    if (pipelined)
        ;  // the Gram ran chunk by chunk above
    else if (c->batched)
        ALN_CHECK(batch_prepare(c));
    else if (f64) {
        ALN_CHECK(ensure(&c->g64_work, &c->g64_work_bytes,
                         gram64_split_bytes(d, n, c->num_sms)));
        ALN_TRY(launch_gram64(c->A, dtype, d, n, lda, c->inv_s, (double*)c->Q, ldq, c->stream,
                              (double*)c->g64_work, c->g64_work_bytes, c->num_sms));
    } else {
        ALN_TRY(launch_gram_tc(c->opt.gram_split, hi, mid, lo, d, n, c->ldk, c->inv_s,
                               (float*)c->Q, ldq, c->flags + 1, c->stream, 0, -1, gpart, gticket,
                               gsplit, skp, skt, c->num_sms));
    }
    ALN_TRY(cudaEventRecord(c->ev[2], c->stream));
    c->launches += 4 + (kc == 0 ? 1 : 0);

    ALN_CHECK(prep_finish(c, k));
    c->prepared = 1;
    return ALN_OK;
}

aln_status aln_prepare_csc(aln_ctx* c, int64_t d, int64_t n, const int64_t* col_ptr,
                           const int32_t* row_idx, const void* vals, int32_t dtype,
                           const void* B, int64_t k, int64_t ldb) {
    if (!c || !col_ptr || !B) return ALN_ERR_INVALID_ARG;
    if (d < 1 || n < 1 || k < 1 || ldb < d) return ALN_ERR_INVALID_ARG;
    if (dtype != ALN_DTYPE_F32 && dtype != ALN_DTYPE_F64) return ALN_ERR_INVALID_ARG;
    if (n > (int64_t)1 << 20 || d > ((int64_t)1 << 31) - 64) return ALN_ERR_INVALID_ARG;
    c->prepared = 0;
    c->grouped = 0;
    c->csc_kkt = 0;
    c->q_tmask = nullptr;
    c->stats.prepare_ms = c->stats.gram_ms = 0.0;
    const size_t esz = elt(dtype);
    const bool dev_ptr = is_device_ptr(col_ptr);
    int64_t* pin = (int64_t*)((uint8_t*)c->host_pool + 1024);  // pinned scratch
    int64_t nnz;
    if (dev_ptr) {
        ALN_TRY(cudaMemcpyAsync(pin, col_ptr + n, 8, cudaMemcpyDeviceToHost, c->stream));
        ALN_TRY(cudaStreamSynchronize(c->stream));
        nnz = pin[0];
    } else {
        nnz = col_ptr[n];
    }
    if (nnz < 0 || nnz > d * n) return ALN_ERR_INVALID_ARG;
    if (nnz > 0 && (!row_idx || !vals)) return ALN_ERR_INVALID_ARG;
    // the three arrays live on the same side (host or device)
    if (nnz > 0 && (is_device_ptr(row_idx) != dev_ptr || is_device_ptr(vals) != dev_ptr))
        return ALN_ERR_INVALID_ARG;

    c->d = d;
    c->n = n;
    c->k = k;
    c->dtype = dtype;
    ALN_CHECK(prep_buffers(c, n, k));
    const bool f64 = fp64(c);
    const int64_t ldq = c->ldq;
    // the sparse Gram serves the single-right-hand-side mixed-precision path;
    // FP64 and the many-right-hand-side solver form Q from the dense copy
    const bool sparse_gram = !f64 && !c->batched;
    const int64_t T = ceil_div(n, 128), KB = ceil_div(d, 64);
    const int W = (int)ceil_div(KB, 32);
    // FP32 values and at most four right-hand sides: nothing after the prepare
    // needs a dense copy of A (the KKT pass reads the CSC arrays and the
    // packed boxes, whose split terms add up exactly to the FP32 entries)
    const bool no_dense = sparse_gram && dtype == ALN_DTYPE_F32 && k <= 4;

    // CSC arrays on the device (host inputs copied; device inputs in place)
    // followed by the occupancy words, word prefixes, tile counts and offsets
    const size_t b_cp = round_up((size_t)(n + 1) * 8, 256);
    const size_t b_ri = round_up((size_t)nnz * 4, 256);
    const size_t b_v = round_up((size_t)nnz * esz, 256);
    const size_t b_occ = sparse_gram ? round_up((size_t)T * W * 4, 256) : 0;
    const size_t b_cnt = sparse_gram ? round_up((size_t)(2 * T + 1) * 8, 256) : 0;
    const size_t b_fp = no_dense ? round_up((size_t)KB * 8, 256) : 0;
    // work list of the block-sparse Gram: pair counts, items, tickets, totals
    const int64_t P = T * (T + 1) / 2;
    const size_t b_lp = sparse_gram ? round_up((size_t)P * 4, 256) : 0;
    const size_t b_it = sparse_gram ? round_up((size_t)(P + c->num_sms + 1) * sizeof(SItem), 256) : 0;
    const size_t b_tk = sparse_gram ? round_up((size_t)P * 4, 256) + 256 : 0;
    const int qtw = (int)ceil_div(T, 32);
    const size_t b_qm = sparse_gram ? round_up((size_t)T * qtw * 4, 256) : 0;
    const size_t b_copy = dev_ptr ? 0 : b_cp + b_ri + b_v;
    ALN_CHECK(ensure(&c->csc_pool, &c->csc_bytes,
                     b_copy + 2 * b_occ + b_cnt + b_fp + b_lp + b_it + b_tk + b_qm + 256));
    uint8_t* cp8 = (uint8_t*)c->csc_pool;
    const int64_t* cp = col_ptr;
    const int32_t* ri = row_idx;
    const void* vv = vals;
    if (!dev_ptr) {
        ALN_TRY(cudaMemcpyAsync(cp8, col_ptr, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice,
                                c->stream));
        cp = (const int64_t*)cp8;
        if (nnz > 0) {
            ALN_TRY(cudaMemcpyAsync(cp8 + b_cp, row_idx, (size_t)nnz * 4, cudaMemcpyHostToDevice,
                                    c->stream));
            ALN_TRY(cudaMemcpyAsync(cp8 + b_cp + b_ri, vals, (size_t)nnz * esz,
                                    cudaMemcpyHostToDevice, c->stream));
        }
        ri = (const int32_t*)(cp8 + b_cp);
        vv = cp8 + b_cp + b_ri;
        cp8 += b_copy;
    }
    uint32_t* occ = (uint32_t*)cp8;
    int32_t* wbase = (int32_t*)(cp8 + b_occ);
    int64_t* cnt = (int64_t*)(cp8 + 2 * b_occ);
    int64_t* toff = cnt + T;
    double* fpart = (double*)(cp8 + 2 * b_occ + b_cnt);
    int32_t* Lp = (int32_t*)(cp8 + 2 * b_occ + b_cnt + b_fp);
    SItem* items = (SItem*)(cp8 + 2 * b_occ + b_cnt + b_fp + b_lp);
    unsigned int* ticket = (unsigned int*)(cp8 + 2 * b_occ + b_cnt + b_fp + b_lp + b_it);
    int64_t* meta = (int64_t*)((uint8_t*)ticket + round_up((size_t)P * 4, 256));
    uint32_t* qmask = (uint32_t*)(cp8 + 2 * b_occ + b_cnt + b_fp + b_lp + b_it + b_tk);

    // dense column-major copy of A (16-byte columns) where a later step reads
    // it: the FP64 Gram, the many-right-hand-side solver, q for k > 4, or the
    // KKT pass of FP64 values
    const int64_t lda = round_up(d, (int64_t)(16 / esz));
    if (!no_dense) {
        ALN_CHECK(ensure(&c->A_copy, &c->A_copy_bytes, (size_t)n * lda * esz));
        c->A = c->A_copy;
    } else {
        c->A = nullptr;
    }
    c->lda = lda;
    ALN_CHECK(resolve_input(c, B, d, k, ldb, esz, &c->B_copy, &c->B_copy_bytes, &c->B));
    c->ldb = ldb;

    // structure first: every later kernel indexes with col_ptr and row_idx
    ALN_TRY(cudaEventRecord(c->ev[0], c->stream));
    ALN_TRY(launch_csc_check(cp, ri, vv, dtype, d, n, nnz, c->flags, c->stream));
    ALN_TRY(launch_check_finite(c->B, dtype, d, k, ldb, c->flags, c->stream));
    ALN_TRY(cudaMemcpyAsync(c->flags_host, c->flags, 3 * sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream));
    ALN_TRY(cudaStreamSynchronize(c->stream));
    if (c->flags_host[2]) return ALN_ERR_INVALID_ARG;
    if (c->flags_host[0]) return ALN_ERR_NONFINITE;

    // Alg. 1: scale factors, q, occupancy (and the scatter)
    if (!no_dense) ALN_TRY(cudaMemsetAsync(c->A_copy, 0, (size_t)n * lda * esz, c->stream));
    if (sparse_gram) ALN_TRY(cudaMemsetAsync(occ, 0, b_occ, c->stream));
    const int kc = k <= 4 ? (int)k : 0;
    ALN_TRY(launch_csc_colstats(cp, ri, vv, dtype, n, c->B, kc, ldb,
                                no_dense ? nullptr : c->A_copy, lda, c->s,
                                c->inv_s, c->q64, ldq, sparse_gram ? occ : nullptr, W,
                                c->stream));
    c->launches += 3;
    if (kc == 0) {
        if (c->batched && dtype == ALN_DTYPE_F32)
            ALN_CHECK(qvec32(c, d, n, lda, k, ldb));
        else
            ALN_TRY(launch_qvec64(c->A, dtype, d, n, lda, c->B, k, ldb, c->inv_s, c->q64, ldq,
                                  c->stream));
        ++c->launches;
    }
    ALN_TRY(launch_denominators(c->q64, n, ldq, k, c->den, c->stream));
    ALN_TRY(cudaEventRecord(c->ev[1], c->stream));
    if (sparse_gram) {
        // number the occupied boxes, size the pack, scatter the split terms
        ALN_TRY(launch_csc_number(occ, W, T, wbase, cnt, toff, c->stream));
        ALN_TRY(launch_csc_worklist(occ, W, T, c->num_sms, Lp, items, meta, c->stream));
        ALN_TRY(launch_csc_qmask(Lp, T, qmask, c->stream));
        ALN_TRY(cudaMemcpyAsync(pin, toff + T, 8, cudaMemcpyDeviceToHost, c->stream));
        ALN_TRY(cudaMemcpyAsync(pin + 1, meta, 16, cudaMemcpyDeviceToHost, c->stream));
        ALN_TRY(cudaStreamSynchronize(c->stream));
        const int64_t boxes = pin[0], nitems = pin[1], nslots = pin[2];
        // partial tiles of the pairs split over several CTAs (≤ 2·num_sms)
        ALN_CHECK(ensure(&c->sp_part, &c->sp_part_bytes,
                         (size_t)std::max<int64_t>(nslots, 1) * 128 * 128 * 4));
        ALN_TRY(cudaMemsetAsync(ticket, 0, (size_t)P * 4, c->stream));
        // tile pairs without a common block have no work item: Q starts at zero
        ALN_TRY(cudaMemsetAsync(c->Q, 0, c->Q_bytes, c->stream));
        const size_t sb = round_up((size_t)std::max<int64_t>(boxes, 1) * 128 * 64 * 2, 1024);
        ALN_CHECK(ensure((void**)&c->A_hi, &c->split_bytes, 3 * sb));
        __nv_bfloat16* hi = c->A_hi;
        __nv_bfloat16* mid = (__nv_bfloat16*)((uint8_t*)c->A_hi + sb);
        __nv_bfloat16* lo = (__nv_bfloat16*)((uint8_t*)c->A_hi + 2 * sb);
        ALN_TRY(cudaMemsetAsync(c->A_hi, 0, 3 * sb, c->stream));
        ALN_TRY(launch_csc_pack(cp, ri, vv, dtype, n, occ, W, wbase, toff, hi, mid, lo,
                                c->stream));
        ALN_TRY(launch_sgram_tc(c->opt.gram_split, items, nitems, occ, W, wbase, toff, hi, mid, lo,
                                n, c->inv_s, (float*)c->Q, ldq, (float*)c->sp_part, ticket,
                                c->flags + 1, c->stream));
        c->launches += 7;
        c->q_tmask = qmask;  // the Alg. 2 products skip Q's zero tiles
        c->q_tw = qtw;
        if (no_dense) {  // the KKT pass reads these until the next prepare
            c->csc_cp = cp;
            c->csc_ri = ri;
            c->csc_v = (const float*)vv;
            c->csc_occ = occ;
            c->csc_wbase = wbase;
            c->csc_toff = toff;
            c->csc_fpart = fpart;
            c->csc_W = W;
            c->csc_box_bytes = sb;
        }
    } else if (c->batched) {
        ALN_CHECK(batch_prepare(c));
    } else {
        ALN_CHECK(ensure(&c->g64_work, &c->g64_work_bytes,
                         gram64_split_bytes(d, n, c->num_sms)));
        ALN_TRY(launch_gram64(c->A, dtype, d, n, lda, c->inv_s, (double*)c->Q, ldq, c->stream,
                              (double*)c->g64_work, c->g64_work_bytes, c->num_sms));
        ++c->launches;
    }
    ALN_TRY(cudaEventRecord(c->ev[2], c->stream));
    ALN_CHECK(prep_finish(c, k));
    c->csc_kkt = no_dense ? 1 : 0;
    c->prepared = 1;
    return ALN_OK;
}

aln_status aln_prepare_grouped(aln_ctx* c, int32_t count, const aln_problem* probs,
                               int32_t dtype) {
    if (!c || !probs || count < 1 || count > (1 << 20)) return ALN_ERR_INVALID_ARG;
    if (dtype != ALN_DTYPE_F32 && dtype != ALN_DTYPE_F64) return ALN_ERR_INVALID_ARG;
    c->csc_kkt = 0;
    c->q_tmask = nullptr;
    int64_t cols = 0;
    for (int32_t p = 0; p < count; ++p) {
        const aln_problem& q = probs[p];
        if (!q.A || !q.b || q.d < 1 || q.n < 1 || q.lda < q.d || q.d > ((int64_t)1 << 30))
            return ALN_ERR_INVALID_ARG;
        cols += q.n;
    }
    if (cols > ((int64_t)1 << 31) / 128) return ALN_ERR_INVALID_ARG;
    if (c->opt.algorithm != ALN_ALG_ANTILOP) return ALN_ERR_UNSUPPORTED;
    c->prepared = 0;
    c->batched = 0;
    c->grouped = 0;
    c->stats.prepare_ms = c->stats.gram_ms = 0.0;
    ALN_CHECK(group_prepare(c, count, probs, dtype));
    c->k = count;
    c->dtype = dtype;
    c->prepared = 1;
    return ALN_OK;
}

aln_status aln_solve(aln_ctx* c, double tol, int32_t max_iter, double* X, int64_t ldx,
                     const double* X0, aln_solve_info* info) {
    if (!c) return ALN_ERR_INVALID_ARG;
    if (!c->prepared) return ALN_ERR_NOT_PREPARED;
    if (c->grouped) {
        if (!X || !(tol > 0.0) || !std::isfinite(tol)) return ALN_ERR_INVALID_ARG;
        if (max_iter <= 0) max_iter = 20000;
        ALN_CHECK(autotune_solve(c, tol, max_iter, X, 0, X0));
        c->stats.solve_ms = c->stats.kkt_ms = c->stats.iterate_ms = 0.0;
        c->stats.passive_rows = c->stats.clipped_rows = 0;
        c->stats.clipped_iterations = 0;
        c->stats.iterations = 0;
        c->stats.product_bytes = 0.0;
        for (double& v : c->stats.phase_us) v = 0.0;
        ALN_TRY(cudaEventRecord(c->ev[4], c->stream));
        ALN_CHECK(group_solve(c, tol, max_iter, X, X0, info));
        ALN_TRY(cudaEventRecord(c->ev[5], c->stream));
        ALN_TRY(cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]) == cudaSuccess) c->stats.solve_ms = ms;
        return ALN_OK;
    }
    if (!X || ldx < c->n || !(tol > 0.0) || !std::isfinite(tol)) return ALN_ERR_INVALID_ARG;
    const int64_t n = c->n;
    if (max_iter <= 0) max_iter = (int32_t)std::max<int64_t>(5 * n, 20000);
    const bool x_dev = is_device_ptr(X);
    const bool x0_dev = X0 ? is_device_ptr(X0) : false;
    const bool f64 = fp64(c);
    ALN_CHECK(autotune_solve(c, tol, max_iter, X, ldx, X0));
    c->stats.solve_ms = c->stats.kkt_ms = c->stats.iterate_ms = 0.0;
    c->stats.passive_rows = c->stats.clipped_rows = 0;
    c->stats.clipped_iterations = 0;
    c->stats.product_bytes = 0.0;
    for (double& v : c->stats.phase_us) v = 0.0;
    c->stats.iterations = 0;
    ALN_TRY(cudaEventRecord(c->ev[4], c->stream));
    if (c->batched) {
        ALN_CHECK(batch_solve(c, tol, max_iter, X, ldx, X0, info));
        ALN_TRY(cudaEventRecord(c->ev[5], c->stream));
        ALN_TRY(cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]) == cudaSuccess) c->stats.solve_ms = ms;
        return ALN_OK;
    }
    if (c->opt.algorithm == ALN_ALG_ANTI_ACC) ALN_CHECK(ensure_lipschitz(c));
    // Inner runs stop a little below tol so that the FP64 check usually passes
    // at once; refinement rounds aim lower still.
    const double first_factor = 0.5, refine_factor = 0.25;

    for (int64_t rhs = 0; rhs < c->k; ++rhs) {
        const double den = c->den_host[rhs];
        auto eps_of = [&](double t) {
            const double a = t * (den > 0.0 ? den : 1.0);
            return a * a;
        };
        const double* x0 = nullptr;
        if (X0) {
            // stage x0 in g64 (free until the first KKT pass)
            ALN_TRY(cudaMemcpyAsync(c->g64, X0 + rhs * ldx, (size_t)n * 8,
                                    x0_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    c->stream));
            int* bad = c->flags;
            ALN_TRY(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
            ALN_TRY(launch_check_finite(c->g64, ALN_DTYPE_F64, n, 1, n, bad, c->stream));
            c->launches += 1;
            ALN_TRY(cudaMemcpyAsync(c->flags_host, bad, sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
            ALN_TRY(cudaStreamSynchronize(c->stream));
            if (c->flags_host[0]) return ALN_ERR_NONFINITE;
            x0 = c->g64;
        }
        const double* q64 = c->q64 + rhs * c->ldq;
        int total = 0, rounds = 0, status = ALN_RHS_MAXITER;
        double rel = 0.0, F = 0.0;
        // the FP64 iteration has no model error to refine away: one run to tol
        const int gain = (f64 || c->opt.refine_gain == 0) ? -1 : c->opt.refine_gain;
        const double t0 = inner_target(tol, first_factor, 1.0, gain);
        ALN_TRY(f64 ? launch_iter_setup<double>(c, q64, x0, eps_of(t0), max_iter)
                    : launch_iter_setup<float>(c, q64, x0, eps_of(t0), max_iter));
        c->launches += x0 ? 4 : 3;
        for (;;) {
            ALN_CHECK(run_until_done(c));
            total += c->st_host->iter;
            const int inner = c->st_host->status;
            ALN_TRY(f64 ? launch_unscale<double>(c, c->x64) : launch_unscale<float>(c, c->x64));
            c->launches += 1;
            ALN_CHECK(kkt_eval(c, rhs, c->x64, &rel, &F));
            if (rel <= tol) {
                status = inner == ALN_RHS_EMPTY_PASSIVE ? ALN_RHS_EMPTY_PASSIVE : ALN_RHS_CONVERGED;
                break;
            }
            if (inner == ALN_RHS_NONFINITE) {
                status = ALN_RHS_NONFINITE;
                break;
            }
            if (total >= max_iter || inner == ALN_RHS_MAXITER) {
                status = ALN_RHS_MAXITER;
                break;
            }
            if (rounds >= c->opt.max_refine) {
                status = inner == ALN_RHS_STAGNATED ? ALN_RHS_STAGNATED : ALN_RHS_MAXITER;
                break;
            }
            // Refinement: restart the inner loop from the current y with the exact
            // FP64 gradient g = Qy + q evaluated from A (left in c->g64 by the KKT pass).
            ++rounds;
            const double tr = inner_target(tol, refine_factor, rel, gain);
            ALN_TRY(f64 ? launch_iter_refresh_from_g64<double>(c, eps_of(tr), max_iter - total)
                        : launch_iter_refresh_from_g64<float>(c, eps_of(tr), max_iter - total));
            c->launches += 2;
        }
        c->stats.iterations += total;
        ALN_TRY(cudaMemcpyAsync(X + rhs * ldx, c->x64, (size_t)n * 8,
                                x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
        if (info) {
            info[rhs].iters = total;
            info[rhs].status = status;
            info[rhs].refine_rounds = rounds;
            info[rhs].reserved = 0;
            info[rhs].rel_kkt = rel;
            info[rhs].objective = F;
        }
    }
    ALN_TRY(cudaEventRecord(c->ev[5], c->stream));
    ALN_TRY(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]) == cudaSuccess) c->stats.solve_ms = ms;
    return ALN_OK;
}

aln_status aln_set_wait_limit(aln_ctx* c, int32_t wait_limit_us, int32_t test_barrier_skew) {
    if (!c || wait_limit_us < 0 || test_barrier_skew < 0 || test_barrier_skew > 1024)
        return ALN_ERR_INVALID_ARG;
    c->opt.wait_limit_us = wait_limit_us;
    c->opt.test_barrier_skew = test_barrier_skew;
    return ALN_OK;
}

aln_status aln_get_stats(aln_ctx* c, aln_stats* out) {
    if (!c || !out) return ALN_ERR_INVALID_ARG;
    *out = c->stats;
    out->kernel_launches = c->launches;
    out->persist_blocks = c->p_G;
    out->iter_kernel = (c->batched || c->grouped || !c->prepared) ? 0
                       : c->p_small                                ? 3
                       : c->p_repl                                 ? 2
                                                                   : 1;
    out->reserved2 = 0;
    return ALN_OK;
}

aln_status aln_kkt_residual(aln_ctx* c, const double* X, int64_t ldx, double* rel_kkt,
                            double* objective) {
    if (!c) return ALN_ERR_INVALID_ARG;
    if (!c->prepared) return ALN_ERR_NOT_PREPARED;
    if (c->grouped) {
        if (!X || !rel_kkt) return ALN_ERR_INVALID_ARG;
        return group_kkt(c, X, rel_kkt, objective);
    }
    if (!X || !rel_kkt || ldx < c->n) return ALN_ERR_INVALID_ARG;
    const bool x_dev = is_device_ptr(X);
    const bool r_dev = is_device_ptr(rel_kkt);
    const bool o_dev = objective ? is_device_ptr(objective) : false;
    for (int64_t rhs = 0; rhs < c->k; ++rhs) {
        ALN_TRY(cudaMemcpyAsync(c->x64, X + rhs * ldx, (size_t)c->n * 8,
                                x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream));
        double rel, F;
        ALN_CHECK(kkt_eval(c, rhs, c->x64, &rel, &F));
        ALN_TRY(cudaMemcpy(rel_kkt + rhs, &rel, 8,
                           r_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
        if (objective)
            ALN_TRY(cudaMemcpy(objective + rhs, &F, 8,
                               o_dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    }
    return ALN_OK;
}

aln_status aln_export_scaled(aln_ctx* c, double* Q, int64_t ldq, double* q, int64_t ldqv,
                             double* s) {
    if (!c) return ALN_ERR_INVALID_ARG;
    if (!c->prepared) return ALN_ERR_NOT_PREPARED;
    if (c->grouped) return group_export(c, Q, q, s);
    const int64_t n = c->n;
    if ((Q && ldq < n) || (q && ldqv < n)) return ALN_ERR_INVALID_ARG;
    if (Q) {
        const bool dev = is_device_ptr(Q);
        double* dst = Q;
        double* tmp = nullptr;
        if (!dev) {
            ALN_TRY(cudaMalloc(&tmp, (size_t)n * n * 8));
            dst = tmp;
        }
        const int64_t ldd = dev ? ldq : n;
        const int blocks = (int)std::min<int64_t>(ceil_div(n * n, 256), 8192);
        if (fp64(c))
            k_copy_to_f64<double><<<blocks, 256, 0, c->stream>>>((const double*)c->Q, c->ldq, dst,
                                                                 ldd, n, n);
        else
            k_copy_to_f64<float><<<blocks, 256, 0, c->stream>>>((const float*)c->Q, c->ldq, dst,
                                                                ldd, n, n);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && !dev)
            e = cudaMemcpy2DAsync(Q, ldq * 8, tmp, n * 8, n * 8, n, cudaMemcpyDeviceToHost,
                                  c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (tmp) cudaFree(tmp);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (q) {
        const bool dev = is_device_ptr(q);
        ALN_TRY(cudaMemcpy2DAsync(q, ldqv * 8, c->q64, c->ldq * 8, n * 8, c->k,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream));
    }
    if (s) {
        const bool dev = is_device_ptr(s);
        ALN_TRY(cudaMemcpyAsync(s, c->s, n * 8,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    }
    ALN_TRY(cudaStreamSynchronize(c->stream));
    return ALN_OK;
}

void aln_default_train_opts(aln_train_opts* o) {
    if (!o) return;
    o->epochs = 10;
    o->batch = 1024;
    o->hidden = 1024;
    o->reserved = 0;
    o->lr = 1e-3;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->seed = 0;
}

static aln_status ws_ready(aln_ctx* c) {
    if (!c) return ALN_ERR_INVALID_ARG;
    if (!c->prepared) return ALN_ERR_NOT_PREPARED;
    if (c->grouped) return ALN_ERR_INVALID_ARG;
    return ALN_OK;
}

aln_status aln_warmstart_init(aln_ctx* c, int32_t hidden, uint64_t seed) {
    ALN_CHECK(ws_ready(c));
    if (hidden < 1 || hidden > (1 << 16)) return ALN_ERR_INVALID_ARG;
    return mlp_init(c, hidden, seed);
}

aln_status aln_warmstart_params(aln_ctx* c, int32_t set, float* W1, float* b1, float* W2,
                                float* b2, float* W3, float* b3, float* e, float* f, float* mu,
                                float* sd, float* muz, float* sdz, float* tau) {
    ALN_CHECK(ws_ready(c));
    if (mlp_n(c) != c->n) return ALN_ERR_INVALID_ARG;
    float* t[13] = {W1, b1, W2, b2, W3, b3, e, f, mu, sd, muz, sdz, tau};
    return mlp_params(c, set ? 1 : 0, t);
}

aln_status aln_warmstart_grad(aln_ctx* c, const double* Qb, const double* Yb, int64_t count,
                              double* loss, float* gW1, float* gb1, float* gW2, float* gb2,
                              float* gW3, float* gb3, float* ge, float* gf) {
    ALN_CHECK(ws_ready(c));
    if (!Qb || !Yb || count < 1 || count > (1 << 20) || mlp_n(c) != c->n)
        return ALN_ERR_INVALID_ARG;
    float* g[8] = {gW1, gb1, gW2, gb2, gW3, gb3, ge, gf};
    return mlp_grad(c, Qb, Yb, count, loss, g);
}

aln_status aln_warmstart_train(aln_ctx* c, const double* Qtrain, const double* Ytrain,
                               int64_t count, const aln_train_opts* opts, double* epoch_loss) {
    ALN_CHECK(ws_ready(c));
    aln_train_opts o;
    aln_default_train_opts(&o);
    if (opts) o = *opts;
    if (!Qtrain || !Ytrain || count < 1 || count > ((int64_t)1 << 31) - 1 || o.epochs < 0 ||
        o.batch < 1 || o.batch > (1 << 16) || o.hidden < 1 || !(o.lr > 0.0) ||
        !(o.beta1 >= 0.0 && o.beta1 < 1.0) || !(o.beta2 >= 0.0 && o.beta2 < 1.0) ||
        !(o.eps > 0.0))
        return ALN_ERR_INVALID_ARG;
    if (mlp_n(c) != c->n) ALN_CHECK(mlp_init(c, o.hidden, o.seed));
    return mlp_train(c, Qtrain, Ytrain, count, o, epoch_loss);
}

aln_status aln_warmstart_predict(aln_ctx* c, double* X0, int64_t ldx, int32_t* kept) {
    ALN_CHECK(ws_ready(c));
    if (!X0 || ldx < c->n || mlp_n(c) != c->n) return ALN_ERR_INVALID_ARG;
    return mlp_predict(c, X0, ldx, kept);
}

}  // extern "C"
