// Host implementation of the C ABI declared in include/gempe.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.cuh"
#include "gempe.h"

#define GEMPE_API extern "C" __attribute__((visibility("default")))

namespace {

using namespace gempe;

thread_local std::string g_last_error;

gempe_status fail(gempe_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

gempe_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? GEMPE_E_OOM : GEMPE_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
    } while (0)

}  // namespace

struct gempe_ctx {
    gempe_params p{};
    int32_t n = 0, d = 0, k = 0, acc_stride = 0;
    int64_t nnz = 0;
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;          // the sampler of the next epoch runs here, beside the sweep
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    bool primed = false;                  // samples of the current epoch are in the buffer
    bool sampled_ahead = false;           // the next epoch's sampler has been launched
    // device memory
    int32_t* row_ptr = nullptr;
    int32_t* col_idx = nullptr;
    unsigned long long* keys = nullptr;
    unsigned long long bucket_mask = 0;
    float* x = nullptr;
    float* acc = nullptr;
    // distance histograms, one allocation: hist_d [bins] u64, hist_e, hist_c [bins] u32, hist_x [bins] f32
    void* hist = nullptr;
    size_t hist_bytes = 0;
    unsigned long long* hist_d = nullptr;
    unsigned int* hist_e = nullptr;
    unsigned int* hist_c = nullptr;
    float* hist_x = nullptr;
    DevState* st = nullptr;
    int4* items = nullptr;
    int32_t n_items = 0;
    int32_t* scratch_i32 = nullptr;   // n*k inspection samples / flags
    int32_t* samples = nullptr;       // [2][n*k] sampled partners, buffer = epoch & 1
    int sampler_grid = 0;
    __nv_bfloat16* xb = nullptr;      // BF16 shadow positions (precision form)
    bool block = false;               // block sampling
    bool tiles = false;               // block samples on the tensor-core tile kernel
    int32_t n_tiles = 0;
    int32_t* block_part = nullptr;    // [2][n_tiles][64]
    unsigned long long* block_mask = nullptr;   // [2][n]
    int4* sampler_units = nullptr;    // block sampler work units {tile, e_lo, e_hi, first}
    int32_t n_sampler_units = 0;
    const MillsCoef* mills = nullptr;
    int32_t slots() const { return block ? kBlockP : k; }
    int sweep_grid = 0, update_grid = 0;
    bool swept = false;               // a sweep ran without the update that clears its sums
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<void*> allocations;

    void* alloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        void* ptr = nullptr;
        if (p.dev_alloc) {
            ptr = p.dev_alloc(bytes, p.alloc_user);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
        }
        if (ptr) allocations.push_back(ptr);
        return ptr;
    }
    void release_all() {
        for (void* ptr : allocations) {
            if (p.dev_free) p.dev_free(ptr, p.alloc_user);
            else cudaFree(ptr);
        }
        allocations.clear();
    }
};

namespace {

EpochArgs epoch_args(const gempe_ctx* c) {
    EpochArgs a{};
    a.row_ptr = c->row_ptr;
    a.col_idx = c->col_idx;
    a.keys = c->keys;
    a.bucket_mask = c->bucket_mask;
    a.x = c->x;
    a.acc = c->acc;
    a.hist_e = c->hist_e;
    a.hist_c = c->hist_c;
    a.hist_d = c->hist_d;
    a.hist_x = c->hist_x;
    a.st = c->st;
    a.items = c->items;
    a.n_items = c->n_items;
    a.n = c->n;
    a.d = c->d;
    a.acc_stride = c->acc_stride;
    a.k = c->k;
    a.max_retries = c->p.max_retries;
    a.symmetric = c->p.symmetric_neg;
    a.w_formula = c->p.w_formula;
    a.clamp_neg_d = c->p.clamp_neg_d;
    a.bins = c->p.hist_bins;
    a.mu = c->p.mu;
    a.hist_scale = (float)c->p.hist_bins / c->p.hist_max;
    a.key_lo = (uint32_t)c->p.seed;
    a.key_hi = (uint32_t)(c->p.seed >> 32);
    a.samples = c->samples;
    a.xb = c->xb;
    a.block_P = c->block ? kBlockP : 0;
    a.block_T = kBlockT;
    a.n_tiles = c->n_tiles;
    a.block_part = c->block_part;
    a.block_mask = c->block_mask;
    a.sweep_samples = c->tiles ? 0 : 1;
    a.mills = c->mills;
    return a;
}

UpdateArgs update_args(const gempe_ctx* c) {
    UpdateArgs u{};
    u.x = c->x;
    u.acc = c->acc;
    u.hist_e = c->hist_e;
    u.hist_c = c->hist_c;
    u.hist_d = c->hist_d;
    u.hist_x = c->hist_x;
    u.k = c->slots();
    u.xb = c->xb;
    u.st = c->st;
    u.n = c->n;
    u.d = c->d;
    u.acc_stride = c->acc_stride;
    u.bins = c->p.hist_bins;
    u.sigma_every = c->p.sigma_every;
    u.z_min = c->p.z_min;
    u.mu = c->p.mu;
    u.hist_max = c->p.hist_max;
    return u;
}

gempe_status check_params(const gempe_params* p, int32_t n, int32_t d) {
    if (!p) return fail(GEMPE_E_INVALID_ARG, "params is null");
    if (n < 2) return fail(GEMPE_E_INVALID_ARG, "n must be at least 2");
    if (!supported_dim(d)) return fail(GEMPE_E_INVALID_ARG, "d must be one of 1,2,3,4,8,16,32,64,128,256");
    if (p->neg_per_vertex < 0 || p->neg_per_vertex > kMaxK)
        return fail(GEMPE_E_INVALID_ARG, "neg_per_vertex must be in [0, 32]");
    if (p->max_retries < 1 || p->max_retries > 4096)
        return fail(GEMPE_E_INVALID_ARG, "max_retries must be in [1, 4096]");
    if (p->hist_bins < 16 || p->hist_bins > 4096)
        return fail(GEMPE_E_INVALID_ARG, "hist_bins must be in [16, 4096]");
    if (!(p->hist_max > 0.0f) || !(p->sigma0 > 0.0f) || !std::isfinite(p->mu) || !(p->init_range > 0.0f) ||
        !(p->z_min > 0.0f))
        return fail(GEMPE_E_INVALID_ARG, "hist_max, sigma0, init_range and z_min must be positive, mu finite");
    if (p->sigma_every < 0) return fail(GEMPE_E_INVALID_ARG, "sigma_every must be >= 0");
    if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr))
        return fail(GEMPE_E_INVALID_ARG, "dev_alloc and dev_free must be given together");
    if (p->precision != 0 && p->precision != 1) return fail(GEMPE_E_INVALID_ARG, "precision must be 0 or 1");
    if (p->precision == 1 && d < 8) return fail(GEMPE_E_INVALID_ARG, "the BF16 form needs d >= 8");
    if (p->block_partners != 0 && p->block_partners != kBlockP)
        return fail(GEMPE_E_INVALID_ARG, "block_partners must be 0 or 64");
    if (p->block_partners && (d < 8 || (p->tile_vertices != 0 && p->tile_vertices != kBlockT)))
        return fail(GEMPE_E_INVALID_ARG, "block sampling needs d >= 8 and tile_vertices 128");
    return GEMPE_OK;
}

// Symmetric, sorted, loop-free, duplicate-free, in-range CSR.
gempe_status validate_csr(const int32_t* rp, const int32_t* ci, int32_t n) {
    if (rp[0] != 0) return fail(GEMPE_E_INVALID_GRAPH, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return fail(GEMPE_E_INVALID_GRAPH, "row_ptr must be non-decreasing");
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            if (j < 0 || j >= n) return fail(GEMPE_E_INVALID_GRAPH, "column index out of range");
            if (j == i) return fail(GEMPE_E_INVALID_GRAPH, "self loop at vertex " + std::to_string(i));
            if (e > rp[i] && ci[e - 1] >= j)
                return fail(GEMPE_E_INVALID_GRAPH, "row " + std::to_string(i) + " not strictly increasing");
        }
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            if (!std::binary_search(ci + rp[j], ci + rp[j + 1], i))
                return fail(GEMPE_E_INVALID_GRAPH, "graph not symmetric: (" + std::to_string(i) + "," +
                                                       std::to_string(j) + ") without its reverse");
        }
    return GEMPE_OK;
}

// Work units of the packed sweep (d <= 4): runs of up to 32 consecutive
// vertices with at most kUnitPairs edge + sample slots in total; a vertex with
// more is cut into kUnitPairs-slot chunks of its row, the last chunk (at most
// kUnitPairs slots plus its k samples) carrying the samples.
std::vector<int4> build_packed_units(const int32_t* rp, int32_t n, int32_t k) {
    std::vector<int4> units;
    units.reserve((size_t)n / 4 + (size_t)(rp[n] / kUnitPairs) + 16);
    const int smp = k > 0 ? kUnitHasSamples : 0;
    int32_t i = 0;
    while (i < n) {
        const int32_t deg = rp[i + 1] - rp[i];
        if (deg + k > kUnitPairs) {
            int32_t e = 0;
            while (deg - e > kUnitPairs) {
                units.push_back(make_int4(i, 1, e, e + kUnitPairs));
                e += kUnitPairs;
            }
            units.push_back(make_int4(i, 1, e, deg | smp));
            ++i;
            continue;
        }
        const int32_t v0 = i;
        int32_t pairs = 0;
        while (i < n && i - v0 < 32) {
            const int32_t di = rp[i + 1] - rp[i] + k;
            if (di > kUnitPairs || pairs + di > kUnitPairs) break;
            pairs += di;
            ++i;
        }
        units.push_back(make_int4(v0, i - v0, -1, smp));
    }
    return units;
}

// Work units of the per-unit sweep (d >= 8): each vertex's CSR slots in
// chunks of kEdgeChunk, the last chunk also carrying the vertex's samples.
std::vector<int4> build_chunk_units(const int32_t* rp, int32_t n) {
    std::vector<int4> items;
    items.reserve((size_t)n + (size_t)(rp[n] / kEdgeChunk) + 1);
    for (int32_t i = 0; i < n; ++i) {
        const int32_t deg = rp[i + 1] - rp[i];
        const int32_t chunks = std::max<int32_t>(1, (deg + kEdgeChunk - 1) / kEdgeChunk);
        for (int32_t c = 0; c < chunks; ++c) {
            const int32_t p0 = c * kEdgeChunk, p1 = std::min(deg, (c + 1) * kEdgeChunk);
            items.push_back(make_int4(i, 1, p0, p1 | (c == chunks - 1 ? kUnitHasSamples : 0)));
        }
    }
    return items;
}

gempe_status create_impl(const int32_t* rp_host, const int32_t* ci_host, int32_t n, int32_t d,
                         const gempe_params* p, void* stream, gempe_ctx** out) {
    gempe_status s = check_params(p, n, d);
    if (s != GEMPE_OK) return s;
    const int64_t nnz = rp_host[n];
    if (nnz < 0) return fail(GEMPE_E_INVALID_GRAPH, "row_ptr[n] negative");
    s = validate_csr(rp_host, ci_host, n);
    if (s != GEMPE_OK) return s;

    gempe_ctx* c = new gempe_ctx();
    c->p = *p;
    c->n = n;
    c->d = d;
    c->k = p->neg_per_vertex;
    c->nnz = nnz;
    c->acc_stride = acc_stride_for(d);
    auto bail = [&](gempe_status st) {
        if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
        if (c->graph) cudaGraphDestroy(c->graph);
        if (c->stream) cudaStreamSynchronize(c->stream);
        if (c->side) cudaStreamSynchronize(c->side);
        c->release_all();
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        if (c->join_ev) cudaEventDestroy(c->join_ev);
        if (c->side) cudaStreamDestroy(c->side);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return st;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    e = ensure_mills_table();
    if (e != cudaSuccess) return bail(cuda_fail(e, "Mills table"));
    e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
        c->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));

    // exact edge set: 2*nnz slots rounded up to a power of two (load <= 1/2), 4-slot buckets
    unsigned long long slots = 16;
    while (slots < 2ull * (unsigned long long)nnz) slots <<= 1;
    c->bucket_mask = slots / 4 - 1;
    c->block = p->block_partners > 0;
    c->tiles = c->block && p->precision == 1 && tile_dim(d);
    c->n_tiles = (n + kBlockT - 1) / kBlockT;
    // the per-block sums of sampled anchors' degrees are 32-bit: slots * nnz must stay below 2^32
    if ((unsigned long long)std::max(p->neg_per_vertex, c->slots()) * (unsigned long long)nnz >= (1ull << 32))
        return bail(fail(GEMPE_E_INVALID_ARG, "sample slots * nnz must be below 2^32"));
    c->mills = mills_table_device();
    if (!c->mills) return bail(fail(GEMPE_E_CUDA, "Mills table address"));
    if (c->tiles) {
        e = prepare_tile_kernel(d, p->hist_bins);
        if (e != cudaSuccess) return bail(cuda_fail(e, "tile kernel attributes"));
    }
    std::vector<int4> items = (d <= kPackedMaxDim) ? build_packed_units(rp_host, n, p->neg_per_vertex)
                                                   : build_chunk_units(rp_host, n);
    c->n_items = (int32_t)items.size();

    c->row_ptr = (int32_t*)c->alloc(sizeof(int32_t) * ((size_t)n + 1));
    c->col_idx = (int32_t*)c->alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    c->keys = (unsigned long long*)c->alloc(sizeof(unsigned long long) * slots);
    c->x = (float*)c->alloc(sizeof(float) * (size_t)n * d);
    c->acc = (float*)c->alloc(sizeof(float) * (size_t)n * c->acc_stride);
    const size_t B = (size_t)p->hist_bins;
    c->hist_bytes = B * (sizeof(unsigned long long) + 2 * sizeof(unsigned int) + sizeof(float));
    c->hist = c->alloc(c->hist_bytes);
    if (c->hist) {
        c->hist_d = (unsigned long long*)c->hist;
        c->hist_e = (unsigned int*)(c->hist_d + B);
        c->hist_c = c->hist_e + B;
        c->hist_x = (float*)(c->hist_c + B);
    }
    c->st = (DevState*)c->alloc(sizeof(DevState));
    c->items = (int4*)c->alloc(sizeof(int4) * items.size());
    c->scratch_i32 = (int32_t*)c->alloc(sizeof(int32_t) * std::max<size_t>((size_t)n * c->k, 1));
    c->samples = (int32_t*)c->alloc(sizeof(int32_t) * std::max<size_t>(c->block ? 1 : 2 * (size_t)n * c->k, 1));
    if (!c->samples) return bail(fail(GEMPE_E_OOM, "device allocation failed"));
    if (p->precision == 1) {
        c->xb = (__nv_bfloat16*)c->alloc(sizeof(__nv_bfloat16) * (size_t)n * d);
        if (!c->xb) return bail(fail(GEMPE_E_OOM, "device allocation failed"));
    }
    std::vector<int4> sunits;
    if (c->block) {
        for (int32_t t = 0; t < c->n_tiles; ++t) {
            const int32_t v0 = t * kBlockT, v1 = std::min(n, v0 + kBlockT);
            const int32_t e0 = rp_host[v0], e1 = rp_host[v1];
            int32_t e = e0;
            do {
                const int32_t eh = std::min(e1, e + kSamplerChunk);
                sunits.push_back(make_int4(t, e, eh, e == e0 ? 1 : 0));
                e = eh;
            } while (e < e1);
        }
        c->n_sampler_units = (int32_t)sunits.size();
        c->block_part = (int32_t*)c->alloc(sizeof(int32_t) * 2 * (size_t)c->n_tiles * kBlockP);
        c->block_mask = (unsigned long long*)c->alloc(sizeof(unsigned long long) * 2 * (size_t)n);
        c->sampler_units = (int4*)c->alloc(sizeof(int4) * sunits.size());
        if (!c->block_part || !c->block_mask || !c->sampler_units)
            return bail(fail(GEMPE_E_OOM, "device allocation failed"));
    }
    if (!c->row_ptr || !c->col_idx || !c->keys || !c->x || !c->acc || !c->hist || !c->st || !c->items ||
        !c->scratch_i32)
        return bail(fail(GEMPE_E_OOM, "device allocation failed"));

    cudaStream_t st = c->stream;
#define CKB(call, what)                                           \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, what));  \
    } while (0)
    CKB(cudaMemcpyAsync(c->row_ptr, rp_host, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st),
        "copy row_ptr");
    if (nnz > 0)
        CKB(cudaMemcpyAsync(c->col_idx, ci_host, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st),
            "copy col_idx");
    CKB(cudaMemcpyAsync(c->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st),
        "copy work units");
    CKB(cudaMemsetAsync(c->keys, 0xFF, sizeof(unsigned long long) * slots, st), "clear hash");
    if (c->block) {
        CKB(cudaMemsetAsync(c->block_mask, 0, sizeof(unsigned long long) * 2 * (size_t)n, st), "clear masks");
        CKB(cudaMemcpyAsync(c->sampler_units, sunits.data(), sizeof(int4) * sunits.size(), cudaMemcpyHostToDevice,
                            st),
            "copy sampler units");
    }
    CKB(cudaMemsetAsync(c->acc, 0, sizeof(float) * (size_t)n * c->acc_stride, st), "clear acc");
    CKB(cudaMemsetAsync(c->hist, 0, c->hist_bytes, st), "clear hist");
    DevState init{};
    init.sigma = p->sigma0;
    CKB(cudaMemcpyAsync(c->st, &init, sizeof(DevState), cudaMemcpyHostToDevice, st), "init state");
    CKB(cudaMemsetAsync(c->scratch_i32, 0, sizeof(int32_t), st), "clear flag");
    CKB(launch_hash_build(c->row_ptr, c->col_idx, n, nnz, c->keys, c->bucket_mask, c->scratch_i32, st),
        "hash build");
    CKB(launch_init_positions(c->x, c->xb, n, d, (uint32_t)p->seed, (uint32_t)(p->seed >> 32), p->init_range, st),
        "init positions");
    int32_t hash_fail = 0;
    CKB(cudaMemcpyAsync(&hash_fail, c->scratch_i32, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "read flag");
    CKB(cudaStreamSynchronize(st), "create");
#undef CKB
    if (hash_fail) return bail(fail(GEMPE_E_INVALID_GRAPH, "edge hash set build failed"));
    c->sweep_grid = sweep_grid(d, p->hist_bins, c->sm_count);
    c->sampler_grid = sampler_grid(n, c->k, c->sm_count);
    c->update_grid = 1 + std::min<int>(c->sm_count * 2, (n + kUpdateThreads - 1) / kUpdateThreads);
    *out = c;
    return GEMPE_OK;
}

// Samples of the current epoch, when the buffer does not hold them yet
// (after create or set_state): drawn on the main stream.
cudaError_t launch_epoch_sampler(gempe_ctx* c, cudaStream_t s) {
    if (c->block) return launch_block_sampler(epoch_args(c), c->sampler_units, c->n_sampler_units, c->sm_count, s);
    return launch_sampler(epoch_args(c), c->sampler_grid, s);
}

gempe_status prime_samples(gempe_ctx* c) {
    if (c->primed || c->slots() == 0) return GEMPE_OK;
    CK(launch_epoch_sampler(c, c->stream), "sampler");
    c->primed = true;
    return GEMPE_OK;
}

// The sweep of the current epoch on the main stream and, forked onto the
// side stream, the sampler of the next epoch (it only needs the graph).
gempe_status enqueue_sweep(gempe_ctx* c) {
    gempe_status s = prime_samples(c);
    if (s != GEMPE_OK) return s;
    if (c->slots() > 0 && !c->sampled_ahead) {
        CK(cudaEventRecord(c->fork_ev, c->stream), "fork");
        CK(cudaStreamWaitEvent(c->side, c->fork_ev, 0), "fork");
        CK(launch_epoch_sampler(c, c->side), "sampler");
        CK(cudaEventRecord(c->join_ev, c->side), "join");
        c->sampled_ahead = true;
    }
    CK(launch_sweep(epoch_args(c), c->sweep_grid, c->stream), "sweep");
    if (c->tiles) CK(launch_tile_bf16(epoch_args(c), c->sm_count, c->stream), "tiles");
    return GEMPE_OK;
}

// The position update, then the join with the side stream.
gempe_status enqueue_update(gempe_ctx* c) {
    CK(launch_update(update_args(c), c->update_grid, c->stream), "update");
    if (c->sampled_ahead) {
        CK(cudaStreamWaitEvent(c->stream, c->join_ev, 0), "join");
        c->sampled_ahead = false;
    }
    return GEMPE_OK;
}

gempe_status read_status(gempe_ctx* c) {
    int32_t status = 0;
    CK(cudaMemcpyAsync(&status, &c->st->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "status");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (status != 0) {
        int32_t zero = 0;
        cudaMemcpyAsync(&c->st->status, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        return fail((gempe_status)status, "a position became non-finite during an update; it kept its old value");
    }
    return GEMPE_OK;
}

}  // namespace

GEMPE_API void gempe_default_params(gempe_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->mu = 1.5f;
    p->sigma0 = 1.0f;
    p->sigma_every = 1;
    p->neg_per_vertex = 5;
    p->max_retries = 32;
    p->symmetric_neg = 1;
    p->w_formula = 0;
    p->clamp_neg_d = 1;
    p->z_min = 1e-30f;
    p->init_range = 1.0f;
    p->seed = 0x6E6D7065ull;
    p->hist_bins = 1024;
    p->hist_max = 12.0f;
    p->precision = 0;
    p->block_partners = 0;
    p->tile_vertices = kBlockT;
}

GEMPE_API gempe_status gempe_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t d,
                                    const gempe_params* p, void* cuda_stream, gempe_ctx** out) {
    if (!out) return fail(GEMPE_E_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!row_ptr || (!col_idx && n > 0)) return fail(GEMPE_E_INVALID_ARG, "null CSR array");
    if (n < 2) return fail(GEMPE_E_INVALID_ARG, "n must be at least 2");
    static const int32_t empty = 0;
    return create_impl(row_ptr, col_idx ? col_idx : &empty, n, d, p, cuda_stream, out);
}

GEMPE_API gempe_status gempe_create_device(const int32_t* d_row_ptr, const int32_t* d_col_idx, int32_t n,
                                           int64_t nnz, int32_t d, const gempe_params* p, void* cuda_stream,
                                           gempe_ctx** out) {
    if (!out) return fail(GEMPE_E_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!d_row_ptr || (!d_col_idx && nnz > 0)) return fail(GEMPE_E_INVALID_ARG, "null CSR array");
    if (n < 2 || nnz < 0 || nnz > INT32_MAX) return fail(GEMPE_E_INVALID_ARG, "n or nnz out of range");
    std::vector<int32_t> rp((size_t)n + 1), ci((size_t)std::max<int64_t>(nnz, 1));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CK(cudaMemcpyAsync(rp.data(), d_row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s),
       "read row_ptr");
    if (nnz > 0)
        CK(cudaMemcpyAsync(ci.data(), d_col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost, s),
           "read col_idx");
    CK(cudaStreamSynchronize(s), "read CSR");
    if (rp[n] != nnz) return fail(GEMPE_E_INVALID_GRAPH, "row_ptr[n] != nnz");
    return create_impl(rp.data(), ci.data(), n, d, p, cuda_stream, out);
}

GEMPE_API void gempe_destroy(gempe_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->release_all();
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

GEMPE_API gempe_status gempe_step(gempe_ctx* c, int32_t iters) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    if (iters < 0) return fail(GEMPE_E_INVALID_ARG, "iters must be >= 0");
    if (iters == 0) return GEMPE_OK;
    if (c->swept) return fail(GEMPE_E_INVALID_ARG, "gempe_step after gempe_sweep: call gempe_update first");
    gempe_status ps = prime_samples(c);
    if (ps != GEMPE_OK) return ps;
    if (!c->graph_exec) {
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        gempe_status s = enqueue_sweep(c);
        if (s == GEMPE_OK) s = enqueue_update(c);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (s != GEMPE_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&c->graph_exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            c->graph_exec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
        c->graph = g;
    }
    for (int32_t it = 0; it < iters; ++it) CK(cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_sweep(gempe_ctx* c, int32_t* host_samples) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    // accumulators and histograms are zero between epochs (the update clears
    // them); only a repeated sweep has to clear its predecessor's sums
    if (c->swept && c->block)
        return fail(GEMPE_E_INVALID_ARG, "block sampling: call gempe_update before the next gempe_sweep");
    if (c->swept) {
        CK(cudaMemsetAsync(c->acc, 0, sizeof(float) * (size_t)c->n * c->acc_stride, c->stream), "clear acc");
        CK(cudaMemsetAsync(c->hist, 0, c->hist_bytes, c->stream), "clear hist");
    }
    std::vector<int32_t> bpart;
    std::vector<unsigned long long> bmask;
    if (host_samples && c->block) {
        // the sweep clears the masks it reads: take the record before it runs
        gempe_status ps = prime_samples(c);
        if (ps != GEMPE_OK) return ps;
        int32_t epoch = 0;
        CK(cudaMemcpyAsync(&epoch, &c->st->epoch, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "epoch");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        bpart.resize((size_t)c->n_tiles * kBlockP);
        bmask.resize((size_t)c->n);
        CK(cudaMemcpyAsync(bpart.data(), c->block_part + (size_t)(epoch & 1) * bpart.size(),
                           sizeof(int32_t) * bpart.size(), cudaMemcpyDeviceToHost, c->stream),
           "copy partners");
        CK(cudaMemcpyAsync(bmask.data(), c->block_mask + (size_t)(epoch & 1) * bmask.size(),
                           sizeof(unsigned long long) * bmask.size(), cudaMemcpyDeviceToHost, c->stream),
           "copy masks");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    gempe_status s = enqueue_sweep(c);
    if (s != GEMPE_OK) return s;
    c->swept = true;
    if (host_samples && c->slots() > 0) {
        int32_t epoch = 0;
        CK(cudaMemcpyAsync(&epoch, &c->st->epoch, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "epoch");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        if (c->block) {
            const std::vector<int32_t>& part = bpart;
            const std::vector<unsigned long long>& mask = bmask;
            for (int32_t i = 0; i < c->n; ++i)
                for (int q = 0; q < kBlockP; ++q)
                    host_samples[(size_t)i * kBlockP + q] =
                        ((mask[i] >> q) & 1ull) ? -1 : part[(size_t)(i / kBlockT) * kBlockP + q];
        } else {
            const size_t nk = (size_t)c->n * c->k;
            CK(cudaMemcpyAsync(host_samples, c->samples + (size_t)(epoch & 1) * nk, sizeof(int32_t) * nk,
                               cudaMemcpyDeviceToHost, c->stream),
               "copy samples");
            CK(cudaStreamSynchronize(c->stream), "synchronize");
        }
    }
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_update(gempe_ctx* c) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    gempe_status s = enqueue_update(c);
    if (s != GEMPE_OK) return s;
    c->swept = false;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_positions(gempe_ctx* c, float* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count != (size_t)c->n * c->d) return fail(GEMPE_E_INVALID_ARG, "count must be n*d");
    CK(cudaMemcpyAsync(host_out, c->x, sizeof(float) * count, cudaMemcpyDeviceToHost, c->stream), "copy x");
    return read_status(c);
}

GEMPE_API gempe_status gempe_positions_device(gempe_ctx* c, const float** d_view) {
    if (!c || !d_view) return fail(GEMPE_E_INVALID_ARG, "null argument");
    *d_view = c->x;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_set_positions(gempe_ctx* c, const float* host_x, size_t count) {
    if (!c || !host_x) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count != (size_t)c->n * c->d) return fail(GEMPE_E_INVALID_ARG, "count must be n*d");
    for (size_t q = 0; q < count; ++q)
        if (!std::isfinite(host_x[q])) return fail(GEMPE_E_INVALID_ARG, "positions must be finite");
    CK(cudaMemcpyAsync(c->x, host_x, sizeof(float) * count, cudaMemcpyHostToDevice, c->stream), "copy x");
    if (c->xb) CK(launch_to_bf16(c->x, c->xb, (long long)count, c->stream), "BF16 shadow");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_set_state(gempe_ctx* c, float sigma, int32_t epoch) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    if (!(sigma > 0.0f) || !std::isfinite(sigma) || epoch < 0)
        return fail(GEMPE_E_INVALID_ARG, "sigma must be positive and finite, epoch >= 0");
    if (c->swept) return fail(GEMPE_E_INVALID_ARG, "gempe_set_state after gempe_sweep: call gempe_update first");
    CK(cudaStreamSynchronize(c->side), "synchronize");
    DevState h{};
    CK(cudaMemcpyAsync(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "read state");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    h.sigma = sigma;
    h.epoch = epoch;
    h.sample_epoch = epoch;     // the buffer is refilled for this epoch before the next sweep
    h.sample_done = 0;
    c->primed = false;
    if (c->block)
        CK(cudaMemsetAsync(c->block_mask, 0, sizeof(unsigned long long) * 2 * (size_t)c->n, c->stream), "clear masks");
    CK(cudaMemcpyAsync(c->st, &h, sizeof(DevState), cudaMemcpyHostToDevice, c->stream), "write state");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_get_state(gempe_ctx* c, float* sigma, int32_t* epoch) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    DevState h{};
    CK(cudaMemcpyAsync(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "read state");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (sigma) *sigma = h.sigma;
    if (epoch) *epoch = h.epoch;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_accumulators(gempe_ctx* c, float* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count != (size_t)c->n * (c->d + 1)) return fail(GEMPE_E_INVALID_ARG, "count must be n*(d+1)");
    std::vector<float> tmp((size_t)c->n * c->acc_stride);
    CK(cudaMemcpyAsync(tmp.data(), c->acc, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, c->stream),
       "copy acc");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    for (int32_t i = 0; i < c->n; ++i)
        std::memcpy(host_out + (size_t)i * (c->d + 1), tmp.data() + (size_t)i * c->acc_stride,
                    sizeof(float) * (c->d + 1));
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_histograms(gempe_ctx* c, float* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count != 2 * (size_t)c->p.hist_bins) return fail(GEMPE_E_INVALID_ARG, "count must be 2*bins");
    const size_t B = (size_t)c->p.hist_bins;
    std::vector<unsigned char> raw(c->hist_bytes);
    CK(cudaMemcpyAsync(raw.data(), c->hist, c->hist_bytes, cudaMemcpyDeviceToHost, c->stream), "copy hist");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    const unsigned long long* hd = (const unsigned long long*)raw.data();
    const unsigned int* he = (const unsigned int*)(hd + B);
    const unsigned int* hc = he + B;
    const float* hx = (const float*)(hc + B);
    const int ks = c->slots();
    for (size_t b = 0; b < B; ++b) {
        host_out[b] = (float)he[b];
        host_out[B + b] = ks > 0 ? (float)(((double)(c->n - 1) * hc[b] - (double)hd[b]) / (2.0 * ks) + hx[b]) : 0.0f;
    }
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_sample(gempe_ctx* c, int32_t stream_id, int32_t* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (stream_id != 0 && stream_id != 1) return fail(GEMPE_E_INVALID_ARG, "stream_id must be 0 or 1");
    if (stream_id == 0 && c->block)
        return fail(GEMPE_E_INVALID_ARG, "block sampling: the epoch's samples come from gempe_sweep's record");
    if (count != (size_t)c->n * c->k) return fail(GEMPE_E_INVALID_ARG, "count must be n*k");
    if (c->k == 0) return GEMPE_OK;
    EpochArgs a = epoch_args(c);
    CK(launch_sample(a, stream_id ? 0x0E000000u : 0x0B000000u, c->scratch_i32, c->stream), "sample");
    CK(cudaMemcpyAsync(host_out, c->scratch_i32, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, c->stream),
       "copy samples");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_is_edge(gempe_ctx* c, const int32_t* host_pairs, size_t count, uint8_t* host_out) {
    if (!c || (count && (!host_pairs || !host_out))) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count == 0) return GEMPE_OK;
    for (size_t q = 0; q < 2 * count; ++q)
        if (host_pairs[q] < 0 || host_pairs[q] >= c->n) return fail(GEMPE_E_INVALID_ARG, "vertex out of range");
    int32_t* dpairs = nullptr;
    uint8_t* dout = nullptr;
    CK(cudaMallocAsync((void**)&dpairs, sizeof(int32_t) * 2 * count, c->stream), "alloc pairs");
    cudaError_t e = cudaMallocAsync((void**)&dout, count, c->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(dpairs, c->stream);
        return cuda_fail(e, "alloc out");
    }
    e = cudaMemcpyAsync(dpairs, host_pairs, sizeof(int32_t) * 2 * count, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_is_edge(c->keys, c->bucket_mask, dpairs, (int64_t)count, dout, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dout, count, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(dpairs, c->stream);
    cudaFreeAsync(dout, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "membership");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_loss(gempe_ctx* c, double* out_pe_bits, float* out_sigma) {
    if (!c || !out_pe_bits) return fail(GEMPE_E_INVALID_ARG, "null argument");
    const double zero = 0.0;
    CK(cudaMemcpyAsync(&c->st->loss_sum, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream), "clear loss");
    CK(launch_loss(epoch_args(c), c->stream), "loss");
    DevState h{};
    CK(cudaMemcpyAsync(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "read loss");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    const double N = 0.5 * (double)c->n * ((double)c->n - 1.0);
    *out_pe_bits = h.loss_sum / N;
    if (out_sigma) *out_sigma = h.sigma;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_fit_sigma(const float* host_hist, int32_t bins, float hist_max, float mu,
                                       void* cuda_stream, float* out_sigma) {
    if (!host_hist || !out_sigma) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (bins < 16 || bins > 4096 || !(hist_max > 0.0f) || !std::isfinite(mu))
        return fail(GEMPE_E_INVALID_ARG, "bins in [16,4096], hist_max > 0, mu finite");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CK(ensure_mills_table(), "Mills table");
    float* dh = nullptr;
    CK(cudaMallocAsync((void**)&dh, sizeof(float) * (2 * (size_t)bins + 1), s), "alloc");
    cudaError_t e = cudaMemcpyAsync(dh, host_hist, sizeof(float) * 2 * (size_t)bins, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_fit_sigma(dh, bins, hist_max, mu, dh + 2 * bins, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_sigma, dh + 2 * bins, sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dh, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "fit sigma");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_stats(gempe_ctx* c, gempe_stats_t* out) {
    if (!c || !out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    DevState h{};
    CK(cudaMemcpyAsync(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "read state");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    out->epoch = h.epoch;
    out->sigma = h.sigma;
    out->accepted = h.accepted;
    out->rejected = h.rejected;
    out->exhausted = h.exhausted;
    out->draws = h.draws;
    out->used = h.used;
    out->n_edges = c->nnz / 2;
    out->n = c->n;
    out->d = c->d;
    out->k = c->k;
    out->sigma_iters = h.sigma_iters;
    return GEMPE_OK;
}

GEMPE_API const char* gempe_last_error(void) { return g_last_error.c_str(); }

namespace gempe {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace gempe
