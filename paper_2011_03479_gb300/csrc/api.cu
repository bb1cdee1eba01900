// Host implementation of the single-graph C ABI declared in include/gempe.h:
// a context is a pack of one graph (pack.cuh) plus its stream and the
// captured epoch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "engine.cuh"
#include "gempe.h"
#include "pack.cuh"

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
    std::unique_ptr<Pack> pk;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int32_t n = 0;
    bool time_kernels = false;   // gempe_kernel_times: record events around directly enqueued kernels
    bool sweep_timed = false;    // the pending sweep recorded its events
    bool timed = false;          // the events hold a whole sweep + update

    ~gempe_ctx() {
        if (stream) cudaStreamSynchronize(stream);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        pk.reset();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

gempe_status create_impl(const int32_t* rp_host, const int32_t* ci_host, int32_t n, int32_t d,
                         const gempe_params* p, void* stream, gempe_ctx** out, int32_t own_lo = 0,
                         int32_t own_hi = -1) {
    gempe_status s = check_params(p, d);
    if (s != GEMPE_OK) return s;
    if (n < 2) return fail(GEMPE_E_INVALID_ARG, "n must be at least 2");
    if (own_hi >= 0) {
        if (own_lo < 0 || own_lo >= own_hi || own_hi > n)
            return fail(GEMPE_E_INVALID_ARG, "shard range must satisfy 0 <= v_begin < v_end <= n");
        if (p->block_partners && (own_lo % kBlockT != 0 || (own_hi % kBlockT != 0 && own_hi != n)))
            return fail(GEMPE_E_INVALID_ARG, "block sampling: a shard range starts and ends on a tile of 128 vertices");
    }
    if (rp_host[n] < 0) return fail(GEMPE_E_INVALID_GRAPH, "row_ptr[n] negative");
    // rows sorted, in range and loop-free on the host, before any device
    // work; the symmetry is checked on the device against the edge set
    s = validate_csr(rp_host, ci_host, n, 0, false);
    if (s != GEMPE_OK) return s;
    std::unique_ptr<gempe_ctx> c(new gempe_ctx());
    c->n = n;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->own_stream = true;
    }
    c->pk.reset(new Pack());
    c->pk->own_lo = own_lo;
    c->pk->own_hi = own_hi;
    std::vector<GraphInput> g(1);
    g[0].row_ptr = rp_host;
    g[0].col_idx = ci_host;
    g[0].n = n;
    g[0].key = p->seed;
    s = c->pk->build(g, d, *p, c->stream, false);
    if (s != GEMPE_OK) return s;
    if (p->autotune) {
        s = c->pk->autotune();
        if (s != GEMPE_OK) return s;
    }
    *out = c.release();
    return GEMPE_OK;
}

GraphState read_graph_state(gempe_ctx* c, gempe_status* rc) {
    GraphState h{};
    cudaError_t e = cudaMemcpyAsync(&h, c->pk->gst, sizeof(GraphState), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    *rc = e == cudaSuccess ? GEMPE_OK : cuda_fail(e, "read state");
    return h;
}

}  // namespace

GEMPE_API gempe_status gempe_validate_csr(const int32_t* row_ptr, const int32_t* col_idx, int32_t n) {
    if (!row_ptr || n < 0) return fail(GEMPE_E_INVALID_ARG, "null row_ptr or negative n");
    if (!col_idx && n > 0 && row_ptr[n] > 0) return fail(GEMPE_E_INVALID_ARG, "null col_idx");
    static const int32_t empty = 0;
    return validate_csr(row_ptr, col_idx ? col_idx : &empty, n);
}

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
    p->autotune = 0;
}

GEMPE_API gempe_status gempe_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t d,
                                    const gempe_params* p, void* cuda_stream, gempe_ctx** out) {
    if (!out) return fail(GEMPE_E_INVALID_ARG, "out is null");
    *out = nullptr;
    if (n < 2) return fail(GEMPE_E_INVALID_ARG, "n must be at least 2");
    if (!row_ptr || (!col_idx && row_ptr[n] > 0)) return fail(GEMPE_E_INVALID_ARG, "null CSR array");
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

GEMPE_API void gempe_destroy(gempe_ctx* c) { delete c; }

GEMPE_API gempe_status gempe_step(gempe_ctx* c, int32_t iters) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    if (iters < 0) return fail(GEMPE_E_INVALID_ARG, "iters must be >= 0");
    if (iters == 0) return GEMPE_OK;
    Pack& pk = *c->pk;
    if (pk.swept) return fail(GEMPE_E_INVALID_ARG, "gempe_step after gempe_sweep: call gempe_update first");
    gempe_status ps = pk.prime();
    if (ps != GEMPE_OK) return ps;
    if (!c->graph_exec) {
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        gempe_status s = pk.enqueue_sweep();
        if (s == GEMPE_OK) s = pk.enqueue_update();
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
    Pack& pk = *c->pk;
    // accumulators and histograms are zero between epochs (the update clears
    // them); only a repeated sweep has to clear its predecessor's sums
    if (pk.swept && pk.block)
        return fail(GEMPE_E_INVALID_ARG, "block sampling: call gempe_update before the next gempe_sweep");
    if (pk.swept) {
        CK(cudaMemsetAsync(pk.acc, 0, sizeof(float) * (size_t)pk.rows * pk.acc_stride, c->stream), "clear acc");
        CK(cudaMemsetAsync(pk.hist, 0, pk.hist_bytes, c->stream), "clear hist");
    }
    const int32_t n = c->n;
    std::vector<int32_t> bpart;
    std::vector<unsigned long long> bmask;
    if (host_samples && pk.block) {
        // the sweep clears the masks it reads: take the record before it runs
        gempe_status ps = pk.prime();
        if (ps != GEMPE_OK) return ps;
        int32_t epoch = 0;
        CK(cudaMemcpyAsync(&epoch, &pk.gst->epoch, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "epoch");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        bpart.resize((size_t)pk.n_tiles * kBlockP);
        bmask.resize((size_t)n);
        CK(cudaMemcpyAsync(bpart.data(), pk.block_part + (size_t)(epoch & 1) * bpart.size(),
                           sizeof(int32_t) * bpart.size(), cudaMemcpyDeviceToHost, c->stream),
           "copy partners");
        CK(cudaMemcpyAsync(bmask.data(), pk.block_mask + (size_t)(epoch & 1) * pk.rows,
                           sizeof(unsigned long long) * bmask.size(), cudaMemcpyDeviceToHost, c->stream),
           "copy masks");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    }
    pk.time_kernels = c->time_kernels;
    gempe_status s = pk.enqueue_sweep();
    pk.time_kernels = false;
    if (s != GEMPE_OK) return s;
    c->sweep_timed = c->time_kernels;
    pk.swept = true;
    if (host_samples && pk.per_slot) {
        int32_t epoch = 0;
        CK(cudaMemcpyAsync(&epoch, &pk.gst->epoch, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "epoch");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        if (pk.slots > 0)
            CK(cudaMemcpyAsync(host_samples, pk.samples + (size_t)(epoch & 1) * pk.slots,
                               sizeof(int32_t) * (size_t)pk.slots, cudaMemcpyDeviceToHost, c->stream),
               "copy samples");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
    } else if (host_samples && pk.slots_per_vertex() > 0) {
        int32_t epoch = 0;
        CK(cudaMemcpyAsync(&epoch, &pk.gst->epoch, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "epoch");
        CK(cudaStreamSynchronize(c->stream), "synchronize");
        if (pk.block) {
            for (int32_t i = 0; i < n; ++i)
                for (int q = 0; q < kBlockP; ++q)
                    host_samples[(size_t)i * kBlockP + q] =
                        ((bmask[i] >> q) & 1ull) ? -1 : bpart[(size_t)(i / kBlockT) * kBlockP + q];
        } else {
            const size_t nk = (size_t)n * pk.k;
            CK(cudaMemcpyAsync(host_samples, pk.samples + (size_t)(epoch & 1) * pk.rows * pk.k, sizeof(int32_t) * nk,
                               cudaMemcpyDeviceToHost, c->stream),
               "copy samples");
            CK(cudaStreamSynchronize(c->stream), "synchronize");
        }
    }
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_update(gempe_ctx* c) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    Pack& pk = *c->pk;
    const bool timed = c->sweep_timed && pk.swept;
    pk.time_kernels = timed;
    gempe_status s = pk.enqueue_update();
    pk.time_kernels = false;
    if (s != GEMPE_OK) return s;
    c->timed = timed;
    c->sweep_timed = false;
    pk.swept = false;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_kernel_times(gempe_ctx* c, int32_t enable, float* out_ms3) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    if (enable != 0 && enable != 1) return fail(GEMPE_E_INVALID_ARG, "enable must be 0 or 1");
    Pack& pk = *c->pk;
    if (out_ms3) {
        out_ms3[0] = out_ms3[1] = out_ms3[2] = 0.0f;
        if (c->timed) {
            CK(cudaEventSynchronize(pk.tev[5]), "synchronize");
            CK(cudaEventElapsedTime(&out_ms3[0], pk.tev[0], pk.tev[1]), "elapsed");
            if (pk.tiles) {
                CK(cudaEventElapsedTime(&out_ms3[1], pk.tev[2], pk.tev[3]), "elapsed");
                CK(cudaEventElapsedTime(&out_ms3[2], pk.tev[4], pk.tev[5]), "elapsed");
            } else {   // no tile kernel: the gap between its events goes to the update's window
                CK(cudaEventElapsedTime(&out_ms3[2], pk.tev[1], pk.tev[5]), "elapsed");
            }
        }
    }
    if (enable && !pk.tev[0])
        for (cudaEvent_t& e : pk.tev) CK(cudaEventCreate(&e), "cudaEventCreate");
    c->time_kernels = enable != 0;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_positions(gempe_ctx* c, float* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count != (size_t)c->n * c->pk->d) return fail(GEMPE_E_INVALID_ARG, "count must be n*d");
    CK(cudaMemcpyAsync(host_out, c->pk->x, sizeof(float) * count, cudaMemcpyDeviceToHost, c->stream), "copy x");
    return c->pk->read_status();
}

GEMPE_API gempe_status gempe_positions_device(gempe_ctx* c, const float** d_view) {
    if (!c || !d_view) return fail(GEMPE_E_INVALID_ARG, "null argument");
    *d_view = c->pk->x;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_set_positions(gempe_ctx* c, const float* host_x, size_t count) {
    if (!c || !host_x) return fail(GEMPE_E_INVALID_ARG, "null argument");
    Pack& pk = *c->pk;
    if (count != (size_t)c->n * pk.d) return fail(GEMPE_E_INVALID_ARG, "count must be n*d");
    for (size_t q = 0; q < count; ++q)
        if (!std::isfinite(host_x[q])) return fail(GEMPE_E_INVALID_ARG, "positions must be finite");
    CK(cudaMemcpyAsync(pk.x, host_x, sizeof(float) * count, cudaMemcpyHostToDevice, c->stream), "copy x");
    if (pk.xb) CK(launch_to_bf16(pk.x, pk.xb, (long long)count, c->stream), "BF16 shadow");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_set_state(gempe_ctx* c, float sigma, int32_t epoch) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    if (!(sigma > 0.0f) || !std::isfinite(sigma) || epoch < 0)
        return fail(GEMPE_E_INVALID_ARG, "sigma must be positive and finite, epoch >= 0");
    Pack& pk = *c->pk;
    if (pk.swept) return fail(GEMPE_E_INVALID_ARG, "gempe_set_state after gempe_sweep: call gempe_update first");
    CK(cudaStreamSynchronize(pk.side), "synchronize");
    gempe_status rc;
    GraphState h = read_graph_state(c, &rc);
    if (rc != GEMPE_OK) return rc;
    h.sigma = sigma;
    h.epoch = epoch;
    h.sample_epoch = epoch;     // the buffer is refilled for this epoch before the next sweep
    pk.primed = false;
    if (pk.block)
        CK(cudaMemsetAsync(pk.block_mask, 0, sizeof(unsigned long long) * 2 * (size_t)pk.rows, c->stream),
           "clear masks");
    CK(cudaMemsetAsync(&pk.ps->sample_done, 0, sizeof(unsigned int), c->stream), "clear sampler count");
    CK(cudaMemcpyAsync(pk.gst, &h, sizeof(GraphState), cudaMemcpyHostToDevice, c->stream), "write state");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_get_state(gempe_ctx* c, float* sigma, int32_t* epoch) {
    if (!c) return fail(GEMPE_E_INVALID_ARG, "ctx is null");
    gempe_status rc;
    GraphState h = read_graph_state(c, &rc);
    if (rc != GEMPE_OK) return rc;
    if (sigma) *sigma = h.sigma;
    if (epoch) *epoch = h.epoch;
    return GEMPE_OK;
}

namespace {

// Checkpoint layout: this header, then the FP32 positions [n][d].  Plain
// fixed-width fields (8-byte aligned, no padding), written and read with
// memcpy.
struct CheckpointHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t n, d;
    int64_t nnz;
    uint64_t seed;
    int32_t k, max_retries, sampling, block_partners;
    int32_t tile_vertices, membership, bytemap_log2, rename_every;
    float sigma;
    int32_t epoch, sigma_iters, reserved;
    uint64_t accepted, rejected, exhausted, draws, used, false_pos;
    // the parameters of the run's arithmetic (version 2)
    float mu, hist_max, z_min;
    int32_t hist_bins, sigma_every, sigma_source, precision;
    int32_t symmetric_neg, w_formula, clamp_neg_d, rng, reserved2;
};
static_assert(sizeof(CheckpointHeader) == 184, "checkpoint header layout");

constexpr char kCheckpointMagic[8] = {'G', 'E', 'M', 'P', 'E', 'C', 'K', '\x01'};
constexpr uint32_t kCheckpointVersion = 2;

size_t checkpoint_bytes(const gempe_ctx* c) {
    return sizeof(CheckpointHeader) + sizeof(float) * (size_t)c->n * c->pk->d;
}

// The checkpoint belongs to a graph of this size and to the parameters that
// key this context's draws.
gempe_status checkpoint_matches(const CheckpointHeader& h, const gempe_ctx* c) {
    const Pack& pk = *c->pk;
    const gempe_params& p = pk.p;
    if (h.n != c->n || h.d != pk.d || h.nnz != pk.nnz[0])
        return fail(GEMPE_E_INVALID_ARG, "checkpoint of another graph: n, d or nnz differ");
    if (h.seed != p.seed || h.k != p.neg_per_vertex || h.max_retries != p.max_retries || h.sampling != p.sampling ||
        h.block_partners != p.block_partners || h.tile_vertices != p.tile_vertices || h.membership != p.membership ||
        h.rng != p.rng)
        return fail(GEMPE_E_INVALID_ARG,
                    "checkpoint of other sampling parameters: seed, neg_per_vertex, max_retries, sampling, "
                    "block_partners, tile_vertices, membership or rng differ");
    if (p.membership == 1 && (h.bytemap_log2 != p.bytemap_log2 || h.rename_every != p.rename_every))
        return fail(GEMPE_E_INVALID_ARG, "checkpoint of another byte map: bytemap_log2 or rename_every differ");
    if (h.mu != p.mu || h.hist_max != p.hist_max || h.z_min != p.z_min || h.hist_bins != p.hist_bins ||
        h.sigma_every != p.sigma_every || h.sigma_source != p.sigma_source || h.precision != p.precision ||
        h.symmetric_neg != p.symmetric_neg || h.w_formula != p.w_formula || h.clamp_neg_d != p.clamp_neg_d)
        return fail(GEMPE_E_INVALID_ARG,
                    "checkpoint of another run: mu, hist_max, z_min, hist_bins, sigma_every, sigma_source, "
                    "precision, symmetric_neg, w_formula or clamp_neg_d differ");
    return GEMPE_OK;
}

}  // namespace

GEMPE_API gempe_status gempe_save(gempe_ctx* c, void* buf, size_t* len) {
    if (!c || !len) return fail(GEMPE_E_INVALID_ARG, "null argument");
    const size_t need = checkpoint_bytes(c);
    if (!buf) {
        *len = need;
        return GEMPE_OK;
    }
    if (*len < need) {
        *len = need;
        return fail(GEMPE_E_INVALID_ARG, "checkpoint buffer too small (*len now holds the size needed)");
    }
    Pack& pk = *c->pk;
    if (pk.swept) return fail(GEMPE_E_INVALID_ARG, "gempe_save after gempe_sweep: call gempe_update first");
    CK(cudaStreamSynchronize(pk.side), "synchronize");
    gempe_status rc;
    const GraphState g = read_graph_state(c, &rc);   // after the context's queued work
    if (rc != GEMPE_OK) return rc;
    unsigned char* out = static_cast<unsigned char*>(buf);
    CK(cudaMemcpyAsync(out + sizeof(CheckpointHeader), pk.x, sizeof(float) * (size_t)c->n * pk.d,
                       cudaMemcpyDeviceToHost, c->stream),
       "copy x");
    rc = pk.read_status();   // synchronises
    if (rc != GEMPE_OK) return rc;
    CheckpointHeader h{};
    std::memcpy(h.magic, kCheckpointMagic, sizeof(h.magic));
    h.version = kCheckpointVersion;
    h.header_bytes = (uint32_t)sizeof(CheckpointHeader);
    h.n = c->n;
    h.d = pk.d;
    h.nnz = pk.nnz[0];
    h.seed = pk.p.seed;
    h.k = pk.p.neg_per_vertex;
    h.max_retries = pk.p.max_retries;
    h.sampling = pk.p.sampling;
    h.block_partners = pk.p.block_partners;
    h.tile_vertices = pk.p.tile_vertices;
    h.membership = pk.p.membership;
    h.bytemap_log2 = pk.p.bytemap_log2;
    h.rename_every = pk.p.rename_every;
    h.sigma = g.sigma;
    h.epoch = g.epoch;
    h.sigma_iters = g.sigma_iters;
    h.accepted = g.accepted;
    h.rejected = g.rejected;
    h.exhausted = g.exhausted;
    h.draws = g.draws;
    h.used = g.used;
    h.false_pos = g.false_pos;
    h.mu = pk.p.mu;
    h.hist_max = pk.p.hist_max;
    h.z_min = pk.p.z_min;
    h.hist_bins = pk.p.hist_bins;
    h.sigma_every = pk.p.sigma_every;
    h.sigma_source = pk.p.sigma_source;
    h.precision = pk.p.precision;
    h.symmetric_neg = pk.p.symmetric_neg;
    h.w_formula = pk.p.w_formula;
    h.clamp_neg_d = pk.p.clamp_neg_d;
    h.rng = pk.p.rng;
    std::memcpy(out, &h, sizeof(h));
    *len = need;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_load(gempe_ctx* c, const void* buf, size_t len) {
    if (!c || !buf) return fail(GEMPE_E_INVALID_ARG, "null argument");
    CheckpointHeader h;
    if (len < sizeof(h)) return fail(GEMPE_E_INVALID_ARG, "not a GEMPE checkpoint: too short");
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kCheckpointMagic, sizeof(h.magic)) != 0 || h.version != kCheckpointVersion ||
        h.header_bytes != sizeof(CheckpointHeader))
        return fail(GEMPE_E_INVALID_ARG, "not a GEMPE checkpoint of this format");
    gempe_status s = checkpoint_matches(h, c);
    if (s != GEMPE_OK) return s;
    if (len < checkpoint_bytes(c)) return fail(GEMPE_E_INVALID_ARG, "checkpoint truncated");
    if (!(h.sigma > 0.0f) || !std::isfinite(h.sigma) || h.epoch < 0)
        return fail(GEMPE_E_INVALID_ARG, "checkpoint holds an invalid sigma or epoch");
    Pack& pk = *c->pk;
    if (pk.swept) return fail(GEMPE_E_INVALID_ARG, "gempe_load after gempe_sweep: call gempe_update first");
    const size_t count = (size_t)c->n * pk.d;
    std::vector<float> x(count);
    std::memcpy(x.data(), static_cast<const unsigned char*>(buf) + sizeof(h), sizeof(float) * count);
    for (size_t q = 0; q < count; ++q)
        if (!std::isfinite(x[q])) return fail(GEMPE_E_INVALID_ARG, "checkpoint holds non-finite positions");
    // positions and their BF16 shadow, as gempe_set_positions
    CK(cudaStreamSynchronize(pk.side), "synchronize");
    CK(cudaMemcpyAsync(pk.x, x.data(), sizeof(float) * count, cudaMemcpyHostToDevice, c->stream), "copy x");
    if (pk.xb) CK(launch_to_bf16(pk.x, pk.xb, (long long)count, c->stream), "BF16 shadow");
    // sigma and the epoch, as gempe_set_state
    gempe_status rc;
    GraphState g = read_graph_state(c, &rc);   // synchronises
    if (rc != GEMPE_OK) return rc;
    g.sigma = h.sigma;
    g.epoch = h.epoch;
    g.sample_epoch = h.epoch;
    g.sigma_iters = h.sigma_iters;
    pk.primed = false;
    if (pk.block)
        CK(cudaMemsetAsync(pk.block_mask, 0, sizeof(unsigned long long) * 2 * (size_t)pk.rows, c->stream),
           "clear masks");
    CK(cudaMemsetAsync(&pk.ps->sample_done, 0, sizeof(unsigned int), c->stream), "clear sampler count");
    CK(cudaMemcpyAsync(pk.gst, &g, sizeof(GraphState), cudaMemcpyHostToDevice, c->stream), "write state");
    // the saved context had drawn the samples of its epoch already (the
    // sampler runs one epoch ahead); draw them again, then restore the
    // statistics as saved, which count those draws once
    s = pk.prime();
    if (s != GEMPE_OK) return s;
    g = read_graph_state(c, &rc);   // synchronises
    if (rc != GEMPE_OK) return rc;
    g.accepted = h.accepted;
    g.rejected = h.rejected;
    g.exhausted = h.exhausted;
    g.draws = h.draws;
    g.used = h.used;
    g.false_pos = h.false_pos;
    CK(cudaMemcpyAsync(pk.gst, &g, sizeof(GraphState), cudaMemcpyHostToDevice, c->stream), "write state");
    return pk.read_status();   // synchronises
}

GEMPE_API gempe_status gempe_accumulators(gempe_ctx* c, float* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    Pack& pk = *c->pk;
    if (count != (size_t)c->n * (pk.d + 1)) return fail(GEMPE_E_INVALID_ARG, "count must be n*(d+1)");
    std::vector<float> tmp((size_t)c->n * pk.acc_stride);
    CK(cudaMemcpyAsync(tmp.data(), pk.acc, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, c->stream),
       "copy acc");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    for (int32_t i = 0; i < c->n; ++i)
        std::memcpy(host_out + (size_t)i * (pk.d + 1), tmp.data() + (size_t)i * pk.acc_stride,
                    sizeof(float) * (pk.d + 1));
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_histograms(gempe_ctx* c, float* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    Pack& pk = *c->pk;
    if (count != 2 * (size_t)pk.bins) return fail(GEMPE_E_INVALID_ARG, "count must be 2*bins");
    const size_t B = (size_t)pk.bins;
    std::vector<unsigned char> raw(pk.hist_bytes);
    CK(cudaMemcpyAsync(raw.data(), pk.hist, pk.hist_bytes, cudaMemcpyDeviceToHost, c->stream), "copy hist");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    // one graph: hist_d [B] u64, hist_e [B] u32, hist_c [B] u32, hist_x [B] f32
    const unsigned long long* hd = (const unsigned long long*)raw.data();
    const unsigned int* he = (const unsigned int*)(hd + B);
    const unsigned int* hc = he + B;
    const float* hx = (const float*)(hc + B);
    const int ks = pk.per_slot ? 0 : pk.slots_per_vertex();   // per-slot weights are all in hist_x
    for (size_t b = 0; b < B; ++b) {
        host_out[b] = (float)he[b];
        host_out[B + b] = ks > 0 ? (float)(((double)(c->n - 1) * hc[b] - (double)hd[b]) / (2.0 * ks) + hx[b])
                                 : (pk.per_slot ? hx[b] : 0.0f);
    }
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_sample(gempe_ctx* c, int32_t stream_id, int32_t* host_out, size_t count) {
    if (!c || !host_out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    Pack& pk = *c->pk;
    if (stream_id < 0 || stream_id > 2) return fail(GEMPE_E_INVALID_ARG, "stream_id must be 0, 1 or 2");
    if (stream_id == 0 && (pk.block || pk.per_slot))
        return fail(GEMPE_E_INVALID_ARG, "block or per-slot sampling: the epoch's samples come from gempe_sweep's record");
    if (count != (size_t)c->n * pk.k) return fail(GEMPE_E_INVALID_ARG, "count must be n*k");
    if (pk.k == 0) return GEMPE_OK;
    const uint32_t tags[3] = {0x0B000000u, 0x0E000000u, 0x0F000000u};   // epoch, loss, histogram pass
    CK(launch_sample(pk.args(), tags[stream_id], pk.scratch, c->stream), "sample");
    CK(cudaMemcpyAsync(host_out, pk.scratch, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, c->stream),
       "copy samples");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_is_edge(gempe_ctx* c, const int32_t* host_pairs, size_t count, uint8_t* host_out) {
    if (!c || (count && (!host_pairs || !host_out))) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (count == 0) return GEMPE_OK;
    for (size_t q = 0; q < 2 * count; ++q)
        if (host_pairs[q] < 0 || host_pairs[q] >= c->n) return fail(GEMPE_E_INVALID_ARG, "vertex out of range");
    Pack& pk = *c->pk;
    int32_t* dpairs = nullptr;
    uint8_t* dout = nullptr;
    CK(cudaMallocAsync((void**)&dpairs, sizeof(int32_t) * 2 * count, c->stream), "alloc pairs");
    cudaError_t e = cudaMallocAsync((void**)&dout, count, c->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(dpairs, c->stream);
        return cuda_fail(e, "alloc out");
    }
    e = cudaMemcpyAsync(dpairs, host_pairs, sizeof(int32_t) * 2 * count, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_is_edge(pk.keys, pk.narrow_keys ? 1 : 0, pk.info[0].key_off, pk.info[0].bucket_mask, dpairs,
                           (int64_t)count, dout, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dout, count, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(dpairs, c->stream);
    cudaFreeAsync(dout, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "membership");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_loss(gempe_ctx* c, double* out_pe_bits, float* out_sigma) {
    if (!c || !out_pe_bits) return fail(GEMPE_E_INVALID_ARG, "null argument");
    Pack& pk = *c->pk;
    CK(cudaMemsetAsync(&pk.gst->loss_sum, 0, sizeof(double), c->stream), "clear loss");
    CK(launch_loss(pk.args(), c->stream), "loss");
    gempe_status rc;
    GraphState h = read_graph_state(c, &rc);
    if (rc != GEMPE_OK) return rc;
    const double N = 0.5 * (double)c->n * ((double)c->n - 1.0);
    *out_pe_bits = h.loss_sum / N;
    if (out_sigma) *out_sigma = h.sigma;
    return GEMPE_OK;
}

namespace {
// {sum dl, F, F'} of the exact Eq. 2 at sigma (one all-pairs pass + the edge pass).
gempe_status exact_eval(gempe_ctx* c, double* dbuf, float sigma, double out[3]) {
    Pack& pk = *c->pk;
    CK(launch_exact_pe(pk.row_ptr, pk.col_idx, pk.x, c->n, pk.d, pk.p.mu, sigma, pk.mills, dbuf, pk.sm_count,
                       c->stream),
       "exact loss");
    CK(cudaMemcpyAsync(out, dbuf, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read sums");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return GEMPE_OK;
}
}  // namespace

GEMPE_API gempe_status gempe_loss_exact(gempe_ctx* c, int32_t fit_sigma, double* out_pe_bits, float* out_sigma) {
    if (!c || !out_pe_bits) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (fit_sigma != 0 && fit_sigma != 1) return fail(GEMPE_E_INVALID_ARG, "fit_sigma must be 0 or 1");
    gempe_status rc;
    const GraphState st = read_graph_state(c, &rc);
    if (rc != GEMPE_OK) return rc;
    double* dbuf = nullptr;
    CK(cudaMallocAsync((void**)&dbuf, 3 * sizeof(double), c->stream), "alloc");
    const double N = 0.5 * (double)c->n * ((double)c->n - 1.0);
    double v[3];
    double t = std::log((double)st.sigma);
    rc = exact_eval(c, dbuf, (float)std::exp(t), v);
    if (rc == GEMPE_OK && fit_sigma) {
        // zero of F (the sign of dPE/dsigma) in t = ln sigma on [ln 1e-3, ln 1e3]:
        // bracket by steps away from the current slope, then Newton steps
        // safeguarded by bisection
        const double t_min = std::log(1e-3), t_max = std::log(1e3);
        double lo = t_min, hi = t_max, f_t = v[1];
        double vt[3] = {v[0], v[1], v[2]};
        bool bracket = false;
        double a = t, fa = f_t, step = 0.25;
        for (int q = 0; q < 40 && rc == GEMPE_OK; ++q) {
            const double b = std::min(t_max, std::max(t_min, a + (fa > 0 ? -step : step)));
            double vb[3];
            rc = exact_eval(c, dbuf, (float)std::exp(b), vb);
            if (rc != GEMPE_OK) break;
            if ((vb[1] > 0) != (fa > 0)) {
                lo = std::min(a, b);
                hi = std::max(a, b);
                // keep the evaluated point closest to the root as the Newton start
                t = b;
                std::memcpy(vt, vb, sizeof(vt));
                bracket = true;
                break;
            }
            if (b == t_min || b == t_max) {   // no sign change: the end with the lower entropy
                t = b;
                std::memcpy(vt, vb, sizeof(vt));
                break;
            }
            a = b;
            fa = vb[1];
            step *= 2.0;
        }
        // F > 0 at hi's side and < 0 at lo's side (dPE/dsigma rises through the minimum)
        for (int q = 0; bracket && q < 60 && rc == GEMPE_OK; ++q) {
            double tn = (vt[2] > 0.0) ? t - vt[1] / vt[2] : 0.5 * (lo + hi);
            if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
            const bool done = std::fabs(tn - t) < 1e-7 || (hi - lo) < 1e-7;
            rc = exact_eval(c, dbuf, (float)std::exp(tn), vt);
            t = tn;
            if (rc != GEMPE_OK || done) break;
            if (vt[1] > 0.0) hi = t; else lo = t;
        }
        std::memcpy(v, vt, sizeof(v));
    }
    cudaFreeAsync(dbuf, c->stream);
    if (rc != GEMPE_OK) return rc;
    *out_pe_bits = v[0] / N;
    if (out_sigma) *out_sigma = (float)std::exp(t);
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

GEMPE_API gempe_status gempe_set_shape(gempe_ctx* c, const int32_t* shape5) {
    if (!c || !shape5) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (c->pk->swept) return fail(GEMPE_E_INVALID_ARG, "gempe_set_shape after gempe_sweep: call gempe_update first");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    PackShape sh;
    sh.unit_pairs = shape5[0];
    sh.edge_chunk = shape5[1];
    sh.lanes = shape5[2];
    sh.blocks_per_sm = shape5[3];
    sh.kernel = shape5[4];
    gempe_status s = c->pk->set_shape(sh);
    if (s != GEMPE_OK) return s;
    // the captured epoch holds the old work list and grid
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_get_shape(gempe_ctx* c, int32_t* out6) {
    if (!c || !out6) return fail(GEMPE_E_INVALID_ARG, "null argument");
    const PackShape& sh = c->pk->shape;
    out6[0] = sh.unit_pairs;
    out6[1] = sh.edge_chunk;
    out6[2] = sh.lanes ? sh.lanes : (c->pk->d <= kPackedMaxDim ? 1 : c->pk->d / 8);
    out6[3] = sh.blocks_per_sm;
    out6[4] = sh.kernel;
    out6[5] = c->pk->sweep_grid;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_stats(gempe_ctx* c, gempe_stats_t* out) {
    if (!c || !out) return fail(GEMPE_E_INVALID_ARG, "null argument");
    gempe_status rc;
    GraphState h = read_graph_state(c, &rc);
    if (rc != GEMPE_OK) return rc;
    const Pack& pk = *c->pk;
    out->epoch = h.epoch;
    out->sigma = h.sigma;
    out->accepted = h.accepted;
    out->rejected = h.rejected;
    out->exhausted = h.exhausted;
    out->draws = h.draws;
    out->used = h.used;
    out->n_edges = pk.nnz[0] / 2;
    out->n = c->n;
    out->d = pk.d;
    out->k = pk.k;
    out->sigma_iters = h.sigma_iters;
    out->false_pos = h.false_pos;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_create_shard(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t d,
                                          int32_t v_begin, int32_t v_end, const gempe_params* p, void* cuda_stream,
                                          gempe_ctx** out) {
    if (!out) return fail(GEMPE_E_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!row_ptr || !p) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (n < 2) return fail(GEMPE_E_INVALID_ARG, "n must be at least 2");
    if (!col_idx && row_ptr[n] > 0) return fail(GEMPE_E_INVALID_ARG, "null col_idx");
    static const int32_t empty = 0;
    if (v_begin < 0 || v_end < 0) return fail(GEMPE_E_INVALID_ARG, "shard range must satisfy 0 <= v_begin < v_end <= n");
    return create_impl(row_ptr, col_idx ? col_idx : &empty, n, d, p, cuda_stream, out, v_begin, v_end);
}

GEMPE_API gempe_status gempe_shard_layout(gempe_ctx* c, int64_t* out4) {
    if (!c || !out4) return fail(GEMPE_E_INVALID_ARG, "null argument");
    const Pack& pk = *c->pk;
    out4[0] = (int64_t)c->n * pk.acc_stride;
    out4[1] = pk.acc_stride;
    out4[2] = pk.bins;
    out4[3] = (int64_t)c->n * pk.d;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_shard_copy(gempe_ctx* c, int32_t what, int32_t direction, void* device_buf) {
    if (!c || !device_buf) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (direction != 0 && direction != 1) return fail(GEMPE_E_INVALID_ARG, "direction must be 0 or 1");
    Pack& pk = *c->pk;
    if (!pk.sharded()) return fail(GEMPE_E_INVALID_ARG, "not a shard context (gempe_create_shard)");
    const size_t bins = (size_t)pk.bins;
    void* src = nullptr;
    size_t bytes = 0;
    switch (what) {
        case 0: src = pk.acc; bytes = sizeof(float) * (size_t)c->n * pk.acc_stride; break;
        case 1: src = pk.hist_e; bytes = sizeof(unsigned int) * bins; break;
        case 2: src = pk.hist_c; bytes = sizeof(unsigned int) * bins; break;
        case 3: src = pk.hist_d; bytes = sizeof(unsigned long long) * bins; break;
        case 4: src = pk.hist_x; bytes = sizeof(float) * bins; break;
        case 5: src = pk.x; bytes = sizeof(float) * (size_t)c->n * pk.d; break;
        default: return fail(GEMPE_E_INVALID_ARG, "what must be in [0, 5]");
    }
    if (what <= 4 && !pk.swept)
        return fail(GEMPE_E_INVALID_ARG, "sums and histograms are exchanged between gempe_sweep and gempe_update");
    if (what == 5 && pk.swept)
        return fail(GEMPE_E_INVALID_ARG, "positions are exchanged after gempe_update");
    if (direction == 0) {
        CK(cudaMemcpyAsync(device_buf, src, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy out");
    } else {
        CK(cudaMemcpyAsync(src, device_buf, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy in");
        if (what == 5 && pk.xb)
            CK(launch_to_bf16(pk.x, pk.xb, (long long)c->n * pk.d, c->stream), "BF16 shadow");
    }
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_test_tile_wait(int32_t poll_limit, int32_t* out_status, int32_t* out_freed) {
    if (!out_status || !out_freed) return fail(GEMPE_E_INVALID_ARG, "null argument");
    if (poll_limit < 1 || poll_limit > (1 << 22)) return fail(GEMPE_E_INVALID_ARG, "poll_limit in [1, 2^22]");
    int32_t* dv = nullptr;
    CK(cudaMalloc((void**)&dv, 2 * sizeof(int32_t)), "alloc");
    int32_t h[2] = {0, 0};
    cudaError_t e = cudaMemset(dv, 0, 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = launch_tile_wait_probe(poll_limit, dv, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(h, dv, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(dv);
    if (e != cudaSuccess) return cuda_fail(e, "tile wait probe");
    *out_status = h[0];
    *out_freed = h[1];
    return GEMPE_OK;
}

GEMPE_API const char* gempe_last_error(void) { return g_last_error.c_str(); }

namespace gempe {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace gempe
