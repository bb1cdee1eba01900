// Batched form of the C ABI (include/gempe.h): many independent graphs,
// grouped by dimension into packs (pack.cuh), stepped by one CUDA-graph
// launch per epoch whose per-pack branches run concurrently.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <vector>

#include "engine.cuh"
#include "gempe.h"
#include "pack.cuh"

#define GEMPE_API extern "C" __attribute__((visibility("default")))

using namespace gempe;

namespace {

#define BK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return pack_cuda_fail(e_, what); \
    } while (0)

}  // namespace

struct gempe_batch {
    std::vector<std::unique_ptr<Pack>> packs;     // ascending d
    std::vector<cudaStream_t> pack_streams;       // owned, one per pack
    std::vector<cudaEvent_t> done_ev;             // owned, one per pack
    std::vector<int> pack_of, index_in_pack;      // per graph of the batch
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t fork_ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool primed = false;

    ~gempe_batch() {
        if (stream) cudaStreamSynchronize(stream);
        for (cudaStream_t s : pack_streams) cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        packs.clear();
        for (cudaEvent_t e : done_ev) cudaEventDestroy(e);
        for (cudaStream_t s : pack_streams) cudaStreamDestroy(s);
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    gempe_status sync() {
        BK(cudaStreamSynchronize(stream), "synchronize");
        for (cudaStream_t s : pack_streams) BK(cudaStreamSynchronize(s), "synchronize");
        return GEMPE_OK;
    }
};

GEMPE_API gempe_status gempe_batch_create(int32_t n_graphs, const gempe_graph_desc* graphs, const gempe_params* p,
                                          void* cuda_stream, gempe_batch** out) {
    if (!out) return pack_fail(GEMPE_E_INVALID_ARG, "out is null");
    *out = nullptr;
    if (n_graphs < 1 || !graphs || !p) return pack_fail(GEMPE_E_INVALID_ARG, "need n_graphs >= 1, graphs and params");
    std::map<int, std::vector<int>> by_dim;
    std::vector<int64_t> slots_before((size_t)n_graphs + 1, 0);
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (!supported_dim(graphs[g].d))
            return pack_fail(GEMPE_E_INVALID_ARG, "graph " + std::to_string(g) + ": unsupported d");
        if (!graphs[g].row_ptr || graphs[g].n < 2 || graphs[g].row_ptr[graphs[g].n] < 0 ||
            (!graphs[g].col_idx && graphs[g].row_ptr[graphs[g].n] > 0))
            return pack_fail(GEMPE_E_INVALID_ARG, "graph " + std::to_string(g) + ": null CSR or n < 2");
        gempe_status rc = check_params(p, graphs[g].d >= 8 ? graphs[g].d : 8);
        if (rc != GEMPE_OK) return rc;
        slots_before[g + 1] = slots_before[g] + graphs[g].row_ptr[graphs[g].n] + graphs[g].n;
        by_dim[graphs[g].d].push_back(g);
    }
    // the rows of every graph on host threads (graphs in ranges of equal
    // size), before device work; the symmetry on the device (Pack::build).
    // The error reported is the lowest failing graph's.
    {
        std::mutex mu;
        int bad = n_graphs;
        gempe_status bad_rc = GEMPE_OK;
        std::string bad_msg;
        parallel_for_weighted(n_graphs, host_threads(slots_before[n_graphs]),
                              [&](int64_t g) { return slots_before[g]; },
                              [&](int64_t g0, int64_t g1) {
                                  for (int64_t g = g0; g < g1; ++g) {
                                      const gempe_status rc =
                                          validate_csr(graphs[g].row_ptr, graphs[g].col_idx, graphs[g].n, 1, false);
                                      if (rc == GEMPE_OK) continue;
                                      std::lock_guard<std::mutex> lock(mu);
                                      if (g < bad) {
                                          bad = (int)g;
                                          bad_rc = rc;
                                          bad_msg = gempe_last_error();   // this thread's message
                                      }
                                      return;
                                  }
                              });
        if (bad < n_graphs) return pack_fail(bad_rc, "graph " + std::to_string(bad) + ": " + bad_msg);
    }
    std::unique_ptr<gempe_batch> b(new gempe_batch());
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        BK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        b->own_stream = true;
    }
    BK(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming), "cudaEventCreate");
    b->pack_of.assign(n_graphs, -1);
    b->index_in_pack.assign(n_graphs, -1);
    for (auto& kv : by_dim) {
        const int d = kv.first;
        gempe_params pp = *p;
        if (d < 8) {   // the BF16 form and block sampling need d >= 8
            pp.precision = 0;
            pp.block_partners = 0;
        }
        std::vector<GraphInput> in;
        for (size_t q = 0; q < kv.second.size(); ++q) {
            const int g = kv.second[q];
            GraphInput gi;
            gi.row_ptr = graphs[g].row_ptr;
            gi.col_idx = graphs[g].col_idx;
            gi.n = graphs[g].n;
            gi.key = p->seed ^ (uint64_t)g;
            gi.label = g;
            in.push_back(gi);
            b->pack_of[g] = (int)b->packs.size();
            b->index_in_pack[g] = (int)q;
        }
        cudaStream_t s = nullptr;
        BK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
        b->pack_streams.push_back(s);
        cudaEvent_t ev = nullptr;
        BK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
        b->done_ev.push_back(ev);
        std::unique_ptr<Pack> pk(new Pack());
        gempe_status rc = pk->build(in, d, pp, s, false);
        if (rc != GEMPE_OK) {
            return pack_fail(rc, "graph group d=" + std::to_string(d) + ": " + std::string(gempe_last_error()));
        }
        if (pp.autotune) {
            rc = pk->autotune();
            if (rc != GEMPE_OK) return rc;
        }
        b->packs.push_back(std::move(pk));
    }
    *out = b.release();
    return GEMPE_OK;
}

GEMPE_API void gempe_batch_destroy(gempe_batch* b) { delete b; }

GEMPE_API gempe_status gempe_batch_step(gempe_batch* b, int32_t iters) {
    if (!b) return pack_fail(GEMPE_E_INVALID_ARG, "batch is null");
    if (iters < 0) return pack_fail(GEMPE_E_INVALID_ARG, "iters must be >= 0");
    if (iters == 0) return GEMPE_OK;
    const size_t P = b->packs.size();
    if (!b->primed) {
        // the first epoch's samples, then the main stream waits for them
        for (size_t q = 0; q < P; ++q) {
            gempe_status rc = b->packs[q]->prime();
            if (rc != GEMPE_OK) return rc;
            BK(cudaEventRecord(b->done_ev[q], b->pack_streams[q]), "record");
            BK(cudaStreamWaitEvent(b->stream, b->done_ev[q], 0), "wait");
        }
        b->primed = true;
    }
    if (!b->exec) {
        BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        gempe_status rc = GEMPE_OK;
        cudaError_t e = cudaEventRecord(b->fork_ev, b->stream);
        for (size_t q = 0; q < P && rc == GEMPE_OK && e == cudaSuccess; ++q) {
            e = cudaStreamWaitEvent(b->pack_streams[q], b->fork_ev, 0);
            if (e != cudaSuccess) break;
            rc = b->packs[q]->enqueue_sweep();
            if (rc == GEMPE_OK) rc = b->packs[q]->enqueue_update();
            if (rc == GEMPE_OK) e = cudaEventRecord(b->done_ev[q], b->pack_streams[q]);
            if (rc == GEMPE_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->done_ev[q], 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
        if (rc != GEMPE_OK || e != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc != GEMPE_OK) return rc;
            return pack_cuda_fail(e != cudaSuccess ? e : ee, "capture");
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            return pack_cuda_fail(e, "graph instantiate");
        }
        b->graph = g;
    }
    for (int32_t it = 0; it < iters; ++it) BK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    return GEMPE_OK;
}

namespace {
gempe_status locate(gempe_batch* b, int32_t graph, Pack** pk, int* idx) {
    if (!b) return pack_fail(GEMPE_E_INVALID_ARG, "batch is null");
    if (graph < 0 || graph >= (int32_t)b->pack_of.size()) return pack_fail(GEMPE_E_INVALID_ARG, "graph out of range");
    *pk = b->packs[b->pack_of[graph]].get();
    *idx = b->index_in_pack[graph];
    return b->sync();
}
}  // namespace

GEMPE_API gempe_status gempe_batch_positions(gempe_batch* b, int32_t graph, float* host_out, size_t count) {
    Pack* pk = nullptr;
    int idx = 0;
    gempe_status rc = locate(b, graph, &pk, &idx);
    if (rc != GEMPE_OK) return rc;
    if (!host_out) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    const GraphInfo& gi = pk->info[idx];
    if (count != (size_t)gi.n * pk->d) return pack_fail(GEMPE_E_INVALID_ARG, "count must be n*d");
    BK(cudaMemcpyAsync(host_out, pk->x + (size_t)gi.v0 * pk->d, sizeof(float) * count, cudaMemcpyDeviceToHost,
                       pk->stream),
       "copy x");
    return pk->read_status();
}

GEMPE_API gempe_status gempe_batch_loss(gempe_batch* b, int32_t graph, double* out_pe_bits, float* out_sigma) {
    Pack* pk = nullptr;
    int idx = 0;
    gempe_status rc = locate(b, graph, &pk, &idx);
    if (rc != GEMPE_OK) return rc;
    if (!out_pe_bits) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    // the loss kernel sums every graph of the pack into its own loss_sum
    std::vector<GraphState> st(pk->G);
    BK(cudaMemcpyAsync(st.data(), pk->gst, sizeof(GraphState) * pk->G, cudaMemcpyDeviceToHost, pk->stream), "state");
    BK(cudaStreamSynchronize(pk->stream), "synchronize");
    for (auto& s : st) s.loss_sum = 0.0;
    BK(cudaMemcpyAsync(pk->gst, st.data(), sizeof(GraphState) * pk->G, cudaMemcpyHostToDevice, pk->stream), "state");
    BK(launch_loss(pk->args(), pk->stream), "loss");
    BK(cudaMemcpyAsync(st.data(), pk->gst, sizeof(GraphState) * pk->G, cudaMemcpyDeviceToHost, pk->stream), "state");
    BK(cudaStreamSynchronize(pk->stream), "synchronize");
    const double n = pk->info[idx].n;
    *out_pe_bits = st[idx].loss_sum / (0.5 * n * (n - 1.0));
    if (out_sigma) *out_sigma = st[idx].sigma;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_batch_stats(gempe_batch* b, int32_t graph, gempe_stats_t* out) {
    Pack* pk = nullptr;
    int idx = 0;
    gempe_status rc = locate(b, graph, &pk, &idx);
    if (rc != GEMPE_OK) return rc;
    if (!out) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    GraphState h{};
    BK(cudaMemcpyAsync(&h, pk->gst + idx, sizeof(GraphState), cudaMemcpyDeviceToHost, pk->stream), "state");
    BK(cudaStreamSynchronize(pk->stream), "synchronize");
    out->epoch = h.epoch;
    out->sigma = h.sigma;
    out->accepted = h.accepted;
    out->rejected = h.rejected;
    out->exhausted = h.exhausted;
    out->draws = h.draws;
    out->used = h.used;
    out->n_edges = pk->nnz[idx] / 2;
    out->n = pk->info[idx].n;
    out->d = pk->d;
    out->k = pk->k;
    out->sigma_iters = h.sigma_iters;
    out->false_pos = h.false_pos;
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_batch_shape(gempe_batch* b, int32_t d, int64_t* out7) {
    if (!b || !out7) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    for (auto& pk : b->packs) {
        if (pk->d != d) continue;
        const bool packed = d <= kPackedMaxDim && pk->shape.kernel == 0;
        out7[0] = packed ? pk->shape.unit_pairs : pk->shape.edge_chunk;
        out7[1] = pk->shape.lanes ? pk->shape.lanes : (d <= kPackedMaxDim ? 1 : d / 8);
        out7[2] = pk->shape.blocks_per_sm;
        out7[3] = pk->sweep_grid;
        out7[4] = pk->G;
        out7[5] = (int64_t)(pk->shape.sweep_us * 1000.0f);
        out7[6] = pk->shape.kernel;
        return GEMPE_OK;
    }
    return pack_fail(GEMPE_E_INVALID_ARG, "no graph of that dimension in the batch");
}
