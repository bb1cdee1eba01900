// Host side of a pack: graphs of one dimension laid out back to back in one
// set of device arrays (layout in engine.cuh), the work lists the kernels
// stride over, and the enqueueing of one epoch.  A single-graph context is
// a pack of one; a batch holds one pack per dimension.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "engine.cuh"
#include "gempe.h"

namespace gempe {

struct GraphInput {
    const int32_t* row_ptr;   // host, n + 1
    const int32_t* col_idx;   // host, row_ptr[n]
    int32_t n;
    uint64_t key;             // Philox key of the graph
    int32_t label = -1;       // index of the graph in the caller's list (error messages), -1: none
};

// Launch shape of the sweep (the autotuner's search space).
struct PackShape {
    int unit_pairs = kUnitPairs;   // d <= 4: pair budget of a packed unit (64 or 128)
    int edge_chunk = kEdgeChunk;   // d >= 8: CSR slots per work unit (32, 64, 128)
    int lanes = 0;                 // d >= 8: lanes per pair (d/8 or d/4; 0 = d/8)
    int blocks_per_sm = 0;         // sweep CTAs per SM (0 = as many as fit)
    int kernel = 0;                // d <= 4: 0 packed units, 1 one lane per vertex; d >= 8 with tiles:
                                   // 2 the sweep (512-thread blocks, one per SM) beside one tile CTA per SM
    float sweep_us = 0.0f;         // measured sweep time of the chosen shape (autotuner)
};

// Message for gempe_last_error() and the status, in one call.
gempe_status pack_fail(gempe_status st, const std::string& msg);
gempe_status pack_cuda_fail(cudaError_t e, const char* what);
gempe_status check_params(const gempe_params* p, int32_t d);
// threads: host threads for the check (0: by the size of the graph);
// symmetry = false leaves the symmetry to the device check of Pack::build.
gempe_status validate_csr(const int32_t* rp, const int32_t* ci, int32_t n, int threads = 0, bool symmetry = true);
// Host threads for O(work) set-up loops: one per 65,536 items, at most 32.
int host_threads(int64_t work);
// fn(begin, end) over [0, count) cut into `parts` ranges of equal weight
// (cum(i): weight of [0, i), non-decreasing), one host thread per range.
void parallel_for_weighted(int64_t count, int parts, const std::function<int64_t(int64_t)>& cum,
                           const std::function<void(int64_t, int64_t)>& fn);

struct Pack {
    gempe_params p{};
    int32_t d = 0, k = 0, acc_stride = 0, bins = 0;
    int32_t G = 0, rows = 0, n_tiles = 0;
    int64_t slots = 0;
    unsigned long long key_slots = 0;
    bool narrow_keys = false;        // every graph has n <= 65536: u32 edge keys
    bool block = false, tiles = false;
    bool per_slot = false;           // Sec. III.C's policy: one sample per CSR slot
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;   // set by the owner (context or batch), not owned
    cudaStream_t side = nullptr;     // owned: the next epoch's sampler runs here
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // launch shape kernel 2 (block form with tiles): the tile kernel runs on
    // tile_stream beside the sweep, forked and joined by these events
    cudaStream_t tile_stream = nullptr;
    cudaEvent_t tile_fork = nullptr, tile_join = nullptr;
    bool primed = false;             // samples of the current epoch are in the buffer
    bool sampled_ahead = false;      // the next epoch's sampler has been enqueued
    bool swept = false;              // a sweep ran without the update that clears its sums
    // per-kernel timing of epochs enqueued directly (not captured): events on
    // `stream` before the sweep, after it, after the tiles, after the update
    // (events: before the sweep, after it, before the tiles, after them, after
    // the join, after the update)
    bool time_kernels = false;
    // shard of one graph (set before build): anchors [own_lo, own_hi) only;
    // own_hi < 0: every vertex
    int32_t own_lo = 0, own_hi = -1;
    bool sharded() const { return own_hi >= 0; }
    cudaEvent_t tev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<GraphInfo> info;     // host copies
    std::vector<int64_t> nnz;
    std::vector<int32_t> row_ptr_h;  // pack CSR offsets, rows + 1
    std::vector<int32_t> orow_ptr_h; // degree-oriented CSR offsets (d <= 4, k-per-vertex policy), else empty
    PackShape shape;

    // device memory
    GraphInfo* graphs = nullptr;
    GraphState* gst = nullptr;
    PackState* ps = nullptr;
    int32_t* row_ptr = nullptr;
    int32_t* col_idx = nullptr;
    int32_t* orow_ptr = nullptr;     // degree-oriented CSR (see orow_ptr_h)
    int32_t* ocol_idx = nullptr;
    void* keys = nullptr;            // edge sets, key_slots keys of 4 (narrow) or 8 bytes
    float* x = nullptr;
    __nv_bfloat16* xb = nullptr;
    float* acc = nullptr;
    void* hist = nullptr;            // hist_d [G][bins] u64, hist_e, hist_c [G][bins] u32, hist_x [G][bins] f32
    size_t hist_bytes = 0;
    unsigned long long* hist_d = nullptr;
    unsigned int* hist_e = nullptr;
    unsigned int* hist_c = nullptr;
    float* hist_x = nullptr;
    int4* items = nullptr;
    int32_t n_items = 0;
    int32_t* task_bounds = nullptr;  // d >= 8: sweep block b takes tasks [bounds[b], bounds[b+1])
    int32_t task_bounds_cap = 0;
    int4* vchunks = nullptr;
    int32_t n_vchunks = 0;
    int32_t* samples = nullptr;      // [2][rows][k], per-slot policy [2][slots]
    int32_t* vacc = nullptr;         // per-slot policy: [2][rows] accepted samples per vertex
    int32_t* block_part = nullptr;   // [2][n_tiles][64]
    unsigned long long* block_mask = nullptr;   // [2][rows]
    int4* sampler_units = nullptr;   // block sampler, one per tile {tile, 0, 0, graph << 1 | 1}
    int32_t n_sampler_units = 0;
    int2* tile_items = nullptr;      // {tile, graph}
    int32_t n_tile_items = 0;
    int32_t* scratch = nullptr;      // rows * max(k, 1) int32: inspection samples, flags
    uint8_t* bytemap = nullptr;      // byte-map membership: the graphs' maps back to back
    size_t bytemap_bytes = 0;
    const MillsCoef* mills = nullptr;
    int sweep_grid = 0, sampler_grid = 0, update_grid = 0, tile_grid = 0;
    std::vector<void*> allocations;

    Pack() = default;
    Pack(const Pack&) = delete;
    Pack& operator=(const Pack&) = delete;
    ~Pack();

    void* alloc(size_t bytes);       // on `stream` (set before the first call)
    void release(void* ptr);
    void free_one(void* ptr);
    void release_all();

    // Lays the graphs out, copies them and builds their edge sets and initial
    // positions on `stream` (synchronised before returning).
    // validate = false: the caller has already run validate_csr on every graph.
    gempe_status build(const std::vector<GraphInput>& graphs, int32_t d, const gempe_params& params,
                       cudaStream_t stream, bool validate = true);
    // Rebuilds the sweep units and grid for another launch shape.
    gempe_status set_shape(const PackShape& s);
    // Times the candidate shapes on this pack's own sweep and keeps the
    // fastest (the epoch state is left as it was).
    gempe_status autotune();

    EpochArgs args() const;
    gempe_status prime();            // samples of the current epoch, if the buffer lacks them
    gempe_status enqueue_sweep();    // sweep (+ tiles); the next epoch's sampler forked to `side`
    gempe_status enqueue_update();   // position update + slope fits; joins `side`
    gempe_status read_status();      // synchronises; reports and clears a device-side error
    int32_t slots_per_vertex() const { return block ? kBlockP : k; }
    bool sampled() const { return per_slot ? slots > 0 : slots_per_vertex() > 0; }

    // log2 of the byte-map size of a graph with nnz CSR slots (the parameter,
    // or nnz rounded up to a power of two times 128, in [2^12, 2^30])
    static int bytemap_log2_for(int64_t nnz, const gempe_params& p);
    // Device bytes a pack of one graph with n vertices and nnz CSR slots
    // allocates (an upper bound: the sweep units are counted at their most).
    static size_t bytes_for(int32_t n, int64_t nnz, int32_t d, const gempe_params& p);
};

}  // namespace gempe
