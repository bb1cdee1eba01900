// Internal interface between the host code (C ABI, packs, batches) and the
// CUDA kernels.
//
// A pack is the unit the kernels run on: one or more graphs of the same
// dimension d, laid out back to back in one set of device arrays.  Graph g
// owns rows [v0, v0 + n) of the vertex arrays (positions, accumulators,
// samples, masks) plus one spare row v0 + n that closes its CSR range; its
// CSR slots are absolute offsets into one column array whose entries are
// pack row ids; its exact edge set is its own table (local vertex ids) at
// key_off in one key array; its Philox key, slope sigma, epoch and
// histograms are its own.  A single graph is a pack of one, and a graph
// gives the same samples and (up to FP32 summation order) the same epoch
// alone or in any pack.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gempe {

// Per-graph constants (read-only while an epoch runs).  48 bytes, 16-byte
// aligned: the kernels read them as one int4 and two ulonglong2.
struct alignas(16) GraphInfo {
    int32_t v0;                       // first row of the graph in the pack
    int32_t n;                        // vertices
    int32_t t0;                       // first tile of the graph (block sampling)
    int32_t n_tiles;                  // tiles of the graph
    uint32_t key_lo, key_hi;          // Philox key
    unsigned long long key_off;       // first slot of the graph's edge table
    unsigned long long bucket_mask;   // buckets - 1 of that table
    unsigned long long map;           // byte-map membership: offset of the graph's map in the pack's
                                      // map array (a multiple of 64) | log2 of its size; 0 without
};
static_assert(sizeof(GraphInfo) == 48, "GraphInfo layout");

// Per-graph scalars that change on the device, so that a captured epoch can
// be replayed without new kernel arguments.
struct GraphState {
    float sigma;
    int32_t epoch;          // epoch of the next sweep
    int32_t sample_epoch;   // epoch whose samples the sampler draws next
    int32_t sigma_iters;    // Newton / halving steps of the last slope fit
    unsigned long long accepted, rejected, exhausted, draws;   // sampler statistics
    unsigned long long used;    // sampled non-edges consumed by sweeps
    double loss_sum;
    int32_t map_period;         // renaming period the byte map holds (-1: none yet)
    int32_t pad;
    unsigned long long false_pos;   // draws the byte map rejected that are not edges
};

// Pack-wide device scalars.
struct PackState {
    int32_t status;             // 0 or a gempe_status set by a kernel
    unsigned int sample_done;   // blocks of the running sampler that finished
};

// Packs whose graphs all have at most this many vertices key their edge
// sets by u32 (min << 16 | max), others by u64.
constexpr int kNarrowKeysMaxN = 65536;

// Chunk size (CSR slots) of the per-unit sweep used for d >= 8 (default;
// the autotuner may pick another).
constexpr int kEdgeChunk = 32;
constexpr int kMaxK = 32;
constexpr int kSweepThreads = 1024;
constexpr int kUpdateThreads = 1024;
constexpr int kSigmaMaxIters = 60;
constexpr int kVChunk = 1024;          // vertices per vertex chunk
constexpr int kSamplerSub = 64;        // vertices per sampler block iteration
constexpr int kGraphShift = 8;         // unit.y = graph << kGraphShift | vertex count

// Work units: int4 {v0, graph << 8 | nv, e_lo, e_hi | flags}.  e_lo < 0: nv
// whole vertices (rows v0 ..); else one vertex's CSR slots [e_lo, e_hi)
// relative to its row start.  kUnitHasSamples: the unit also carries the
// sampled non-edges of its vertices.  Units never cross graphs.
constexpr int kUnitHasSamples = 1 << 30;
constexpr int kUnitPairs = 128;          // pair budget of a packed unit (d <= 4, default)
constexpr int kUnitSampleCap = 128;      // samples one packed unit may hold
constexpr int kPackedMaxDim = 4;
constexpr int kPackedThreads = 512;

// Sampled-partner layout of block sampling.
constexpr int kBlockP = 64;
constexpr int kBlockT = 128;

// he, hc, hd (u32) and hw (f32, the per-slot policy's sample weights)
inline size_t hist_smem_bytes(int bins) { return (size_t)bins * 4 * sizeof(unsigned int); }

constexpr uint32_t kTagSlot = 0x0C000000u;   // counter tag of the per-slot samples
constexpr uint32_t kTagLcg = 0x08000000u;    // LCG seeds of the per-vertex sample slots (rng 1)
constexpr uint32_t kTagLcgSlot = 0x07000000u;   // LCG seeds of the per-slot samples (rng 1)

inline size_t packed_smem_bytes(int d, int bins) {
    const int as = ((d + 1) + 3) / 4 * 4;
    return hist_smem_bytes(bins) + (size_t)(kPackedThreads / 32) * (kUnitSampleCap * sizeof(int) + 32 * as * sizeof(float));
}

struct EpochArgs {
    // graphs
    const GraphInfo* graphs;
    GraphState* gst;
    PackState* ps;
    int32_t n_graphs;
    // CSR, edge sets, positions, accumulators
    const int32_t* row_ptr;   // [rows + 1] absolute slot offsets
    const int32_t* col_idx;   // pack row ids
    // degree-oriented CSR (d <= 4, k-per-vertex policy): each undirected edge
    // once, in the row of its endpoint with the larger (degree, id)
    const int32_t* orow_ptr;
    const int32_t* ocol_idx;
    int32_t oriented;         // 1: the packed sweep takes its edge slots from it
    const void* keys;         // edge sets: u32 keys when narrow_keys, else u64 (device_math.cuh)
    int32_t narrow_keys;
    float* x;
    __nv_bfloat16* xb;        // BF16 shadow of x (precision form), else null
    float* acc;               // [rows][acc_stride]: d values of y - z x, then z
    // histograms, [n_graphs][bins] each
    unsigned int* hist_e;         // edge counts
    unsigned int* hist_c;         // sample counts
    unsigned long long* hist_d;   // sums of the samples' anchor degrees
    float* hist_x;                // weight corrections of vertices with dropped samples
    // work lists
    const int4* items;        // sweep units
    int32_t n_items;
    const int32_t* task_bounds;   // d >= 8: first task of each sweep block (grid + 1 entries)
    int32_t blocked;          // 1: block b takes a contiguous range of units (packs of several graphs)
    const int4* vchunks;      // {row begin, count <= kVChunk, graph, 0}
    int32_t n_vchunks;
    int32_t rows, d, acc_stride, k, max_retries, symmetric, w_formula, clamp_neg_d, bins;
    float mu, hist_scale;     // hist_scale = bins / hist_max
    int32_t* samples;         // [2][rows][k] accepted partners (-1 = dropped), buffer = epoch & 1;
                              // per-slot policy: [2][n_slots], one partner per CSR slot
    int32_t per_slot;         // 1: Sec. III.C's policy, one sample per CSR slot of the anchor's row
    int32_t n_slots;          // CSR slots of the pack
    int32_t* vacc;            // per-slot policy: [2][rows] accepted samples per vertex
    // block sampling: tiles of kBlockT rows share kBlockP partners
    int32_t block_P, n_tiles;
    int32_t* block_part;             // [2][n_tiles][kBlockP] partner rows, buffer = epoch & 1
    unsigned long long* block_mask;  // [2][rows] bit p set: partner p of the row's tile is masked
    const int2* tile_items;          // {tile, graph} of the tile kernel
    int32_t n_tile_items;
    int32_t sweep_samples;           // 0: the sweep leaves the sampled non-edges to the tile kernel
    // update
    int32_t sigma_every;
    int32_t sigma_source;     // 0: histograms from the sweep; 1: a separate pass after the update (Sec. III.F)
    int32_t sweep_hist;       // 1: the sweep kernels bin their distances
    float z_min, hist_max;
    const struct MillsCoef* mills;   // Mills-ratio table on this device
    // byte-map membership (Sec. III.C): the sampler tests draws against the
    // graph's byte map under the renaming of period sample_epoch / rename_every
    int32_t membership;       // 0: the exact edge sets; 1: the byte maps
    int32_t rename_every;     // 0: one renaming (period 0) for the whole run
    uint8_t* bytemap;
    int32_t rng;              // 1: Sec. III.C's LCG draws the epoch's sampled non-edges
    int32_t own_n;            // shard of one graph: vertices whose anchors this pack evaluates (0: all)
};

int acc_stride_for(int d);
bool supported_dim(int d);

// Per-graph set-up (rows and slots of one graph of the pack).
cudaError_t launch_hash_build(const int32_t* row_ptr, const int32_t* col_idx, int32_t v0, int32_t n, int64_t nnz,
                              void* keys, int narrow, unsigned long long bucket_mask,
                              int32_t* fail_flag, cudaStream_t s);
// Symmetry check of one graph of the pack against its edge set (rows sorted
// and in range): counts3 += {slots above the diagonal, below, below without
// their reverse}; symmetric iff above == below and none missing.
cudaError_t launch_check_symmetric(const int32_t* row_ptr, const int32_t* col_idx, int32_t v0, int32_t n, int64_t nnz,
                                   const void* keys, int narrow, unsigned long long key_off,
                                   unsigned long long bucket_mask, unsigned long long* counts3, cudaStream_t s);
// v[0..count) += off (a graph's column indices to pack rows).
cudaError_t launch_add_offset(int32_t* v, int64_t count, int32_t off, cudaStream_t s);
// Degree-oriented CSR of the pack (rows + 1 offsets, kept slots in row
// order); scratch: orient_scratch_ints(rows) ints.
size_t orient_scratch_ints(int rows);
cudaError_t launch_orient(const int32_t* row_ptr, const int32_t* col_idx, int rows, int32_t* orow_ptr,
                          int32_t* ocol_idx, int32_t* scratch, int sm_count, cudaStream_t s);
cudaError_t launch_init_positions(float* x, __nv_bfloat16* xb, int32_t n, int32_t d, uint32_t key_lo,
                                  uint32_t key_hi, float range, cudaStream_t s);

// Sweep launch shape (chosen per pack, autotuned).
struct SweepShape {
    int grid = 0;
    int lanes = 0;      // d >= 8: lanes per pair (0: d / 8)
    int kernel = 0;     // d <= 4: 0 packed units, 1 one lane per vertex (the d >= 8 kernel with G = 1);
                        // d >= 8 with tiles: 2 the sweep beside the tile kernel (kSweepThreadsBeside per block)
};
// Threads of a d >= 8 sweep block that shares its SM with a tile CTA: half the
// register file, so that one block of each kernel is resident on every SM.
constexpr int kSweepThreadsBeside = 512;
cudaError_t launch_sweep(const EpochArgs& a, const SweepShape& shape, cudaStream_t s);
int sweep_grid(int d, int lanes, int bins, int sm_count, int blocks_per_sm, int kernel);
bool sweep_lanes_supported(int d, int lanes);
cudaError_t launch_update(const EpochArgs& a, int grid, cudaStream_t s);
cudaError_t prepare_update_kernels(int bins);   // shared-memory size of the slope-fit blocks
// Raises the dynamic shared-memory limit of `func` on the current device to
// at least `bytes`.  The limit is one per function and device, shared by
// every context, batch and server of the process, so it is only ever raised
// (a running maximum under a lock): a pack built with fewer histogram bins
// never lowers the limit another pack's launches rely on.
cudaError_t raise_smem_limit(const void* func, int bytes);
// sigma_source 1: the separate histogram pass at the updated positions, then
// the per-graph slope fits on it
cudaError_t launch_hist_pass(const EpochArgs& a, cudaStream_t s);
cudaError_t launch_fit_graphs(const EpochArgs& a, cudaStream_t s);
cudaError_t launch_sample(const EpochArgs& a, uint32_t tag, int32_t* out, cudaStream_t s);
cudaError_t launch_sampler(const EpochArgs& a, int grid, cudaStream_t s);   // k per vertex, or one per slot
// Byte maps of the graphs whose map does not hold the renaming period of their
// sample epoch (all graphs when force): cleared, then every edge marked.
cudaError_t launch_bytemap_build(const EpochArgs& a, int force, int sm_count, cudaStream_t s);
cudaError_t launch_block_sampler(const EpochArgs& a, const int4* units, int n_units, int sm_count,
                                 cudaStream_t s);
cudaError_t launch_tile_bf16(const EpochArgs& a, int grid, cudaStream_t s);
// FP32 tiles of block-sampled non-edges (precision 0, d in {16, 32, 64, 128}).
bool tile_dim_f32(int d);
size_t tile_f32_smem_bytes(int d, int bins);
cudaError_t prepare_tile_f32_kernel(int d, int bins);
int tile_f32_blocks_per_sm(int d, int bins);
cudaError_t launch_tile_f32(const EpochArgs& a, int grid, cudaStream_t s);
int tile_grid(int n_tile_items, int sm_count, int blocks_per_sm);
bool tile_dim(int d);
size_t tile_smem_bytes(int d, int bins);
cudaError_t prepare_tile_kernel(int d, int bins);
int tile_bf16_blocks_per_sm(int d, int bins);
// Test only: one tile-shaped CTA whose mbarrier wait (limit polls) runs out;
// dev_out[0] = the status it records, dev_out[1] = 1 after it freed its TMEM.
cudaError_t launch_tile_wait_probe(int limit, int32_t* dev_out, cudaStream_t s);
cudaError_t launch_to_bf16(const float* x, __nv_bfloat16* xb, long long count, cudaStream_t s);
int sampler_grid(int rows, int k, int sm_count);
cudaError_t launch_loss(const EpochArgs& a, cudaStream_t s);
cudaError_t launch_is_edge(const void* keys, int narrow, unsigned long long key_off, unsigned long long bucket_mask,
                           const int32_t* pairs, int64_t count, uint8_t* out, cudaStream_t s);
// Kernels on an epoch's critical path (sweeps, tiles, update, slope fit)
// launch at the device's highest stream priority, so that when SMs free up
// their blocks are dispatched ahead of those of the next epoch's sampler,
// which runs beside them on the side stream and has until the next sweep.
int critical_priority();
// dependent: launched as a programmatic dependent of the previous kernel in
// the stream (the kernel waits with griddepcontrol.wait before it reads what
// that kernel wrote; the previous kernel lets it be scheduled early with
// griddepcontrol.launch_dependents).
template <typename... KArgs, typename... Args>
cudaError_t launch_critical(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            bool dependent, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = critical_priority();
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Message for gempe_last_error() on the calling thread.
void set_last_error(const char* msg);

// Mills-ratio table (host side): builds the coefficients and uploads them to
// the current device once.
cudaError_t ensure_mills_table();
const struct MillsCoef* mills_table_device();
cudaError_t upload_mills_table(const void* host_coefs, size_t bytes);
cudaError_t launch_fit_sigma(const float* hist, int32_t bins, float hist_max, float mu,
                             float* sigma_inout, cudaStream_t s);
// Exact Eq. 2 at sigma over all pairs of one graph (rows 0..n-1): out3 = {sum dl,
// F, dF/d ln sigma} (FP64; F has the sign of dPE/dsigma).
cudaError_t launch_exact_pe(const int32_t* row_ptr, const int32_t* col_idx, const float* x, int n, int d, float mu,
                            float sigma, const struct MillsCoef* tab, double* out3, int sm_count, cudaStream_t s);

}  // namespace gempe
