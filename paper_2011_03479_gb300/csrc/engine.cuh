// Internal interface between the C-ABI host code and the CUDA kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gempe {

// Per-context scalars that change on the device (so a captured epoch graph
// can be replayed without new kernel arguments).
struct DevState {
    float sigma;
    int32_t epoch;          // epoch of the next sweep
    int32_t status;         // 0 or a gempe_status set by a kernel
    int32_t sample_epoch;   // epoch whose samples the sampler draws next
    unsigned int sample_done;   // blocks of the running sampler that finished
    int32_t sigma_iters;        // Newton / halving steps of the last slope fit
    unsigned long long accepted, rejected, exhausted, draws;   // sampler statistics
    unsigned long long used;    // sampled non-edges consumed by sweeps
    double loss_sum;
};

// Chunk size (CSR slots) of the per-unit sweep used for d >= 8.
constexpr int kEdgeChunk = 64;
constexpr int kMaxK = 32;
constexpr int kSweepThreads = 1024;
constexpr int kUpdateThreads = 1024;
constexpr int kSigmaMaxIters = 60;

// Work units: int4 {v0, nv, e_lo, e_hi | flags}.  e_lo < 0: nv whole vertices;
// else one vertex's CSR slots [e_lo, e_hi).  kUnitHasSamples: the unit also
// carries the sampled non-edges of its vertices.
constexpr int kUnitHasSamples = 1 << 30;
constexpr int kUnitPairs = 128;          // pair budget of a packed unit (d <= 4)
constexpr int kUnitSampleCap = 128;      // samples one packed unit may hold
constexpr int kPackedMaxDim = 4;
constexpr int kPackedThreads = 512;

inline size_t hist_smem_bytes(int bins) { return (size_t)bins * 3 * sizeof(unsigned int); }

inline size_t packed_smem_bytes(int d, int bins) {
    const int as = ((d + 1) + 3) / 4 * 4;
    return hist_smem_bytes(bins) + (size_t)(kPackedThreads / 32) * (kUnitSampleCap * sizeof(int) + 32 * as * sizeof(float));
}

struct EpochArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const unsigned long long* keys;
    unsigned long long bucket_mask;
    const float* x;
    float* acc;           // [n][acc_stride]: d values of y - z x, then z
    unsigned int* hist_e;         // [bins] edge counts
    unsigned int* hist_c;         // [bins] sample counts
    unsigned long long* hist_d;   // [bins] sums of the samples' anchor degrees
    float* hist_x;                // [bins] weight corrections of vertices with dropped samples
    DevState* st;
    const int4* items;
    int32_t n_items;
    int32_t n, d, acc_stride, k, max_retries, symmetric, w_formula, clamp_neg_d, bins;
    float mu, hist_scale;  // hist_scale = bins / hist_max
    uint32_t key_lo, key_hi;
    int32_t* samples;      // [2][n][k] accepted partners (-1 = dropped), buffer = epoch & 1
    // precision form: BF16 shadow of x (null in the FP32 form)
    __nv_bfloat16* xb;
    // block sampling: tiles of block_T vertices share block_P partners
    int32_t block_P, block_T, n_tiles;
    int32_t* block_part;             // [2][n_tiles][block_P], buffer = epoch & 1
    unsigned long long* block_mask;  // [2][n] bit p set: partner p of the vertex's tile is masked
    int32_t sweep_samples;           // 0: the sweep leaves the sampled non-edges to the tile kernel
    const struct MillsCoef* mills;   // Mills-ratio table on this device
};

// Sampled-partner layout of block sampling.
constexpr int kBlockP = 64;
constexpr int kBlockT = 128;

struct UpdateArgs {
    float* x;
    __nv_bfloat16* xb;     // BF16 shadow, or null
    float* acc;
    unsigned int* hist_e;
    unsigned int* hist_c;
    unsigned long long* hist_d;
    float* hist_x;
    DevState* st;
    int32_t n, d, acc_stride, bins, sigma_every, k;
    float z_min, mu, hist_max;
};

int acc_stride_for(int d);
bool supported_dim(int d);

cudaError_t launch_hash_build(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                              unsigned long long* keys, unsigned long long bucket_mask,
                              int32_t* fail_flag, cudaStream_t s);
cudaError_t launch_init_positions(float* x, __nv_bfloat16* xb, int32_t n, int32_t d, uint32_t key_lo,
                                  uint32_t key_hi, float range, cudaStream_t s);
cudaError_t launch_sweep(const EpochArgs& a, int grid, cudaStream_t s);
int sweep_grid(int d, int bins, int sm_count);
cudaError_t launch_update(const UpdateArgs& a, int grid, cudaStream_t s);
cudaError_t launch_sample(const EpochArgs& a, uint32_t tag, int32_t* out, cudaStream_t s);
cudaError_t launch_sampler(const EpochArgs& a, int grid, cudaStream_t s);
cudaError_t launch_block_sampler(const EpochArgs& a, const int4* units, int n_units, int sm_count,
                                 cudaStream_t s);
constexpr int kSamplerChunk = 1024;   // CSR slots per block-sampler work unit
cudaError_t launch_tile_bf16(const EpochArgs& a, int sm_count, cudaStream_t s);
bool tile_dim(int d);
size_t tile_smem_bytes(int d, int bins);
cudaError_t prepare_tile_kernel(int d, int bins);
cudaError_t launch_to_bf16(const float* x, __nv_bfloat16* xb, long long count, cudaStream_t s);
int sampler_grid(int n, int k, int sm_count);
cudaError_t launch_loss(const EpochArgs& a, cudaStream_t s);
cudaError_t launch_is_edge(const unsigned long long* keys, unsigned long long bucket_mask,
                           const int32_t* pairs, int64_t count, uint8_t* out, cudaStream_t s);
// Message for gempe_last_error() on the calling thread.
void set_last_error(const char* msg);

// Mills-ratio table (host side): builds the coefficients and uploads them to
// the current device once.
cudaError_t ensure_mills_table();
const struct MillsCoef* mills_table_device();
cudaError_t upload_mills_table(const void* host_coefs, size_t bytes);
cudaError_t launch_fit_sigma(const float* hist, int32_t bins, float hist_max, float mu,
                             float* sigma_inout, cudaStream_t s);

}  // namespace gempe
