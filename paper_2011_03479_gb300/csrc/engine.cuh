// Internal interface between the C-ABI host code and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gempe {

// Per-context scalars that change on the device (so a captured epoch graph
// can be replayed without new kernel arguments).
struct DevState {
    float sigma;
    int32_t epoch;
    int32_t status;        // 0 or a gempe_status set by a kernel
    int32_t pad;
    unsigned long long accepted, rejected, exhausted, draws;
    double loss_sum;
};

// One unit of sweep work: vertex v, its CSR slots [p0, p1) relative to the
// row start, and (flags & 1) whether the unit also carries v's samples.
// Hubs are cut into several units of at most kEdgeChunk slots; a vertex's
// samples always stay in one unit (its last).
constexpr int kEdgeChunk = 64;
constexpr int kMaxK = 32;
constexpr int kSweepThreads = 256;
constexpr int kUpdateThreads = 256;
constexpr int kSigmaIters = 32;

struct EpochArgs {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const unsigned long long* keys;
    unsigned long long bucket_mask;
    const float* x;
    float* acc;           // [n][acc_stride]: d values of y - z x, then z
    float* hist;          // [2][bins]
    DevState* st;
    const int4* items;
    int32_t n_items;
    int32_t n, d, acc_stride, k, max_retries, symmetric, w_formula, clamp_neg_d, bins;
    float mu, hist_scale;  // hist_scale = bins / hist_max
    uint32_t key_lo, key_hi;
    int32_t* record;       // null, or [n][k] accepted partners (-1 = dropped)
};

struct UpdateArgs {
    float* x;
    float* acc;
    float* hist;
    DevState* st;
    int32_t n, d, acc_stride, bins, sigma_every;
    float z_min, mu, hist_max;
};

int acc_stride_for(int d);
bool supported_dim(int d);

cudaError_t launch_hash_build(const int32_t* row_ptr, const int32_t* col_idx, int32_t n,
                              unsigned long long* keys, unsigned long long bucket_mask,
                              int32_t* fail_flag, cudaStream_t s);
cudaError_t launch_init_positions(float* x, int32_t n, int32_t d, uint32_t key_lo, uint32_t key_hi,
                                  float range, cudaStream_t s);
cudaError_t launch_sweep(const EpochArgs& a, int grid, cudaStream_t s);
int sweep_grid(int d, int bins, int sm_count);
cudaError_t launch_update(const UpdateArgs& a, int grid, cudaStream_t s);
cudaError_t launch_sample(const EpochArgs& a, uint32_t tag, int32_t* out, cudaStream_t s);
cudaError_t launch_loss(const EpochArgs& a, cudaStream_t s);
cudaError_t launch_is_edge(const unsigned long long* keys, unsigned long long bucket_mask,
                           const int32_t* pairs, int64_t count, uint8_t* out, cudaStream_t s);
cudaError_t launch_fit_sigma(const float* hist, int32_t bins, float hist_max, float mu,
                             float* sigma_inout, cudaStream_t s);

}  // namespace gempe
