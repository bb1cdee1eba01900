// CUDA kernels of the GEMPE epoch (sm_103a).
//
//  k_hash_build    exact edge set (replaces the lossy byte map of Sec. III.C)
//  k_init          initial positions, uniform random (Fig. 4)
//  k_sweep         one epoch's pair sweep: edge parabolas (Eq. 4/5), sampled
//                  non-edges with retry-until-non-edge (Fig. 2), Eq. 3 terms
//                  reduced per vertex, distance histograms (Sec. III.F)
//  k_update        x_i := y_i / z_i (Fig. 4), sigma bisection (Sec. III.F)
//  k_loss          sampled predictive entropy (Eq. 2) with FP64 sums
//  k_sample        the sampler alone (inspection)
//  k_is_edge       membership probes (inspection)
#include "device_math.cuh"
#include "engine.cuh"

namespace gempe {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Graph set-up
// ---------------------------------------------------------------------------
__global__ void k_hash_build(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                             int32_t n, unsigned long long* keys, unsigned long long bucket_mask,
                             int32_t* fail_flag) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const unsigned long long slot_mask = 4ull * bucket_mask + 3ull;
    for (int i = warp; i < n; i += n_warps) {
        const int b = row_ptr[i], e = row_ptr[i + 1];
        for (int s = b + lane; s < e; s += 32) {
            const unsigned long long key = edge_key(i, col_idx[s]);
            unsigned long long slot = 4ull * (mix64(key) & bucket_mask);
            bool done = false;
            for (unsigned long long probe = 0; probe <= slot_mask; ++probe) {
                const unsigned long long prev = atomicCAS(keys + slot, kEmptyKey, key);
                if (prev == kEmptyKey || prev == key) { done = true; break; }
                slot = (slot + 1) & slot_mask;
            }
            if (!done) atomicExch(fail_flag, 1);
        }
    }
}

__global__ void k_init(float* __restrict__ x, int32_t n, int32_t d, uint32_t key_lo, uint32_t key_hi,
                       float range) {
    const int quads = (d + 3) / 4;
    const long long total = (long long)n * quads;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / quads), q = (int)(t % quads);
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)q, 0u, kTagInit), key_lo, key_hi);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int c = 4 * q + w;
            if (c < d) {
                // (r >> 8) * 2^-23 - 1 is exact in FP32; one rounding for the range
                const float unit = (float)(word_of(r, w) >> 8) * 1.1920928955078125e-7f - 1.0f;
                x[(size_t)i * d + c] = unit * range;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Coordinate chunks: a pair is handled by G lanes, lane gl owning the P = D/G
// coordinates [gl*P, gl*P + P).
// ---------------------------------------------------------------------------
template <int D, int P>
__device__ __forceinline__ void load_chunk(const float* __restrict__ x, int row, int gl, float* out) {
    const float* p = x + (size_t)row * D + gl * P;
    if constexpr (P % 4 == 0) {
#pragma unroll
        for (int c = 0; c < P; c += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p + c));
            out[c] = v.x; out[c + 1] = v.y; out[c + 2] = v.z; out[c + 3] = v.w;
        }
    } else if constexpr (P == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        out[0] = v.x; out[1] = v.y;
    } else {
#pragma unroll
        for (int c = 0; c < P; ++c) out[c] = __ldg(p + c);
    }
}

// acc row layout: D values then z, padded to a multiple of 4 floats.
template <int D, int G, int P>
__device__ __forceinline__ void acc_add(float* row, int gl, const float* v, float z) {
    if constexpr (D <= 3) {   // G == 1: the whole row is one float4 {v..., z, 0...}
        float4 q;
        q.x = v[0];
        q.y = (D > 1) ? v[(D > 1) ? 1 : 0] : z;
        q.z = (D > 2) ? v[(D > 2) ? 2 : 0] : (D == 2 ? z : 0.0f);
        q.w = (D == 3) ? z : 0.0f;
        atomicAdd(reinterpret_cast<float4*>(row), q);
    } else {
        float* p = row + gl * P;
        if constexpr (P % 4 == 0) {
#pragma unroll
            for (int c = 0; c < P; c += 4)
                atomicAdd(reinterpret_cast<float4*>(p + c), make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]));
        } else if constexpr (P == 2) {
            atomicAdd(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
        } else {
#pragma unroll
            for (int c = 0; c < P; ++c) atomicAdd(p + c, v[c]);
        }
        if (gl == 0) atomicAdd(row + D, z);
    }
}

// Draw the accepted partner of sample slot t of vertex i (Fig. 2: redraw while
// the pair is an edge; also redraw g == i), or -1 after max_retries draws.
__device__ __forceinline__ int sample_partner(const EpochArgs& a, int i, int epoch, int t, uint32_t tag,
                                              unsigned& rejected) {
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    for (int att = 0; att < a.max_retries; ++att) {
        if ((att & 3) == 0)
            r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)epoch, (uint32_t)t, tag | ((uint32_t)att >> 2)),
                              a.key_lo, a.key_hi);
        const int g = draw_vertex(word_of(r, att & 3), (uint32_t)a.n);
        if (g != i && !hash_contains(a.keys, a.bucket_mask, edge_key(i, g))) return g;
        ++rejected;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// The pair sweep (one warp per work unit).
// ---------------------------------------------------------------------------
template <int D, int G, bool REC>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(const EpochArgs a) {
    constexpr int P = D / G;
    constexpr int PAIRS = 32 / G;
    extern __shared__ float s_hist[];   // [2][bins]
    __shared__ unsigned long long s_stats[3];
    for (int t = threadIdx.x; t < 2 * a.bins; t += blockDim.x) s_hist[t] = 0.0f;
    if (threadIdx.x < 3) s_stats[threadIdx.x] = 0ull;
    __syncthreads();

    const float sigma = a.st->sigma;
    const int epoch = a.st->epoch;
    const PairConsts K = make_pair_consts(a.mu, sigma, a.w_formula == 1, a.clamp_neg_d);
    const int lane = threadIdx.x & 31;
    const int grp = lane / G;
    const int gl = lane % G;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    unsigned n_acc = 0, n_rej = 0, n_exh = 0;

    for (int it = warp; it < a.n_items; it += n_warps) {
        const int4 item = __ldg(a.items + it);
        const int i = item.x, p0 = item.y, p1 = item.z;
        const bool has_samples = (item.w & 1) && a.k > 0;
        const int e0 = __ldg(a.row_ptr + i);
        const int deg = __ldg(a.row_ptr + i + 1) - e0;
        float xi[P];
        load_chunk<D, P>(a.x, i, gl, xi);

        // Sampled non-edges of this vertex: lane t < k owns slot t.
        int g_mine = -1;
        float omega = 0.0f;
        if (has_samples) {
            if (lane < a.k) {
                g_mine = sample_partner(a, i, epoch, lane, kTagEpoch, n_rej);
                if (g_mine < 0) ++n_exh;
            }
            const int k_acc = __popc(__ballot_sync(kFull, g_mine >= 0));
            n_acc += (lane == 0) ? k_acc : 0;
            // histogram weight: sum over samples estimates the unordered non-edge count
            omega = k_acc ? (float)(a.n - 1 - deg) / (2.0f * (float)k_acc) : 0.0f;
            if (REC && lane < a.k) a.record[(size_t)i * a.k + lane] = g_mine;
        }

        const int ne = p1 - p0;
        const int total = ne + (has_samples ? a.k : 0);
        float dacc[P];
#pragma unroll
        for (int c = 0; c < P; ++c) dacc[c] = 0.0f;
        float zacc = 0.0f;
        for (int base = 0; base < total; base += PAIRS) {
            const int q = base + grp;
            const bool active = q < total;
            const bool is_edge = q < ne;
            const int sidx = q - ne;
            const int gs = __shfl_sync(kFull, g_mine, (sidx >= 0 && sidx < 32) ? sidx : 0);
            int j = -1;
            if (active) j = is_edge ? __ldg(a.col_idx + e0 + p0 + q) : gs;
            const bool valid = active && j >= 0;
            float xj[P];
            if (valid) {
                load_chunk<D, P>(a.x, j, gl, xj);
            } else {
#pragma unroll
                for (int c = 0; c < P; ++c) xj[c] = xi[c];
            }
            float diff[P];
            float ss = 0.0f;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                diff[c] = xi[c] - xj[c];
                ss = fmaf(diff[c], diff[c], ss);
            }
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
            if (valid) {
                const float delta = sqrtf(ss);
                const PairTerm t = pair_term(delta, is_edge, K);
#pragma unroll
                for (int c = 0; c < P; ++c) dacc[c] = fmaf(t.c, diff[c], dacc[c]);
                if (gl == 0) zacc += t.w;
                if (!is_edge && a.symmetric) {
                    float pv[P];
#pragma unroll
                    for (int c = 0; c < P; ++c) pv[c] = -t.c * diff[c];
                    acc_add<D, G, P>(a.acc + (size_t)j * a.acc_stride, gl, pv, t.w);
                }
                if (gl == 0) {
                    const int bin = min((int)(delta * a.hist_scale), a.bins - 1);
                    if (is_edge) {
                        if (j > i) atomicAdd(s_hist + bin, 1.0f);
                    } else {
                        atomicAdd(s_hist + a.bins + bin, omega);
                    }
                }
            }
        }
        // per-vertex reduction: coordinates over lanes with equal gl, z over all
#pragma unroll
        for (int o = 16; o >= G; o >>= 1)
#pragma unroll
            for (int c = 0; c < P; ++c) dacc[c] += __shfl_xor_sync(kFull, dacc[c], o);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) zacc += __shfl_xor_sync(kFull, zacc, o);
        if (lane < G) acc_add<D, G, P>(a.acc + (size_t)i * a.acc_stride, gl, dacc, zacc);
    }

    // statistics: warp sums, then one shared atomic per warp
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        n_acc += __shfl_xor_sync(kFull, n_acc, o);
        n_rej += __shfl_xor_sync(kFull, n_rej, o);
        n_exh += __shfl_xor_sync(kFull, n_exh, o);
    }
    if (lane == 0) {
        atomicAdd(&s_stats[0], (unsigned long long)n_acc);
        atomicAdd(&s_stats[1], (unsigned long long)n_rej);
        atomicAdd(&s_stats[2], (unsigned long long)n_exh);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * a.bins; t += blockDim.x) {
        const float v = s_hist[t];
        if (v != 0.0f) atomicAdd(a.hist + t, v);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&a.st->accepted, s_stats[0]);
        atomicAdd(&a.st->rejected, s_stats[1]);
        atomicAdd(&a.st->exhausted, s_stats[2]);
        atomicAdd(&a.st->draws, s_stats[0] + s_stats[1]);
    }
}

// ---------------------------------------------------------------------------
// Sec. III.F: dPE/dsigma on the histogram (sign only matters) and bisection
// in log sigma, executed by one whole block.
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q];
    return s;
}

// sum_b c_e[b] (-u h(u)) + c_n[b] (u g(u)),  u = (centre_b - mu)/sigma, g(u) = h(-u)
__device__ double dpe_sign_sum(const float* hist, int bins, float bin_w, float mu, float sigma, double* red) {
    double part = 0.0;
    const float inv_s = 1.0f / sigma;
    for (int b = threadIdx.x; b < bins; b += blockDim.x) {
        const float ce = hist[b], cn = hist[bins + b];
        if (ce == 0.0f && cn == 0.0f) continue;
        const float u = (((float)b + 0.5f) * bin_w - mu) * inv_s;
        float h, T;
        if (ce != 0.0f) {
            mills(u, h, T);
            part += (double)ce * (double)(-u * h);
        }
        if (cn != 0.0f) {
            mills(-u, h, T);
            part += (double)cn * (double)(u * h);
        }
    }
    return block_sum(part, red);
}

__device__ float block_fit_sigma(const float* hist, int bins, float hist_max, float mu, double* red) {
    const float bin_w = hist_max / (float)bins;
    double lo = 1e-3, hi = 1e3;
    const double flo = dpe_sign_sum(hist, bins, bin_w, mu, (float)lo, red);
    const double fhi = dpe_sign_sum(hist, bins, bin_w, mu, (float)hi, red);
    if ((flo > 0.0) == (fhi > 0.0)) return (float)((flo > 0.0) ? lo : hi);
    const bool lo_pos = flo > 0.0;
    for (int it = 0; it < kSigmaIters; ++it) {
        const double mid = sqrt(lo * hi);
        const double fm = dpe_sign_sum(hist, bins, bin_w, mu, (float)mid, red);
        if ((fm > 0.0) == lo_pos) lo = mid; else hi = mid;
    }
    return (float)sqrt(lo * hi);
}

__global__ void __launch_bounds__(kUpdateThreads) k_update(const UpdateArgs a) {
    if (blockIdx.x == 0) {
        __shared__ double red[32];
        const int epoch = a.st->epoch;
        if (a.sigma_every > 0 && ((epoch + 1) % a.sigma_every) == 0) {
            const float s = block_fit_sigma(a.hist, a.bins, a.hist_max, a.mu, red);
            __syncthreads();
            if (threadIdx.x == 0) a.st->sigma = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * a.bins; t += blockDim.x) a.hist[t] = 0.0f;
        if (threadIdx.x == 0) a.st->epoch = epoch + 1;
        return;
    }
    const int stride = (gridDim.x - 1) * blockDim.x;
    for (int v = (blockIdx.x - 1) * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        float* row = a.acc + (size_t)v * a.acc_stride;
        float* xv = a.x + (size_t)v * a.d;
        const float z = row[a.d];
        if (z >= a.z_min) {
            const float inv_z = 1.0f / z;
            bool bad = false;
            for (int c = 0; c < a.d; ++c) {
                const float xn = fmaf(row[c], inv_z, xv[c]);
                if (!isfinite(xn)) bad = true;
            }
            if (!bad) {
                for (int c = 0; c < a.d; ++c) xv[c] = fmaf(row[c], inv_z, xv[c]);
            } else {
                atomicCAS(&a.st->status, 0, -6 /* GEMPE_E_NUMERIC */);
            }
        }
        for (int c = 0; c < a.acc_stride; c += 4)
            *reinterpret_cast<float4*>(row + c) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

__global__ void k_fit_sigma(const float* hist, int bins, float hist_max, float mu, float* sigma) {
    __shared__ double red[32];
    const float s = block_fit_sigma(hist, bins, hist_max, mu, red);
    if (threadIdx.x == 0) *sigma = s;
}

// ---------------------------------------------------------------------------
// Inspection kernels and the loss estimator
// ---------------------------------------------------------------------------
__global__ void k_sample(const EpochArgs a, uint32_t tag, int32_t* out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int epoch = a.st->epoch;
    for (int i = warp; i < a.n; i += n_warps) {
        unsigned rej = 0;
        if (lane < a.k) out[(size_t)i * a.k + lane] = sample_partner(a, i, epoch, lane, tag, rej);
    }
}

template <int D, int G>
__global__ void __launch_bounds__(256) k_loss(const EpochArgs a) {
    constexpr int P = D / G;
    constexpr int PAIRS = 32 / G;
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const float sigma = a.st->sigma;
    const int epoch = a.st->epoch;
    const float inv_sigma = 1.0f / sigma;
    double sum = 0.0;
    for (int i = warp; i < a.n; i += n_warps) {
        const int e0 = __ldg(a.row_ptr + i);
        const int deg = __ldg(a.row_ptr + i + 1) - e0;
        float xi[P];
        load_chunk<D, P>(a.x, i, gl, xi);
        int g_mine = -1;
        unsigned rej = 0;
        if (lane < a.k) g_mine = sample_partner(a, i, epoch, lane, kTagLoss, rej);
        const int k_acc = __popc(__ballot_sync(kFull, g_mine >= 0));
        const double omega = k_acc ? (double)(a.n - 1 - deg) / (2.0 * k_acc) : 0.0;
        const int total = deg + a.k;
        for (int base = 0; base < total; base += PAIRS) {
            const int q = base + grp;
            const bool is_edge = q < deg;
            const int sidx = q - deg;
            const int gs = __shfl_sync(kFull, g_mine, (sidx >= 0 && sidx < 32) ? sidx : 0);
            int j = -1;
            if (q < total) j = is_edge ? __ldg(a.col_idx + e0 + q) : gs;
            const bool valid = (q < total) && j >= 0 && (!is_edge || j > i);
            float xj[P];
            if (valid) {
                load_chunk<D, P>(a.x, j, gl, xj);
            } else {
#pragma unroll
                for (int c = 0; c < P; ++c) xj[c] = xi[c];
            }
            float ss = 0.0f;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const float df = xi[c] - xj[c];
                ss = fmaf(df, df, ss);
            }
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
            if (valid && gl == 0) {
                const float u = (sqrtf(ss) - a.mu) * inv_sigma;
                const float dl = neg_log2_Q(is_edge ? u : -u);
                sum += is_edge ? (double)dl : omega * (double)dl;
            }
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if (lane == 0 && sum != 0.0) atomicAdd(&a.st->loss_sum, sum);
}

__global__ void k_is_edge(const unsigned long long* keys, unsigned long long bucket_mask,
                          const int32_t* pairs, int64_t count, uint8_t* out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = hash_contains(keys, bucket_mask, edge_key(pairs[2 * p], pairs[2 * p + 1])) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Dispatch on the dimension: lanes per pair G grows with d so that each lane
// gathers at most 8 coordinates (16-byte vector loads from d = 8 on).
// ---------------------------------------------------------------------------
#define GEMPE_DIMS(X) X(1, 1) X(2, 1) X(3, 1) X(4, 1) X(8, 2) X(16, 4) X(32, 8) X(64, 16) X(128, 32) X(256, 32)

template <int D, int G>
cudaError_t sweep_for(const EpochArgs& a, int grid, cudaStream_t s) {
    // at most 2 x 4096 bins x 4 B = 32 KiB: within the default dynamic shared memory limit
    const size_t smem = 2 * (size_t)a.bins * sizeof(float);
    if (a.record) k_sweep<D, G, true><<<grid, kSweepThreads, smem, s>>>(a);
    else k_sweep<D, G, false><<<grid, kSweepThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int D, int G>
cudaError_t loss_for(const EpochArgs& a, int grid, cudaStream_t s) {
    k_loss<D, G><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int acc_stride_for(int d) { return ((d + 1) + 3) / 4 * 4; }

bool supported_dim(int d) {
    switch (d) {
#define GEMPE_CASE(D, G) case D:
        GEMPE_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        return true;
        default: return false;
    }
}

template <int D, int G>
int sweep_blocks_per_sm(int bins) {
    int blocks = 0;
    const size_t smem = 2 * (size_t)bins * sizeof(float);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep<D, G, false>, kSweepThreads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        blocks = 1;
    }
    return blocks < 1 ? 1 : blocks;
}

// One resident wave: SM count x blocks that fit per SM (the sweep strides
// over its work units, so a second wave would only add histogram merges).
int sweep_grid(int d, int bins, int sm_count) {
    switch (d) {
#define GEMPE_CASE(D, G) case D: return sm_count * sweep_blocks_per_sm<D, G>(bins);
        GEMPE_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        default: return sm_count;
    }
}

cudaError_t launch_hash_build(const int32_t* row_ptr, const int32_t* col_idx, int32_t n,
                              unsigned long long* keys, unsigned long long bucket_mask,
                              int32_t* fail_flag, cudaStream_t s) {
    const int warps = 8;
    int grid = (n + warps - 1) / warps;
    if (grid > 65535) grid = 65535;
    if (grid < 1) grid = 1;
    k_hash_build<<<grid, 32 * warps, 0, s>>>(row_ptr, col_idx, n, keys, bucket_mask, fail_flag);
    return cudaGetLastError();
}

cudaError_t launch_init_positions(float* x, int32_t n, int32_t d, uint32_t key_lo, uint32_t key_hi,
                                  float range, cudaStream_t s) {
    const long long total = (long long)n * ((d + 3) / 4);
    long long grid = (total + 255) / 256;
    if (grid > 65535) grid = 65535;
    if (grid < 1) grid = 1;
    k_init<<<(int)grid, 256, 0, s>>>(x, n, d, key_lo, key_hi, range);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const EpochArgs& a, int grid, cudaStream_t s) {
    switch (a.d) {
#define GEMPE_CASE(D, G) case D: return sweep_for<D, G>(a, grid, s);
        GEMPE_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_loss(const EpochArgs& a, cudaStream_t s) {
    int grid = (a.n + 7) / 8;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    switch (a.d) {
#define GEMPE_CASE(D, G) case D: return loss_for<D, G>(a, grid, s);
        GEMPE_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_update(const UpdateArgs& a, int grid, cudaStream_t s) {
    k_update<<<grid, kUpdateThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sample(const EpochArgs& a, uint32_t tag, int32_t* out, cudaStream_t s) {
    int grid = (a.n + 7) / 8;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    k_sample<<<grid, 256, 0, s>>>(a, tag, out);
    return cudaGetLastError();
}

cudaError_t launch_is_edge(const unsigned long long* keys, unsigned long long bucket_mask,
                           const int32_t* pairs, int64_t count, uint8_t* out, cudaStream_t s) {
    long long grid = (count + 255) / 256;
    if (grid > 65535) grid = 65535;
    if (grid < 1) grid = 1;
    k_is_edge<<<(int)grid, 256, 0, s>>>(keys, bucket_mask, pairs, count, out);
    return cudaGetLastError();
}

cudaError_t launch_fit_sigma(const float* hist, int32_t bins, float hist_max, float mu,
                             float* sigma_inout, cudaStream_t s) {
    k_fit_sigma<<<1, kUpdateThreads, 0, s>>>(hist, bins, hist_max, mu, sigma_inout);
    return cudaGetLastError();
}

}  // namespace gempe
