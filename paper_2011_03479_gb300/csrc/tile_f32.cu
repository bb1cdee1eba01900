// FP32 tiles of block-sampled non-edges: the plain FP32 form of the
// representation-learning workload (block sampling, Sec. III.C's non-edge
// sampling cut into tiles; pair terms of Eq. 3-5).
//
// Each tile of kBlockT = 128 consecutive vertices meets the kBlockP = 64
// partners k_block_sampler drew for it; a pair is masked when the partner is
// the vertex itself or a neighbour.  One CTA of 256 threads per tile:
//
//   (1) the anchors' rows X_T (128 x D) and the partners' rows X_P (64 x D),
//       FP32, are staged in shared memory (cp.async);
//   (2) every pair's squared distance is summed from coordinate differences,
//       as the sweep and the oracle form it (no |x|^2 + |y|^2 - 2 x.y
//       cancellation): thread (ta, tp) holds the pairs of anchors ta + 16 r
//       and partners tp + 16 j, in two passes of 4 x 4 pairs, with packed
//       FP32 pairs (f32x2.cuh: even and odd coordinates in the two halves);
//   (3) after each pass, the pair terms (c, w) of its unmasked pairs (c the
//       coefficient of x_self - x_other in y - z x, w the weight added to z),
//       C into shared memory, the row sums of C and W by shuffles; the column
//       sums by one shared-memory addition per warp and partner; the
//       distances go to the histograms;
//   (4) A = C X_P and B = C^T X_T by register tiles of packed FP32 FMAs, then
//         y_i - z_i x_i += x_i rowsum(C)_i - A_i,   z_i += rowsum(W)_i,
//         y_g - z_g x_g += x_g colsum(C)_g - B_g,   z_g += colsum(W)_g
//       by vector atomics (partners only in the symmetric form).
//
// Every product and sum is FP32 on the CUDA cores; only the order of the
// additions differs from the per-pair evaluation of the sweep.  The global
// words of the next tile's staging are loaded while a tile runs, and the
// pair-term loop stays rolled over anchor rows (its squared distances wait
// in C's slots), which keeps the kernel's code small.
#include <algorithm>

#include "device_math.cuh"
#include "engine.cuh"
#include "f32x2.cuh"
#include "hist.cuh"
#include "tile_ahead.cuh"

namespace gempe {

namespace {

constexpr int kF32Threads = 256;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void copy16_async(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem));
}
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}

template <int D>
struct TileF32 {
    static constexpr int R = D + 4;          // row stride of XT and XP (floats): conflict-free float4 rows
    static constexpr int RC = kBlockP + 4;   // row stride of C
    float xt[kBlockT * R];
    float xp[kBlockP * R];
    float c[kBlockT * RC];
    float rsum_c[kBlockT], rsum_w[kBlockT];
    float csum_c[kBlockP], csum_w[kBlockP];
    unsigned long long mask[kBlockT];
    int deg[kBlockT], kacc[kBlockT];
    int part[kBlockP];
    MillsCoef mills[kMillsIntervals];   // the Mills-ratio table (pair terms)
};

// CK consecutive floats of shared memory (CK = 1, 2, 4 or 8; 4-float chunks aligned).
template <int CK>
__device__ __forceinline__ void load_chunk(const float* p, float (&v)[CK]) {
    if constexpr (CK == 1) {
        v[0] = p[0];
    } else if constexpr (CK == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < CK / 4; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(p + 4 * q);
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    }
}

// acc[0 .. CK) += v by vector atomics.
template <int CK>
__device__ __forceinline__ void atomic_add_chunk(float* acc, const float (&v)[CK]) {
    if constexpr (CK == 1) {
        atomicAdd(acc, v[0]);
    } else if constexpr (CK == 2) {
        atomicAdd(reinterpret_cast<float2*>(acc), make_float2(v[0], v[1]));
    } else {
#pragma unroll
        for (int q = 0; q < CK / 4; ++q)
            atomicAdd(reinterpret_cast<float4*>(acc + 4 * q), make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    }
}

__device__ __forceinline__ float comp(const float4& v, int q) { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); }

template <int D>
__global__ void __launch_bounds__(kF32Threads, D <= 64 ? 2 : 1) k_tile_f32(const EpochArgs a) {
    using L = TileF32<D>;
    constexpr int R = L::R, RC = L::RC;
    constexpr int CK = D / 16;   // coordinates per thread in the two sums
    extern __shared__ __align__(16) unsigned char smem_raw[];
    L& sm = *reinterpret_cast<L*>(smem_raw);
    unsigned int* hist_base = reinterpret_cast<unsigned int*>(smem_raw + sizeof(L));
    int it0, it1, istep, home;
    if (a.blocked) {
        it0 = (int)((long long)a.n_tile_items * blockIdx.x / gridDim.x);
        it1 = (int)((long long)a.n_tile_items * (blockIdx.x + 1) / gridDim.x);
        istep = 1;
        home = it0 < it1 ? __ldg(&a.tile_items[it0].y) : -1;
    } else {
        it0 = blockIdx.x;
        it1 = a.n_tile_items;
        istep = gridDim.x;
        home = a.n_graphs == 1 ? 0 : -1;
    }
    const BlockHist hist = block_hist(hist_base, a.bins, home);
    __shared__ unsigned int s_used, s_tile_used;
    const int tid = threadIdx.x, lane = tid & 31;
    const int ta = tid >> 4, tp = tid & 15;   // anchor group / partner (or coordinate) group
    for (int t = tid; t < kMillsIntervals; t += blockDim.x) sm.mills[t].lh = __ldg(&a.mills[t].lh);
    for (int t = tid; t < a.bins; t += blockDim.x) {
        hist.he[t] = 0u;
        hist.hc[t] = 0u;
        hist.hd[t] = 0u;
    }
    if (tid == 0) {
        s_used = 0u;
        s_tile_used = 0u;
    }

    constexpr int CH = D / 4;   // 16-byte chunks of a row
    using Ahead = TileAhead<CH, kF32Threads>;
    Ahead nxt;
    if (it0 < it1) nxt = tile_ahead<CH, kF32Threads>(a, it0, tid);
    for (int it = it0; it < it1; it += istep) {
        const Ahead cur = nxt;
        const int graph = cur.graph, v0 = cur.v0, nv = cur.nv;
        const float sigma = a.gst[graph].sigma;
        const int epoch = a.gst[graph].epoch;
        const NonEdgeConsts NK =
            make_nonedge_consts(make_pair_consts(a.mu, sigma, a.w_formula == 1, a.clamp_neg_d, sm.mills));
        unsigned long long* bmask = a.block_mask + (size_t)(epoch & 1) * (size_t)a.rows;

        // ---- (1) stage rows, partners, masks ----
        __syncthreads();   // the previous tile's shared data is no longer read
        if (tid < kBlockP) {
            sm.part[tid] = cur.part;
            sm.csum_c[tid] = 0.0f;
            sm.csum_w[tid] = 0.0f;
        }
        for (int q = tid; q < kBlockT * CH; q += blockDim.x) {
            const int r = q / CH, c4 = q - r * CH;
            float* dst = sm.xt + r * R + 4 * c4;
            if (r < nv) copy16_async(dst, a.x + (size_t)(v0 + r) * D + 4 * c4);
            else *reinterpret_cast<float4*>(dst) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int j = 0; j < Ahead::kChunks; ++j) {
            const int q = tid + kF32Threads * j;
            if (q < kBlockP * CH) {
                const int r = q / CH, c4 = q - r * CH;
                copy16_async(sm.xp + r * R + 4 * c4, a.x + (size_t)cur.pid[j] * D + 4 * c4);
            }
        }
        if (tid < kBlockT) {
            const int v = tid;
            if (v < nv) {
                const unsigned long long m = cur.m;
                bmask[v0 + v] = 0ull;   // read once: the buffer starts empty for the epoch two ahead
                sm.mask[v] = m;
                sm.deg[v] = cur.deg;
                sm.kacc[v] = kBlockP - __popcll(m);
                atomicAdd(&s_tile_used, (unsigned)(kBlockP - __popcll(m)));
            } else {
                sm.mask[v] = ~0ull;
                sm.deg[v] = 0;
                sm.kacc[v] = 0;
            }
        }
        if (it + istep < it1) nxt = tile_ahead<CH, kF32Threads>(a, it + istep, tid);
        copy_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            if (s_tile_used) {
                if (graph == home) s_used += s_tile_used;
                else atomicAdd(&a.gst[graph].used, (unsigned long long)s_tile_used);
            }
            s_tile_used = 0u;
        }

        // ---- (2, 3) in two passes over anchor halves h: anchors ta + 16 (4 h + r),
        // partners tp + 16 j; squared distances summed in packed pairs (even and odd
        // coordinates in the two halves), then the pair terms, C, row sums and the
        // histograms of the half ----
        float cc[4], cw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cc[j] = cw[j] = 0.0f;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            f2 acc2[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc2[r][j] = 0ull;
#pragma unroll 2
            for (int kc = 0; kc < D / 4; ++kc) {
                ulonglong2 b[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    b[j] = *reinterpret_cast<const ulonglong2*>(sm.xp + (tp + 16 * j) * R + 4 * kc);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const ulonglong2 av =
                        *reinterpret_cast<const ulonglong2*>(sm.xt + (ta + 16 * (4 * h + r)) * R + 4 * kc);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        f2 t = f2_sub(av.x, b[j].x);
                        acc2[r][j] = f2_fma(t, t, acc2[r][j]);
                        t = f2_sub(av.y, b[j].y);
                        acc2[r][j] = f2_fma(t, t, acc2[r][j]);
                    }
                }
            }
            // the squared distances wait in C's slots (each thread reads back
            // only its own), so that the term loop below stays rolled over r
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float lo, hi;
                    f2_unpack(acc2[r][j], lo, hi);
                    sm.c[(ta + 16 * (4 * h + r)) * RC + tp + 16 * j] = lo + hi;
                }
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
                const int i = ta + 16 * (4 * h + r);
                const unsigned long long mk = sm.mask[i];
                const int di = sm.deg[i], ki = sm.kacc[i];
                float cv[4], wv[4];
                int bn[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {   // the four terms without branches (masked pairs give 0)
                    const int p = tp + 16 * j;
                    const bool live = !((mk >> p) & 1ull);
                    float delta, inv_delta;
                    dist_of(sm.c[i * RC + p], delta, inv_delta);
                    const PairTerm pt = nonedge_term<false>(delta, inv_delta, NK);
                    cv[j] = live ? pt.c : 0.0f;
                    wv[j] = live ? pt.w : 0.0f;
                    bn[j] = live ? min((int)(delta * a.hist_scale), a.bins - 1) : -1;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (bn[j] >= 0) hist_sample(hist, a, graph, bn[j], di, ki, kBlockP);
                float rc = 0.0f, rw = 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    sm.c[i * RC + tp + 16 * j] = cv[j];
                    rc += cv[j];
                    rw += wv[j];
                    cc[j] += cv[j];
                    cw[j] += wv[j];
                }
                // row sums over the 16 lanes of a half-warp (one anchor group)
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    rc += __shfl_xor_sync(0xFFFFFFFFu, rc, o);
                    rw += __shfl_xor_sync(0xFFFFFFFFu, rw, o);
                }
                if (tp == 0) {
                    sm.rsum_c[i] = rc;
                    sm.rsum_w[i] = rw;
                }
            }
        }
        // column sums: the warp's two anchor groups, then one shared-memory
        // addition per warp and partner
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cc[j] += __shfl_xor_sync(0xFFFFFFFFu, cc[j], 16);
            cw[j] += __shfl_xor_sync(0xFFFFFFFFu, cw[j], 16);
        }
        if (lane < 16) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                atomicAdd(&sm.csum_c[tp + 16 * j], cc[j]);
                atomicAdd(&sm.csum_w[tp + 16 * j], cw[j]);
            }
        }
        __syncthreads();   // C for the products

        // ---- (4a) A = C X_P: anchors ta + 16 r, coordinates CK tp .. ----
        {
            float A[8][CK];
            if constexpr (CK >= 2) {   // packed coordinate pairs, c broadcast to both halves
                f2 A2[8][CK / 2];
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int e = 0; e < CK / 2; ++e) A2[r][e] = 0ull;
#pragma unroll 8
                for (int pc = 0; pc < kBlockP / 4; ++pc) {
                    f2 xr[4][CK / 2];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int e = 0; e < CK / 2; ++e)
                            xr[q][e] = *reinterpret_cast<const f2*>(sm.xp + (4 * pc + q) * R + CK * tp + 2 * e);
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const float4 c4 = *reinterpret_cast<const float4*>(sm.c + (ta + 16 * r) * RC + 4 * pc);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float cq = comp(c4, q);
                            const f2 cc = f2_pack(cq, cq);
#pragma unroll
                            for (int e = 0; e < CK / 2; ++e) A2[r][e] = f2_fma(cc, xr[q][e], A2[r][e]);
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int e = 0; e < CK / 2; ++e) f2_unpack(A2[r][e], A[r][2 * e], A[r][2 * e + 1]);
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r) A[r][0] = 0.0f;
#pragma unroll 2
                for (int pc = 0; pc < kBlockP / 4; ++pc) {
                    float xr[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) xr[q] = sm.xp[(4 * pc + q) * R + tp];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const float4 c4 = *reinterpret_cast<const float4*>(sm.c + (ta + 16 * r) * RC + 4 * pc);
#pragma unroll
                        for (int q = 0; q < 4; ++q) A[r][0] = fmaf(comp(c4, q), xr[q], A[r][0]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = ta + 16 * r;
                if (i >= nv || sm.kacc[i] == 0) continue;
                const float rs = sm.rsum_c[i];
                float xi[CK], o[CK];
                load_chunk<CK>(sm.xt + i * R + CK * tp, xi);
#pragma unroll
                for (int e = 0; e < CK; ++e) o[e] = xi[e] * rs - A[r][e];
                float* row = a.acc + (size_t)(v0 + i) * a.acc_stride;
                atomic_add_chunk<CK>(row + CK * tp, o);
                if (tp == 0) atomicAdd(row + D, sm.rsum_w[i]);
            }
        }

        // ---- (4b) B = C^T X_T: partners 4 ta .. 4 ta + 3, coordinates CK tp .. ----
        if (a.symmetric) {
            float Bv[4][CK];
            if constexpr (CK >= 2) {
                f2 B2[4][CK / 2];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < CK / 2; ++e) B2[q][e] = 0ull;
#pragma unroll 4
                for (int i = 0; i < nv; ++i) {   // rows of vertices past the graph have c = 0
                    const float4 c4 = *reinterpret_cast<const float4*>(sm.c + i * RC + 4 * ta);
                    f2 xi[CK / 2];
#pragma unroll
                    for (int e = 0; e < CK / 2; ++e) xi[e] = *reinterpret_cast<const f2*>(sm.xt + i * R + CK * tp + 2 * e);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float cq = comp(c4, q);
                        const f2 cc = f2_pack(cq, cq);
#pragma unroll
                        for (int e = 0; e < CK / 2; ++e) B2[q][e] = f2_fma(cc, xi[e], B2[q][e]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < CK / 2; ++e) f2_unpack(B2[q][e], Bv[q][2 * e], Bv[q][2 * e + 1]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) Bv[q][0] = 0.0f;
#pragma unroll 4
                for (int i = 0; i < nv; ++i) {
                    const float4 c4 = *reinterpret_cast<const float4*>(sm.c + i * RC + 4 * ta);
                    const float xi = sm.xt[i * R + tp];
#pragma unroll
                    for (int q = 0; q < 4; ++q) Bv[q][0] = fmaf(comp(c4, q), xi, Bv[q][0]);
                }
            }
            __syncthreads();   // the column sums
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int p = 4 * ta + q;
                const float cs = sm.csum_c[p], ws = sm.csum_w[p];
                if (cs == 0.0f && ws == 0.0f) continue;   // every pair of the partner masked
                float xg[CK], o[CK];
                load_chunk<CK>(sm.xp + p * R + CK * tp, xg);
#pragma unroll
                for (int e = 0; e < CK; ++e) o[e] = xg[e] * cs - Bv[q][e];
                float* row = a.acc + (size_t)sm.part[p] * a.acc_stride;
                atomic_add_chunk<CK>(row + CK * tp, o);
                if (tp == 0) atomicAdd(row + D, ws);
            }
        }
    }
    __syncthreads();
    hist_merge(hist, a);
    if (tid == 0 && s_used && home >= 0) atomicAdd(&a.gst[home].used, (unsigned long long)s_used);
}

template <int D>
size_t f32_smem(int bins) {
    return sizeof(TileF32<D>) + hist_smem_bytes(bins) / 4 * 3;   // no per-slot weights in block sampling
}

}  // namespace

bool tile_dim_f32(int d) { return d == 16 || d == 32 || d == 64 || d == 128; }

size_t tile_f32_smem_bytes(int d, int bins) {
    switch (d) {
        case 16: return f32_smem<16>(bins);
        case 32: return f32_smem<32>(bins);
        case 64: return f32_smem<64>(bins);
        case 128: return f32_smem<128>(bins);
        default: return 0;
    }
}

cudaError_t prepare_tile_f32_kernel(int d, int bins) {
    const int smem = (int)tile_f32_smem_bytes(d, bins);
    switch (d) {
        case 16: return raise_smem_limit((const void*)k_tile_f32<16>, smem);
        case 32: return raise_smem_limit((const void*)k_tile_f32<32>, smem);
        case 64: return raise_smem_limit((const void*)k_tile_f32<64>, smem);
        case 128: return raise_smem_limit((const void*)k_tile_f32<128>, smem);
        default: return cudaErrorInvalidValue;
    }
}

int tile_f32_blocks_per_sm(int d, int bins) {
    const size_t smem = tile_f32_smem_bytes(d, bins);
    int blocks = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (d) {
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_tile_f32<16>, kF32Threads, smem); break;
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_tile_f32<32>, kF32Threads, smem); break;
        case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_tile_f32<64>, kF32Threads, smem); break;
        case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_tile_f32<128>, kF32Threads, smem); break;
        default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return blocks < 1 ? 1 : blocks;
}

cudaError_t launch_tile_f32(const EpochArgs& a, int grid, cudaStream_t s) {
    if (a.n_tile_items == 0) return cudaSuccess;
    const size_t smem = tile_f32_smem_bytes(a.d, a.bins);
    switch (a.d) {
        case 16: return launch_critical(k_tile_f32<16>, grid, kF32Threads, smem, s, false, a);
        case 32: return launch_critical(k_tile_f32<32>, grid, kF32Threads, smem, s, false, a);
        case 64: return launch_critical(k_tile_f32<64>, grid, kF32Threads, smem, s, false, a);
        case 128: return launch_critical(k_tile_f32<128>, grid, kF32Threads, smem, s, false, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gempe
