// Block-sampled non-edges (the representation-learning form).
//
// Vertices are cut into tiles of kBlockT = 128 consecutive ids; per epoch,
// every tile draws kBlockP = 64 partners from Philox (counter (tile, epoch,
// p >> 2, 0x0D000000), word p & 3), and every vertex of the tile meets every
// partner.  A pair is masked -- skipped, not redrawn -- when the partner is
// the vertex itself or one of its neighbours (Fig. 2's membership test, here
// done by intersecting the tile's CSR rows with the partner list, which gives
// the same exact answer as probing the edge set).
//
//  k_block_sampler  partners and per-vertex masks of the next epoch (runs on
//                   the side stream beside the current epoch's sweep)
//  k_tile_bf16      one CTA per tile: with BF16 positions X_T (128 x d) and
//                   X_P (64 x d), tensor-core tiles (mma.sync m16n8k16, FP32
//                   accumulation) give
//                     S = X_T X_P^T,  delta^2 = |x_i|^2 + |x_g|^2 - 2 S,
//                   the pair terms (c, w) of Eq. 3-5 per (i, g), then
//                     A = C X_P    -> y_i - z_i x_i += x_i rowsum(C) - A_i
//                     B = C^T X_T  -> y_g - z_g x_g += x_g colsum(C) - B_g
//                   and z_i += rowsum(W), z_g += colsum(W).
#include <cuda_bf16.h>

#include "device_math.cuh"
#include "engine.cuh"
#include "hist.cuh"

namespace gempe {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kTagBlock = 0x0D000000u;
constexpr int kTileThreads = 256;          // 8 warps, 16 tile rows each
constexpr int kSamplerWarps = 8;
constexpr int kMiniHash = 128;             // slots of the per-warp partner hash

// ---------------------------------------------------------------------------
// k_block_sampler: one warp per tile.
// ---------------------------------------------------------------------------
struct WarpHash {
    int key[kMiniHash];
    unsigned int lo[kMiniHash];   // bits of partner positions 0..31
    unsigned int hi[kMiniHash];   // bits of positions 32..63
};

__device__ __forceinline__ unsigned hash_slot(int g) { return ((unsigned)g * 0x9E3779B1u) >> 25; }   // 7 bits

// Positions p whose partner equals j (as a 64-bit mask).
__device__ __forceinline__ unsigned long long partner_bits(const WarpHash& h, int j) {
    unsigned s = hash_slot(j);
    for (int probe = 0; probe < kMiniHash; ++probe) {
        const int k = h.key[s];
        if (k == j) return ((unsigned long long)h.hi[s] << 32) | h.lo[s];
        if (k < 0) return 0ull;
        s = (s + 1) & (kMiniHash - 1);
    }
    return 0ull;
}

// One warp per work unit {tile, e_lo, e_hi, graph << 1 | first}: the unit
// recomputes its tile's 64 partners into a small shared hash (partner row ->
// positions), the tile's first unit writes the partners and the self-pair
// bits, and every unit tests absolute CSR slots [e_lo, e_hi) of the tile's
// rows against the partners, OR-ing hits into the vertices' masks (cleared
// before the launch).  Hub tiles are thereby spread over many warps.  The
// Philox counter takes the tile's index within its graph and the graph's
// key, so a graph draws the same partners alone or in a pack.
__global__ void __launch_bounds__(kSamplerWarps * 32) k_block_sampler(const EpochArgs a, const int4* units,
                                                                      int n_units) {
    __shared__ WarpHash s_hash[kSamplerWarps];
    __shared__ int s_rp[kSamplerWarps][kBlockT + 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpHash& h = s_hash[wib];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;

    for (int it = warp; it < n_units; it += n_warps) {
        const int4 u = __ldg(units + it);
        const int tile = u.x, e_lo = u.y, e_hi = u.z, first = u.w & 1, graph = u.w >> 1;
        const int gv0 = __ldg(&a.graphs[graph].v0), gn = __ldg(&a.graphs[graph].n);
        const int gt0 = __ldg(&a.graphs[graph].t0);
        const uint32_t key_lo = __ldg(&a.graphs[graph].key_lo), key_hi = __ldg(&a.graphs[graph].key_hi);
        const int se = a.gst[graph].sample_epoch;
        const int lt = tile - gt0;                 // tile within the graph
        const int v0 = gv0 + lt * kBlockT;         // pack row of the tile's first vertex
        const int nv = min(kBlockT, gn - lt * kBlockT);
        int32_t* part_out = a.block_part + (size_t)(se & 1) * (size_t)a.n_tiles * kBlockP;
        unsigned long long* mask_out = a.block_mask + (size_t)(se & 1) * (size_t)a.rows;
        unsigned c_rej = 0;
        for (int q = lane; q < kMiniHash; q += 32) {
            h.key[q] = -1;
            h.lo[q] = 0u;
            h.hi[q] = 0u;
        }
        for (int v = lane; v <= nv; v += 32) s_rp[wib][v] = __ldg(a.row_ptr + v0 + v);
        __syncwarp();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int p = lane + 32 * half;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)lt, (uint32_t)se, (uint32_t)(p >> 2), kTagBlock),
                                          key_lo, key_hi);
            const int g = gv0 + draw_vertex(word_of(r, p & 3), (uint32_t)gn);
            if (first) part_out[(size_t)tile * kBlockP + p] = g;
            unsigned s = hash_slot(g);
            for (int probe = 0; probe < kMiniHash; ++probe) {
                const int prev = atomicCAS(&h.key[s], -1, g);
                if (prev == -1 || prev == g) break;
                s = (s + 1) & (kMiniHash - 1);
            }
            if (half == 0) atomicOr(&h.lo[s], 1u << lane);
            else atomicOr(&h.hi[s], 1u << lane);
        }
        __syncwarp();
        if (first) {   // self pairs
            for (int v = lane; v < nv; v += 32) {
                const unsigned long long b = partner_bits(h, v0 + v);
                if (b) {
                    atomicOr(mask_out + v0 + v, b);
                    c_rej += __popcll(b);
                }
            }
        }
        for (int e = e_lo + lane; e < e_hi; e += 32) {
            const unsigned long long b = partner_bits(h, __ldg(a.col_idx + e));
            if (b) {
                int lo = 0, hi = nv - 1;   // row of slot e: last v with rp[v] <= e
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_rp[wib][mid] <= e) lo = mid; else hi = mid - 1;
                }
                atomicOr(mask_out + v0 + lo, b);
                c_rej += __popcll(b);
            }
        }
        // every masked bit is set by exactly one event (a slot or the self
        // pair): accepted = slots - masked, the slots added at completion
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) c_rej += __shfl_xor_sync(kFull, c_rej, o);
        if (lane == 0 && c_rej) {
            atomicAdd(&a.gst[graph].rejected, (unsigned long long)c_rej);
            atomicAdd(&a.gst[graph].accepted, (unsigned long long)(-(long long)c_rej));
        }
        __syncwarp();
    }
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.ps->sample_done, 1u);
        s_last = (prev == gridDim.x - 1) ? 1 : 0;   // every block has read the sample epochs by now
    }
    __syncthreads();
    if (s_last) {
        for (int graph = threadIdx.x; graph < a.n_graphs; graph += blockDim.x) {
            GraphState* st = a.gst + graph;
            const unsigned long long slots = (unsigned long long)__ldg(&a.graphs[graph].n) * kBlockP;
            atomicAdd(&st->accepted, slots);
            atomicAdd(&st->draws, slots);
            st->sample_epoch = st->sample_epoch + 1;
        }
        if (threadIdx.x == 0) a.ps->sample_done = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// Tensor-core helpers (mma.sync m16n8k16, BF16 inputs, FP32 accumulation)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_at(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Shared-memory layout of k_tile_bf16 (rows padded by 8 BF16 so that the
// eight 16-byte rows an ldmatrix reads fall into distinct banks).
template <int D>
struct TileSmem {
    static constexpr int kXS = D + 8;          // row stride (elements) of X_T, X_P
    static constexpr int kCS = kBlockP + 8;    // row stride of C
    __nv_bfloat16 xt[2][kBlockT * kXS];   // double buffer: the next tile's rows load during this one
    __nv_bfloat16 xp[2][kBlockP * kXS];
    __nv_bfloat16 cs[kBlockT * kCS];
    float nt[kBlockT], np[kBlockP];
    float row_c[kBlockT], row_w[kBlockT];
    float col_c[8][kBlockP], col_w[8][kBlockP];
    unsigned long long mask[kBlockT];
    int deg[kBlockT], kacc[kBlockT];
    int part[2][kBlockP];
};

// Start the asynchronous loads of tile item `it` (if below `end`) into
// buffer b: its partner list, X_T (zero rows past the graph's end) and X_P;
// always commits one cp.async group.
template <int D>
__device__ __forceinline__ void stage_tile(const EpochArgs& a, TileSmem<D>& sm, int it, int end, int b) {
    constexpr int XS = TileSmem<D>::kXS;
    constexpr int CH = D / 8;   // 16-byte chunks per row
    if (it < end) {
        const int2 ti = __ldg(a.tile_items + it);
        const int tile = ti.x, graph = ti.y;
        const int gv0 = __ldg(&a.graphs[graph].v0), gn = __ldg(&a.graphs[graph].n);
        const int lt = tile - __ldg(&a.graphs[graph].t0);
        const int v0 = gv0 + lt * kBlockT;
        const int nv = min(kBlockT, gn - lt * kBlockT);
        const int epoch = a.gst[graph].epoch;
        const int32_t* part = a.block_part + ((size_t)(epoch & 1) * (size_t)a.n_tiles + tile) * kBlockP;
        if (threadIdx.x < kBlockP) sm.part[b][threadIdx.x] = __ldg(part + threadIdx.x);
        for (int c = threadIdx.x; c < kBlockT * CH; c += blockDim.x) {
            const int r = c / CH, q = c - r * CH;
            __nv_bfloat16* dst = sm.xt[b] + r * XS + q * 8;
            if (r < nv) cp_async16(dst, a.xb + (size_t)(v0 + r) * D + q * 8);
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
        for (int c = threadIdx.x; c < kBlockP * CH; c += blockDim.x) {
            const int r = c / CH, q = c - r * CH;
            cp_async16(sm.xp[b] + r * XS + q * 8, a.xb + (size_t)__ldg(part + r) * D + q * 8);
        }
    }
    cp_async_commit();
}

// ---------------------------------------------------------------------------
// k_tile_bf16: block-sampled non-edges of one tile per CTA iteration; the
// next tile's rows are staged (cp.async) while the current one computes.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kTileThreads) k_tile_bf16(const EpochArgs a) {
    constexpr int KS = D / 16;          // k-steps of S = X_T X_P^T
    constexpr int ND = D / 8;           // n-tiles over the dimensions
    constexpr int XS = TileSmem<D>::kXS, CS = TileSmem<D>::kCS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<D>& sm = *reinterpret_cast<TileSmem<D>*>(smem_raw);
    unsigned int* hist_base = reinterpret_cast<unsigned int*>(smem_raw + sizeof(TileSmem<D>));
    // tile items: a contiguous range per block in packs of several graphs
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
    for (int t = threadIdx.x; t < a.bins; t += blockDim.x) {
        hist.he[t] = 0u;
        hist.hc[t] = 0u;
        hist.hd[t] = 0u;
    }
    if (threadIdx.x == 0) {
        s_used = 0u;
        s_tile_used = 0u;
    }

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;

    stage_tile<D>(a, sm, it0, it1, 0);
    int buf = 0;
    for (int it = it0; it < it1; it += istep, buf ^= 1) {
        const int2 ti = __ldg(a.tile_items + it);
        const int tile = ti.x, graph = ti.y;
        const int gv0 = __ldg(&a.graphs[graph].v0), gn = __ldg(&a.graphs[graph].n);
        const int lt = tile - __ldg(&a.graphs[graph].t0);
        const int v0 = gv0 + lt * kBlockT;
        const int nv = min(kBlockT, gn - lt * kBlockT);
        const float sigma = a.gst[graph].sigma;
        const int epoch = a.gst[graph].epoch;
        const PairConsts K = make_pair_consts(a.mu, sigma, a.w_formula == 1, a.clamp_neg_d, a.mills);
        unsigned long long* bmask = a.block_mask + (size_t)(epoch & 1) * (size_t)a.rows;
        __syncthreads();   // the previous tile's shared data (and buffer buf ^ 1) is no longer read
        stage_tile<D>(a, sm, it + istep, it1, buf ^ 1);
        const __nv_bfloat16* xt = sm.xt[buf];
        const __nv_bfloat16* xp = sm.xp[buf];
        const int* prt = sm.part[buf];
        // ---- masks and degrees (X_T, X_P and the partners were staged one tile ahead) ----
        for (int v = threadIdx.x; v < kBlockT; v += blockDim.x) {
            if (v < nv) {
                const unsigned long long m = bmask[v0 + v];
                bmask[v0 + v] = 0ull;   // read once: the buffer starts empty for the epoch two ahead
                sm.mask[v] = m;
                sm.deg[v] = __ldg(a.row_ptr + v0 + v + 1) - __ldg(a.row_ptr + v0 + v);
                sm.kacc[v] = kBlockP - __popcll(m);
                atomicAdd(&s_tile_used, (unsigned)(kBlockP - __popcll(m)));
            } else {
                sm.mask[v] = ~0ull;
                sm.deg[v] = 0;
                sm.kacc[v] = 0;
            }
        }
        cp_async_wait_prev();   // this tile's group has landed (the next one may still be loading)
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_tile_used) {
                if (graph == home) s_used += s_tile_used;
                else atomicAdd(&a.gst[graph].used, (unsigned long long)s_tile_used);
            }
            s_tile_used = 0u;
        }
        for (int r = threadIdx.x; r < kBlockT + kBlockP; r += blockDim.x) {
            const __nv_bfloat16* row = (r < kBlockT) ? xt + r * XS : xp + (r - kBlockT) * XS;
            float s = 0.0f;
#pragma unroll 8
            for (int c = 0; c < D; ++c) {
                const float v = bf16_at(row + c);
                s = fmaf(v, v, s);
            }
            if (r < kBlockT) sm.nt[r] = s; else sm.np[r - kBlockT] = s;
        }
        __syncthreads();

        // ---- S = X_T X_P^T for rows 16w..16w+15 ----
        const int r0 = 16 * w;
        float S[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) S[j][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            uint32_t af[4];
            {
                const int mat = lane >> 3, rr = lane & 7;
                ldsm_x4(af, xt + (r0 + rr + 8 * (mat & 1)) * XS + 16 * ks + 8 * (mat >> 1));
            }
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                uint32_t bf[4];
                const int mat = lane >> 3, rr = lane & 7;
                ldsm_x4(bf, xp + (8 * (j + (mat >> 1)) + rr) * XS + 16 * ks + 8 * (mat & 1));
                mma_16816(S[j], af, bf[0], bf[1]);
                mma_16816(S[j + 1], af, bf[2], bf[3]);
            }
        }

        // ---- pair terms per (i, p); C to registers (bf16) and shared memory ----
        // Af[kk]: A fragments of C for C X_P, k-step kk (partners 16kk..16kk+15):
        // {C(g, 16kk+2t..), C(g+8, 16kk+2t..), C(g, 16kk+8+2t..), C(g+8, 16kk+8+2t..)}
        uint32_t Af[4][4];
        float rc[2] = {0.0f, 0.0f}, rw[2] = {0.0f, 0.0f};    // row sums for rows g, g + 8
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float cv[4], col_c[2] = {0.0f, 0.0f}, col_w[2] = {0.0f, 0.0f};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int il = r0 + g + 8 * (e >> 1);
                const int p = 8 * j + 2 * t4 + (e & 1);
                const bool valid = !((sm.mask[il] >> p) & 1ull);
                float c = 0.0f, wv = 0.0f;
                if (valid) {
                    const float d2 = fmaxf(sm.nt[il] + sm.np[p] - 2.0f * S[j][e], 0.0f);
                    float delta, inv_delta;
                    dist_of(d2, delta, inv_delta);
                    const PairTerm pt = pair_term(delta, inv_delta, false, K);
                    c = pt.c;
                    wv = pt.w;
                    const int bin = min((int)(delta * a.hist_scale), a.bins - 1);
                    hist_sample(hist, a, graph, bin, sm.deg[il], sm.kacc[il], kBlockP);
                }
                cv[e] = c;
                rc[e >> 1] += c;
                rw[e >> 1] += wv;
                col_c[e & 1] += c;
                col_w[e & 1] += wv;
            }
            const uint32_t top = pack_bf16(cv[0], cv[1]), bot = pack_bf16(cv[2], cv[3]);
            Af[j >> 1][(j & 1) * 2 + 0] = top;
            Af[j >> 1][(j & 1) * 2 + 1] = bot;
            *reinterpret_cast<uint32_t*>(sm.cs + (r0 + g) * CS + 8 * j + 2 * t4) = top;
            *reinterpret_cast<uint32_t*>(sm.cs + (r0 + g + 8) * CS + 8 * j + 2 * t4) = bot;
            // column sums over the warp's 16 rows (lanes with equal t4)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    col_c[e] += __shfl_xor_sync(kFull, col_c[e], o);
                    col_w[e] += __shfl_xor_sync(kFull, col_w[e], o);
                }
                if (g == 0) {
                    sm.col_c[w][8 * j + 2 * t4 + e] = col_c[e];
                    sm.col_w[w][8 * j + 2 * t4 + e] = col_w[e];
                }
            }
        }
        // row sums over the quad
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            rc[h] += __shfl_xor_sync(kFull, rc[h], 1);
            rc[h] += __shfl_xor_sync(kFull, rc[h], 2);
            rw[h] += __shfl_xor_sync(kFull, rw[h], 1);
            rw[h] += __shfl_xor_sync(kFull, rw[h], 2);
        }
        if (t4 == 0) {
            sm.row_c[r0 + g] = rc[0];
            sm.row_c[r0 + g + 8] = rc[1];
            sm.row_w[r0 + g] = rw[0];
            sm.row_w[r0 + g + 8] = rw[1];
        }
        __syncwarp();

        // ---- A = C X_P: anchors of rows 16w..16w+15 ----
#pragma unroll
        for (int jd = 0; jd < ND; jd += 2) {
            float A0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, A1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                uint32_t bf[4];
                const int mat = lane >> 3, rr = lane & 7;
                ldsm_x4_t(bf, xp + (16 * kk + 8 * (mat & 1) + rr) * XS + 8 * (jd + (mat >> 1)));
                mma_16816(A0, Af[kk], bf[0], bf[1]);
                mma_16816(A1, Af[kk], bf[2], bf[3]);
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const float* Ar = hh ? A1 : A0;
                const int dim = 8 * (jd + hh) + 2 * t4;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int il = r0 + g + 8 * h;
                    if (il < nv && sm.kacc[il] > 0) {
                        const float s = sm.row_c[il];
                        const float v0f = bf16_at(xt + il * XS + dim) * s - Ar[2 * h];
                        const float v1f = bf16_at(xt + il * XS + dim + 1) * s - Ar[2 * h + 1];
                        atomicAdd(reinterpret_cast<float2*>(a.acc + (size_t)(v0 + il) * a.acc_stride + dim),
                                  make_float2(v0f, v1f));
                    }
                }
            }
        }
        if (t4 == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int il = r0 + g + 8 * h;
                if (il < nv && sm.kacc[il] > 0) atomicAdd(a.acc + (size_t)(v0 + il) * a.acc_stride + D, sm.row_w[il]);
            }
        }
        __syncthreads();   // C in shared memory and the column sums are complete

        // ---- B = C^T X_T: partners; warp w -> partners 16*(w>>1).., dims half (w&1) ----
        if (a.symmetric) {
            const int m0 = 16 * (w >> 1);
            constexpr int NW = ND / 2;     // n-tiles per warp
            float Bacc[NW][4];
#pragma unroll
            for (int j = 0; j < NW; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) Bacc[j][e] = 0.0f;
            const int nbase = (w & 1) * NW;
#pragma unroll
            for (int kk = 0; kk < kBlockT / 16; ++kk) {
                uint32_t af[4];
                {
                    const int mat = lane >> 3, rr = lane & 7;
                    ldsm_x4_t(af, sm.cs + (16 * kk + 8 * (mat >> 1) + rr) * CS + m0 + 8 * (mat & 1));
                }
#pragma unroll
                for (int j = 0; j < NW; j += 2) {
                    uint32_t bf[4];
                    const int mat = lane >> 3, rr = lane & 7;
                    ldsm_x4_t(bf, xt + (16 * kk + 8 * (mat & 1) + rr) * XS + 8 * (nbase + j + (mat >> 1)));
                    mma_16816(Bacc[j], af, bf[0], bf[1]);
                    if (j + 1 < NW) mma_16816(Bacc[j + 1], af, bf[2], bf[3]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = m0 + g + 8 * h;
                float csum = 0.0f, wsum = 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    csum += sm.col_c[q][p];
                    wsum += sm.col_w[q][p];
                }
                if (wsum == 0.0f && csum == 0.0f) continue;   // every pair of this partner masked or underflowed
                const int gv = prt[p];
#pragma unroll
                for (int j = 0; j < NW; ++j) {
                    const int dim = 8 * (nbase + j) + 2 * t4;
                    const float v0f = bf16_at(xp + p * XS + dim) * csum - Bacc[j][2 * h];
                    const float v1f = bf16_at(xp + p * XS + dim + 1) * csum - Bacc[j][2 * h + 1];
                    atomicAdd(reinterpret_cast<float2*>(a.acc + (size_t)gv * a.acc_stride + dim), make_float2(v0f, v1f));
                }
                if (t4 == 0 && (w & 1) == 0) atomicAdd(a.acc + (size_t)gv * a.acc_stride + D, wsum);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    hist_merge(hist, a);
    if (threadIdx.x == 0 && s_used && home >= 0) atomicAdd(&a.gst[home].used, (unsigned long long)s_used);
}

}  // namespace

bool tile_dim(int d) { return d == 16 || d == 32 || d == 64; }

size_t tile_smem_bytes(int d, int bins) {
    size_t base = 0;
    switch (d) {
        case 16: base = sizeof(TileSmem<16>); break;
        case 32: base = sizeof(TileSmem<32>); break;
        case 64: base = sizeof(TileSmem<64>); break;
        default: return 0;
    }
    return base + hist_smem_bytes(bins);
}

cudaError_t prepare_tile_kernel(int d, int bins) {
    const int smem = (int)tile_smem_bytes(d, bins);
    switch (d) {
        case 16: return cudaFuncSetAttribute(k_tile_bf16<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        case 32: return cudaFuncSetAttribute(k_tile_bf16<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        case 64: return cudaFuncSetAttribute(k_tile_bf16<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_block_sampler(const EpochArgs& a, const int4* units, int n_units, int sm_count,
                                 cudaStream_t s) {
    // the masks of the epoch being drawn start empty (their consumers clear them)
    int grid = (n_units + kSamplerWarps - 1) / kSamplerWarps;
    if (grid > sm_count * 8) grid = sm_count * 8;
    if (grid < 1) grid = 1;
    k_block_sampler<<<grid, kSamplerWarps * 32, 0, s>>>(a, units, n_units);
    return cudaGetLastError();
}

// blocks_per_sm: 0 = two CTAs per SM (what fits with the histogram bins)
int tile_grid(int n_tile_items, int sm_count, int blocks_per_sm) {
    const int per_sm = blocks_per_sm > 0 ? blocks_per_sm : 2;
    int grid = n_tile_items < sm_count * per_sm ? n_tile_items : sm_count * per_sm;
    return grid < 1 ? 1 : grid;
}

cudaError_t launch_tile_bf16(const EpochArgs& a, int grid, cudaStream_t s) {
    if (a.n_tile_items == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(a.d, a.bins);
    switch (a.d) {
        case 16: return launch_critical(k_tile_bf16<16>, grid, kTileThreads, smem, s, a);
        case 32: return launch_critical(k_tile_bf16<32>, grid, kTileThreads, smem, s, a);
        case 64: return launch_critical(k_tile_bf16<64>, grid, kTileThreads, smem, s, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gempe
