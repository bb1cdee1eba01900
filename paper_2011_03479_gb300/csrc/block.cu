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
//  k_tile_tc        one CTA per tile: with BF16 positions X_T (128 x d) and
//                   X_P (64 x d), 5th-generation tensor cores (tcgen05.mma,
//                   operands in shared memory, FP32 accumulators in TMEM) give
//                     S = X_T X_P^T,  delta^2 = |x_i|^2 + |x_g|^2 - 2 S,
//                   the pair terms (c, w) of Eq. 3-5 per (i, g) (rounded to
//                   BF16 for the next products), then
//                     A = C X_P    -> y_i - z_i x_i += x_i rowsum(C) - A_i
//                     B = C^T X_T  -> y_g - z_g x_g += x_g colsum(C) - B_g
//                   and z_i += rowsum(W), z_g += colsum(W).
#include <cuda_bf16.h>

#include <algorithm>

#include "device_math.cuh"
#include "engine.cuh"
#include "hist.cuh"
#include "tile_ahead.cuh"

namespace gempe {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kTagBlock = 0x0D000000u;
constexpr int kTileThreads = 256;          // 8 warps, 16 tile rows each
constexpr int kSamplerWarps = 8;
constexpr int kTileWaitLimit = 1 << 22;    // mbarrier polls before a tile CTA gives up
constexpr int32_t kStatusTimeout = -5;     // gempe_status of a bounded device wait that gave up
constexpr int kTileCtasPerSm = 2;          // 256 TMEM columns and about 113 KB of shared memory each
constexpr size_t kTileMinSmem = 80 * 1024; // at most two tile CTAs per SM: never more TMEM columns than 512

// ---------------------------------------------------------------------------
// k_block_sampler: one warp per tile {tile, -, -, graph << 1 | 1}.  Lane l
// draws the tile's partners p = l and l + 32 (the Philox counter takes the
// tile's index within its graph and the graph's key, so a graph draws the
// same partners alone or in a pack), writes them, and the warp builds the
// tile's 128 mask words in shared memory: bit p of anchor v is set when
// partner p is v itself or a neighbour of v.  As the CSR is symmetric, the
// neighbours are found from the partners' side: every id of partner p's row
// that falls inside the tile's anchor range [v0, v0 + nv) marks that anchor
// (64 rows of random vertices per tile, a range test per slot, where the
// anchors' own rows would need a membership probe per slot).  Rows of up to
// kSamplerRowLane slots are scanned by their lane, longer ones by the whole
// warp.  Each tile has one warp, so the mask words are stored, not merged.
// ---------------------------------------------------------------------------
constexpr int kSamplerRowLane = 32;

__global__ void __launch_bounds__(kSamplerWarps * 32) k_block_sampler(const EpochArgs a, const int4* units,
                                                                      int n_units) {
    __shared__ unsigned long long s_mask[kSamplerWarps][kBlockT];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned long long* sm = s_mask[wib];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;

    for (int it = warp; it < n_units; it += n_warps) {
        const int4 u = __ldg(units + it);
        const int tile = u.x, graph = u.w >> 1;
        const int gv0 = __ldg(&a.graphs[graph].v0), gn = __ldg(&a.graphs[graph].n);
        const int gt0 = __ldg(&a.graphs[graph].t0);
        const uint32_t key_lo = __ldg(&a.graphs[graph].key_lo), key_hi = __ldg(&a.graphs[graph].key_hi);
        const int se = a.gst[graph].sample_epoch;
        const int lt = tile - gt0;                 // tile within the graph
        const int v0 = gv0 + lt * kBlockT;         // pack row of the tile's first vertex
        const int nv = min(kBlockT, gn - lt * kBlockT);
        int32_t* part_out = a.block_part + (size_t)(se & 1) * (size_t)a.n_tiles * kBlockP;
        unsigned long long* mask_out = a.block_mask + (size_t)(se & 1) * (size_t)a.rows;
        for (int v = lane; v < kBlockT; v += 32) sm[v] = 0ull;
        int rb[2], re[2];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int p = lane + 32 * half;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)lt, (uint32_t)se, (uint32_t)(p >> 2), kTagBlock),
                                          key_lo, key_hi);
            const int g = gv0 + draw_vertex(word_of(r, p & 3), (uint32_t)gn);
            part_out[(size_t)tile * kBlockP + p] = g;
            rb[half] = __ldg(a.row_ptr + g);
            re[half] = __ldg(a.row_ptr + g + 1);
            __syncwarp();
            const unsigned self = (unsigned)(g - v0);   // the partner is an anchor of the tile
            if (self < (unsigned)nv) atomicOr(&sm[self], 1ull << p);
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const unsigned long long bit = 1ull << (lane + 32 * half);
            if (re[half] - rb[half] <= kSamplerRowLane) {
                for (int e = rb[half]; e < re[half]; ++e) {
                    const unsigned o = (unsigned)(__ldg(a.col_idx + e) - v0);
                    if (o < (unsigned)nv) atomicOr(&sm[o], bit);
                }
            }
            unsigned longs = __ballot_sync(kFull, re[half] - rb[half] > kSamplerRowLane);
            while (longs) {
                const int src = __ffs(longs) - 1;
                longs &= longs - 1;
                const int e0 = __shfl_sync(kFull, rb[half], src), e1 = __shfl_sync(kFull, re[half], src);
                const unsigned long long sbit = 1ull << (src + 32 * half);
                for (int e = e0 + lane; e < e1; e += 32) {
                    const unsigned o = (unsigned)(__ldg(a.col_idx + e) - v0);
                    if (o < (unsigned)nv) atomicOr(&sm[o], sbit);
                }
            }
        }
        __syncwarp();
        // every masked bit is set by exactly one event (the self pair or one
        // edge): accepted = slots - masked, the slots added at completion
        unsigned c_rej = 0;
        for (int v = lane; v < nv; v += 32) {
            const unsigned long long m = sm[v];
            mask_out[v0 + v] = m;
            c_rej += __popcll(m);
        }
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
            const int own = a.own_n > 0 ? a.own_n : __ldg(&a.graphs[graph].n);   // a shard draws for its range
            const unsigned long long slots = (unsigned long long)own * kBlockP;
            atomicAdd(&st->accepted, slots);
            atomicAdd(&st->draws, slots);
            st->sample_epoch = st->sample_epoch + 1;
        }
        if (threadIdx.x == 0) a.ps->sample_done = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): operands in shared memory, the
// accumulators in tensor memory (TMEM).
//
// Operand layout: every BF16 matrix of the tile kernel is stored in 8-row x
// 16-byte core matrices; element (r, c) of an R x W buffer sits at byte
//   (r / 8) * (W / 8) * 128 + (c / 8) * 128 + (r % 8) * 16 + (c % 8) * 2.
// Read with K along c (K-major) its shared-memory descriptor has leading
// byte offset (between core matrices along K) 128 and stride byte offset
// (between 8-row groups) (W / 8) * 128; read with K along r (MN-major, the
// 16-byte rows running along M or N) the leading offset is (W / 8) * 128 and
// the stride offset 128.  No swizzling.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__host__ __device__ constexpr uint32_t core_off(int r, int c, int W) {
    return (uint32_t)((r >> 3) * (W / 8) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// A / B major (0 K-major, 1 MN-major), N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = A B (+ D when accumulate); issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// The mbarrier completes one phase when every MMA issued so far by this
// thread has finished.
__device__ __forceinline__ void tc_commit(unsigned long long* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(mbar)));
}

// Bounded wait for phase `parity` of an mbarrier; false when it gave up
// after `limit` polls.  The give-up path of the tile kernel (leave the tile
// loop, free the TMEM, record GEMPE_E_TIMEOUT) assumes that nothing the CTA
// committed is still running: it is meant for the hang where the arrival
// never comes.  Were an MMA only slow, it could still write the TMEM and
// read the shared memory the CTA gives up, so a context whose status reads
// GEMPE_E_TIMEOUT must be destroyed, not stepped again.
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, uint32_t parity, int limit = kTileWaitLimit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity));
    return done != 0;
}

// 8 consecutive FP32 columns of this thread's TMEM lane (the warp's quadrant).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}

// Shared memory of the tile kernel, in two stages: the tile being computed
// and the next one, whose rows are copied in while the current tile's pair
// terms run.  Per stage, XT: the tile's BF16 rows (128 x D), XP: its
// partners' rows (64 x D), their squared norms, masks, degrees and partner
// ids.  CW: the pair coefficients, C in columns 0..63, W in 64..127 (W fills
// the 128 rows the B product needs; its row and column sums come from the
// epilogue and from CW).  TMEM, per stage: S in columns 0..63, then A in
// 0..D-1 once the epilogue has read S, B in 64..64+D-1 (2 x 128 columns per
// CTA, two CTAs per SM).
template <int D>
struct TileTc {
    static constexpr int DP = D;
    static constexpr uint32_t kStageCols = 128;
    static constexpr uint32_t kCols = 2 * kStageCols;        // TMEM columns of a CTA
    static constexpr uint32_t kColS = 0, kColA = 0, kColB = 64;
    struct alignas(128) Stage {
        __nv_bfloat16 xt[kBlockT * DP];
        __nv_bfloat16 xp[kBlockP * DP];
        float nt[kBlockT], np[kBlockP];
        unsigned long long mask[kBlockT];
        int deg[kBlockT], kacc[kBlockT];
        int part[kBlockP];
    };
    Stage st[2];
    __nv_bfloat16 cw[kBlockT * 2 * kBlockP];
    float row_w[2][kBlockT], row_c[2][kBlockT];   // per partner half: sums of w and of the rounded c
    float col[2][2 * kBlockP];                    // per anchor half: column sums of the rounded C | W
    MillsCoef mills[kMillsIntervals];             // the Mills-ratio table (pair terms)
    unsigned long long mbar_s, mbar_ab;           // completions of the S products / of A and B
    uint32_t tmem;
    int abort;
};

// ---------------------------------------------------------------------------
// k_tile_tc: block-sampled non-edges, 8 warps per CTA, tiles in a pipeline
// of two stages.  For tile t (stage b):
//   (0) the rows, masks and partners of tile t + 1 are copied into stage
//       1 - b (cp.async; the global words they need were loaded a tile
//       earlier still);
//   (1) S = X_T X_P^T (M 128, N 64, K d), issued at the end of tile t - 1,
//       is waited for;
//   (2) warp w reads rows 32 (w % 4) .. of S, partner columns 32 (w / 4) ..,
//       forms the pair terms (c, w) with the masks and histograms, writes
//       them rounded to BF16 into CW and sums, per anchor and partner half,
//       w and the rounded c (the row sums);
//   (3) A = C X_P (K 64) gives sum_g c_ig x_g; B = [C | W]^T X_T (M 128,
//       K 128) gives sum_i c_ig x_i in rows 0..63; meanwhile the column
//       sums of the rounded C and W are added up from CW, then tile t + 1's
//       rows are waited for, their norms taken, and its S issued behind A
//       and B on the tensor cores;
//   (4) x_i rowsum(C) - A_i and the row sums of W go to the anchors'
//       accumulators, x_g colsum(C) - B_g and colsum(W) to the partners'.
// One thread issues the MMAs; their completions are signalled on two
// mbarriers (bounded waits: a timeout sets the pack's status and ends the
// kernel).  The pair-term loop over the four 8-partner chunks is kept rolled
// (the unrolled kernel stalled on instruction fetch).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kTileThreads, kTileCtasPerSm) k_tile_tc(const EpochArgs a) {
    using L = TileTc<D>;
    using Stage = typename L::Stage;
    constexpr int DP = L::DP;
    constexpr int CH = D / 8;                     // 16-byte chunks of a row
    constexpr uint32_t kSbT = (DP / 8) * 128;     // stride of 8-row groups of XT, XP
    constexpr uint32_t kSbC = (2 * kBlockP / 8) * 128;
    extern __shared__ __align__(128) unsigned char smem_raw[];
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
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int quad = w & 3, half = w >> 2;
    for (int t = tid; t < a.bins; t += blockDim.x) {
        hist.he[t] = 0u;
        hist.hc[t] = 0u;
        hist.hd[t] = 0u;
    }
    for (int t = tid; t < kMillsIntervals; t += blockDim.x) sm.mills[t].lh = __ldg(&a.mills[t].lh);
    if (tid == 0) {
        s_used = 0u;
        s_tile_used = 0u;
        sm.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sm.mbar_s)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sm.mbar_ab)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&sm.tmem)), "r"(L::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;   // this warp's TMEM lanes
    uint32_t ph_s = 0, ph_ab = 0;
    using Ahead = TileAhead<CH, kTileThreads>;

    // Copy a tile's rows into stage s (no wait) and set its masks.
    auto stage_tile = [&](const Ahead& t, Stage& s) {
        const int v0 = t.v0, nv = t.nv;
        unsigned long long* bmask = a.block_mask + (size_t)(a.gst[t.graph].epoch & 1) * (size_t)a.rows;
        if (tid < kBlockP) s.part[tid] = t.part;
        for (int c = tid; c < kBlockT * CH; c += blockDim.x) {
            const int r = c / CH, q = c - r * CH;
            unsigned char* dst = reinterpret_cast<unsigned char*>(s.xt) + core_off(r, 8 * q, DP);
            if (r < nv) cp_async16(dst, a.xb + (size_t)(v0 + r) * D + 8 * q);
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < Ahead::kChunks; ++j) {
            const int c = tid + kTileThreads * j;
            if (c < kBlockP * CH) {
                const int r = c / CH, q = c - r * CH;
                cp_async16(reinterpret_cast<unsigned char*>(s.xp) + core_off(r, 8 * q, DP),
                           a.xb + (size_t)t.pid[j] * D + 8 * q);
            }
        }
        if (tid < kBlockT) {
            const int v = tid;
            if (v < nv) {
                const unsigned long long m = t.m;
                bmask[v0 + v] = 0ull;   // read once: the buffer starts empty for the epoch two ahead
                s.mask[v] = m;
                s.deg[v] = t.deg;
                s.kacc[v] = kBlockP - __popcll(m);
                atomicAdd(&s_tile_used, (unsigned)(kBlockP - __popcll(m)));
            } else {
                s.mask[v] = ~0ull;
                s.deg[v] = 0;
                s.kacc[v] = 0;
            }
        }
    };
    // Wait for stage s's rows, book its accepted samples, take the squared
    // norms of its BF16 rows (what S is made of) and hand the rows to the
    // tensor cores.
    auto finish_stage = [&](Stage& s, int graph) {
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            if (s_tile_used) {
                if (graph == home) s_used += s_tile_used;
                else atomicAdd(&a.gst[graph].used, (unsigned long long)s_tile_used);
            }
            s_tile_used = 0u;
        }
        for (int r = tid; r < kBlockT + kBlockP; r += blockDim.x) {
            const unsigned char* base = reinterpret_cast<const unsigned char*>(r < kBlockT ? s.xt : s.xp);
            const int rr = r < kBlockT ? r : r - kBlockT;
            float s2 = 0.0f;
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                const uint4 u = *reinterpret_cast<const uint4*>(base + core_off(rr, 8 * q, DP));
                const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float lo = __uint_as_float(wd[e] << 16), hi = __uint_as_float(wd[e] & 0xFFFF0000u);
                    s2 = fmaf(lo, lo, fmaf(hi, hi, s2));
                }
            }
            if (r < kBlockT) s.nt[rr] = s2; else s.np[rr] = s2;
        }
        asm volatile("fence.proxy.async.shared::cta;");   // the staged rows, for the tensor cores
        __syncthreads();
    };
    // S = X_T X_P^T of stage s into TMEM columns col0 .. col0 + 63.
    auto issue_s = [&](const Stage& s, uint32_t col0) {
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t at = smem_u32(s.xt), ap = smem_u32(s.xp);
#pragma unroll
            for (int k = 0; k < D / 16; ++k)
                tc_mma(tmem + col0 + L::kColS, smem_desc(at + 256 * k, 128, kSbT), smem_desc(ap + 256 * k, 128, kSbT),
                       mma_idesc(128, kBlockP, 0, 0), k > 0);
            tc_commit(&sm.mbar_s);
        }
    };

    Ahead cur, nxt;
    if (it0 < it1) {
        cur = tile_ahead<CH, kTileThreads>(a, it0, tid);
        if (it0 + istep < it1) nxt = tile_ahead<CH, kTileThreads>(a, it0 + istep, tid);
        stage_tile(cur, sm.st[0]);
        finish_stage(sm.st[0], cur.graph);
        issue_s(sm.st[0], 0);
    }
    int b = 0;
    for (int it = it0; it < it1; it += istep, b ^= 1) {
        Stage& S0 = sm.st[b];
        Stage& S1 = sm.st[b ^ 1];
        const uint32_t col0 = (uint32_t)b * L::kStageCols, col1 = (uint32_t)(b ^ 1) * L::kStageCols;
        const int graph = cur.graph, v0 = cur.v0, nv = cur.nv;
        const bool has_next = it + istep < it1;
        const int next_graph = nxt.graph;
        const NonEdgeConsts NK =
            make_nonedge_consts(make_pair_consts(a.mu, a.gst[graph].sigma, a.w_formula == 1, a.clamp_neg_d, sm.mills));

        // ---- (0) the next tile's rows into the other stage ----
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();   // the tile before this one no longer reads the other stage or its TMEM
        if (has_next) stage_tile(nxt, S1);
        Ahead after;
        if (it + 2 * istep < it1) after = tile_ahead<CH, kTileThreads>(a, it + 2 * istep, tid);

        // ---- (1) S of this tile ----
        if (!mbar_wait(&sm.mbar_s, ph_s)) atomicExch(&sm.abort, 1);
        ph_s ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (sm.abort) break;

        // ---- (2) pair terms: anchor i = 32 quad + lane, partners 32 half .. 32 half + 31 ----
        {
            const int i = 32 * quad + lane;
            const unsigned long long mk = S0.mask[i];
            const float ni = S0.nt[i];
            const int di = S0.deg[i], ki = S0.kacc[i];
            float rw = 0.0f, rc = 0.0f;
#pragma unroll 1
            for (int c8 = 0; c8 < 4; ++c8) {
                const int p0 = 32 * half + 8 * c8;
                float sv[8];
                tmem_ld8(tmem + lane_base + col0 + L::kColS + (uint32_t)p0, sv);
                // the eight terms without branches (masked pairs give 0),
                // then their histogram counts
                float cv[8], wv[8];
                int bn[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const bool live = !((mk >> (p0 + e)) & 1ull);
                    const float d2 = fmaxf(ni + S0.np[p0 + e] - 2.0f * sv[e], 0.0f);
                    float delta, inv_delta;
                    dist_of(d2, delta, inv_delta);
                    const PairTerm pt = nonedge_term<false>(delta, inv_delta, NK);
                    cv[e] = live ? pt.c : 0.0f;
                    wv[e] = live ? pt.w : 0.0f;
                    bn[e] = live ? min((int)(delta * a.hist_scale), a.bins - 1) : -1;
                    rw += wv[e];
                }
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (bn[e] >= 0) hist_sample(hist, a, graph, bn[e], di, ki, kBlockP);
                unsigned char* cw = reinterpret_cast<unsigned char*>(sm.cw);
                const uint4 cpk = make_uint4(pack_bf16(cv[0], cv[1]), pack_bf16(cv[2], cv[3]), pack_bf16(cv[4], cv[5]),
                                             pack_bf16(cv[6], cv[7]));
                // the row sum of C as the products see it: of the rounded terms
                rc += ((__uint_as_float(cpk.x << 16) + __uint_as_float(cpk.x & 0xFFFF0000u)) +
                       (__uint_as_float(cpk.y << 16) + __uint_as_float(cpk.y & 0xFFFF0000u))) +
                      ((__uint_as_float(cpk.z << 16) + __uint_as_float(cpk.z & 0xFFFF0000u)) +
                       (__uint_as_float(cpk.w << 16) + __uint_as_float(cpk.w & 0xFFFF0000u)));
                *reinterpret_cast<uint4*>(cw + core_off(i, p0, 2 * kBlockP)) = cpk;
                *reinterpret_cast<uint4*>(cw + core_off(i, kBlockP + p0, 2 * kBlockP)) =
                    make_uint4(pack_bf16(wv[0], wv[1]), pack_bf16(wv[2], wv[3]), pack_bf16(wv[4], wv[5]),
                               pack_bf16(wv[6], wv[7]));
            }
            sm.row_w[half][i] = rw;
            sm.row_c[half][i] = rc;
        }
        asm volatile("fence.proxy.async.shared::cta;");   // CW, for the tensor cores
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();

        // ---- (3) A = C X_P,  B = [C | W]^T X_T ----
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t at = smem_u32(S0.xt), ap = smem_u32(S0.xp), ac = smem_u32(sm.cw);
#pragma unroll
            for (int k = 0; k < kBlockP / 16; ++k)   // K = partners: C K-major, X_P MN-major
                tc_mma(tmem + col0 + L::kColA, smem_desc(ac + 256 * k, 128, kSbC),
                       smem_desc(ap + 2 * k * kSbT, kSbT, 128), mma_idesc(128, DP, 0, 1), k > 0);
#pragma unroll
            for (int k = 0; k < kBlockT / 16; ++k)   // K = anchors: [C | W] and X_T both MN-major
                tc_mma(tmem + col0 + L::kColB, smem_desc(ac + 2 * k * kSbC, kSbC, 128),
                       smem_desc(at + 2 * k * kSbT, kSbT, 128), mma_idesc(128, DP, 1, 1), k > 0);
            tc_commit(&sm.mbar_ab);
        }
        {
            // beside the products: the column sums of the rounded C and W.
            // Eight lanes read rows 8 rb + j (j = lane % 8) of one 8-column
            // group (128 contiguous bytes: no bank conflicts), over half of
            // the row blocks; three halving exchanges leave lane j with the
            // sum of column j of its group.
            const int j = lane & 7, gid = 4 * w + (lane >> 3);   // 32 = 16 column groups x 2 anchor halves
            const int cg = gid & 15, ah = gid >> 4;
            const unsigned char* cwb = reinterpret_cast<const unsigned char*>(sm.cw);
            float sv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int rb = 8 * ah; rb < 8 * ah + 8; ++rb) {
                const uint4 u = *reinterpret_cast<const uint4*>(cwb + core_off(8 * rb + j, 8 * cg, 2 * kBlockP));
                const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    sv[2 * e] += __uint_as_float(wd[e] << 16);
                    sv[2 * e + 1] += __uint_as_float(wd[e] & 0xFFFF0000u);
                }
            }
            const bool b4 = (j & 4) != 0, b2 = (j & 2) != 0, b1 = (j & 1) != 0;
            float t4[4], t2[2];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                t4[q] = (b4 ? sv[4 + q] : sv[q]) + __shfl_xor_sync(0xffffffffu, b4 ? sv[q] : sv[4 + q], 4);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                t2[q] = (b2 ? t4[2 + q] : t4[q]) + __shfl_xor_sync(0xffffffffu, b2 ? t4[q] : t4[2 + q], 2);
            sm.col[ah][8 * cg + j] = (b1 ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? t2[0] : t2[1], 1);
        }
        // the next tile's rows: wait, norms, and its S behind A and B
        if (has_next) {
            finish_stage(S1, next_graph);
            issue_s(S1, col1);
        }
        if (!mbar_wait(&sm.mbar_ab, ph_ab)) atomicExch(&sm.abort, 1);
        ph_ab ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (sm.abort) break;

        // ---- (4) accumulators ----
        {
            // anchors: dims [half * D/2, (half + 1) * D/2)
            const int i = 32 * quad + lane;
            const float rsum = sm.row_c[0][i] + sm.row_c[1][i];   // rowsum of C (rounded terms)
            const bool live = i < nv && S0.kacc[i] > 0;
            float* row = a.acc + (size_t)(v0 + i) * a.acc_stride;
#pragma unroll
            for (int c8 = 0; c8 < D / 16; ++c8) {
                const int d0 = half * (D / 2) + 8 * c8;
                float av[8];
                tmem_ld8(tmem + lane_base + col0 + L::kColA + (uint32_t)d0, av);
                if (live) {
                    const uint4 u = *reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(S0.xt) +
                                                                    core_off(i, d0, DP));
                    const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
                    float o[8];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        o[2 * e] = __uint_as_float(wd[e] << 16) * rsum - av[2 * e];
                        o[2 * e + 1] = __uint_as_float(wd[e] & 0xFFFF0000u) * rsum - av[2 * e + 1];
                    }
                    atomicAdd(reinterpret_cast<float4*>(row + d0), make_float4(o[0], o[1], o[2], o[3]));
                    atomicAdd(reinterpret_cast<float4*>(row + d0 + 4), make_float4(o[4], o[5], o[6], o[7]));
                }
            }
            if (live && half == 0) atomicAdd(row + D, sm.row_w[0][i] + sm.row_w[1][i]);
        }
        if (a.symmetric && quad < 2) {
            // partners g = 32 quad + lane, dims [half * D/2, (half + 1) * D/2)
            const int g = 32 * quad + lane;
            const float csum = sm.col[0][g] + sm.col[1][g];
            const float wsum = sm.col[0][kBlockP + g] + sm.col[1][kBlockP + g];
            const int gv = S0.part[g];
            float* row = a.acc + (size_t)gv * a.acc_stride;
#pragma unroll
            for (int c8 = 0; c8 < D / 16; ++c8) {
                const int d0 = half * (D / 2) + 8 * c8;
                float bv[8];
                tmem_ld8(tmem + lane_base + col0 + L::kColB + (uint32_t)d0, bv);
                if (wsum != 0.0f || csum != 0.0f) {
                    const uint4 u = *reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(S0.xp) +
                                                                    core_off(g, d0, DP));
                    const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
                    float o[8];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        o[2 * e] = __uint_as_float(wd[e] << 16) * csum - bv[2 * e];
                        o[2 * e + 1] = __uint_as_float(wd[e] & 0xFFFF0000u) * csum - bv[2 * e + 1];
                    }
                    atomicAdd(reinterpret_cast<float4*>(row + d0), make_float4(o[0], o[1], o[2], o[3]));
                    atomicAdd(reinterpret_cast<float4*>(row + d0 + 4), make_float4(o[4], o[5], o[6], o[7]));
                }
            }
            if (half == 0 && (wsum != 0.0f || csum != 0.0f)) atomicAdd(row + D, wsum);
        }
        cur = nxt;
        nxt = after;
    }
    cp_async_wait_all();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (sm.abort && tid == 0) atomicExch(&a.ps->status, kStatusTimeout);
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(L::kCols));
    hist_merge(hist, a);
    if (tid == 0 && s_used && home >= 0) atomicAdd(&a.gst[home].used, (unsigned long long)s_used);
}

// ---------------------------------------------------------------------------
// k_tile_wait_probe (test only): one CTA set up like a tile CTA -- TMEM
// allocated, mbarrier initialised -- waits for a barrier phase that nothing
// completes (no MMA is issued, nothing committed) with `limit` polls, then
// takes the tile kernel's give-up path: out[0] = the status it records,
// out[1] = 1 once the TMEM is freed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTileThreads) k_tile_wait_probe(int limit, int32_t* out) {
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, w = tid >> 5;
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    if (!mbar_wait(&mbar, 0u, limit)) atomicExch(&abort_flag, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) out[0] = abort_flag ? kStatusTimeout : 0;
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(256));
    __syncthreads();
    if (tid == 0) out[1] = 1;
}

}  // namespace

cudaError_t launch_tile_wait_probe(int limit, int32_t* dev_out, cudaStream_t s) {
    k_tile_wait_probe<<<1, kTileThreads, 0, s>>>(limit, dev_out);
    return cudaGetLastError();
}

bool tile_dim(int d) { return d == 16 || d == 32 || d == 64; }

// Shared memory of the tile kernel: its layout and three of the four
// histogram arrays (edge counts stay zero, the per-slot weights are never
// used: block sampling excludes that policy), at least kTileMinSmem so that
// no more than two CTAs of any tile kernel share an SM (each holds 256 of the
// SM's 512 TMEM columns for the whole launch).
size_t tile_smem_bytes(int d, int bins) {
    size_t base = 0;
    switch (d) {
        case 16: base = sizeof(TileTc<16>); break;
        case 32: base = sizeof(TileTc<32>); break;
        case 64: base = sizeof(TileTc<64>); break;
        default: return 0;
    }
    return std::max<size_t>(base + hist_smem_bytes(bins) / 4 * 3, kTileMinSmem);
}

// CTAs of the tile kernel per SM: what its registers, shared memory and
// TMEM columns allow, at most kTileCtasPerSm.  Worked out here because the
// runtime's occupancy query answers one CTA per SM for this kernel at any
// shared-memory size, although two fit and run side by side (measured: the
// launch with two per SM takes 0.64 of the time of the one with one).
int tile_bf16_blocks_per_sm(int d, int bins) {
    const void* f = nullptr;
    int cols = 0;
    switch (d) {
        case 16: f = (const void*)k_tile_tc<16>; cols = (int)TileTc<16>::kCols; break;
        case 32: f = (const void*)k_tile_tc<32>; cols = (int)TileTc<32>::kCols; break;
        case 64: f = (const void*)k_tile_tc<64>; cols = (int)TileTc<64>::kCols; break;
        default: return 1;
    }
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const size_t smem_cta = tile_smem_bytes(d, bins) + fa.sharedSizeBytes + (size_t)reserved;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;   // allocated per warp in units of 256
    const int by_regs = regs_sm / (regs_warp * (kTileThreads / 32));
    const int by_smem = (int)((size_t)smem_sm / smem_cta);
    const int by_tmem = 512 / cols;
    const int blocks = std::min(std::min(by_regs, by_smem), std::min(by_tmem, kTileCtasPerSm));
    return blocks < 1 ? 1 : blocks;
}

cudaError_t prepare_tile_kernel(int d, int bins) {
    const int smem = (int)tile_smem_bytes(d, bins);
    switch (d) {
        case 16: return raise_smem_limit((const void*)k_tile_tc<16>, smem);
        case 32: return raise_smem_limit((const void*)k_tile_tc<32>, smem);
        case 64: return raise_smem_limit((const void*)k_tile_tc<64>, smem);
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

// blocks_per_sm: CTAs per SM (0: two)
int tile_grid(int n_tile_items, int sm_count, int blocks_per_sm) {
    const int per_sm = blocks_per_sm > 0 ? blocks_per_sm : 2;
    int grid = n_tile_items < sm_count * per_sm ? n_tile_items : sm_count * per_sm;
    return grid < 1 ? 1 : grid;
}

cudaError_t launch_tile_bf16(const EpochArgs& a, int grid, cudaStream_t s) {
    if (a.n_tile_items == 0) return cudaSuccess;
    const size_t smem = tile_smem_bytes(a.d, a.bins);
    switch (a.d) {
        case 16: return launch_critical(k_tile_tc<16>, grid, kTileThreads, smem, s, false, a);
        case 32: return launch_critical(k_tile_tc<32>, grid, kTileThreads, smem, s, false, a);
        case 64: return launch_critical(k_tile_tc<64>, grid, kTileThreads, smem, s, false, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gempe
