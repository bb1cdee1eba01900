// CUDA kernels of the GEMPE epoch (sm_103a).  Every kernel runs on a pack:
// one or more graphs of one dimension in shared device arrays, each work
// unit naming its graph (see engine.cuh).
//
//  k_hash_build    exact edge set (replaces the lossy byte map of Sec. III.C)
//  k_init          initial positions, uniform random (Fig. 4)
//  k_sampler       one epoch's sampled non-edges (Fig. 2 semantics: redraw
//                  while the pair is an edge), drawn ahead of the sweep
//  k_sweep_packed  one epoch's pair sweep for d <= 4: edge parabolas
//  k_sweep         (Eq. 4/5) and sampled non-edges, Eq. 3 terms reduced per
//                  vertex, distance histograms (Sec. III.F); k_sweep for d >= 8
//  k_update        x_i := y_i / z_i (Fig. 4), slope fit per graph (Sec. III.F)
//  k_loss          sampled predictive entropy (Eq. 2) with FP64 sums
//  k_sample        the sampler alone (inspection)
//  k_is_edge       membership probes (inspection)
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "device_math.cuh"
#include "engine.cuh"
#include "f32x2.cuh"
#include "hist.cuh"

namespace gempe {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Mills-ratio interpolation table (identical on every device; filled once
// per device by init_mills_table before the first kernel that reads it).
__device__ MillsCoef g_mills[kMillsIntervals];

// ---------------------------------------------------------------------------
// Graph set-up (one graph of the pack per launch)
// ---------------------------------------------------------------------------
template <bool kNarrow>
__global__ void k_hash_build(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t v0,
                             int32_t n, void* keys_v, unsigned long long bucket_mask, int32_t* fail_flag) {
    using Key = typename std::conditional<kNarrow, unsigned int, unsigned long long>::type;
    constexpr int kPerBucket = kNarrow ? 8 : 4;
    constexpr Key kEmpty = (Key)~0ull;
    Key* keys = static_cast<Key*>(keys_v);
    const int32_t* rp = row_ptr + v0;
    const int64_t e0 = __ldg(rp), e1 = __ldg(rp + n);
    const unsigned long long slot_mask = (unsigned long long)kPerBucket * bucket_mask + (kPerBucket - 1);
    for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = __ldg(col_idx + e) - v0;
        // local row of CSR slot e: the last i with rp[i] <= e
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(rp + mid) <= e) lo = mid; else hi = mid - 1;
        }
        if (j <= lo) continue;   // each undirected edge once, from its lower end
        const Key key = kNarrow ? (Key)edge_key32(lo, j) : (Key)edge_key(lo, j);
        unsigned long long slot = (unsigned long long)kPerBucket * (mix64(key) & bucket_mask);
        bool done = false;
        for (unsigned long long probe = 0; probe <= slot_mask; ++probe) {
            const Key prev = atomicCAS(keys + slot, kEmpty, key);
            if (prev == kEmpty || prev == key) { done = true; break; }
            slot = (slot + 1) & slot_mask;
        }
        if (!done) atomicExch(fail_flag, 1);
    }
}

__global__ void k_init(float* __restrict__ x, __nv_bfloat16* __restrict__ xb, int32_t n, int32_t d,
                       uint32_t key_lo, uint32_t key_hi, float range) {
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
                if (xb) xb[(size_t)i * d + c] = __float2bfloat16_rn(unit * range);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Coordinate chunks: a pair is handled by G = D/P lanes, each owning P of the
// row's coordinates.  The row is cut into 16-byte units (U = 4 coordinates of
// FP32 positions, 8 of BF16 ones); when P is a multiple of U, lane gl owns
// the units gl, gl + G, gl + 2G, ..., so that each load instruction of the
// G lanes reads one contiguous stretch of the row (whole 32-byte sectors);
// otherwise lane gl owns the coordinates [gl*P, gl*P + P).  chunk_unit_off
// gives the first coordinate of the lane's unit q.
// ---------------------------------------------------------------------------
template <int D, int P, int U>
__device__ __forceinline__ int chunk_unit_off(int gl, int q) {
    return U * gl + U * (D / P) * q;
}

template <int D, int P>
__device__ __forceinline__ void load_chunk(const float* __restrict__ x, int row, int gl, float* out) {
    const float* p = x + (size_t)row * D + gl * P;
    if constexpr (P % 4 == 0) {
        const float* r = x + (size_t)row * D;
#pragma unroll
        for (int c = 0; c < P; c += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(r + chunk_unit_off<D, P, 4>(gl, c / 4)));
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

// The same chunk from BF16 positions, widened to FP32 (exact).
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

template <int D, int P>
__device__ __forceinline__ void load_chunk(const __nv_bfloat16* __restrict__ x, int row, int gl, float* out) {
    const __nv_bfloat16* p = x + (size_t)row * D + gl * P;
    if constexpr (P % 8 == 0) {
        const __nv_bfloat16* r = x + (size_t)row * D;
#pragma unroll
        for (int c = 0; c < P; c += 8) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(r + chunk_unit_off<D, P, 8>(gl, c / 8)));
            out[c] = bf16_lo(v.x); out[c + 1] = bf16_hi(v.x); out[c + 2] = bf16_lo(v.y); out[c + 3] = bf16_hi(v.y);
            out[c + 4] = bf16_lo(v.z); out[c + 5] = bf16_hi(v.z); out[c + 6] = bf16_lo(v.w); out[c + 7] = bf16_hi(v.w);
        }
    } else if constexpr (P == 4) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        out[0] = bf16_lo(v.x); out[1] = bf16_hi(v.x); out[2] = bf16_lo(v.y); out[3] = bf16_hi(v.y);
    } else {
        const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
#pragma unroll
        for (int c = 0; c < P; ++c) out[c] = __uint_as_float((uint32_t)__ldg(q + c) << 16);
    }
}

// The same chunks as packed FP32 pairs (P even): coordinates 2c, 2c + 1 in
// the two halves of out[c].
template <int D, int P>
__device__ __forceinline__ void load_pairs(const float* __restrict__ x, int row, int gl, f2* out) {
    static_assert(P % 2 == 0, "packed pairs need an even chunk");
    const float* p = x + (size_t)row * D + gl * P;
    if constexpr (P % 4 == 0) {
        const float* r = x + (size_t)row * D;
#pragma unroll
        for (int c = 0; c < P; c += 4) {
            const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(r + chunk_unit_off<D, P, 4>(gl, c / 4)));
            out[c / 2] = v.x;
            out[c / 2 + 1] = v.y;
        }
    } else {
        out[0] = __ldg(reinterpret_cast<const unsigned long long*>(p));
    }
}

template <int D, int P>
__device__ __forceinline__ void load_pairs(const __nv_bfloat16* __restrict__ x, int row, int gl, f2* out) {
    static_assert(P % 2 == 0, "packed pairs need an even chunk");
    float v[P];
    load_chunk<D, P>(x, row, gl, v);
#pragma unroll
    for (int c = 0; c < P / 2; ++c) out[c] = f2_pack(v[2 * c], v[2 * c + 1]);
}

// acc row layout: D values then z, padded to a multiple of 4 floats.  U:
// the 16-byte unit of the positions the lane's coordinates were loaded with
// (4 for FP32, 8 for BF16), so that v[] maps to the same coordinates.
template <int D, int G, int P, int U = 4>
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
        if constexpr (P % U == 0) {
#pragma unroll
            for (int c = 0; c < P; c += 4) {
                const int off = chunk_unit_off<D, P, U>(gl, c / U) + c % U;
                atomicAdd(reinterpret_cast<float4*>(row + off), make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]));
            }
        } else if constexpr (P % 4 == 0) {
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

__device__ __forceinline__ GraphInfo load_graph(const EpochArgs& a, int g) {
    GraphInfo gi;
    const int4 w0 = __ldg(reinterpret_cast<const int4*>(a.graphs + g));
    const ulonglong2 w1 = __ldg(reinterpret_cast<const ulonglong2*>(a.graphs + g) + 1);
    const ulonglong2 w2 = __ldg(reinterpret_cast<const ulonglong2*>(a.graphs + g) + 2);
    gi.v0 = w0.x;
    gi.n = w0.y;
    gi.t0 = w0.z;
    gi.n_tiles = w0.w;
    gi.key_lo = (uint32_t)w1.x;
    gi.key_hi = (uint32_t)(w1.x >> 32);
    gi.key_off = w1.y;
    gi.bucket_mask = w2.x;
    gi.map = w2.y;
    return gi;
}

// The pack's exact edge sets (key array and width).
struct EdgeSets {
    const void* keys;
    int narrow;
};

__device__ __forceinline__ EdgeSets edge_sets(const EpochArgs& a) { return EdgeSets{a.keys, a.narrow_keys}; }

// ---------------------------------------------------------------------------
// Membership as the sampler sees it (Sec. III.C).  Exact: the graph's edge
// hash set.  Byte map: a byte array of s = 2^b entries in which every edge
// (i, j) marks address ((pi(i) n + pi(j)) * 1103515245) & (s - 1), in 32-bit
// arithmetic with wrap-around, pi a random renaming pi(v) = (alpha v + beta)
// mod n with alpha coprime to n; a draw whose address is marked is taken
// for an edge.  No edge is missed; a non-edge that collides with an edge is
// rejected too, and counted as a false positive against the exact set.
// ---------------------------------------------------------------------------
struct Membership {
    const uint8_t* map;   // null: exact
    uint32_t mask, n, alpha, beta;
};

__device__ __forceinline__ uint32_t gcd_u32(uint32_t x, uint32_t y) {
    while (y != 0u) {
        const uint32_t t = x % y;
        x = y;
        y = t;
    }
    return x;
}

// The renaming of `period`: alpha = 1 + (w0 mod (n - 1)), stepped up (past
// n - 1 back to 1) to the first value coprime to n, beta = w1 mod n, with
// (w0, w1) the first two words of counter (period, 0, 0, kTagRename).
__device__ __forceinline__ void renaming(uint32_t key_lo, uint32_t key_hi, int period, uint32_t n,
                                         uint32_t& alpha, uint32_t& beta) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)period, 0u, 0u, kTagRename), key_lo, key_hi);
    uint32_t al = 1u + (n > 1u ? r.x % (n - 1u) : 0u);
    while (gcd_u32(al, n) != 1u) al = (al + 1u >= n) ? 1u : al + 1u;   // ends at alpha = 1 at the latest
    alpha = al;
    beta = r.y % n;
}

__device__ __forceinline__ int map_period_of(const EpochArgs& a, int sample_epoch) {
    return a.rename_every > 0 ? sample_epoch / a.rename_every : 0;
}

__device__ __forceinline__ Membership membership_of(const EpochArgs& a, const GraphInfo& gi, int sample_epoch) {
    Membership m{nullptr, 0u, (uint32_t)gi.n, 1u, 0u};
    if (!a.membership) return m;
    m.map = a.bytemap + (gi.map & ~63ull);
    m.mask = (uint32_t)((1ull << (gi.map & 63ull)) - 1ull);
    renaming(gi.key_lo, gi.key_hi, map_period_of(a, sample_epoch), m.n, m.alpha, m.beta);
    return m;
}

__device__ __forceinline__ uint32_t renamed(const Membership& m, uint32_t v) {
    return (uint32_t)(((unsigned long long)m.alpha * v + m.beta) % m.n);
}

__device__ __forceinline__ uint32_t map_address(const Membership& m, uint32_t name_i, uint32_t name_j) {
    return ((name_i * m.n + name_j) * 1103515245u) & m.mask;
}

// Is the draw (i, g) taken for an edge?  name_i = pi(i) (byte map only).
__device__ __forceinline__ bool taken_for_edge(const GraphInfo& gi, const EdgeSets& es, const Membership& m,
                                               uint32_t name_i, int i, int g, unsigned& false_pos) {
    if (!m.map) return edge_set_contains(es.keys, es.narrow, gi.key_off, gi.bucket_mask, i, g);
    if (!__ldg(m.map + map_address(m, name_i, renamed(m, (uint32_t)g)))) return false;
    if (!edge_set_contains(es.keys, es.narrow, gi.key_off, gi.bucket_mask, i, g)) ++false_pos;
    return true;
}

// Attempts of sample slot t of local vertex i of a graph: attempt a is word
// t & 3 of counter (i, epoch, t >> 2, tag | a), so one Philox call gives
// attempt a of four consecutive slots.
__device__ __forceinline__ int draw_attempt(const GraphInfo& gi, int i, int epoch, int t, uint32_t tag, int att) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)epoch, (uint32_t)t >> 2, tag | (uint32_t)att),
                                  gi.key_lo, gi.key_hi);
    return draw_vertex(word_of(r, t & 3), (uint32_t)gi.n);
}

// Attempts att0, att0 + 1, ... of slot t of local vertex i (Fig. 2: redraw
// while the pair is taken for an edge; also redraw g == i); the accepted
// partner (local id), or -1 after max_retries attempts in all.  att0 >= 1:
// the caller drew and counted the earlier attempts.
__device__ __forceinline__ int sample_partner_from(const GraphInfo& gi, const EdgeSets& keys, int max_retries,
                                                   int i, int epoch, int t, uint32_t tag, int att0,
                                                   unsigned& rejected, const Membership& m, unsigned& false_pos) {
    const uint32_t name_i = m.map ? renamed(m, (uint32_t)i) : 0u;
    for (int att = att0; att < max_retries; ++att) {
        const int g = draw_attempt(gi, i, epoch, t, tag, att);
        if (g != i && !taken_for_edge(gi, keys, m, name_i, i, g, false_pos)) return g;
        ++rejected;
    }
    return -1;
}

// The LCG form (rng 1) of sample_partner_from: the slot's state after the
// attempts before att0; each further attempt advances it once and draws.
__device__ __forceinline__ int lcg_partner_from(const GraphInfo& gi, const EdgeSets& keys, int max_retries, int i,
                                                uint32_t state, int att0, unsigned& rejected, const Membership& m,
                                                unsigned& false_pos) {
    const uint32_t name_i = m.map ? renamed(m, (uint32_t)i) : 0u;
    for (int att = att0; att < max_retries; ++att) {
        state = lcg_next(state);
        const int g = lcg_vertex(state, gi.n);
        if (g != i && !taken_for_edge(gi, keys, m, name_i, i, g, false_pos)) return g;
        ++rejected;
    }
    return -1;
}

// All attempts of slot t of local vertex i.
__device__ __forceinline__ int sample_partner(const GraphInfo& gi, const EdgeSets& keys, int max_retries, int i,
                                              int epoch, int t, uint32_t tag, unsigned& rejected,
                                              const Membership& m, unsigned& false_pos) {
    return sample_partner_from(gi, keys, max_retries, i, epoch, t, tag, 0, rejected, m, false_pos);
}

// The same with the exact edge set (loss, slope-pass and inspection draws).
__device__ __forceinline__ int sample_partner(const GraphInfo& gi, const EdgeSets& keys, int max_retries,
                                              int i, int epoch, int t, uint32_t tag, unsigned& rejected) {
    unsigned unused = 0u;
    const Membership exact{nullptr, 0u, (uint32_t)gi.n, 1u, 0u};
    return sample_partner_from(gi, keys, max_retries, i, epoch, t, tag, 0, rejected, exact, unused);
}

// Sec. III.C's policy: attempt a of CSR slot e_local of the graph (anchored
// at local vertex i, the slot's row) is word e_local & 3 of counter
// (e_local >> 2, epoch, 0, kTagSlot | a); the partner, or -1 after
// max_retries attempts.  att0 >= 1: the earlier attempts were drawn and
// counted by the caller.
__device__ __forceinline__ int slot_partner_from(const GraphInfo& gi, const EdgeSets& keys, int max_retries,
                                                 int i, int e_local, int epoch, int att0, unsigned& rejected,
                                                 const Membership& m, unsigned& false_pos) {
    const uint32_t name_i = m.map ? renamed(m, (uint32_t)i) : 0u;
    for (int att = att0; att < max_retries; ++att) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)e_local >> 2, (uint32_t)epoch, 0u, kTagSlot | (uint32_t)att),
                                      gi.key_lo, gi.key_hi);
        const int g = draw_vertex(word_of(r, e_local & 3), (uint32_t)gi.n);
        if (g != i && !taken_for_edge(gi, keys, m, name_i, i, g, false_pos)) return g;
        ++rejected;
    }
    return -1;
}

// Sum of the per-thread sampler counters {accepted, rejected, exhausted,
// false positives} over the block, added to a graph's statistics by thread 0
// (all threads must call it).
__device__ __forceinline__ void block_count4(unsigned (&v)[4], unsigned* s_cnt, GraphState* st) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[q] += __shfl_xor_sync(kFull, v[q], o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (v[q]) atomicAdd(&s_cnt[q], v[q]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned acc = s_cnt[0], rej = s_cnt[1], exh = s_cnt[2], fp = s_cnt[3];
        if (acc) atomicAdd(&st->accepted, (unsigned long long)acc);
        if (rej) atomicAdd(&st->rejected, (unsigned long long)rej);
        if (exh) atomicAdd(&st->exhausted, (unsigned long long)exh);
        if (fp) atomicAdd(&st->false_pos, (unsigned long long)fp);
        if (acc + rej) atomicAdd(&st->draws, (unsigned long long)(acc + rej));
        s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = 0u;
}

// Sampler completion: the last block to finish advances every stepped
// graph's sample_epoch (every block has read them by then).
__device__ __forceinline__ void sampler_done(const EpochArgs& a) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.ps->sample_done, 1u);
        s_last = (prev == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        for (int t = threadIdx.x; t < a.n_graphs; t += blockDim.x) {
            GraphState* st = a.gst + t;
            st->sample_epoch = st->sample_epoch + 1;
        }
        if (threadIdx.x == 0) a.ps->sample_done = 0u;
        __threadfence();
    }
}

template <typename PT> __device__ __forceinline__ const PT* pos_of(const EpochArgs& a);
template <> __device__ __forceinline__ const float* pos_of<float>(const EpochArgs& a) { return a.x; }
template <> __device__ __forceinline__ const __nv_bfloat16* pos_of<__nv_bfloat16>(const EpochArgs& a) { return a.xb; }

// ---------------------------------------------------------------------------
// The sampler: for every graph of the pack, the k samples of each vertex for
// the graph's epoch sample_epoch, written to samples[sample_epoch & 1] as pack
// rows.  It depends on the graph and the epoch only, so it runs beside the
// previous epoch's sweep.  A thread takes one vertex's group of (up to) four
// consecutive slots, whose first attempts come from one Philox call; a
// rejected slot draws its further attempts alone.  Blocks take pieces of
// sampler_piece(k) vertices of the vertex chunks (one graph each).
// ---------------------------------------------------------------------------
__host__ __device__ inline int sampler_groups(int k) { return (k + 3) / 4; }
__host__ __device__ inline int sampler_piece(int k) {
    const int g = sampler_groups(k);
    return g > 0 ? 256 / g : 256;
}

template <bool kMap>
__global__ void __launch_bounds__(256, kMap ? 3 : 5) k_sampler(const EpochArgs a) {
    __shared__ unsigned s_cnt[4];
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int k = a.k;
    const int groups = sampler_groups(k), piece = sampler_piece(k);
    const int per_chunk = (kVChunk + piece - 1) / piece;
    const int n_sub = a.n_vchunks * per_chunk;
    const EdgeSets es = edge_sets(a);
    unsigned c[4] = {0u, 0u, 0u, 0u};   // accepted, rejected, exhausted, false positives of graph cur
    int cur = -1;                       // block-uniform
    Membership m{nullptr, 0u, 0u, 1u, 0u};
    for (int s = blockIdx.x; s < n_sub; s += gridDim.x) {
        const int4 ch = __ldg(a.vchunks + s / per_chunk);
        const int sub = s % per_chunk;
        const int cnt = min(piece, ch.y - sub * piece);
        if (cnt <= 0) continue;   // uniform over the block
        const int graph = ch.z;
        const GraphInfo gi = load_graph(a, graph);
        const int se = a.gst[graph].sample_epoch;
        if (graph != cur) {
            // the counts go to the graph's statistics once per run of pieces of one graph
            if (cur >= 0) block_count4(c, s_cnt, a.gst + cur);
            cur = graph;
            if (kMap) m = membership_of(a, gi, se);
            // the map holds this period now (the map builders, which read it, ran before)
            if (kMap && threadIdx.x == 0) a.gst[graph].map_period = map_period_of(a, se);
        }
        const int row0 = ch.x + sub * piece;
        const int vi = threadIdx.x / groups, q = threadIdx.x - vi * groups;
        if (vi < cnt) {
            const int i = row0 - gi.v0 + vi;
            const uint32_t name_i = kMap ? renamed(m, (uint32_t)i) : 0u;
            // Philox: attempt 0 of the four slots; LCG (rng 1): the four slots' seeds
            const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)se, (uint32_t)q, a.rng ? kTagLcg : kTagEpoch),
                                          gi.key_lo, gi.key_hi);
            int32_t* out = a.samples + ((size_t)(se & 1) * a.rows + row0 + vi) * k;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int t = 4 * q + w;
                if (t >= k) break;
                uint32_t st = word_of(r, w);
                int g;
                if (a.rng) {
                    st = lcg_next(st);
                    g = lcg_vertex(st, gi.n);
                } else {
                    g = draw_vertex(st, (uint32_t)gi.n);
                }
                if (g == i || taken_for_edge(gi, es, m, name_i, i, g, c[3])) {
                    ++c[1];
                    g = a.rng ? lcg_partner_from(gi, es, a.max_retries, i, st, 1, c[1], m, c[3])
                              : sample_partner_from(gi, es, a.max_retries, i, se, t, kTagEpoch, 1, c[1], m, c[3]);
                }
                out[t] = g >= 0 ? gi.v0 + g : -1;
                if (g >= 0) ++c[0]; else ++c[2];
            }
        }
    }
    if (cur >= 0) block_count4(c, s_cnt, a.gst + cur);
    sampler_done(a);
}

// ---------------------------------------------------------------------------
// Byte-map (re)build for the renaming period of each graph's sample epoch,
// run before the sampler on the sampler's stream.  A graph's map is rebuilt
// when it does not hold that period (the sampler records the period it used)
// or when force is set (at create): k_bytemap_clear zeroes it, then
// k_bytemap_mark sets the byte of every CSR slot (i, j) -- both orientations
// of each edge, one warp per row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool map_due(const EpochArgs& a, int graph, int force) {
    if (force) return true;
    const GraphState* st = a.gst + graph;
    return st->map_period != map_period_of(a, st->sample_epoch);
}

__global__ void __launch_bounds__(256) k_bytemap_clear(const EpochArgs a, int force) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int g = 0; g < a.n_graphs; ++g) {
        if (!map_due(a, g, force)) continue;
        const unsigned long long mp = a.graphs[g].map;
        uint4* p = reinterpret_cast<uint4*>(a.bytemap + (mp & ~63ull));
        const size_t words = (1ull << (mp & 63ull)) / sizeof(uint4);
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < words; q += stride)
            p[q] = make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void __launch_bounds__(256) k_bytemap_mark(const EpochArgs a, int force) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int c = blockIdx.x; c < a.n_vchunks; c += gridDim.x) {
        const int4 ch = __ldg(a.vchunks + c);
        const int graph = ch.z;
        if (!map_due(a, graph, force)) continue;
        const GraphInfo gi = load_graph(a, graph);
        const Membership m = membership_of(a, gi, a.gst[graph].sample_epoch);
        uint8_t* map = a.bytemap + (gi.map & ~63ull);
        for (int v = warp; v < ch.y; v += warps) {
            const int row = ch.x + v;
            const uint32_t name_i = renamed(m, (uint32_t)(row - gi.v0));
            const int e1 = __ldg(a.row_ptr + row + 1);
            for (int e = __ldg(a.row_ptr + row) + lane; e < e1; e += 32) {
                const uint32_t j = (uint32_t)(__ldg(a.col_idx + e) - gi.v0);
                map[map_address(m, name_i, renamed(m, j))] = 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The per-slot sampler (Sec. III.C's policy) over 64-vertex pieces: a thread
// takes a group of four consecutive CSR slots (graph-local slot numbers 4g ..
// 4g + 3, cut to the piece), whose first attempts come from one Philox call;
// each slot's row is found by a binary search in the piece's row offsets
// (shared memory) and advanced from slot to slot.  The accepted count of
// every vertex of the piece goes to vacc for the sweep's histogram weights.
// ---------------------------------------------------------------------------
template <bool kMap>
__global__ void __launch_bounds__(256) k_sampler_slots(const EpochArgs a) {
    __shared__ unsigned s_cnt[4];
    __shared__ int s_rp[kSamplerSub + 1];
    __shared__ int s_acc[kSamplerSub];
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0u;
    constexpr int kSubs = kVChunk / kSamplerSub;
    const int n_sub = a.n_vchunks * kSubs;
    const EdgeSets es = edge_sets(a);
    unsigned c[4] = {0u, 0u, 0u, 0u};   // accepted, rejected, exhausted, false positives of graph cur
    int cur = -1;                       // block-uniform
    Membership m{nullptr, 0u, 0u, 1u, 0u};
    for (int s = blockIdx.x; s < n_sub; s += gridDim.x) {
        const int4 ch = __ldg(a.vchunks + s / kSubs);
        const int sub = s % kSubs;
        const int cnt = min(kSamplerSub, ch.y - sub * kSamplerSub);
        if (cnt <= 0) continue;   // uniform over the block
        const int graph = ch.z;
        const GraphInfo gi = load_graph(a, graph);
        const int se = a.gst[graph].sample_epoch;
        if (graph != cur) {
            if (cur >= 0) block_count4(c, s_cnt, a.gst + cur);
            cur = graph;
            if (kMap) m = membership_of(a, gi, se);
            if (kMap && threadIdx.x == 0) a.gst[graph].map_period = map_period_of(a, se);
        }
        const int row0 = ch.x + sub * kSamplerSub;
        __syncthreads();   // the previous piece's shared data is no longer read
        for (int t = threadIdx.x; t <= cnt; t += blockDim.x) s_rp[t] = __ldg(a.row_ptr + row0 + t);
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) s_acc[t] = 0;
        __syncthreads();
        const int s0 = __ldg(a.row_ptr + gi.v0);   // the graph's first CSR slot
        int32_t* out = a.samples + (size_t)(se & 1) * (size_t)a.n_slots;
        const int e0 = s_rp[0], e1 = s_rp[cnt];
        const int g_first = (e0 - s0) >> 2, g_last = e1 > e0 ? (e1 - 1 - s0) >> 2 : g_first - 1;
        for (int grp = g_first + (int)threadIdx.x; grp <= g_last; grp += blockDim.x) {
            const int ea = max(e0, s0 + 4 * grp), eb = min(e1, s0 + 4 * grp + 4);
            int lo = 0, hi = cnt - 1;   // row of slot ea: the last r with s_rp[r] <= ea
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_rp[mid] <= ea) lo = mid; else hi = mid - 1;
            }
            const uint4 r = philox4x32_10(make_uint4((uint32_t)grp, (uint32_t)se, 0u, a.rng ? kTagLcgSlot : kTagSlot),
                                          gi.key_lo, gi.key_hi);
            for (int e = ea; e < eb; ++e) {
                while (s_rp[lo + 1] <= e) ++lo;   // rows may be empty
                const int i = row0 + lo - gi.v0, el = e - s0;
                const uint32_t name_i = kMap ? renamed(m, (uint32_t)i) : 0u;
                uint32_t st = word_of(r, el & 3);
                int g;
                if (a.rng) {
                    st = lcg_next(st);
                    g = lcg_vertex(st, gi.n);
                } else {
                    g = draw_vertex(st, (uint32_t)gi.n);
                }
                if (g == i || taken_for_edge(gi, es, m, name_i, i, g, c[3])) {
                    ++c[1];
                    g = a.rng ? lcg_partner_from(gi, es, a.max_retries, i, st, 1, c[1], m, c[3])
                              : slot_partner_from(gi, es, a.max_retries, i, el, se, 1, c[1], m, c[3]);
                }
                out[e] = g >= 0 ? gi.v0 + g : -1;
                if (g >= 0) {
                    ++c[0];
                    atomicAdd(&s_acc[lo], 1);
                } else {
                    ++c[2];
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) a.vacc[(size_t)(se & 1) * a.rows + row0 + t] = s_acc[t];
    }
    if (cur >= 0) block_count4(c, s_cnt, a.gst + cur);
    sampler_done(a);
}

// ---------------------------------------------------------------------------
// Packed pair sweep for d <= 4 (one lane per pair).
//
// A work unit is either up to 32 consecutive vertices of one graph whose edge
// slots plus sample slots number at most the unit pair budget, or one chunk
// of a hub's CSR row (the hub's samples ride in its last chunk).  The warp
// lays the unit's pairs out vertex by vertex, 32 per round; a lane finds its
// vertex by a shuffle binary search over the per-vertex offsets.  Per-vertex
// sums are formed by a segmented warp scan and kept in a per-warp shared row
// until the unit ends, then added to the global accumulator with one vector
// atomic per vertex.  Sampled partners receive their term by vector atomics.
//
// Oriented form (a.oriented, the k-per-vertex policy): the edge slots are
// those of the degree-oriented CSR, in which each undirected edge appears
// once, at the endpoint with the larger (degree, id); that endpoint
// evaluates the pair and the other receives its term by a vector atomic,
// like a sampled partner.  Each edge's term is then evaluated once instead
// of once per endpoint, and no vertex receives more atomics than it has
// neighbours of larger degree, so hubs (which process their whole rows)
// see few.
// ---------------------------------------------------------------------------
template <int D>
struct PackedAcc {
    static constexpr int kStride = ((D + 1) + 3) / 4 * 4;   // floats per vertex row
};

template <int D, bool kOriented>
__global__ void __launch_bounds__(kPackedThreads, 3) k_sweep_packed(const EpochArgs a) {
    constexpr int AS = PackedAcc<D>::kStride;
    constexpr int kWarps = kPackedThreads / 32;
    extern __shared__ unsigned int s_u32[];
    const BlockHist hist = block_hist(s_u32, a.bins, home_graph(a));
    int* s_g_all = reinterpret_cast<int*>(s_u32 + 3 * a.bins);            // [warps][kUnitSampleCap]
    float* s_acc_all = reinterpret_cast<float*>(s_g_all + kWarps * kUnitSampleCap);   // [warps][32][AS]
    __shared__ unsigned int s_used;
    hist_clear(hist, a.bins);
    if (threadIdx.x == 0) s_used = 0u;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int* s_g = s_g_all + wib * kUnitSampleCap;
    float* s_acc = s_acc_all + wib * 32 * AS;
    const int k = a.k;
    const UnitRange ur = warp_units(a);

    for (int it = ur.begin; it < ur.end; it += ur.step) {
        const int4 unit = __ldg(a.items + it);
        const int v0 = unit.x, nv = unit.y & ((1 << kGraphShift) - 1), graph = unit.y >> kGraphShift;
        const bool whole_rows = unit.z < 0;
        const bool slots = !kOriented && a.per_slot != 0;   // Sec. III.C's policy: one sample per CSR slot
        const bool has_s = (unit.w & kUnitHasSamples) && (k > 0 || slots);
        const int e_lo = whole_rows ? 0 : unit.z;
        const int e_hi = unit.w & ~kUnitHasSamples;
        const float sigma = a.gst[graph].sigma;
        const int epoch = a.gst[graph].epoch;
        const PairConsts K = make_pair_consts(a.mu, sigma, a.w_formula == 1, a.clamp_neg_d, g_mills);
        const int32_t* samples =
            a.samples + (size_t)(epoch & 1) * (slots ? (size_t)a.n_slots : (size_t)a.rows * k);

        // per-vertex layout: lane l < nv describes vertex v0 + l (edge slots
        // from the oriented CSR in the oriented form; deg is the full degree)
        const int32_t* erow = kOriented ? a.orow_ptr : a.row_ptr;
        int rs = 0, deg = 0, ne = 0;
        if (lane < nv) {
            rs = __ldg(erow + v0 + lane);
            const int deg_e = __ldg(erow + v0 + lane + 1) - rs;
            deg = kOriented ? __ldg(a.row_ptr + v0 + lane + 1) - __ldg(a.row_ptr + v0 + lane) : deg_e;
            ne = whole_rows ? deg_e : e_hi - e_lo;
        }
        const int ebase = rs + e_lo;
        const int np = (lane < nv) ? ne + (has_s ? (slots ? ne : k) : 0) : 0;
        int incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - np;
        const int total = __shfl_sync(kFull, incl, 31);
        if (lane < nv) {
#pragma unroll
            for (int c = 0; c < AS; ++c) s_acc[lane * AS + c] = 0.0f;
        }

        // the unit's sampled partners (contiguous in the sample buffer); in the
        // per-slot policy they are read pair by pair and counted per vertex
        // by the sampler
        int k_acc = 0;
        if (has_s && slots) {
            if (lane < nv) k_acc = __ldg(a.vacc + (size_t)(epoch & 1) * a.rows + v0 + lane);
        } else if (has_s) {
            const int ns = nv * k;
            const int32_t* src = samples + (size_t)v0 * k;
            for (int s = lane; s < ns; s += 32) s_g[s] = __ldg(src + s);
            __syncwarp();
            if (lane < nv)
                for (int t = 0; t < k; ++t) k_acc += (s_g[lane * k + t] >= 0);
            int unit_used = k_acc;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) unit_used += __shfl_xor_sync(kFull, unit_used, o);
            if (lane == 0 && unit_used) {
                if (graph == hist.home) atomicAdd(&s_used, (unsigned)unit_used);
                else atomicAdd(&a.gst[graph].used, (unsigned long long)unit_used);
            }
        }
        __syncwarp();
        int slot_used = 0;   // per-slot policy: accepted samples this lane processed

        for (int base = 0; base < total; base += 32) {
            const int q = base + lane;
            const bool active = q < total;
            // vertex of pair q: the last lane l with excl_l <= q
            int l = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = l + step;
                const int e = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && e <= q) l = cand;
            }
            const int r = q - __shfl_sync(kFull, excl, l);
            const int ne_l = __shfl_sync(kFull, ne, l);
            const int eb_l = __shfl_sync(kFull, ebase, l);
            const int deg_l = __shfl_sync(kFull, deg, l);
            const int kacc_l = __shfl_sync(kFull, k_acc, l);
            const int v = v0 + l;
            const bool is_edge = r < ne_l;
            int j = -1;
            if (active) {
                if (is_edge) j = __ldg((kOriented ? a.ocol_idx : a.col_idx) + eb_l + r);
                else j = slots ? __ldg(samples + eb_l + (r - ne_l)) : s_g[l * k + (r - ne_l)];
            }
            const bool valid = active && j >= 0;
            slot_used += (slots && valid && !is_edge) ? 1 : 0;

            float val[D + 1];
#pragma unroll
            for (int c = 0; c <= D; ++c) val[c] = 0.0f;
            if (valid) {
                float xv[D], xj[D];
                load_chunk<D, D>(a.x, v, 0, xv);
                load_chunk<D, D>(a.x, j, 0, xj);
                float diff[D];
                float ss = 0.0f;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    diff[c] = xv[c] - xj[c];
                    ss = fmaf(diff[c], diff[c], ss);
                }
                float delta, inv_delta;
                dist_of(ss, delta, inv_delta);
                const PairTerm t = pair_term(delta, inv_delta, is_edge, K);
#pragma unroll
                for (int c = 0; c < D; ++c) val[c] = t.c * diff[c];
                val[D] = t.w;
                const int bin = min((int)(delta * a.hist_scale), a.bins - 1);
                if (is_edge) {
                    if (kOriented || j > v) hist_edge(hist, a, graph, bin);
                } else {
                    if (slots) hist_sample_w(hist, a, graph, bin, deg_l, kacc_l);
                    else hist_sample(hist, a, graph, bin, deg_l, kacc_l, k);
                }
                // the other endpoint of an oriented edge, or a sampled partner
                if (is_edge ? kOriented : a.symmetric) {
                    float pv[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) pv[c] = -val[c];
                    acc_add<D, 1, D>(a.acc + (size_t)j * a.acc_stride, 0, pv, t.w);
                }
            }
            // segmented inclusive scan over lanes of the same vertex
            const int seg = active ? l : 32 + lane;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int seg_up = __shfl_up_sync(kFull, seg, o);
#pragma unroll
                for (int c = 0; c <= D; ++c) {
                    const float t = __shfl_up_sync(kFull, val[c], o);
                    if (lane >= o && seg_up == seg) val[c] += t;
                }
            }
            const int seg_next = __shfl_down_sync(kFull, seg, 1);
            if (active && (lane == 31 || seg_next != seg)) {
#pragma unroll
                for (int c = 0; c <= D; ++c) s_acc[l * AS + c] += val[c];
            }
            __syncwarp();
        }
        if (slots) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) slot_used += __shfl_xor_sync(kFull, slot_used, o);
            if (lane == 0 && slot_used) {
                if (graph == hist.home) atomicAdd(&s_used, (unsigned)slot_used);
                else atomicAdd(&a.gst[graph].used, (unsigned long long)slot_used);
            }
        }
        // one vector atomic per vertex into the global accumulator
        if (lane < nv && s_acc[lane * AS + D] != 0.0f) {
            float row[D];
#pragma unroll
            for (int c = 0; c < D; ++c) row[c] = s_acc[lane * AS + c];
            acc_add<D, 1, D>(a.acc + (size_t)(v0 + lane) * a.acc_stride, 0, row, s_acc[lane * AS + D]);
        }
        __syncwarp();
    }
    asm volatile("griddepcontrol.launch_dependents;");   // the update may be scheduled (it waits for this grid)
    __syncthreads();
    hist_merge(hist, a);
    if (threadIdx.x == 0 && s_used && hist.home >= 0) atomicAdd(&a.gst[hist.home].used, (unsigned long long)s_used);
}

// ---------------------------------------------------------------------------
// Pair sweep for d >= 8.  A warp is 32/G lane groups of G lanes; each group
// owns one work unit (a vertex with its samples, or one chunk of a hub's
// row), lane gl of the group owning P = D/G coordinates of every row (the
// 16-byte units gl, gl + G, ... of the row when P is a multiple of a unit:
// each load instruction of the group then reads a contiguous stretch).  The host packs the units into warp tasks of 32/G units of
// similar size, so the groups of a warp run the same number of rounds.
//
// A round takes G pairs of the group's vertex, one per lane:
//   (A) G sub-rounds: the group gathers pair s's row chunk by chunk and sums
//       the squared differences over its lanes; lane s keeps the distance;
//   (B) every lane evaluates the pair term of its own pair (one math pass
//       per G pairs per group, 32 per warp);
//   (C) G sub-rounds: the group gathers pair s's row again (an L1 hit) and
//       adds c (x_i - x_j) to its own coordinates of the vertex's sum, and
//       the negated term to a sampled partner's accumulator row.
// Each lane's vertex sum covers its own coordinates, so no reduction across
// lanes is needed except for z.
// ---------------------------------------------------------------------------
template <int D, int G, typename PT>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(const EpochArgs a) {
    constexpr int P = D / G;
    constexpr int PG = 32 / G;            // groups (units) per warp task
    constexpr int kU = sizeof(PT) == 2 ? 8 : 4;   // coordinates per 16-byte unit of the positions
    const PT* X = pos_of<PT>(a);
    extern __shared__ unsigned int s_u32[];
    // block b takes the tasks [bounds[b], bounds[b+1]) (ranges of equal
    // estimated work, cut on the host) and hands them to its warps one at a
    // time (a shared counter), so that its warps finish together
    const int t_lo = __ldg(a.task_bounds + blockIdx.x);
    const int t_end = __ldg(a.task_bounds + blockIdx.x + 1);
    const int home = (a.n_graphs == 1) ? 0 : (t_lo < t_end ? (__ldg(&a.items[(size_t)t_lo * PG].y) >> kGraphShift) : -1);
    const BlockHist hist = block_hist(s_u32, a.bins, home);
    __shared__ unsigned int s_used;
    __shared__ int s_next;
    hist_clear(hist, a.bins);
    if (threadIdx.x == 0) {
        s_used = 0u;
        s_next = t_lo;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int gl = lane % G;               // lane within the group
    const int gbase = lane - gl;           // first lane of the group
    const bool block = a.block_P > 0;
    const bool slots = a.per_slot != 0;          // Sec. III.C's policy: one sample per CSR slot
    const int k_eff = block ? kBlockP : a.k;     // sample slots per vertex (k and block forms)

    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(&s_next, 1);
        task = __shfl_sync(kFull, task, 0);
        if (task >= t_end) break;
        const int4 item = __ldg(a.items + (size_t)task * PG + lane / G);
        const int i = item.x;                              // -1: padding
        const int graph = item.y >> kGraphShift;
        const bool live = i >= 0;
        const bool has_samples = live && (item.w & kUnitHasSamples) && (k_eff > 0 || slots) && a.sweep_samples;
        const int p0 = item.z, p1 = item.w & ~kUnitHasSamples;
        const float sigma = a.gst[graph].sigma;
        const int epoch = a.gst[graph].epoch;
        const PairConsts K = make_pair_consts(a.mu, sigma, a.w_formula == 1, a.clamp_neg_d, g_mills);
        int e0 = 0, deg = 0;
        float xi[P];
        if (live) {
            e0 = __ldg(a.row_ptr + i);
            deg = __ldg(a.row_ptr + i + 1) - e0;
            load_chunk<D, P>(X, i, gl, xi);
        } else {
#pragma unroll
            for (int c = 0; c < P; ++c) xi[c] = 0.0f;
        }
        const int ne = live ? p1 - p0 : 0;
        // the vertex's sampled partners: masks / buffer, accepted count
        int k_acc = 0;
        unsigned long long bmask_v = 0ull;
        const int32_t* tp = nullptr;
        const int32_t* sp = nullptr;
        if (has_samples && slots) {
            sp = a.samples + (size_t)(epoch & 1) * (size_t)a.n_slots + e0 + p0;   // this unit's slots
            k_acc = __ldg(a.vacc + (size_t)(epoch & 1) * a.rows + i);
        } else if (has_samples) {
            if (block) {
                unsigned long long* bm = a.block_mask + (size_t)(epoch & 1) * (size_t)a.rows + i;
                bmask_v = *bm;
                const int gv0 = __ldg(&a.graphs[graph].v0), gt0 = __ldg(&a.graphs[graph].t0);
                const int tile = gt0 + (i - gv0) / kBlockT;
                tp = a.block_part + ((size_t)(epoch & 1) * (size_t)a.n_tiles + tile) * kBlockP;
                k_acc = kBlockP - __popcll(bmask_v);
            } else {
                sp = a.samples + ((size_t)(epoch & 1) * (size_t)a.rows + i) * a.k;
                for (int t = gl; t < a.k; t += G) k_acc += (__ldg(sp + t) >= 0);
            }
        }
        // group sum of the per-vertex count: every lane of the warp takes part
        // (groups without samples add zeros); the block form's count is
        // already complete in every lane of its group
        if (!block && !slots) {
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) k_acc += __shfl_xor_sync(kFull, k_acc, o);
        }
        __syncwarp();
        if (has_samples && !slots && gl == 0) {
            if (block) a.block_mask[(size_t)(epoch & 1) * (size_t)a.rows + i] = 0ull;   // read once
            if (k_acc) {
                if (graph == home) atomicAdd(&s_used, (unsigned)k_acc);
                else atomicAdd(&a.gst[graph].used, (unsigned long long)k_acc);
            }
        }
        const int total = ne + (has_samples ? (slots ? ne : k_eff) : 0);
        int slot_used = 0;   // per-slot policy: accepted samples this lane evaluated
        const int rounds = (total + G - 1) / G;
        const int rmax = (int)__reduce_max_sync(kFull, (unsigned)rounds);
        // the partners' weights travel only when some group of the warp has
        // samples whose terms go to the partners as well
        const bool pass_w = a.symmetric && __any_sync(kFull, has_samples);

        // even chunks run on packed FP32 pairs (coordinates 2c, 2c + 1 in the
        // two halves of a 64-bit register: the same roundings, half the
        // instructions); odd ones (d <= 4 with one lane per vertex) on scalars
        constexpr bool kPk = (P % 2 == 0);
        constexpr int PH = kPk ? P / 2 : 1;
        f2 xi2[PH], dacc2[PH];
#pragma unroll
        for (int c = 0; c < PH; ++c) {
            xi2[c] = kPk ? f2_pack(xi[2 * c], xi[(2 * c + 1) % P]) : 0ull;
            dacc2[c] = 0ull;
        }
        float dacc[P];
#pragma unroll
        for (int c = 0; c < P; ++c) dacc[c] = 0.0f;
        float zacc = 0.0f;
        for (int r = 0; r < rmax; ++r) {
            // this lane's pair of the round
            const int q = r * G + gl;
            int my_j = -1;
            if (q < ne) {
                my_j = __ldg(a.col_idx + e0 + p0 + q);
            } else if (q < total) {
                const int t = q - ne;
                if (block) my_j = ((bmask_v >> t) & 1ull) ? -1 : __ldg(tp + t);
                else my_j = __ldg(sp + t);
            }
            // the lane's partner row on its way to L1 before the group's
            // gathers reach it
            if (my_j >= 0) {
                const char* rp = reinterpret_cast<const char*>(X + (size_t)my_j * D);
#pragma unroll
                for (int b = 0; b < D * (int)sizeof(PT); b += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(rp + b));
            }
            // (A) distances
            float my_ss = 0.0f;
#pragma unroll
            for (int s2 = 0; s2 < G; ++s2) {
                const int j = __shfl_sync(kFull, my_j, gbase + s2);
                float ss = 0.0f;
                if constexpr (kPk) {
                    f2 a2 = 0ull;
                    if (j >= 0) {
                        f2 xj2[PH];
                        load_pairs<D, P>(X, j, gl, xj2);
#pragma unroll
                        for (int c = 0; c < PH; ++c) {
                            const f2 t = f2_sub(xi2[c], xj2[c]);
                            a2 = f2_fma(t, t, a2);
                        }
                    }
                    float lo, hi;
                    f2_unpack(a2, lo, hi);
                    ss = lo + hi;
                } else {
                    float xj[P];
                    if (j >= 0) {
                        load_chunk<D, P>(X, j, gl, xj);
                    } else {
#pragma unroll
                        for (int c = 0; c < P; ++c) xj[c] = xi[c];
                    }
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        const float df = xi[c] - xj[c];
                        ss = fmaf(df, df, ss);
                    }
                }
#pragma unroll
                for (int o = G / 2; o >= 1; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
                if (gl == s2) my_ss = ss;
            }
            
            // (B) the pair term of this lane's pair
            const bool my_edge = q < ne;
            float my_c = 0.0f, my_w = 0.0f;
            if (my_j >= 0) {
                float delta, inv_delta;
                dist_of(my_ss, delta, inv_delta);
                const PairTerm t = pair_term(delta, inv_delta, my_edge, K);
                my_c = t.c;
                my_w = t.w;
                zacc += t.w;
                const int bin = min((int)(delta * a.hist_scale), a.bins - 1);
                if (my_edge) {
                    if (my_j > i) hist_edge(hist, a, graph, bin);
                } else if (slots) {
                    hist_sample_w(hist, a, graph, bin, deg, k_acc);
                    ++slot_used;
                } else {
                    hist_sample(hist, a, graph, bin, deg, k_acc, k_eff);
                }
            }
            // (C) the vertex's sum and the sampled partners' terms
#pragma unroll
            for (int s2 = 0; s2 < G; ++s2) {
                const int j = __shfl_sync(kFull, my_j, gbase + s2);
                const float c = __shfl_sync(kFull, my_c, gbase + s2);
                const float wv = pass_w ? __shfl_sync(kFull, my_w, gbase + s2) : 0.0f;
                if constexpr (kPk) {
                  if (j >= 0) {
                    f2 xj2[PH], d2[PH];
                    load_pairs<D, P>(X, j, gl, xj2);
                    const f2 c2 = f2_pack(c, c);
#pragma unroll
                    for (int cc = 0; cc < PH; ++cc) {
                        d2[cc] = f2_sub(xi2[cc], xj2[cc]);
                        dacc2[cc] = f2_fma(c2, d2[cc], dacc2[cc]);
                    }
                    if (r * G + s2 >= ne && a.symmetric) {
                        float pv[P];
                        const f2 nc2 = f2_pack(-c, -c);
#pragma unroll
                        for (int cc = 0; cc < PH; ++cc) f2_unpack(f2_mul(nc2, d2[cc]), pv[2 * cc], pv[(2 * cc + 1) % P]);
                        acc_add<D, G, P, kU>(a.acc + (size_t)j * a.acc_stride, gl, pv, wv);
                    }
                  }
                } else if (j >= 0) {
                    float xj[P];
                    load_chunk<D, P>(X, j, gl, xj);
                    float diff[P];
#pragma unroll
                    for (int cc = 0; cc < P; ++cc) {
                        diff[cc] = xi[cc] - xj[cc];
                        dacc[cc] = fmaf(c, diff[cc], dacc[cc]);
                    }
                    if (r * G + s2 >= ne && a.symmetric) {
                        float pv[P];
#pragma unroll
                        for (int cc = 0; cc < P; ++cc) pv[cc] = -c * diff[cc];
                        acc_add<D, G, P, kU>(a.acc + (size_t)j * a.acc_stride, gl, pv, wv);
                    }
                }
            }
        }
        // z over the group; each lane adds its own coordinates of the sum
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) zacc += __shfl_xor_sync(kFull, zacc, o);
        if (slots) {
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) slot_used += __shfl_xor_sync(kFull, slot_used, o);
            if (gl == 0 && slot_used) {
                if (graph == home) atomicAdd(&s_used, (unsigned)slot_used);
                else atomicAdd(&a.gst[graph].used, (unsigned long long)slot_used);
            }
        }
        if constexpr (kPk) {
#pragma unroll
            for (int c = 0; c < PH; ++c) f2_unpack(dacc2[c], dacc[2 * c], dacc[(2 * c + 1) % P]);
        }
        if (total > 0) acc_add<D, G, P, kU>(a.acc + (size_t)i * a.acc_stride, gl, dacc, zacc);
    }
    asm volatile("griddepcontrol.launch_dependents;");   // the update may be scheduled (it waits for this grid)
    __syncthreads();
    hist_merge(hist, a);
    if (threadIdx.x == 0 && s_used && home >= 0) atomicAdd(&a.gst[home].used, (unsigned long long)s_used);
}

// ---------------------------------------------------------------------------
// Sec. III.F: the slope sigma at which dPE/dsigma = 0 on the histograms.
//
// With t = ln sigma and u = (centre - mu)/sigma (du/dt = -u), the sign of
// dPE/dsigma is the sign of
//   F(t)  = sum_b c_e[b] (-u h(u)) + c_n[b] (u g(u)),     g(u) = h(-u),
// and, from h' = h (h - u) = h T,
//   F'(t) = sum_b c_e[b] u h (1 + u T(u)) - c_n[b] u g (1 - u T(-u)).
// The paper bisects in log sigma on [1e-3, 1e3] (no sign change: the end
// with the lower entropy).  The same root is found here by Newton steps in t
// from the previous sigma, with that bracket as the fallback (see
// block_fit_sigma).  One whole block runs the search on a shared-memory copy
// of the histograms: per-bin terms in FP32, block sums by warp shuffles, the
// step by one thread.
// ---------------------------------------------------------------------------
struct SigmaSmem {
    float4 part[32];
    float inv_s;
    int done;
    int iters;
};

// F and F' terms of one bin at 1/sigma = inv_s (F without the positive
// factor); tab: the Mills-ratio table copied to shared memory.
__device__ __forceinline__ float2 dpe_bin(float ce, float cn, float centre, float mu, float inv_s,
                                          const MillsCoef* tab) {
    const float u = (centre - mu) * inv_s;
    float h, T, g, Tn;
    mills_t<false>(u, h, T, tab);     // edge side: h(u), T(u)
    mills_t<false>(-u, g, Tn, tab);   // non-edge side: g(u) = h(-u), T(-u) = g + u
    const float uh = u * h, ug = u * g;
    return make_float2(fmaf(ce, -uh, cn * ug),
                       fmaf(ce * uh, fmaf(u, T, 1.0f), -cn * ug * fmaf(-u, Tn, 1.0f)));
}

// Block sum of a float4 held by every thread; the result is valid in warp 0.
__device__ __forceinline__ float4 block_sum4(float4 v, SigmaSmem& sm) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        v.x += __shfl_xor_sync(kFull, v.x, o);
        v.y += __shfl_xor_sync(kFull, v.y, o);
        v.z += __shfl_xor_sync(kFull, v.z, o);
        v.w += __shfl_xor_sync(kFull, v.w, o);
    }
    if (lane == 0) sm.part[w] = v;
    __syncthreads();
    float4 t = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (w == 0) {
        if (lane < nw) t = sm.part[lane];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            t.x += __shfl_xor_sync(kFull, t.x, o);
            t.y += __shfl_xor_sync(kFull, t.y, o);
            t.z += __shfl_xor_sync(kFull, t.z, o);
            t.w += __shfl_xor_sync(kFull, t.w, o);
        }
    }
    return t;
}

// The root search's state, kept by one thread: the sign-change bracket
// [lo, hi] with F at both ends, the side that was moved last (for the
// Illinois rule) and the current point t.
struct SigmaSearch {
    float lo, hi, f_lo, f_hi, t;
    int side;   // -1: lo moved last, +1: hi moved last, 0: none yet
};

// One step: F(t) = f, F'(t) = df have been evaluated.  Newton's step is
// taken when it stays inside the bracket; otherwise a regula-falsi step on
// the bracket with the Illinois rule (the value at an end kept twice in a row
// is halved), which keeps convergence superlinear where Newton overshoots.
// The search stops when the step, or the bracket, is below 1e-5 in ln sigma:
// the FP32 evaluation of F leaves the root uncertain at about 1e-6, so
// smaller thresholds only make the steps follow the rounding.  Run by one
// thread.
__device__ __forceinline__ void newton_update(float f, float df, bool lo_pos, SigmaSearch& q, SigmaSmem& sm,
                                              int iter) {
    if ((f > 0.0f) == lo_pos) {
        q.lo = q.t;
        q.f_lo = f;
        if (q.side == -1) q.f_hi *= 0.5f;
        q.side = -1;
    } else {
        q.hi = q.t;
        q.f_hi = f;
        if (q.side == 1) q.f_lo *= 0.5f;
        q.side = 1;
    }
    float tn = q.t - f / df;
    if (!(tn > q.lo && tn < q.hi)) {
        const float den = q.f_hi - q.f_lo;
        tn = (den != 0.0f) ? (q.lo * q.f_hi - q.hi * q.f_lo) / den : 0.5f * (q.lo + q.hi);
        if (!(tn > q.lo && tn < q.hi)) tn = 0.5f * (q.lo + q.hi);
    }
    sm.done = (fabsf(tn - q.t) < 1e-5f || (q.hi - q.lo) < 1e-5f) ? 1 : 0;
    sm.iters = iter;
    q.t = tn;
    sm.inv_s = expf(-tn);
}

// Block sums of F and F' at t = -ln(inv_s) over the non-empty bins.
__device__ __forceinline__ float4 block_dpe(const float* he, const float* hn, int bins, float bin_w, float mu,
                                            float inv_s, const MillsCoef* tab, SigmaSmem& sm) {
    float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int b = threadIdx.x; b < bins; b += blockDim.x) {
        if (he[b] == 0.0f && hn[b] == 0.0f) continue;
        const float2 fd = dpe_bin(he[b], hn[b], ((float)b + 0.5f) * bin_w, mu, inv_s, tab);
        p.x += fd.x;
        p.y += fd.y;
    }
    return block_sum4(p, sm);
}

// Returns the new sigma (valid in every thread).  he/hn: shared-memory bins;
// tab: the Mills-ratio table in shared memory.  Empty bins contribute
// nothing and are skipped.
//
// Newton steps in t from the previous sigma come first: while F' > 0 (F
// rises through the root, the minimum of PE in sigma), each step is at most
// 2 in t and stays in [ln 1e-3, ln 1e3], they converge to the root the
// bracketed search would find, at one evaluation of (F, F') per step.  If
// a step breaks one of those conditions, or 8 steps do not converge, the
// bracketed search runs: F at both ends of [1e-3, 1e3] (no sign change: the
// end with the lower entropy, as the paper's bisection does), then Newton
// inside the bracket with the Illinois fallback.
__device__ float block_fit_sigma(const float* he, const float* hn, int bins, float hist_max, float mu,
                                 float sigma_prev, const MillsCoef* tab, SigmaSmem& sm) {
    constexpr int kFreeSteps = 8;
    const float bin_w = hist_max / (float)bins;
    const bool lead = threadIdx.x == 0;
    const float t_lo = -6.9077553f, t_hi = 6.9077553f;   // ln 1e-3, ln 1e3
    float t0 = (sigma_prev > 0.0f) ? logf(sigma_prev) : 0.0f;
    if (!(t0 > t_lo && t0 < t_hi)) t0 = 0.0f;
    float t = t0;
    if (lead) {
        sm.inv_s = expf(-t0);
        sm.done = 0;
        sm.iters = 0;
    }
    __syncthreads();
    int it = 0;
    bool bracketed = true;
    while (it < kFreeSteps) {
        ++it;
        const float4 fd = block_dpe(he, hn, bins, bin_w, mu, sm.inv_s, tab, sm);
        if (lead) {
            const float step = -fd.x / fd.y;
            const float tn = t + step;
            if (!(fd.y > 0.0f) || !(fabsf(step) <= 2.0f) || !(tn > t_lo && tn < t_hi)) {
                sm.done = 2;   // leave the search to the bracket
            } else {
                sm.done = fabsf(step) < 1e-5f ? 1 : 0;
                t = tn;
                sm.inv_s = expf(-tn);
                sm.iters = it;
            }
        }
        __syncthreads();
        const int done = sm.done;
        __syncthreads();   // every thread has read sm.done before it changes
        if (done == 1) {
            bracketed = false;
            break;
        }
        if (done == 2) break;
    }
    if (!bracketed) return 1.0f / sm.inv_s;

    // the bracketed search from the previous sigma
    SigmaSearch q{t_lo, t_hi, 0.0f, 0.0f, t0, 0};
    const float inv_s0 = expf(-t0);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int b = threadIdx.x; b < bins; b += blockDim.x) {
        const float ce = he[b], cn = hn[b], c = ((float)b + 0.5f) * bin_w;
        if (ce == 0.0f && cn == 0.0f) continue;
        acc.x += dpe_bin(ce, cn, c, mu, 1e3f, tab).x;     // sigma = 1e-3
        acc.y += dpe_bin(ce, cn, c, mu, 1e-3f, tab).x;    // sigma = 1e3
        const float2 f0 = dpe_bin(ce, cn, c, mu, inv_s0, tab);
        acc.z += f0.x;
        acc.w += f0.y;
    }
    const float4 tot = block_sum4(acc, sm);
    bool lo_pos = false;
    ++it;
    if (lead) {
        lo_pos = tot.x > 0.0f;
        if ((tot.x > 0.0f) == (tot.y > 0.0f)) {
            // no sign change: the bracket end with the lower entropy
            sm.inv_s = lo_pos ? 1e3f : 1e-3f;
            sm.done = 1;
            sm.iters = it;
        } else {
            q.f_lo = tot.x;
            q.f_hi = tot.y;
            newton_update(tot.z, tot.w, lo_pos, q, sm, it);
        }
    }
    __syncthreads();
    for (++it; it <= kSigmaMaxIters && !sm.done; ++it) {
        const float4 fd = block_dpe(he, hn, bins, bin_w, mu, sm.inv_s, tab, sm);
        if (lead) newton_update(fd.x, fd.y, lo_pos, q, sm, it);
        __syncthreads();
    }
    return 1.0f / sm.inv_s;
}

// Copy the Mills-ratio table into shared memory (all threads of the block).
__device__ __forceinline__ void load_mills_smem(MillsCoef* dst) {
    const float4* src = reinterpret_cast<const float4*>(g_mills);
    float4* d4 = reinterpret_cast<float4*>(dst);
    constexpr int kQuads = (int)(sizeof(MillsCoef) / sizeof(float4)) * kMillsIntervals;
    for (int q = threadIdx.x; q < kQuads; q += blockDim.x) d4[q] = __ldg(src + q);
}

// Shared memory of the slope-fit blocks: [2][bins] floats, then the table.
__host__ __device__ inline size_t fit_smem_bytes(int bins) {
    return ((2 * (size_t)bins * sizeof(float) + 15) / 16) * 16 + sizeof(MillsCoef) * kMillsIntervals;
}

// Load one graph's histograms into shared memory as floats: edge counts, and
// the non-edge weights ((n-1) hc - hd) / (2k) + hx.
__device__ void load_hist_smem(const EpochArgs& a, size_t off, int n, int k_slots, float* he, float* hn) {
    const float inv2k = k_slots > 0 ? 0.5f / (float)k_slots : 0.0f;
    for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
        he[b] = (float)a.hist_e[off + b];
        hn[b] = fmaf((float)(n - 1), (float)a.hist_c[off + b], -(float)a.hist_d[off + b]) * inv2k + a.hist_x[off + b];
    }
    __syncthreads();
}

// Blocks [0, n_graphs): the slope fit, histogram reset and epoch advance of
// one stepped graph each.  The other blocks: x_i := y_i / z_i over the vertex
// chunks, accumulators cleared for the next epoch.
__global__ void __launch_bounds__(kUpdateThreads) k_update(const EpochArgs a) {
    // Launched as a programmatic dependent of the sweep (or the tiles): the
    // slope-fit blocks copy the Mills table, which the sweep does not write,
    // then every block waits for the sweep's grid to finish and its writes to
    // be visible before it reads the sums and histograms.
    extern __shared__ __align__(16) float s_bins[];   // slope fit: [2][bins], then the Mills table
    MillsCoef* s_tab = reinterpret_cast<MillsCoef*>(reinterpret_cast<unsigned char*>(s_bins) +
                                                    ((2 * (size_t)a.bins * sizeof(float) + 15) / 16) * 16);
    const bool fit_block = (int)blockIdx.x < a.n_graphs && a.sigma_source == 0 && a.sigma_every > 0;
    if (fit_block) load_mills_smem(s_tab);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if ((int)blockIdx.x < a.n_graphs) {
        __shared__ SigmaSmem sm;
        const int graph = blockIdx.x;
        GraphState* st = a.gst + graph;
        const size_t off = (size_t)graph * a.bins;
        const int epoch = st->epoch;
        const float sigma_prev = st->sigma;
        // sigma_source 1: the fit follows in k_fit_graphs on the separate pass's histograms
        const bool fit = a.sigma_source == 0 &&
                         (a.sigma_every == 1 || (a.sigma_every > 1 && ((epoch + 1) % a.sigma_every) == 0));
        if (fit) {
            const int k_slots = a.block_P > 0 ? kBlockP : a.k;
            load_hist_smem(a, off, __ldg(&a.graphs[graph].n), k_slots, s_bins, s_bins + a.bins);   // syncs the block
            const float s =
                block_fit_sigma(s_bins, s_bins + a.bins, a.bins, a.hist_max, a.mu, sigma_prev, s_tab, sm);
            if (threadIdx.x == 0) {
                st->sigma = s;
                st->sigma_iters = sm.iters;
            }
        }
        for (int t = threadIdx.x; t < a.bins; t += blockDim.x) {
            a.hist_e[off + t] = 0u;
            a.hist_c[off + t] = 0u;
            a.hist_d[off + t] = 0ull;
            a.hist_x[off + t] = 0.0f;
        }
        if (threadIdx.x == 0) st->epoch = epoch + 1;
        return;
    }
    const int vblk = blockIdx.x - a.n_graphs, n_vblk = gridDim.x - a.n_graphs;
    if (a.d >= 8) {
        // L = min(32, d/4) lanes per vertex, float4 over the dimensions (at most 2 per lane)
        const int lane = threadIdx.x & 31;
        const int nq = a.d >> 2, sq = a.acc_stride >> 2;
        const int L = nq < 32 ? nq : 32;
        const int vpw = 32 / L;                       // vertices per warp
        const int sub = lane / L, ql = lane - sub * L;
        const unsigned group = (L == 32) ? kFull : (((1u << L) - 1u) << (sub * L));
        const int per_pass = (blockDim.x >> 5) * vpw;
        for (int c = vblk; c < a.n_vchunks; c += n_vblk) {
            const int4 ch = __ldg(a.vchunks + c);
            // two batches of the warp's vertices per pass: all their loads
            // are in flight before either batch is updated
            for (int vb0 = (threadIdx.x >> 5) * vpw; vb0 < ch.y; vb0 += 2 * per_pass) {
                float4 dv[2][2], xo[2][2];
                float z[2];
                bool live[2];
                int v[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int vb = vb0 + u * per_pass;
                    live[u] = vb + sub < ch.y;
                    v[u] = ch.x + vb + sub;
                    const float4* row = reinterpret_cast<const float4*>(a.acc + (size_t)v[u] * a.acc_stride);
                    const float4* xv = reinterpret_cast<const float4*>(a.x + (size_t)v[u] * a.d);
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int q = ql + L * r;
                        dv[u][r] = xo[u][r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (live[u] && q < nq) {
                            dv[u][r] = row[q];
                            xo[u][r] = xv[q];
                        }
                    }
                    z[u] = live[u] ? a.acc[(size_t)v[u] * a.acc_stride + a.d] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float4* row = reinterpret_cast<float4*>(a.acc + (size_t)v[u] * a.acc_stride);
                    float4* xv = reinterpret_cast<float4*>(a.x + (size_t)v[u] * a.d);
                    const bool upd = live[u] && z[u] >= a.z_min;
                    float4 xn[2];
                    bool finite = true;
                    if (upd) {
                        const float inv_z = 1.0f / z[u];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const int q = ql + L * r;
                            if (q < nq) {
                                xn[r] = make_float4(fmaf(dv[u][r].x, inv_z, xo[u][r].x), fmaf(dv[u][r].y, inv_z, xo[u][r].y),
                                                    fmaf(dv[u][r].z, inv_z, xo[u][r].z), fmaf(dv[u][r].w, inv_z, xo[u][r].w));
                                finite = finite && isfinite(xn[r].x) && isfinite(xn[r].y) && isfinite(xn[r].z) &&
                                         isfinite(xn[r].w);
                            }
                        }
                    }
                    const bool all_finite = (__ballot_sync(kFull, !finite) & group) == 0u;
                    if (upd) {
                        if (all_finite) {
#pragma unroll
                            for (int r = 0; r < 2; ++r) {
                                const int q = ql + L * r;
                                if (q < nq) {
                                    xv[q] = xn[r];
                                    if (a.xb) {
                                        __nv_bfloat162* bp =
                                            reinterpret_cast<__nv_bfloat162*>(a.xb + (size_t)v[u] * a.d + 4 * q);
                                        bp[0] = __floats2bfloat162_rn(xn[r].x, xn[r].y);
                                        bp[1] = __floats2bfloat162_rn(xn[r].z, xn[r].w);
                                    }
                                }
                            }
                        } else if (ql == 0) {
                            atomicCAS(&a.ps->status, 0, -6 /* GEMPE_E_NUMERIC */);
                        }
                    }
                    if (live[u])
                        for (int q = ql; q < sq; q += L) row[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
            }
        }
        return;
    }
    for (int c = vblk; c < a.n_vchunks; c += n_vblk) {
        const int4 ch = __ldg(a.vchunks + c);
        // d <= 4 here (the dimensions below 8); the sums and the position are
        // loaded with z, not after it
        for (int vi = threadIdx.x; vi < ch.y; vi += blockDim.x) {
            const int v = ch.x + vi;
            float* row = a.acc + (size_t)v * a.acc_stride;
            float* xv = a.x + (size_t)v * a.d;
            float dv[kPackedMaxDim], xo[kPackedMaxDim];
#pragma unroll
            for (int c2 = 0; c2 < kPackedMaxDim; ++c2) {
                dv[c2] = c2 < a.d ? row[c2] : 0.0f;
                xo[c2] = c2 < a.d ? xv[c2] : 0.0f;
            }
            const float z = row[a.d];
            if (z >= a.z_min) {
                const float inv_z = 1.0f / z;
                float xn[kPackedMaxDim];
                bool bad = false;
#pragma unroll
                for (int c2 = 0; c2 < kPackedMaxDim; ++c2) {
                    xn[c2] = fmaf(dv[c2], inv_z, xo[c2]);
                    if (c2 < a.d && !isfinite(xn[c2])) bad = true;
                }
                if (!bad) {
#pragma unroll
                    for (int c2 = 0; c2 < kPackedMaxDim; ++c2) {
                        if (c2 >= a.d) break;
                        xv[c2] = xn[c2];
                        if (a.xb) a.xb[(size_t)v * a.d + c2] = __float2bfloat16_rn(xn[c2]);
                    }
                } else {
                    atomicCAS(&a.ps->status, 0, -6 /* GEMPE_E_NUMERIC */);
                }
            }
            for (int c2 = 0; c2 < a.acc_stride; c2 += 4)
                *reinterpret_cast<float4*>(row + c2) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
}

__global__ void __launch_bounds__(kUpdateThreads) k_fit_sigma(const float* hist, int bins, float hist_max, float mu,
                                                               float* sigma) {
    __shared__ SigmaSmem sm;
    extern __shared__ __align__(16) float s_bins[];
    MillsCoef* s_tab = reinterpret_cast<MillsCoef*>(reinterpret_cast<unsigned char*>(s_bins) +
                                                    ((2 * (size_t)bins * sizeof(float) + 15) / 16) * 16);
    load_mills_smem(s_tab);
    for (int b = threadIdx.x; b < 2 * bins; b += blockDim.x) s_bins[b] = hist[b];
    __syncthreads();
    const float s = block_fit_sigma(s_bins, s_bins + bins, bins, hist_max, mu, 1.0f, s_tab, sm);
    if (threadIdx.x == 0) *sigma = s;
}

// ---------------------------------------------------------------------------
// Sec. III.F's separate histogram pass (sigma_source 1), after the update:
// every edge once and k fresh samples per vertex (stream kTagSlope, drawn for
// the epoch just completed) at the new positions.  One block per vertex
// chunk, a warp per vertex, G lanes per pair; shared bins per chunk, merged
// into the chunk's graph.
// ---------------------------------------------------------------------------
template <int D, int G>
__global__ void __launch_bounds__(256) k_hist_pass(const EpochArgs a) {
    constexpr int P = D / G;
    constexpr int PAIRS = 32 / G;
    extern __shared__ unsigned int s_u32[];
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x; c < a.n_vchunks; c += gridDim.x) {
        const int4 ch = __ldg(a.vchunks + c);
        const int graph = ch.z;
        const BlockHist hist = block_hist(s_u32, a.bins, graph);
        __syncthreads();   // the previous chunk's bins are merged
        hist_clear(hist, a.bins);
        __syncthreads();
        const GraphInfo gi = load_graph(a, graph);
        const int epoch = a.gst[graph].epoch - 1;   // the epoch just completed
        for (int vi = wib; vi < ch.y; vi += wpb) {
            const int i = ch.x + vi;
            const int e0 = __ldg(a.row_ptr + i);
            const int deg = __ldg(a.row_ptr + i + 1) - e0;
            float xi[P];
            load_chunk<D, P>(a.x, i, gl, xi);
            int g_mine = -1;
            unsigned rej = 0;
            if (lane < a.k) {
                const int g = sample_partner(gi, edge_sets(a), a.max_retries, i - gi.v0, epoch, lane, kTagSlope, rej);
                g_mine = g >= 0 ? gi.v0 + g : -1;
            }
            const int k_acc = __popc(__ballot_sync(kFull, g_mine >= 0));
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
                    for (int cc = 0; cc < P; ++cc) xj[cc] = xi[cc];
                }
                float ss = 0.0f;
#pragma unroll
                for (int cc = 0; cc < P; ++cc) {
                    const float df = xi[cc] - xj[cc];
                    ss = fmaf(df, df, ss);
                }
#pragma unroll
                for (int o = G / 2; o >= 1; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
                if (valid && gl == 0) {
                    const int bin = min((int)(sqrtf(ss) * a.hist_scale), a.bins - 1);
                    if (is_edge) hist_edge(hist, a, graph, bin);
                    else hist_sample(hist, a, graph, bin, deg, k_acc, a.k);
                }
            }
        }
        __syncthreads();
        hist_merge(hist, a);
    }
}

// The slope fits of the stepped graphs on the separate pass's histograms
// (one block per graph; the epoch counter has already advanced).
__global__ void __launch_bounds__(kUpdateThreads) k_fit_graphs(const EpochArgs a) {
    __shared__ SigmaSmem sm;
    extern __shared__ __align__(16) float s_bins[];   // [2][bins], then the Mills table
    MillsCoef* s_tab = reinterpret_cast<MillsCoef*>(reinterpret_cast<unsigned char*>(s_bins) +
                                                    ((2 * (size_t)a.bins * sizeof(float) + 15) / 16) * 16);
    const int graph = blockIdx.x;
    GraphState* st = a.gst + graph;
    const size_t off = (size_t)graph * a.bins;
    if (a.sigma_every > 0 && (st->epoch % a.sigma_every) == 0) {
        load_mills_smem(s_tab);
        load_hist_smem(a, off, __ldg(&a.graphs[graph].n), a.k, s_bins, s_bins + a.bins);
        const float s = block_fit_sigma(s_bins, s_bins + a.bins, a.bins, a.hist_max, a.mu, st->sigma, s_tab, sm);
        if (threadIdx.x == 0) {
            st->sigma = s;
            st->sigma_iters = sm.iters;
        }
    }
    for (int t = threadIdx.x; t < a.bins; t += blockDim.x) {
        a.hist_e[off + t] = 0u;
        a.hist_c[off + t] = 0u;
        a.hist_d[off + t] = 0ull;
        a.hist_x[off + t] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Inspection kernels and the loss estimator
// ---------------------------------------------------------------------------
// Samples of the current epoch (tag kTagEpoch) or of the loss stream, as
// pack rows, one warp per vertex.
__global__ void k_sample(const EpochArgs a, uint32_t tag, int32_t* out) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x; c < a.n_vchunks; c += gridDim.x) {
        const int4 ch = __ldg(a.vchunks + c);
        const GraphInfo gi = load_graph(a, ch.z);
        const int epoch = a.gst[ch.z].epoch;
        for (int vi = wib; vi < ch.y; vi += wpb) {
            const int v = ch.x + vi;
            unsigned rej = 0;
            if (lane < a.k) {
                int g;
                if (tag == kTagEpoch && a.rng) {   // the epoch's draws come from the LCG (rng 1)
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)(v - gi.v0), (uint32_t)epoch,
                                                             (uint32_t)lane >> 2, kTagLcg), gi.key_lo, gi.key_hi);
                    const Membership exact{nullptr, 0u, (uint32_t)gi.n, 1u, 0u};
                    unsigned fp = 0u;
                    g = lcg_partner_from(gi, edge_sets(a), a.max_retries, v - gi.v0, word_of(r, lane & 3), 0, rej,
                                         exact, fp);
                } else {
                    g = sample_partner(gi, edge_sets(a), a.max_retries, v - gi.v0, epoch, lane, tag, rej);
                }
                out[(size_t)v * a.k + lane] = g >= 0 ? gi.v0 + g : -1;
            }
        }
    }
}

// Sampled predictive entropy (Eq. 2) of each graph at its current sigma:
// the graph's edges once each plus k fresh samples per vertex weighted by
// (n-1-deg)/(2 k_acc); one block per vertex chunk, FP64 sums, one FP64
// atomic per chunk into the graph's loss_sum.
template <int D, int G>
__global__ void __launch_bounds__(256) k_loss(const EpochArgs a) {
    constexpr int P = D / G;
    constexpr int PAIRS = 32 / G;
    __shared__ double s_part[8];
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane % G;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x; c < a.n_vchunks; c += gridDim.x) {
        const int4 ch = __ldg(a.vchunks + c);
        const int graph = ch.z;
        const GraphInfo gi = load_graph(a, graph);
        const float sigma = a.gst[graph].sigma;
        const int epoch = a.gst[graph].epoch;
        const float inv_sigma = 1.0f / sigma;
        double sum = 0.0;
        for (int vi = wib; vi < ch.y; vi += wpb) {
            const int i = ch.x + vi;
            const int e0 = __ldg(a.row_ptr + i);
            const int deg = __ldg(a.row_ptr + i + 1) - e0;
            float xi[P];
            load_chunk<D, P>(a.x, i, gl, xi);
            int g_mine = -1;
            unsigned rej = 0;
            if (lane < a.k) {
                const int g = sample_partner(gi, edge_sets(a), a.max_retries, i - gi.v0, epoch, lane, kTagLoss, rej);
                g_mine = g >= 0 ? gi.v0 + g : -1;
            }
            const int k_acc = __popc(__ballot_sync(kFull, g_mine >= 0));
            const double omega = k_acc ? (double)(gi.n - 1 - deg) / (2.0 * k_acc) : 0.0;
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
                    for (int cc = 0; cc < P; ++cc) xj[cc] = xi[cc];
                }
                float ss = 0.0f;
#pragma unroll
                for (int cc = 0; cc < P; ++cc) {
                    const float df = xi[cc] - xj[cc];
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
        if (lane == 0) s_part[wib] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < wpb; ++w) t += s_part[w];
            if (t != 0.0) atomicAdd(&a.gst[graph].loss_sum, t);
        }
        __syncthreads();
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ xb, long long count) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        xb[t] = __float2bfloat16_rn(x[t]);
}

__global__ void k_is_edge(const void* keys, int narrow, unsigned long long key_off, unsigned long long bucket_mask,
                          const int32_t* pairs, int64_t count, uint8_t* out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = pairs[2 * p], j = pairs[2 * p + 1];
        out[p] = (i != j && edge_set_contains(keys, narrow, key_off, bucket_mask, i, j)) ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// Dispatch on the dimension.  d <= 4: the packed sweep.  d >= 8: G lanes per
// pair, each lane gathering D/G coordinates; two lane counts per dimension
// (8 or 4 coordinates per lane) for the autotuner, the first the default.
// ---------------------------------------------------------------------------
#define GEMPE_PACKED_DIMS(X) X(1) X(2) X(3) X(4)
// d <= 4 also has the per-unit kernel with one lane per vertex (G = 1)
#define GEMPE_LANE_DIMS(X) X(1, 1) X(2, 1) X(3, 1) X(4, 1)
#define GEMPE_WIDE(X) X(8, 1) X(8, 2) X(16, 2) X(16, 4) X(32, 4) X(32, 8) X(64, 8) X(64, 16) X(128, 16) X(128, 32) X(256, 32)
#define GEMPE_LOSS_DIMS(X) X(1, 1) X(2, 1) X(3, 1) X(4, 1) X(8, 1) X(16, 2) X(32, 4) X(64, 8) X(128, 16) X(256, 32)

template <int D, int G>
cudaError_t wide_sweep(const EpochArgs& a, int grid, cudaStream_t s, int threads = kSweepThreads) {
    if (a.xb) return launch_critical(k_sweep<D, G, __nv_bfloat16>, grid, threads, hist_smem_bytes(a.bins), s, false, a);
    return launch_critical(k_sweep<D, G, float>, grid, threads, hist_smem_bytes(a.bins), s, false, a);
}

template <int D>
cudaError_t packed_sweep(const EpochArgs& a, int grid, cudaStream_t s) {
    if (a.oriented) return launch_critical(k_sweep_packed<D, true>, grid, kPackedThreads, packed_smem_bytes(D, a.bins), s, false, a);
    return launch_critical(k_sweep_packed<D, false>, grid, kPackedThreads, packed_smem_bytes(D, a.bins), s, false, a);
}

template <int D, int G>
cudaError_t loss_for(const EpochArgs& a, int grid, cudaStream_t s) {
    k_loss<D, G><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int D>
int packed_blocks_per_sm(int bins) {
    int blocks = 0;
    const size_t smem = packed_smem_bytes(D, bins);
    raise_smem_limit((const void*)k_sweep_packed<D, true>, (int)smem);
    raise_smem_limit((const void*)k_sweep_packed<D, false>, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep_packed<D, false>, kPackedThreads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        blocks = 1;
    }
    return blocks < 1 ? 1 : blocks;
}

template <int D, int G>
int wide_blocks_per_sm(int bins) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep<D, G, float>, kSweepThreads,
                                                      hist_smem_bytes(bins)) != cudaSuccess) {
        cudaGetLastError();
        blocks = 1;
    }
    return blocks < 1 ? 1 : blocks;
}

}  // namespace

int acc_stride_for(int d) { return ((d + 1) + 3) / 4 * 4; }

bool supported_dim(int d) {
    switch (d) {
#define GEMPE_CASE(D, G) case D:
        GEMPE_LOSS_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        return true;
        default: return false;
    }
}

bool sweep_lanes_supported(int d, int lanes) {
    if (d <= kPackedMaxDim) return lanes == 0 || lanes == 1;
    if (lanes == 0) lanes = d / 8;
#define GEMPE_CASE(D, G) \
    if (d == D && lanes == G) return true;
    GEMPE_WIDE(GEMPE_CASE)
#undef GEMPE_CASE
    return false;
}

// One resident wave (SM count x blocks per SM, at most what fits): the
// sweep strides over its work units, so a second wave would only add
// histogram merges.
int sweep_grid(int d, int lanes, int bins, int sm_count, int blocks_per_sm, int kernel) {
    int fit = 1;
    if (lanes == 0) lanes = d <= kPackedMaxDim ? 1 : d / 8;
    if (d <= kPackedMaxDim && kernel == 1) {
        switch (d) {
#define GEMPE_CASE(D, G) \
    case D: fit = wide_blocks_per_sm<D, G>(bins); break;
            GEMPE_LANE_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
            default: break;
        }
    } else {
        switch (d) {
#define GEMPE_CASE(D) \
    case D: fit = packed_blocks_per_sm<D>(bins); break;
            GEMPE_PACKED_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
            default:
#define GEMPE_CASE(D, G) \
    if (d == D && lanes == G) fit = wide_blocks_per_sm<D, G>(bins);
                GEMPE_WIDE(GEMPE_CASE)
#undef GEMPE_CASE
                break;
        }
    }
    const int b = (blocks_per_sm > 0 && blocks_per_sm < fit) ? blocks_per_sm : fit;
    return sm_count * b;
}

cudaError_t launch_hash_build(const int32_t* row_ptr, const int32_t* col_idx, int32_t v0, int32_t n, int64_t nnz,
                              void* keys, int narrow, unsigned long long bucket_mask, int32_t* fail_flag,
                              cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    long long grid = (nnz + 255) / 256;
    if (grid > 65535) grid = 65535;
    if (narrow) k_hash_build<true><<<(int)grid, 256, 0, s>>>(row_ptr, col_idx, v0, n, keys, bucket_mask, fail_flag);
    else k_hash_build<false><<<(int)grid, 256, 0, s>>>(row_ptr, col_idx, v0, n, keys, bucket_mask, fail_flag);
    return cudaGetLastError();
}

cudaError_t launch_init_positions(float* x, __nv_bfloat16* xb, int32_t n, int32_t d, uint32_t key_lo,
                                  uint32_t key_hi, float range, cudaStream_t s) {
    const long long total = (long long)n * ((d + 3) / 4);
    long long grid = (total + 255) / 256;
    if (grid > 65535) grid = 65535;
    if (grid < 1) grid = 1;
    k_init<<<(int)grid, 256, 0, s>>>(x, xb, n, d, key_lo, key_hi, range);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const EpochArgs& a, const SweepShape& shape, cudaStream_t s) {
    if (a.n_items == 0) return cudaSuccess;
    const int lanes = shape.lanes ? shape.lanes : (a.d <= kPackedMaxDim ? 1 : a.d / 8);
    if (a.d <= kPackedMaxDim && shape.kernel == 1) {
        switch (a.d) {
#define GEMPE_CASE(D, G) \
    case D: return wide_sweep<D, G>(a, shape.grid, s);
            GEMPE_LANE_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.d) {
#define GEMPE_CASE(D) \
    case D: return packed_sweep<D>(a, shape.grid, s);
        GEMPE_PACKED_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        default:
#define GEMPE_CASE(D, G) \
    if (a.d == D && lanes == G) \
        return wide_sweep<D, G>(a, shape.grid, s, shape.kernel == 2 ? kSweepThreadsBeside : kSweepThreads);
            GEMPE_WIDE(GEMPE_CASE)
#undef GEMPE_CASE
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_loss(const EpochArgs& a, cudaStream_t s) {
    int grid = a.n_vchunks;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    switch (a.d) {
#define GEMPE_CASE(D, G) \
    case D: return loss_for<D, G>(a, grid, s);
        GEMPE_LOSS_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t raise_smem_limit(const void* func, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> limit;   // (device, function) -> bytes set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int& cur = limit[std::make_pair(dev, func)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

cudaError_t prepare_update_kernels(int bins) {
    const int smem = (int)fit_smem_bytes(bins);
    cudaError_t e = raise_smem_limit((const void*)k_update, smem);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)k_fit_sigma, smem);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)k_fit_graphs, smem);
    return e;
}

template <int D, int G>
cudaError_t hist_pass_for(const EpochArgs& a, int grid, cudaStream_t s) {
    EpochArgs b = a;
    b.sweep_hist = 1;          // this pass bins its own distances
    b.per_slot = 0;            // with the integer sample weights of k samples per vertex
    const cudaError_t e = launch_critical(k_hist_pass<D, G>, grid, 256, hist_smem_bytes(a.bins), s, false, b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_hist_pass(const EpochArgs& a, cudaStream_t s) {
    int grid = a.n_vchunks;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    switch (a.d) {
#define GEMPE_CASE(D, G) \
    case D: return hist_pass_for<D, G>(a, grid, s);
        GEMPE_LOSS_DIMS(GEMPE_CASE)
#undef GEMPE_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fit_graphs(const EpochArgs& a, cudaStream_t s) {
    const cudaError_t e = launch_critical(k_fit_graphs, a.n_graphs, kUpdateThreads, fit_smem_bytes(a.bins), s, false, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_update(const EpochArgs& a, int grid, cudaStream_t s) {
    const cudaError_t e = launch_critical(k_update, grid, kUpdateThreads, fit_smem_bytes(a.bins), s, true, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int sampler_grid(int rows, int k, int sm_count) {
    const long long subs = ((long long)rows + sampler_piece(k) - 1) / sampler_piece(k) + 1;
    long long grid = subs;
    const long long cap = (long long)sm_count * 8;
    if (grid > cap) grid = cap;
    return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_sampler(const EpochArgs& a, int grid, cudaStream_t s) {
    if (a.per_slot) {
        if (a.membership) k_sampler_slots<true><<<grid, 256, 0, s>>>(a);
        else k_sampler_slots<false><<<grid, 256, 0, s>>>(a);
    } else {
        if (a.membership) k_sampler<true><<<grid, 256, 0, s>>>(a);
        else k_sampler<false><<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int critical_priority() {
    static const int prio = [] {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return greatest;
    }();
    return prio;
}

cudaError_t launch_bytemap_build(const EpochArgs& a, int force, int sm_count, cudaStream_t s) {
    if (!a.membership) return cudaSuccess;
    k_bytemap_clear<<<sm_count * 4, 256, 0, s>>>(a, force);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int grid = a.n_vchunks < sm_count * 8 ? a.n_vchunks : sm_count * 8;
    if (grid < 1) grid = 1;
    k_bytemap_mark<<<grid, 256, 0, s>>>(a, force);
    return cudaGetLastError();
}

cudaError_t launch_sample(const EpochArgs& a, uint32_t tag, int32_t* out, cudaStream_t s) {
    int grid = a.n_vchunks;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    k_sample<<<grid, 256, 0, s>>>(a, tag, out);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* x, __nv_bfloat16* xb, long long count, cudaStream_t s) {
    long long grid = (count + 255) / 256;
    if (grid > 65535) grid = 65535;
    if (grid < 1) grid = 1;
    k_to_bf16<<<(int)grid, 256, 0, s>>>(x, xb, count);
    return cudaGetLastError();
}

cudaError_t launch_is_edge(const void* keys, int narrow, unsigned long long key_off, unsigned long long bucket_mask,
                           const int32_t* pairs, int64_t count, uint8_t* out, cudaStream_t s) {
    long long grid = (count + 255) / 256;
    if (grid > 65535) grid = 65535;
    if (grid < 1) grid = 1;
    k_is_edge<<<(int)grid, 256, 0, s>>>(keys, narrow, key_off, bucket_mask, pairs, count, out);
    return cudaGetLastError();
}

const MillsCoef* mills_table_device() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mills) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (const MillsCoef*)p;
}

cudaError_t upload_mills_table(const void* host_coefs, size_t bytes) {
    if (bytes != sizeof(MillsCoef) * kMillsIntervals) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbol(g_mills, host_coefs, bytes);
}

cudaError_t launch_fit_sigma(const float* hist, int32_t bins, float hist_max, float mu,
                             float* sigma_inout, cudaStream_t s) {
    cudaError_t e = prepare_update_kernels(bins);
    if (e != cudaSuccess) return e;
    k_fit_sigma<<<1, kUpdateThreads, fit_smem_bytes(bins), s>>>(hist, bins, hist_max, mu, sigma_inout);
    return cudaGetLastError();
}

}  // namespace gempe
