// Device arithmetic of the GEMPE epoch: counter-based random numbers, the
// edge-set hash, and the Eq. 3-5 pair term in FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gempe {

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 multiplications with Weyl-sequence key increments.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& r, int w) {
    return w == 0 ? r.x : (w == 1 ? r.y : (w == 2 ? r.z : r.w));
}

// Random 32-bit word -> vertex in [0, n): floor(r * n / 2^32).
__device__ __forceinline__ int32_t draw_vertex(uint32_t r, uint32_t n) { return (int32_t)__umulhi(r, n); }

// Sec. III.C's 32-bit linear congruential generator (multiplier 1103515245,
// increment 1), advanced before each draw as in Fig. 2.
__device__ __forceinline__ uint32_t lcg_next(uint32_t s) { return s * 1103515245u + 1u; }

// Fig. 2's vertex of a state: the low 23 bits as the mantissa of f in [1, 2),
// then f * n - n and a round to nearest (ties to even), each an FP32
// operation with one rounding; the value n that rounding can reach is
// vertex 0.
__device__ __forceinline__ int32_t lcg_vertex(uint32_t s, int32_t n) {
    const float f = __uint_as_float(0x3F800000u | (s & 0x007FFFFFu));
    const float nf = __int2float_rn(n);
    const float t = __fsub_rn(__fmul_rn(f, nf), nf);
    const int32_t g = __float2int_rn(t);
    return g >= n ? g - n : g;
}

// Stream tags in the fourth counter word.
constexpr uint32_t kTagInit = 0x0A000000u;
constexpr uint32_t kTagEpoch = 0x0B000000u;
constexpr uint32_t kTagLoss = 0x0E000000u;
constexpr uint32_t kTagSlope = 0x0F000000u;   // the separate histogram pass of the slope fit
constexpr uint32_t kTagRename = 0x09000000u;  // the byte map's random renaming (Sec. III.C)

// --------------------------------------------------------------------------
// Exact edge set: every undirected edge {i, j} once, keyed by (min, max),
// open addressing with linear probing bucket by bucket over 32-byte buckets
// (one sector).  Narrow sets (every graph of the pack has n <= 65536) hold
// u32 keys min << 16 | max, eight per bucket; wide sets u64 keys
// min << 32 | max, four per bucket.  All-ones marks an empty slot (never a
// key: min < max).
// --------------------------------------------------------------------------
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr uint32_t kEmptyKey32 = ~0u;

__device__ __forceinline__ unsigned long long edge_key(int32_t i, int32_t j) {
    return ((unsigned long long)(uint32_t)min(i, j) << 32) | (uint32_t)max(i, j);
}

__device__ __forceinline__ uint32_t edge_key32(int32_t i, int32_t j) {
    return ((uint32_t)min(i, j) << 16) | (uint32_t)max(i, j);
}

// splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) as the bucket hash.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Membership of key in a wide table of (bucket_mask + 1) buckets.
__device__ __forceinline__ bool hash_contains(const unsigned long long* __restrict__ keys,
                                              unsigned long long bucket_mask, unsigned long long key) {
    unsigned long long b = mix64(key) & bucket_mask;
    for (unsigned long long probe = 0; probe <= bucket_mask; ++probe) {
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(keys + 4 * b);
        const ulonglong2 s01 = __ldg(p), s23 = __ldg(p + 1);
        if (s01.x == key || s01.y == key || s23.x == key || s23.y == key) return true;
        if (s01.x == kEmptyKey || s01.y == kEmptyKey || s23.x == kEmptyKey || s23.y == kEmptyKey)
            return false;
        b = (b + 1) & bucket_mask;
    }
    return false;
}

// Membership of key in a narrow table of (bucket_mask + 1) buckets.
__device__ __forceinline__ bool hash_contains32(const uint32_t* __restrict__ keys, unsigned long long bucket_mask,
                                                uint32_t key) {
    unsigned long long b = mix64(key) & bucket_mask;
    for (unsigned long long probe = 0; probe <= bucket_mask; ++probe) {
        const uint4* p = reinterpret_cast<const uint4*>(keys + 8 * b);
        const uint4 s03 = __ldg(p), s47 = __ldg(p + 1);
        if (s03.x == key || s03.y == key || s03.z == key || s03.w == key || s47.x == key || s47.y == key ||
            s47.z == key || s47.w == key)
            return true;
        if (s03.x == kEmptyKey32 || s03.y == kEmptyKey32 || s03.z == kEmptyKey32 || s03.w == kEmptyKey32 ||
            s47.x == kEmptyKey32 || s47.y == kEmptyKey32 || s47.z == kEmptyKey32 || s47.w == kEmptyKey32)
            return false;
        b = (b + 1) & bucket_mask;
    }
    return false;
}

// Is {i, j} (local ids) an edge of the graph whose table starts at slot
// key_off of the pack's key array?
__device__ __forceinline__ bool edge_set_contains(const void* keys, int narrow, unsigned long long key_off,
                                                  unsigned long long bucket_mask, int32_t i, int32_t j) {
    if (narrow) return hash_contains32(static_cast<const uint32_t*>(keys) + key_off, bucket_mask, edge_key32(i, j));
    return hash_contains(static_cast<const unsigned long long*>(keys) + key_off, bucket_mask, edge_key(i, j));
}

// --------------------------------------------------------------------------
// Pair arithmetic (Sec. II.B/C) in FP32.
//
// With u = (delta - mu)/sigma, the edge sigmoid is s+ = Q(u) (upper normal
// tail) and the non-edge one s- = Q(-u).  Writing v = u for an edge and
// v = -u for a non-edge, both cases use h = phi(v)/Q(v) and T = h - v > 0:
//   dl'(delta)  = +-h / (sigma ln2)            (+ edge, - non-edge)
//   w (derived) = h T / (2 ln2 sigma^2)        (matches dl'' as Sec. II.C asks)
//   w (printed) = h (h + T) / (2 ln2 sigma^2)  (Eq. 4 with its first term as printed)
//   d           = delta - dl' / (2 w)          (Eq. 5, both readings)
// Eq. 3 adds w (x_j + s (x_i - x_j)) to y_i, s = d/delta.  The engine keeps
// y_i - z_i x_i instead of y_i, i.e. adds c (x_i - x_j) with
//   c = w (s - 1) = -dl' / (2 delta),
// which avoids the cancellation of forming y_i - z_i x_i at the end; when
// delta = 0, or when d < 0 is clamped to 0, s = 0 and c = -w.
// --------------------------------------------------------------------------
// Mills-ratio table: on [kMillsV0, kMillsV1) with kMillsStepsPerUnit
// intervals per unit of v, interval i holds the cubic coefficients (in the
// local coordinate x in [0, 1)) of log2 h(v), the Hermite interpolant built
// on the host from the values and the slopes (log2 h)' = T / ln2.  Since
// h' = h T, T itself is ln2 times the derivative of that cubic in v: one
// 16-byte entry per interval gives both h and T (FP32 relative error about
// 1.6e-7 for either, the same as a second table of log2 T would give).
constexpr float kMillsV0 = -14.0f;
constexpr float kMillsV1 = 8.0f;
constexpr int kMillsStepsPerUnit = 32;
constexpr int kMillsIntervals = (int)((kMillsV1 - kMillsV0) * kMillsStepsPerUnit);

struct MillsCoef {
    float4 lh;   // log2 h: c0 + x (c1 + x (c2 + x c3))
};

struct PairConsts {
    float mu, inv_sigma;
    float w_scale;    // 1 / (2 ln2 sigma^2)
    float g_scale;    // 1 / (2 ln2 sigma)
    int printed;      // w_formula == 1
    int clamp;        // clamp_neg_d
    const MillsCoef* mills;
};

__device__ __forceinline__ PairConsts make_pair_consts(float mu, float sigma, int printed, int clamp,
                                                       const MillsCoef* mills) {
    PairConsts k;
    const float ln2 = 0.69314718055994531f;
    k.mu = mu;
    k.inv_sigma = 1.0f / sigma;
    k.w_scale = 1.0f / (2.0f * ln2 * sigma * sigma);
    k.g_scale = 1.0f / (2.0f * ln2 * sigma);
    k.printed = printed;
    k.clamp = clamp;
    k.mills = mills;
    return k;
}

// T(v) = h(v) - v by Laplace's continued fraction T = 1/(v + 2/(v + 3/(v + ...))),
// truncated after the 8th partial denominator (relative error < 2e-8 for v >= 6;
// it is used from v = kMillsV1 = 8 on).
__device__ __forceinline__ float mills_tail_T(float v) {
    float t = v;
#pragma unroll
    for (int k = 8; k >= 2; --k) t = v + __fdividef((float)k, t);
    return 1.0f / t;
}

// h(v) = phi(v)/Q(v) and T(v) = h(v) - v > 0.  On the table range h comes
// from the interpolated logarithm and T from its slope, T = ln2 d(log2 h)/dv;
// from kMillsV1 on, T by the continued fraction and h = v + T; below
// kMillsV0, h is below the FP32 range (h = 0, T = -v).
// kGlobal: the table is in global memory (read through the read-only
// cache); otherwise it is a copy in shared memory.
template <bool kGlobal>
__device__ __forceinline__ void mills_t(float v, float& h, float& T, const MillsCoef* tab) {
    if (v < kMillsV1) {
        const float pos = (fmaxf(v, kMillsV0) - kMillsV0) * (float)kMillsStepsPerUnit;
        const int i = min((int)pos, kMillsIntervals - 1);
        const float x = pos - (float)i;
        const float4 a = kGlobal ? __ldg(&tab[i].lh) : tab[i].lh;
        const float lh = fmaf(fmaf(fmaf(a.w, x, a.z), x, a.y), x, a.x);
        const float dlh = fmaf(fmaf(3.0f * a.w, x, 2.0f * a.z), x, a.y);   // d(log2 h)/dx
        constexpr float kTScale = 0.69314718055994531f * (float)kMillsStepsPerUnit;
        h = (v < kMillsV0) ? 0.0f : exp2f(lh);
        T = (v < kMillsV0) ? -v : dlh * kTScale;
    } else {
        T = mills_tail_T(v);
        h = v + T;
    }
}

__device__ __forceinline__ void mills(float v, float& h, float& T, const MillsCoef* tab) {
    mills_t<true>(v, h, T, tab);
}

struct PairTerm {
    float c;   // coefficient of (x_self - x_other)
    float w;   // weight added to z_self
};

// delta = sqrt(ss), inv_delta = 1/delta (0 when delta = 0).  kGlobal: the
// table K.mills is in global memory, else a copy in shared memory.
template <bool kGlobal = true>
__device__ __forceinline__ PairTerm pair_term(float delta, float inv_delta, bool edge, const PairConsts& K) {
    const float u = (delta - K.mu) * K.inv_sigma;
    const float v = edge ? u : -u;
    float h, T;
    mills_t<kGlobal>(v, h, T, K.mills);
    const float w = h * (K.printed ? (h + T) : T) * K.w_scale;
    const float g = h * K.g_scale;                   // |dl'| / 2
    // d = delta - g/w (edge) < 0  <=>  g > w delta
    const bool s_zero = !(delta > 0.0f) || (K.clamp && edge && g > w * delta);
    PairTerm r;
    r.w = w;
    r.c = s_zero ? -w : (edge ? -g : g) * inv_delta;
    return r;
}

// 2^x by the hardware's base-2 exponential, results below the FP32 normal
// range flushed to zero.
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Non-edge pair terms with the epoch's constants folded in (the tile
// kernels, where every pair is a sampled non-edge).  With v = (mu - delta) /
// sigma, the table coordinate pos = (v - kMillsV0) * kMillsStepsPerUnit is
// one FMA of delta; pos < 0 is v < kMillsV0 (h = 0, T = -v), pos past the
// last interval is v >= kMillsV1 (the continued fraction).  The same h, T,
// w, c as pair_term(delta, inv_delta, false, K) up to rounding; an h below
// the FP32 normal range (v < -13.2) is taken as 0.
struct NonEdgeConsts {
    float pos_a, pos_b;   // pos = pos_a - pos_b * delta
    float w_scale, g_scale;
    int printed;
    const MillsCoef* mills;
};

__device__ __forceinline__ NonEdgeConsts make_nonedge_consts(const PairConsts& K) {
    NonEdgeConsts n;
    n.pos_b = K.inv_sigma * (float)kMillsStepsPerUnit;
    n.pos_a = (K.mu * K.inv_sigma - kMillsV0) * (float)kMillsStepsPerUnit;
    n.w_scale = K.w_scale;
    n.g_scale = K.g_scale;
    n.printed = K.printed;
    n.mills = K.mills;
    return n;
}

template <bool kGlobal>
__device__ __forceinline__ PairTerm nonedge_term(float delta, float inv_delta, const NonEdgeConsts& N) {
    constexpr float kInvSteps = 1.0f / (float)kMillsStepsPerUnit;
    const float pos_raw = fmaf(-N.pos_b, delta, N.pos_a);
    float h, T;
    if (pos_raw < (float)kMillsIntervals) {
        const float pos = fmaxf(pos_raw, 0.0f);
        const int i = (int)pos;   // < kMillsIntervals
        const float x = pos - (float)i;
        const float4 c = kGlobal ? __ldg(&N.mills[i].lh) : N.mills[i].lh;
        const float lh = fmaf(fmaf(fmaf(c.w, x, c.z), x, c.y), x, c.x);
        const float dlh = fmaf(fmaf(3.0f * c.w, x, 2.0f * c.z), x, c.y);
        constexpr float kTScale = 0.69314718055994531f * (float)kMillsStepsPerUnit;
        const bool below = pos_raw < 0.0f;
        h = below ? 0.0f : ex2_ftz(lh);
        T = below ? -fmaf(pos_raw, kInvSteps, kMillsV0) : dlh * kTScale;
    } else {
        const float v = fmaf(pos_raw, kInvSteps, kMillsV0);
        T = mills_tail_T(v);
        h = v + T;
    }
    PairTerm r;
    r.w = h * (N.printed ? (h + T) : T) * N.w_scale;
    r.c = delta > 0.0f ? h * N.g_scale * inv_delta : -r.w;
    return r;
}

// sqrt and reciprocal of a squared distance (both 0 for ss = 0)
__device__ __forceinline__ void dist_of(float ss, float& delta, float& inv_delta) {
    const float r = rsqrtf(ss);
    inv_delta = (ss > 0.0f) ? r : 0.0f;
    delta = ss * inv_delta;
}

// -log2 Q(v): the description length of an edge (v = u) or non-edge (v = -u).
__device__ __forceinline__ float neg_log2_Q(float v) {
    const float inv_ln2 = 1.4426950408889634f;
    if (v > 0.0f) {
        const float ex = erfcxf(v * 0.70710678118654752f);
        return (0.5f * v * v - logf(0.5f * ex)) * inv_ln2;
    }
    return -log1pf(-0.5f * erfcf(-v * 0.70710678118654752f)) * inv_ln2;
}

}  // namespace gempe
