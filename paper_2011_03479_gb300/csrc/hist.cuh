// Block-private distance histograms of the sweep kernels (Sec. III.F).
#pragma once
#include "engine.cuh"

namespace gempe {

// ---------------------------------------------------------------------------
// Block-private distance histograms (Sec. III.F), all 32-bit integer bins so
// that every update is a native shared-memory atomic:
//   he[b]  edge count (each undirected edge once, j > i)
//   hc[b]  sample count
//   hd[b]  sum of the anchor degrees of those samples
// A sample anchored at i weighs (n-1-deg_i)/(2 k_acc_i); while no sample of
// i was dropped (k_acc_i = k) the non-edge bin is ((n-1) hc - hd) / (2k).
// Samples of vertices with dropped slots add their weight's difference to
// that value into hx (global float, rare).
// ---------------------------------------------------------------------------
struct BlockHist {
    unsigned int* he;
    unsigned int* hc;
    unsigned int* hd;
};

__device__ __forceinline__ BlockHist block_hist(unsigned int* base, int bins) {
    BlockHist h;
    h.he = base;
    h.hc = base + bins;
    h.hd = base + 2 * bins;
    return h;
}

__device__ __forceinline__ void hist_clear(const BlockHist& h, int bins) {
    for (int t = threadIdx.x; t < bins; t += blockDim.x) {
        h.he[t] = 0u;
        h.hc[t] = 0u;
        h.hd[t] = 0u;
    }
}

__device__ __forceinline__ void hist_merge(const BlockHist& h, const EpochArgs& a) {
    for (int t = threadIdx.x; t < a.bins; t += blockDim.x) {
        const unsigned int e = h.he[t], c = h.hc[t], d = h.hd[t];
        if (e) atomicAdd(a.hist_e + t, e);
        if (c) atomicAdd(a.hist_c + t, c);
        if (d) atomicAdd(a.hist_d + t, (unsigned long long)d);
    }
}

// k_slots: sample slots per vertex (k, or the block partner count)
__device__ __forceinline__ void hist_sample(const BlockHist& h, const EpochArgs& a, int bin, int deg, int k_acc,
                                            int k_slots) {
    atomicAdd(h.hc + bin, 1u);
    atomicAdd(h.hd + bin, (unsigned int)deg);
    if (k_acc < k_slots && k_acc > 0) {
        const float base = (float)(a.n - 1 - deg);
        atomicAdd(a.hist_x + bin, base / (2.0f * (float)k_acc) - base / (2.0f * (float)k_slots));
    }
}


}  // namespace gempe
