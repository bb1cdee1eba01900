// Distance histograms of the sweep kernels (Sec. III.F).
#pragma once
#include "engine.cuh"

namespace gempe {

// ---------------------------------------------------------------------------
// Distance histograms (Sec. III.F), all 32-bit integer bins so that every
// block-level update is a native shared-memory atomic:
//   he[b]  edge count (each undirected edge once, j > i)
//   hc[b]  sample count
//   hd[b]  sum of the anchor degrees of those samples
// A sample anchored at i weighs (n-1-deg_i)/(2 k_acc_i); while no sample of
// i was dropped (k_acc_i = k) the non-edge bin is ((n-1) hc - hd) / (2k).
// Samples of vertices with dropped slots add their weight's difference to
// that value into hx (global float, rare).
//
// A block keeps shared bins for one graph, its home graph (the graph of its
// first work unit); pairs of other graphs go to that graph's global bins
// directly.  In a pack of one graph every pair lands in shared bins.
// ---------------------------------------------------------------------------
struct BlockHist {
    unsigned int* he;
    unsigned int* hc;
    unsigned int* hd;
    float* hw;        // per-slot policy: sums of the samples' weights
    int home;
};

__device__ __forceinline__ BlockHist block_hist(unsigned int* base, int bins, int home) {
    BlockHist h;
    h.he = base;
    h.hc = base + bins;
    h.hd = base + 2 * bins;
    h.hw = reinterpret_cast<float*>(base + 3 * bins);
    h.home = home;
    return h;
}

__device__ __forceinline__ void hist_clear(const BlockHist& h, int bins) {
    for (int t = threadIdx.x; t < bins; t += blockDim.x) {
        h.he[t] = 0u;
        h.hc[t] = 0u;
        h.hd[t] = 0u;
        h.hw[t] = 0.0f;
    }
}

__device__ __forceinline__ void hist_merge(const BlockHist& h, const EpochArgs& a) {
    if (h.home < 0) return;
    const size_t off = (size_t)h.home * a.bins;
    for (int t = threadIdx.x; t < a.bins; t += blockDim.x) {
        const unsigned int e = h.he[t], c = h.hc[t], d = h.hd[t];
        if (e) atomicAdd(a.hist_e + off + t, e);
        if (c) atomicAdd(a.hist_c + off + t, c);
        if (d) atomicAdd(a.hist_d + off + t, (unsigned long long)d);
        if (a.per_slot && h.hw[t] != 0.0f) atomicAdd(a.hist_x + off + t, h.hw[t]);
    }
}

// A per-slot sample anchored at a vertex of degree deg with k_acc accepted
// samples weighs (n-1-deg)/(2 k_acc): added as a float.
__device__ __forceinline__ void hist_sample_w(const BlockHist& h, const EpochArgs& a, int graph, int bin, int deg,
                                              int k_acc) {
    if (!a.sweep_hist) return;
    const float w = (float)(__ldg(&a.graphs[graph].n) - 1 - deg) / (2.0f * (float)k_acc);
    if (graph == h.home) atomicAdd(h.hw + bin, w);
    else atomicAdd(a.hist_x + (size_t)graph * a.bins + bin, w);
}

__device__ __forceinline__ void hist_edge(const BlockHist& h, const EpochArgs& a, int graph, int bin) {
    if (!a.sweep_hist) return;
    if (graph == h.home) atomicAdd(h.he + bin, 1u);
    else atomicAdd(a.hist_e + (size_t)graph * a.bins + bin, 1u);
}

// k_slots: sample slots per vertex (k, or the block partner count)
__device__ __forceinline__ void hist_sample(const BlockHist& h, const EpochArgs& a, int graph, int bin, int deg,
                                            int k_acc, int k_slots) {
    if (!a.sweep_hist) return;
    if (graph == h.home) {
        atomicAdd(h.hc + bin, 1u);
        atomicAdd(h.hd + bin, (unsigned int)deg);
    } else {
        const size_t off = (size_t)graph * a.bins + bin;
        atomicAdd(a.hist_c + off, 1u);
        atomicAdd(a.hist_d + off, (unsigned long long)deg);
    }
    if (k_acc < k_slots && k_acc > 0) {
        const float base = (float)(__ldg(&a.graphs[graph].n) - 1 - deg);
        atomicAdd(a.hist_x + (size_t)graph * a.bins + bin, base / (2.0f * (float)k_acc) - base / (2.0f * (float)k_slots));
    }
}

// Work units of one warp: block b takes units [b U / B, (b+1) U / B) when
// a.blocked (its warps striding through them), else the grid strides.
struct UnitRange {
    int begin, end, step;
};

__device__ __forceinline__ UnitRange warp_units(const EpochArgs& a) {
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    UnitRange r;
    if (a.blocked) {
        const int lo = (int)((long long)a.n_items * blockIdx.x / gridDim.x);
        r.begin = lo + wib;
        r.end = (int)((long long)a.n_items * (blockIdx.x + 1) / gridDim.x);
        r.step = wpb;
    } else {
        r.begin = blockIdx.x * wpb + wib;
        r.end = a.n_items;
        r.step = gridDim.x * wpb;
    }
    return r;
}

// The home graph of this block (-1: none).
__device__ __forceinline__ int home_graph(const EpochArgs& a) {
    if (!a.blocked) return a.n_graphs == 1 ? 0 : -1;
    const int lo = (int)((long long)a.n_items * blockIdx.x / gridDim.x);
    return lo < a.n_items ? (__ldg(&a.items[lo].y) >> kGraphShift) : -1;
}

}  // namespace gempe
