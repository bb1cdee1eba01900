// The global words that staging one tile of block-sampled non-edges needs,
// loaded one tile ahead so that their latency hides behind the tile before:
// the tile and its graph, the mask word and degree of anchor t (thread
// t < kBlockT stages anchor t), partner t (t < kBlockP), and the partner ids
// of the 16-byte row chunks this thread copies (chunk c = t + kThreads j of
// the kBlockP x CH chunks of the partners' rows).
#pragma once
#include "engine.cuh"

namespace gempe {

template <int CH, int kThreads>
struct TileAhead {
    static constexpr int kChunks = (kBlockP * CH + kThreads - 1) / kThreads;
    int tile, graph, v0, nv;
    unsigned long long m;
    int deg, part;
    int pid[kChunks];
};

template <int CH, int kThreads>
__device__ __forceinline__ TileAhead<CH, kThreads> tile_ahead(const EpochArgs& a, int it, int tid) {
    TileAhead<CH, kThreads> t;
    const int2 ti = __ldg(a.tile_items + it);
    t.tile = ti.x;
    t.graph = ti.y;
    const int gv0 = __ldg(&a.graphs[t.graph].v0), gn = __ldg(&a.graphs[t.graph].n);
    const int lt = t.tile - __ldg(&a.graphs[t.graph].t0);
    t.v0 = gv0 + lt * kBlockT;
    t.nv = min(kBlockT, gn - lt * kBlockT);
    const int epoch = a.gst[t.graph].epoch;
    const int32_t* part = a.block_part + ((size_t)(epoch & 1) * (size_t)a.n_tiles + t.tile) * kBlockP;
    t.m = ~0ull;
    t.deg = 0;
    if (tid < t.nv) {   // nv <= kBlockT
        t.m = a.block_mask[(size_t)(epoch & 1) * (size_t)a.rows + t.v0 + tid];
        t.deg = __ldg(a.row_ptr + t.v0 + tid + 1) - __ldg(a.row_ptr + t.v0 + tid);
    }
#pragma unroll
    for (int j = 0; j < TileAhead<CH, kThreads>::kChunks; ++j) {
        const int c = tid + kThreads * j;
        t.pid[j] = c < kBlockP * CH ? __ldg(part + c / CH) : 0;
    }
    t.part = tid < kBlockP ? __ldg(part + tid) : 0;
    return t;
}

}  // namespace gempe
