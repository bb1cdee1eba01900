// Host side of a pack (see pack.cuh): layout, device copies, work lists,
// epoch enqueueing and the sweep autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "pack.cuh"

namespace gempe {

gempe_status pack_fail(gempe_status st, const std::string& msg) {
    set_last_error(msg.c_str());
    return st;
}

gempe_status pack_cuda_fail(cudaError_t e, const char* what) {
    return pack_fail(e == cudaErrorMemoryAllocation ? GEMPE_E_OOM : GEMPE_E_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

#define PK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return pack_cuda_fail(e_, what); \
    } while (0)

gempe_status check_params(const gempe_params* p, int32_t d) {
    if (!p) return pack_fail(GEMPE_E_INVALID_ARG, "params is null");
    if (!supported_dim(d)) return pack_fail(GEMPE_E_INVALID_ARG, "d must be one of 1,2,3,4,8,16,32,64,128,256");
    if (p->neg_per_vertex < 0 || p->neg_per_vertex > kMaxK)
        return pack_fail(GEMPE_E_INVALID_ARG, "neg_per_vertex must be in [0, 32]");
    if (p->max_retries < 1 || p->max_retries > 4096)
        return pack_fail(GEMPE_E_INVALID_ARG, "max_retries must be in [1, 4096]");
    if (p->hist_bins < 16 || p->hist_bins > 4096)
        return pack_fail(GEMPE_E_INVALID_ARG, "hist_bins must be in [16, 4096]");
    if (!(p->hist_max > 0.0f) || !(p->sigma0 > 0.0f) || !std::isfinite(p->mu) || !(p->init_range > 0.0f) ||
        !(p->z_min > 0.0f))
        return pack_fail(GEMPE_E_INVALID_ARG,
                         "hist_max, sigma0, init_range and z_min must be positive, mu finite");
    if (p->sigma_every < 0) return pack_fail(GEMPE_E_INVALID_ARG, "sigma_every must be >= 0");
    if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr))
        return pack_fail(GEMPE_E_INVALID_ARG, "dev_alloc and dev_free must be given together");
    if (p->precision != 0 && p->precision != 1) return pack_fail(GEMPE_E_INVALID_ARG, "precision must be 0 or 1");
    if (p->precision == 1 && d < 8) return pack_fail(GEMPE_E_INVALID_ARG, "the BF16 form needs d >= 8");
    if (p->block_partners != 0 && p->block_partners != kBlockP)
        return pack_fail(GEMPE_E_INVALID_ARG, "block_partners must be 0 or 64");
    if (p->block_partners && (d < 8 || (p->tile_vertices != 0 && p->tile_vertices != kBlockT)))
        return pack_fail(GEMPE_E_INVALID_ARG, "block sampling needs d >= 8 and tile_vertices 128");
    if (p->autotune != 0 && p->autotune != 1) return pack_fail(GEMPE_E_INVALID_ARG, "autotune must be 0 or 1");
    if (p->sampling != 0 && p->sampling != 1) return pack_fail(GEMPE_E_INVALID_ARG, "sampling must be 0 or 1");
    if (p->sigma_source != 0 && p->sigma_source != 1)
        return pack_fail(GEMPE_E_INVALID_ARG, "sigma_source must be 0 or 1");
    if (p->sampling == 1 && p->block_partners)
        return pack_fail(GEMPE_E_INVALID_ARG, "the per-slot sampling policy excludes block sampling");
    if (p->membership != 0 && p->membership != 1) return pack_fail(GEMPE_E_INVALID_ARG, "membership must be 0 or 1");
    if (p->membership == 1 && p->block_partners)
        return pack_fail(GEMPE_E_INVALID_ARG, "byte-map membership applies to the sampled non-edges, not block sampling");
    if (p->bytemap_log2 != 0 && (p->bytemap_log2 < 6 || p->bytemap_log2 > 32))
        return pack_fail(GEMPE_E_INVALID_ARG, "bytemap_log2 must be 0 (automatic) or in [6, 32]");
    if (p->rename_every < 0) return pack_fail(GEMPE_E_INVALID_ARG, "rename_every must be >= 0");
    if (p->rng != 0 && p->rng != 1) return pack_fail(GEMPE_E_INVALID_ARG, "rng must be 0 or 1");
    if (p->rng == 1 && p->block_partners)
        return pack_fail(GEMPE_E_INVALID_ARG, "the LCG draws the sampled non-edges, not block partners");
    return GEMPE_OK;
}

int host_threads(int64_t work) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t by_work = work / (1 << 16) + 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 32, by_work}));
}

namespace {

// Runs fn(begin, end) over [0, count) cut into `parts` consecutive ranges of
// (roughly) equal weight, one thread per range (the caller runs the first).
// cum(i): the weight of [0, i), non-decreasing.
template <typename Cum, typename F>
void parallel_ranges(int64_t count, int parts, Cum cum, F fn) {
    if (parts <= 1 || count < 2) {
        fn((int64_t)0, count);
        return;
    }
    std::vector<int64_t> cut(parts + 1, 0);
    const int64_t total = cum(count);
    for (int t = 1; t < parts; ++t) {
        const int64_t target = total * t / parts;
        int64_t lo = cut[t - 1], hi = count;   // first i with cum(i) >= target
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (cum(mid) < target) lo = mid + 1; else hi = mid;
        }
        cut[t] = lo;
    }
    cut[parts] = count;
    std::vector<std::thread> th;
    th.reserve(parts - 1);
    for (int t = 1; t < parts; ++t) th.emplace_back(fn, cut[t], cut[t + 1]);
    fn(cut[0], cut[1]);
    for (auto& x : th) x.join();
}

}  // namespace

void parallel_for_weighted(int64_t count, int parts, const std::function<int64_t(int64_t)>& cum,
                           const std::function<void(int64_t, int64_t)>& fn) {
    parallel_ranges(count, parts, cum, fn);
}

// Symmetric, sorted, loop-free, duplicate-free, in-range CSR.  The rows are
// checked in parallel (ranges of equal CSR slots); the error reported is the
// one of the lowest row, as a row-by-row check would find it: first the
// per-row checks of every row, then (symmetry) the symmetry by a binary
// search of (j, i) in row j for every slot (i, j).
gempe_status validate_csr(const int32_t* rp, const int32_t* ci, int32_t n, int threads, bool symmetry) {
    if (rp[0] != 0) return pack_fail(GEMPE_E_INVALID_GRAPH, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return pack_fail(GEMPE_E_INVALID_GRAPH, "row_ptr must be non-decreasing");
    const int parts = threads > 0 ? threads : host_threads(rp[n]);
    auto cum = [&](int64_t i) { return (int64_t)rp[i] + i; };
    std::mutex mu;
    int32_t bad_row = n, bad_kind = 0, bad_j = 0;
    auto report = [&](int32_t i, int kind, int32_t j) {
        std::lock_guard<std::mutex> lock(mu);
        if (i < bad_row) {
            bad_row = i;
            bad_kind = kind;
            bad_j = j;
        }
    };
    parallel_ranges(n, parts, cum, [&](int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; ++i)
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t j = ci[e];
                const int kind = (j < 0 || j >= n) ? 1 : (j == i) ? 2 : (e > rp[i] && ci[e - 1] >= j) ? 3 : 0;
                if (kind) {
                    report((int32_t)i, kind, j);
                    return;
                }
            }
    });
    if (bad_kind == 1) return pack_fail(GEMPE_E_INVALID_GRAPH, "column index out of range");
    if (bad_kind == 2) return pack_fail(GEMPE_E_INVALID_GRAPH, "self loop at vertex " + std::to_string(bad_row));
    if (bad_kind == 3)
        return pack_fail(GEMPE_E_INVALID_GRAPH, "row " + std::to_string(bad_row) + " not strictly increasing");
    if (!symmetry) return GEMPE_OK;
    parallel_ranges(n, parts, cum, [&](int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; ++i)
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t j = ci[e];
                if (!std::binary_search(ci + rp[j], ci + rp[j + 1], (int32_t)i)) {
                    report((int32_t)i, 4, j);
                    return;
                }
            }
    });
    if (bad_kind == 4)
        return pack_fail(GEMPE_E_INVALID_GRAPH, "graph not symmetric: (" + std::to_string(bad_row) + "," +
                                                    std::to_string(bad_j) + ") without its reverse");
    return GEMPE_OK;
}

namespace {

// Work units of the packed sweep (d <= 4) for rows [v0, v0 + n) of graph g:
// runs of up to 32 consecutive vertices with at most `budget` edge + sample
// slots in total; a vertex with more is cut into `budget`-slot chunks of its
// row, the last chunk carrying the samples.
// per_slot: Sec. III.C's policy, every CSR slot carries its own sample, so a
// vertex has 2 deg pairs and a hub chunk of c slots carries c samples.
void packed_units(const int32_t* rp, int32_t v0, int32_t n, int32_t k, int budget, int32_t g, bool per_slot,
                  std::vector<int4>& units) {
    const int smp = (k > 0 || per_slot) ? kUnitHasSamples : 0;
    const int gy = g << kGraphShift;
    int32_t i = v0;
    const int32_t end = v0 + n;
    while (i < end) {
        const int32_t deg = rp[i + 1] - rp[i];
        const int32_t pairs_i = per_slot ? 2 * deg : deg + k;
        if (pairs_i > budget) {
            const int32_t chunk = per_slot ? budget / 2 : budget;
            int32_t e = 0;
            while (deg - e > chunk) {
                units.push_back(make_int4(i, gy | 1, e, (e + chunk) | (per_slot ? smp : 0)));
                e += chunk;
            }
            units.push_back(make_int4(i, gy | 1, e, deg | smp));
            ++i;
            continue;
        }
        const int32_t u0 = i;
        int32_t pairs = 0;
        while (i < end && i - u0 < 32) {
            const int32_t di = per_slot ? 2 * (rp[i + 1] - rp[i]) : rp[i + 1] - rp[i] + k;
            if (di > budget || pairs + di > budget) break;
            pairs += di;
            ++i;
        }
        units.push_back(make_int4(u0, gy | (i - u0), -1, smp));
    }
}

// Work units of the per-unit sweep (d >= 8): each vertex's CSR slots in
// chunks of `chunk`, the last chunk also carrying the vertex's samples.
// per_slot: every chunk carries the samples of its own slots.
void chunk_units(const int32_t* rp, int32_t v0, int32_t n, int chunk, int32_t g, bool per_slot,
                 std::vector<int4>& units) {
    const int gy = (g << kGraphShift) | 1;
    for (int32_t i = v0; i < v0 + n; ++i) {
        const int32_t deg = rp[i + 1] - rp[i];
        const int32_t chunks = std::max<int32_t>(1, (deg + chunk - 1) / chunk);
        for (int32_t c = 0; c < chunks; ++c) {
            const int32_t p0 = c * chunk, p1 = std::min(deg, (c + 1) * chunk);
            units.push_back(make_int4(i, gy, p0, p1 | ((per_slot || c == chunks - 1) ? kUnitHasSamples : 0)));
        }
    }
}

// Warp tasks of the d >= 8 sweep: groups of `pg` units (one per lane group)
// of similar size, so that the groups of a warp run the same number of
// rounds.  Within windows of 16 * pg consecutive units the units are sorted
// by their pair count, then cut into consecutive tasks; the list is padded to
// a multiple of pg with empty units (vertex -1).
int unit_pairs_of(const int4& u, int k_slots, bool per_slot) {
    const int ne = (u.w & ~kUnitHasSamples) - u.z;
    return ne + ((u.w & kUnitHasSamples) ? (per_slot ? ne : k_slots) : 0);
}

void wide_tasks(std::vector<int4>& units, int pg, int k_slots, bool per_slot) {
    if (pg <= 1) return;
    const size_t window = 16 * (size_t)pg;
    const int64_t n_windows = (int64_t)((units.size() + window - 1) / window);
    // each window ordered by decreasing pair count, ties in their original
    // order (a stable sort, without the per-call buffer of std::stable_sort);
    // the windows are independent and split over host threads
    parallel_ranges(n_windows, host_threads((int64_t)units.size()), [](int64_t i) { return i; },
                    [&](int64_t wlo, int64_t whi) {
                        std::vector<std::pair<int, int>> key(window);
                        std::vector<int4> tmp(window);
                        for (int64_t wi = wlo; wi < whi; ++wi) {
                            const size_t w0 = (size_t)wi * window;
                            const size_t w1 = std::min(units.size(), w0 + window), len = w1 - w0;
                            for (size_t q = 0; q < len; ++q)
                                key[q] = {-unit_pairs_of(units[w0 + q], k_slots, per_slot), (int)q};
                            std::sort(key.begin(), key.begin() + len);
                            for (size_t q = 0; q < len; ++q) tmp[q] = units[w0 + key[q].second];
                            std::copy(tmp.begin(), tmp.begin() + len, units.begin() + w0);
                        }
                    });
    while (units.size() % pg) units.push_back(make_int4(-1, 0, 0, 0));
}

// Slots of a graph's edge set: every undirected edge once (nnz / 2 keys) at
// a load of at most 1/2.
unsigned long long table_slots(int64_t nnz) {
    unsigned long long s = 16;
    while (s < (unsigned long long)std::max<int64_t>(nnz, 0)) s <<= 1;
    return s;
}

}  // namespace

Pack::~Pack() {
    if (stream) cudaStreamSynchronize(stream);
    if (side) cudaStreamSynchronize(side);
    if (tile_stream) cudaStreamSynchronize(tile_stream);
    release_all();
    if (tile_fork) cudaEventDestroy(tile_fork);
    if (tile_join) cudaEventDestroy(tile_join);
    if (tile_stream) cudaStreamDestroy(tile_stream);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    for (cudaEvent_t& e : tev)
        if (e) cudaEventDestroy(e);
    if (side) cudaStreamDestroy(side);
}

namespace {
// The default allocation path is stream-ordered (the device's default memory
// pool, cudaMallocAsync on the pack's stream): a context that is created
// and destroyed per job reuses the pool's memory instead of mapping and
// unmapping it (and synchronising the device) every time.  The pool keeps
// what it holds between jobs (release threshold: unlimited) for the life of
// the process.
void keep_pool_memory(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), device) != done.end()) return;
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(device);
}
}  // namespace

void* Pack::alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    if (p.dev_alloc) {
        ptr = p.dev_alloc(bytes, p.alloc_user);
    } else {
        keep_pool_memory(device);
        if (cudaMallocAsync(&ptr, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
        }
    }
    if (ptr) allocations.push_back(ptr);
    return ptr;
}

void Pack::free_one(void* ptr) {
    if (p.dev_free) p.dev_free(ptr, p.alloc_user);
    else cudaFreeAsync(ptr, stream);
}

void Pack::release(void* ptr) {
    if (!ptr) return;
    auto it = std::find(allocations.begin(), allocations.end(), ptr);
    if (it == allocations.end()) return;
    allocations.erase(it);
    free_one(ptr);
}

void Pack::release_all() {
    for (void* ptr : allocations) free_one(ptr);
    allocations.clear();
    if (!p.dev_free && stream) cudaStreamSynchronize(stream);
}

gempe_status Pack::build(const std::vector<GraphInput>& gs, int32_t dim, const gempe_params& params,
                         cudaStream_t s, bool validate) {
    gempe_status rc = check_params(&params, dim);
    if (rc != GEMPE_OK) return rc;
    if (gs.empty()) return pack_fail(GEMPE_E_INVALID_ARG, "a pack needs at least one graph");
    if (gs.size() >= (1u << (31 - kGraphShift))) return pack_fail(GEMPE_E_INVALID_ARG, "too many graphs");
    p = params;
    d = dim;
    k = p.neg_per_vertex;
    acc_stride = acc_stride_for(d);
    bins = p.hist_bins;
    G = (int32_t)gs.size();
    stream = s;
    block = p.block_partners > 0;
    tiles = block && (p.precision == 1 ? tile_dim(d) : tile_dim_f32(d));
    per_slot = p.sampling == 1;
    narrow_keys = true;
    for (const GraphInput& in : gs) narrow_keys = narrow_keys && in.n <= kNarrowKeysMaxN;
    const unsigned long long per_bucket = narrow_keys ? 8 : 4;

    // layout
    long long rows_ll = 0, slots_ll = 0, tiles_ll = 0;
    unsigned long long kslots = 0, map_off = 0;
    info.assign(G, GraphInfo{});
    nnz.assign(G, 0);
    for (int32_t g = 0; g < G; ++g) {
        const GraphInput& in = gs[g];
        if (!in.row_ptr || (!in.col_idx && in.n > 0 && in.row_ptr[in.n] > 0))
            return pack_fail(GEMPE_E_INVALID_ARG, "null CSR array");
        if (in.n < 2) return pack_fail(GEMPE_E_INVALID_ARG, "n must be at least 2");
        if (in.row_ptr[in.n] < 0) return pack_fail(GEMPE_E_INVALID_GRAPH, "row_ptr[n] negative");
        if (validate) {
            rc = validate_csr(in.row_ptr, in.col_idx, in.n);
            if (rc != GEMPE_OK) return rc;
        }
        nnz[g] = in.row_ptr[in.n];
        // the per-block sums of sampled anchors' degrees are 32-bit
        if (!per_slot && (unsigned long long)std::max(k, slots_per_vertex()) * (unsigned long long)nnz[g] >= (1ull << 32))
            return pack_fail(GEMPE_E_INVALID_ARG, "sample slots * nnz must be below 2^32");
        GraphInfo& gi = info[g];
        gi.v0 = (int32_t)rows_ll;
        gi.n = in.n;
        gi.t0 = (int32_t)tiles_ll;
        gi.n_tiles = block ? (in.n + kBlockT - 1) / kBlockT : 0;
        gi.key_lo = (uint32_t)in.key;
        gi.key_hi = (uint32_t)(in.key >> 32);
        gi.key_off = kslots;
        const unsigned long long ts = table_slots(nnz[g]);
        gi.bucket_mask = ts / per_bucket - 1;
        if (p.membership == 1) {
            // each map's size is a power of two >= 64, so every offset is a multiple of 64
            const int lg = bytemap_log2_for(nnz[g], p);
            gi.map = map_off | (unsigned long long)lg;
            map_off += 1ull << lg;
        }
        rows_ll += (long long)in.n + 1;
        slots_ll += nnz[g];
        tiles_ll += gi.n_tiles;
        kslots += ts;
    }
    if (rows_ll >= INT32_MAX || slots_ll >= INT32_MAX)
        return pack_fail(GEMPE_E_INVALID_ARG, "a pack holds below 2^31 vertices and CSR slots");
    rows = (int32_t)rows_ll;
    slots = slots_ll;
    n_tiles = (int32_t)tiles_ll;
    key_slots = kslots;
    bytemap_bytes = (size_t)map_off;

    PK(cudaGetDevice(&device), "cudaGetDevice");
    PK(ensure_mills_table(), "Mills table");
    PK(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device), "cudaDeviceGetAttribute");
    PK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking), "cudaStreamCreate");
    if (tiles) {
        PK(cudaStreamCreateWithPriority(&tile_stream, cudaStreamNonBlocking, critical_priority()), "cudaStreamCreate");
        PK(cudaEventCreateWithFlags(&tile_fork, cudaEventDisableTiming), "cudaEventCreate");
        PK(cudaEventCreateWithFlags(&tile_join, cudaEventDisableTiming), "cudaEventCreate");
    }
    PK(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming), "cudaEventCreate");
    PK(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming), "cudaEventCreate");
    mills = mills_table_device();
    if (!mills) return pack_fail(GEMPE_E_CUDA, "Mills table address");
    if (tiles)
        PK(p.precision == 1 ? prepare_tile_kernel(d, bins) : prepare_tile_f32_kernel(d, bins), "tile kernel attributes");
    PK(prepare_update_kernels(bins), "update kernel attributes");

    // host copy of the pack's row offsets (the column arrays go to the
    // device as they are and are shifted to pack rows there)
    row_ptr_h.assign((size_t)rows + 1, 0);
    std::vector<int32_t> slot0(G);   // first CSR slot of each graph
    for (int32_t g = 0; g < G; ++g) {
        const GraphInput& in = gs[g];
        const GraphInfo& gi = info[g];
        const int32_t s0 = (int32_t)(g == 0 ? 0 : row_ptr_h[gi.v0]);
        slot0[g] = s0;
        for (int32_t i = 0; i <= in.n; ++i) row_ptr_h[(size_t)gi.v0 + i] = s0 + in.row_ptr[i];
        // the spare row v0 + n closes the range; the next graph starts there
        if (g + 1 < G) row_ptr_h[(size_t)gi.v0 + in.n + 1] = s0 + (int32_t)nnz[g];
    }
    row_ptr_h[(size_t)rows] = (int32_t)slots;
    // the degree-oriented CSR of the packed sweep is built on the device
    // (setup.cu); its row offsets come back to orow_ptr_h for the work units
    const bool oriented_csr = d <= kPackedMaxDim && !per_slot && !block;
    orow_ptr_h.clear();
    // vertex chunks and tile lists
    std::vector<int4> vch;
    std::vector<int2> titems;
    std::vector<int4> sunits;
    for (int32_t g = 0; g < G; ++g) {
        const GraphInfo& gi = info[g];
        // a shard takes the chunks and tiles of its own vertex range only
        const int32_t lo = sharded() ? own_lo : 0, hi = sharded() ? own_hi : gi.n;
        for (int32_t o = lo; o < hi; o += kVChunk) vch.push_back(make_int4(gi.v0 + o, std::min(kVChunk, hi - o), g, 0));
        for (int32_t t = lo / kBlockT; t < (block ? (hi + kBlockT - 1) / kBlockT : 0); ++t) {
            titems.push_back(make_int2(gi.t0 + t, g));
            sunits.push_back(make_int4(gi.t0 + t, 0, 0, (g << 1) | 1));
        }
    }
    n_vchunks = (int32_t)vch.size();
    n_tile_items = tiles ? (int32_t)titems.size() : 0;
    n_sampler_units = (int32_t)sunits.size();

    // device memory
    const size_t R = (size_t)rows;
    row_ptr = (int32_t*)alloc(sizeof(int32_t) * (R + 1));
    col_idx = (int32_t*)alloc(sizeof(int32_t) * std::max<size_t>((size_t)slots, 1));
    keys = alloc((narrow_keys ? 4 : 8) * key_slots);
    // set-up scratch: per graph {slots above, below, below without reverse}
    // of the symmetry check, then the oriented rows' counts and scan sums
    unsigned long long* sym = (unsigned long long*)alloc(sizeof(unsigned long long) * 3 * (size_t)G);
    int32_t* oscratch = nullptr;
    if (!sym) return pack_fail(GEMPE_E_OOM, "device allocation failed");
    if (oriented_csr) {
        // ocol_idx holds every slot at most (exactly half of them for a
        // symmetric graph, which is checked only after the build)
        orow_ptr = (int32_t*)alloc(sizeof(int32_t) * (R + 1));
        ocol_idx = (int32_t*)alloc(sizeof(int32_t) * std::max<size_t>((size_t)slots, 1));
        oscratch = (int32_t*)alloc(sizeof(int32_t) * orient_scratch_ints(rows));
        if (!orow_ptr || !ocol_idx || !oscratch) return pack_fail(GEMPE_E_OOM, "device allocation failed");
    }
    x = (float*)alloc(sizeof(float) * R * d);
    acc = (float*)alloc(sizeof(float) * R * acc_stride);
    const size_t GB = (size_t)G * bins;
    hist_bytes = GB * (sizeof(unsigned long long) + 2 * sizeof(unsigned int) + sizeof(float));
    hist = alloc(hist_bytes);
    if (hist) {
        hist_d = (unsigned long long*)hist;
        hist_e = (unsigned int*)(hist_d + GB);
        hist_c = hist_e + GB;
        hist_x = (float*)(hist_c + GB);
    }
    graphs = (GraphInfo*)alloc(sizeof(GraphInfo) * G);
    gst = (GraphState*)alloc(sizeof(GraphState) * G);
    ps = (PackState*)alloc(sizeof(PackState));
    vchunks = (int4*)alloc(sizeof(int4) * vch.size());
    scratch = (int32_t*)alloc(sizeof(int32_t) * std::max<size_t>(R * std::max(k, 1), 1));
    samples = (int32_t*)alloc(sizeof(int32_t) *
                              std::max<size_t>(block ? 1 : (per_slot ? 2 * (size_t)slots : 2 * R * k), 1));
    if (per_slot) {
        vacc = (int32_t*)alloc(sizeof(int32_t) * 2 * R);
        if (!vacc) return pack_fail(GEMPE_E_OOM, "device allocation failed");
    }
    if (p.precision == 1) xb = (__nv_bfloat16*)alloc(sizeof(__nv_bfloat16) * R * d);
    if (bytemap_bytes) {
        bytemap = (uint8_t*)alloc(bytemap_bytes);
        if (!bytemap) return pack_fail(GEMPE_E_OOM, "device allocation failed (byte maps)");
    }
    if (block) {
        block_part = (int32_t*)alloc(sizeof(int32_t) * 2 * (size_t)std::max(n_tiles, 1) * kBlockP);
        block_mask = (unsigned long long*)alloc(sizeof(unsigned long long) * 2 * R);
        sampler_units = (int4*)alloc(sizeof(int4) * std::max<size_t>(sunits.size(), 1));
        tile_items = (int2*)alloc(sizeof(int2) * std::max<size_t>(titems.size(), 1));
        if (!block_part || !block_mask || !sampler_units || !tile_items)
            return pack_fail(GEMPE_E_OOM, "device allocation failed");
    }
    if (!row_ptr || !col_idx || !keys || !x || !acc || !hist || !graphs || !gst || !ps || !vchunks ||
        !scratch || !samples || (p.precision == 1 && !xb))
        return pack_fail(GEMPE_E_OOM, "device allocation failed");

    std::vector<GraphState> st0(G);
    std::memset(st0.data(), 0, sizeof(GraphState) * G);
    for (auto& st : st0) {
        st.sigma = p.sigma0;
        st.map_period = bytemap ? 0 : -1;   // the maps are built below for period 0
    }
    PK(cudaMemcpyAsync(row_ptr, row_ptr_h.data(), sizeof(int32_t) * (R + 1), cudaMemcpyHostToDevice, s), "copy row_ptr");
    for (int32_t g = 0; g < G; ++g) {
        if (nnz[g] == 0) continue;
        PK(cudaMemcpyAsync(col_idx + slot0[g], gs[g].col_idx, sizeof(int32_t) * (size_t)nnz[g], cudaMemcpyHostToDevice, s),
           "copy col_idx");
        if (info[g].v0 != 0) PK(launch_add_offset(col_idx + slot0[g], nnz[g], info[g].v0, s), "col_idx to pack rows");
    }
    PK(cudaMemsetAsync(sym, 0, sizeof(unsigned long long) * 3 * (size_t)G, s), "clear counts");
    PK(cudaMemcpyAsync(graphs, info.data(), sizeof(GraphInfo) * G, cudaMemcpyHostToDevice, s), "copy graph table");
    PK(cudaMemcpyAsync(gst, st0.data(), sizeof(GraphState) * G, cudaMemcpyHostToDevice, s), "init graph state");
    PK(cudaMemsetAsync(ps, 0, sizeof(PackState), s), "init pack state");
    PK(cudaMemcpyAsync(vchunks, vch.data(), sizeof(int4) * vch.size(), cudaMemcpyHostToDevice, s), "copy chunks");
    PK(cudaMemsetAsync(keys, 0xFF, (narrow_keys ? 4 : 8) * key_slots, s), "clear edge sets");
    PK(cudaMemsetAsync(x, 0, sizeof(float) * R * d, s), "clear x");
    if (xb) PK(cudaMemsetAsync(xb, 0, sizeof(__nv_bfloat16) * R * d, s), "clear xb");
    PK(cudaMemsetAsync(acc, 0, sizeof(float) * R * acc_stride, s), "clear acc");
    PK(cudaMemsetAsync(hist, 0, hist_bytes, s), "clear hist");
    if (block) {
        PK(cudaMemsetAsync(block_mask, 0, sizeof(unsigned long long) * 2 * R, s), "clear masks");
        PK(cudaMemcpyAsync(sampler_units, sunits.data(), sizeof(int4) * sunits.size(), cudaMemcpyHostToDevice, s),
           "copy sampler units");
        PK(cudaMemcpyAsync(tile_items, titems.data(), sizeof(int2) * titems.size(), cudaMemcpyHostToDevice, s),
           "copy tile list");
    }
    PK(cudaMemsetAsync(scratch, 0, sizeof(int32_t), s), "clear flag");
    for (int32_t g = 0; g < G; ++g) {
        const GraphInfo& gi = info[g];
        PK(launch_hash_build(row_ptr, col_idx, gi.v0, gi.n, nnz[g],
                             static_cast<char*>(keys) + (narrow_keys ? 4 : 8) * gi.key_off, narrow_keys ? 1 : 0,
                             gi.bucket_mask, scratch, s),
           "hash build");
        PK(launch_init_positions(x + (size_t)gi.v0 * d, xb ? xb + (size_t)gi.v0 * d : nullptr, gi.n, d, gi.key_lo,
                                 gi.key_hi, p.init_range, s),
           "init positions");
    }
    for (int32_t g = 0; g < G; ++g) {
        const GraphInfo& gi = info[g];
        PK(launch_check_symmetric(row_ptr, col_idx, gi.v0, gi.n, nnz[g], keys, narrow_keys ? 1 : 0, gi.key_off,
                                  gi.bucket_mask, sym + 3 * (size_t)g, s),
           "symmetry check");
    }
    if (oriented_csr) {
        PK(launch_orient(row_ptr, col_idx, rows, orow_ptr, ocol_idx, oscratch, sm_count, s), "oriented CSR");
        orow_ptr_h.assign((size_t)rows + 1, 0);
        PK(cudaMemcpyAsync(orow_ptr_h.data(), orow_ptr, sizeof(int32_t) * (R + 1), cudaMemcpyDeviceToHost, s),
           "read oriented row_ptr");
    }
    if (bytemap) PK(launch_bytemap_build(args(), 1, sm_count, s), "byte-map build");
    int32_t hash_fail = 0;
    std::vector<unsigned long long> sym_h(3 * (size_t)G);
    PK(cudaMemcpyAsync(&hash_fail, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read flag");
    PK(cudaMemcpyAsync(sym_h.data(), sym, sizeof(unsigned long long) * sym_h.size(), cudaMemcpyDeviceToHost, s),
       "read counts");
    PK(cudaStreamSynchronize(s), "create");
    release(sym);
    if (oscratch) release(oscratch);
    if (hash_fail) return pack_fail(GEMPE_E_INVALID_GRAPH, "edge hash set build failed");
    for (int32_t g = 0; g < G; ++g) {
        if (sym_h[3 * g] == sym_h[3 * g + 1] && sym_h[3 * g + 2] == 0) continue;
        // not symmetric: the host check names the lowest row with a slot whose reverse is missing
        const gempe_status vs = validate_csr(gs[g].row_ptr, gs[g].col_idx, gs[g].n);
        std::string msg = vs != GEMPE_OK ? std::string(gempe_last_error()) : std::string("graph not symmetric");
        if (gs[g].label >= 0) msg = "graph " + std::to_string(gs[g].label) + ": " + msg;
        return pack_fail(GEMPE_E_INVALID_GRAPH, msg);
    }

    sampler_grid = gempe::sampler_grid(rows, k, sm_count);
    update_grid = G + std::min<int>(sm_count * 2, std::max(n_vchunks, 1));
    // with autotuning the shape is set by autotune(), which the owner calls next
    return p.autotune ? GEMPE_OK : set_shape(PackShape{});
}

int Pack::bytemap_log2_for(int64_t nnz, const gempe_params& p) {
    if (p.bytemap_log2 > 0) return p.bytemap_log2;
    int lg = 0;
    while ((1ll << lg) < std::max<int64_t>(nnz, 1)) ++lg;
    return std::min(30, std::max(12, lg + 7));
}

size_t Pack::bytes_for(int32_t n, int64_t nnz, int32_t d, const gempe_params& p) {
    auto al = [](size_t b) { return (b + 511) / 512 * 512; };   // allocation granularity
    const bool blk = p.block_partners > 0 && d >= 8;
    const size_t R = (size_t)n + 1, k = (size_t)p.neg_per_vertex, bins = (size_t)p.hist_bins;
    const size_t tiles = blk ? ((size_t)n + kBlockT - 1) / kBlockT : 0;
    const size_t units_max = (size_t)n + (size_t)nnz / 8 + 16;
    size_t b = 0;
    b += al(4 * (R + 1)) + al(4 * std::max<size_t>((size_t)nnz, 1)) + al((n <= kNarrowKeysMaxN ? 4 : 8) * table_slots(nnz));
    b += al(4 * R * d) + al(4 * R * acc_stride_for(d));
    if (p.precision == 1 && d >= 8) b += al(2 * R * d);
    b += al(bins * 20) + al(sizeof(GraphInfo)) + al(sizeof(GraphState)) + al(sizeof(PackState)) + al(4);
    b += al(16 * (((size_t)n + kVChunk - 1) / kVChunk)) + al(4 * R * std::max<size_t>(k, 1));
    const bool ps = p.sampling == 1;
    b += al(4 * std::max<size_t>(blk ? 1 : (ps ? 2 * (size_t)nnz : 2 * R * k), 1)) + al(16 * units_max) + al(4 * 4097);
    if (ps) b += al(8 * R);
    if (d <= kPackedMaxDim && !ps && !blk) b += al(4 * (R + 1)) + al(4 * std::max<size_t>((size_t)nnz, 1));
    if (p.membership == 1 && !blk) b += al((size_t)1 << bytemap_log2_for(nnz, p));
    if (blk) b += al(8 * tiles * kBlockP) + al(16 * R) + al(16 * (tiles + 1)) + al(8 * tiles);
    return b;
}

gempe_status Pack::set_shape(const PackShape& s) {
    PackShape sh = s;
    if (!sweep_lanes_supported(d, sh.lanes)) return pack_fail(GEMPE_E_INVALID_ARG, "unsupported lanes per pair");
    if (sh.kernel == 2 && !tiles)
        return pack_fail(GEMPE_E_INVALID_ARG, "kernel 2 (the sweep beside the tiles) needs block sampling with tiles");
    if (sh.kernel != 0 && sh.kernel != 2 && (sh.kernel != 1 || d > kPackedMaxDim))
        return pack_fail(GEMPE_E_INVALID_ARG, "kernel 1 (one lane per vertex) is for d <= 4");
    if (sh.unit_pairs != 64 && sh.unit_pairs != 128) return pack_fail(GEMPE_E_INVALID_ARG, "unit pairs: 64 or 128");
    if (sh.edge_chunk < 8 || sh.edge_chunk > 1024) return pack_fail(GEMPE_E_INVALID_ARG, "edge chunk in [8, 1024]");
    if (sh.blocks_per_sm < 0 || sh.blocks_per_sm > 8) return pack_fail(GEMPE_E_INVALID_ARG, "blocks per SM in [0, 8]");
    std::vector<int4> units;
    units.reserve((size_t)rows + (size_t)slots / 32 + 16);
    const bool per_unit = d > kPackedMaxDim || sh.kernel == 1;   // the kernel with lane groups per unit
    for (int32_t g = 0; g < G; ++g) {
        const GraphInfo& gi = info[g];
        const int32_t v0 = sharded() ? gi.v0 + own_lo : gi.v0, nv = sharded() ? own_hi - own_lo : gi.n;
        if (!per_unit)
            packed_units(orow_ptr_h.empty() ? row_ptr_h.data() : orow_ptr_h.data(), v0, nv, k, sh.unit_pairs, g,
                         per_slot, units);
        else chunk_units(row_ptr_h.data(), v0, nv, sh.edge_chunk, g, per_slot, units);
    }
    // kernel 2: one sweep block of kSweepThreadsBeside threads per SM (the
    // tile kernel takes the other half of every SM's registers)
    const int grid = sh.kernel == 2 ? sm_count : gempe::sweep_grid(d, sh.lanes, bins, sm_count, sh.blocks_per_sm, sh.kernel);
    std::vector<int32_t> bounds;
    if (per_unit) {
        const int lanes = sh.lanes ? sh.lanes : (d <= kPackedMaxDim ? 1 : d / 8);
        const int pg = 32 / lanes;
        const int k_slots = tiles ? 0 : slots_per_vertex();
        wide_tasks(units, pg, k_slots, per_slot);
        // per-block task ranges of equal estimated work: a task costs its
        // longest unit's rounds plus a fixed set-up
        const size_t n_tasks = units.size() / pg;
        std::vector<double> cum(n_tasks + 1, 0.0);
        for (size_t t = 0; t < n_tasks; ++t) {
            int rounds = 0;
            for (int g2 = 0; g2 < pg; ++g2) {
                const int4& u = units[t * pg + g2];
                if (u.x < 0) continue;
                const int pairs = unit_pairs_of(u, k_slots, per_slot);
                rounds = std::max(rounds, (pairs + lanes - 1) / lanes);
            }
            cum[t + 1] = cum[t] + rounds + 1.0;
        }
        bounds.assign(grid + 1, 0);
        size_t t = 0;
        for (int b = 1; b < grid; ++b) {
            const double target = cum[n_tasks] * b / grid;
            while (t < n_tasks && cum[t + 1] <= target) ++t;
            bounds[b] = (int32_t)t;
        }
        bounds[grid] = (int32_t)n_tasks;
    }
    if (items && (size_t)n_items < units.size()) {
        release(items);
        items = nullptr;
    }
    if (!items) {
        items = (int4*)alloc(sizeof(int4) * std::max<size_t>(units.size(), 1));
        if (!items) return pack_fail(GEMPE_E_OOM, "device allocation failed");
    }
    n_items = (int32_t)units.size();
    if (!units.empty())
        PK(cudaMemcpyAsync(items, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice, stream),
           "copy work units");
    if (!bounds.empty()) {
        if (task_bounds && task_bounds_cap < (int32_t)bounds.size()) {
            release(task_bounds);
            task_bounds = nullptr;
        }
        if (!task_bounds) {
            task_bounds = (int32_t*)alloc(sizeof(int32_t) * bounds.size());
            if (!task_bounds) return pack_fail(GEMPE_E_OOM, "device allocation failed");
            task_bounds_cap = (int32_t)bounds.size();
        }
        PK(cudaMemcpyAsync(task_bounds, bounds.data(), sizeof(int32_t) * bounds.size(), cudaMemcpyHostToDevice,
                           stream),
           "copy task ranges");
    }
    PK(cudaStreamSynchronize(stream), "copy work units");
    sweep_grid = grid;
    tile_grid = gempe::tile_grid(n_tile_items, sm_count,
                                 sh.kernel == 2 ? 1
                                 : (p.precision == 1 ? tile_bf16_blocks_per_sm(d, bins) : tile_f32_blocks_per_sm(d, bins)));
    shape = sh;
    return GEMPE_OK;
}

EpochArgs Pack::args() const {
    EpochArgs a{};
    a.graphs = graphs;
    a.gst = gst;
    a.ps = ps;
    a.n_graphs = G;
    a.row_ptr = row_ptr;
    a.col_idx = col_idx;
    a.orow_ptr = orow_ptr;
    a.ocol_idx = ocol_idx;
    a.oriented = (orow_ptr && shape.kernel == 0) ? 1 : 0;
    a.keys = keys;
    a.narrow_keys = narrow_keys ? 1 : 0;
    a.x = x;
    a.xb = xb;
    a.acc = acc;
    a.hist_e = hist_e;
    a.hist_c = hist_c;
    a.hist_d = hist_d;
    a.hist_x = hist_x;
    a.items = items;
    a.n_items = n_items;
    a.task_bounds = task_bounds;
    a.blocked = G > 1 ? 1 : 0;
    a.vchunks = vchunks;
    a.n_vchunks = n_vchunks;
    a.rows = rows;
    a.d = d;
    a.acc_stride = acc_stride;
    a.k = k;
    a.max_retries = p.max_retries;
    a.symmetric = p.symmetric_neg;
    a.w_formula = p.w_formula;
    a.clamp_neg_d = p.clamp_neg_d;
    a.bins = bins;
    a.mu = p.mu;
    a.hist_scale = (float)bins / p.hist_max;
    a.samples = samples;
    a.per_slot = per_slot ? 1 : 0;
    a.n_slots = (int32_t)slots;
    a.vacc = vacc;
    a.block_P = block ? kBlockP : 0;
    a.n_tiles = n_tiles;
    a.block_part = block_part;
    a.block_mask = block_mask;
    a.tile_items = tile_items;
    a.n_tile_items = n_tile_items;
    a.sweep_samples = tiles ? 0 : 1;
    a.sigma_every = p.sigma_every;
    a.sigma_source = p.sigma_source;
    a.sweep_hist = p.sigma_source == 0 ? 1 : 0;
    a.z_min = p.z_min;
    a.hist_max = p.hist_max;
    a.mills = mills;
    a.membership = bytemap ? 1 : 0;
    a.rename_every = p.rename_every;
    a.rng = p.rng;
    a.own_n = sharded() ? own_hi - own_lo : 0;
    a.bytemap = bytemap;
    return a;
}

namespace {
cudaError_t launch_epoch_sampler(const Pack& pk, cudaStream_t s) {
    if (pk.block) return launch_block_sampler(pk.args(), pk.sampler_units, pk.n_sampler_units, pk.sm_count, s);
    if (pk.bytemap && pk.p.rename_every > 0) {
        // a new renaming period: rebuild the maps that hold another one
        const cudaError_t e = launch_bytemap_build(pk.args(), 0, pk.sm_count, s);
        if (e != cudaSuccess) return e;
    }
    return launch_sampler(pk.args(), pk.sampler_grid, s);
}
}  // namespace

gempe_status Pack::prime() {
    if (primed || !sampled()) return GEMPE_OK;
    PK(launch_epoch_sampler(*this, stream), "sampler");
    primed = true;
    return GEMPE_OK;
}

// The sweep of the current epoch on the stream and, forked onto the side
// stream, the sampler of the next epoch (it only needs the graph).
gempe_status Pack::enqueue_sweep() {
    gempe_status s = prime();
    if (s != GEMPE_OK) return s;
    // the sweep is launched first (at high priority), the sampler after it
    // from the same point of the stream, so that the sweep's resident wave
    // takes the SMs and the sampler fills them as the sweep's blocks retire
    const bool fork = sampled() && !sampled_ahead;
    if (fork) PK(cudaEventRecord(fork_ev, stream), "fork");
    SweepShape ss;
    ss.grid = sweep_grid;
    ss.lanes = shape.lanes;
    ss.kernel = shape.kernel;
    // kernel 2: the tiles on tile_stream, beside the sweep (both only add into
    // the sums and bins, by atomics), joined before the update
    const bool beside = tiles && shape.kernel == 2;
    cudaStream_t ts = beside ? tile_stream : stream;
    if (beside) {
        PK(cudaEventRecord(tile_fork, stream), "fork");
        PK(cudaStreamWaitEvent(tile_stream, tile_fork, 0), "fork");
    }
    if (time_kernels) PK(cudaEventRecord(tev[0], stream), "timing event");
    PK(launch_sweep(args(), ss, stream), "sweep");
    if (time_kernels) PK(cudaEventRecord(tev[1], stream), "timing event");
    if (time_kernels) PK(cudaEventRecord(tev[2], ts), "timing event");
    if (tiles)
        PK(p.precision == 1 ? launch_tile_bf16(args(), tile_grid, ts) : launch_tile_f32(args(), tile_grid, ts),
           "tiles");
    if (time_kernels) PK(cudaEventRecord(tev[3], ts), "timing event");
    if (beside) {
        PK(cudaEventRecord(tile_join, tile_stream), "join");
        PK(cudaStreamWaitEvent(stream, tile_join, 0), "join");
    }
    if (time_kernels) PK(cudaEventRecord(tev[4], stream), "timing event");
    if (fork) {
        PK(cudaStreamWaitEvent(side, fork_ev, 0), "fork");
        PK(launch_epoch_sampler(*this, side), "sampler");
        PK(cudaEventRecord(join_ev, side), "join");
        sampled_ahead = true;
    }
    return GEMPE_OK;
}

// The position update and slope fits, then the join with the side stream.
gempe_status Pack::enqueue_update() {
    PK(launch_update(args(), update_grid, stream), "update");
    if (sharded()) {
        // the update clears the sums of the shard's own rows; the rows of the
        // other shards' vertices held this shard's partner terms (and, after
        // the exchange, everyone's) and start the next epoch at zero too
        const size_t row = sizeof(float) * (size_t)acc_stride;
        if (own_lo > 0) PK(cudaMemsetAsync(acc, 0, row * own_lo, stream), "clear sums");
        if (own_hi < rows) PK(cudaMemsetAsync(acc + (size_t)own_hi * acc_stride, 0, row * (rows - own_hi), stream), "clear sums");
    }
    if (time_kernels) PK(cudaEventRecord(tev[5], stream), "timing event");
    if (p.sigma_source == 1 && p.sigma_every > 0) {
        PK(launch_hist_pass(args(), stream), "histogram pass");
        PK(launch_fit_graphs(args(), stream), "slope fit");
    }
    if (sampled_ahead) {
        PK(cudaStreamWaitEvent(stream, join_ev, 0), "join");
        sampled_ahead = false;
    }
    return GEMPE_OK;
}

gempe_status Pack::read_status() {
    int32_t status = 0;
    PK(cudaMemcpyAsync(&status, &ps->status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream), "status");
    PK(cudaStreamSynchronize(stream), "synchronize");
    if (status != 0) {
        int32_t zero = 0;
        cudaMemcpyAsync(&ps->status, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, stream);
        cudaStreamSynchronize(stream);
        return pack_fail((gempe_status)status,
                         status == GEMPE_E_TIMEOUT
                             ? "a tensor-core tile gave up waiting for its MMAs (bounded wait); the epoch is incomplete"
                             : "a position became non-finite during an update; it kept its old value");
    }
    return GEMPE_OK;
}

// ---------------------------------------------------------------------------
// Autotuner.  The candidates are the launch shapes the kernels support: for
// d <= 4 the pair budget of a packed unit and the CTAs per SM; for d >= 8
// the CSR slots per unit and the lanes per pair.  Each candidate's sweep is
// timed (CUDA events, best of 3 after one warm-up) on the pack's own graphs
// and current positions; the sums it leaves are cleared, the block masks it
// consumes restored, and the graph statistics put back, so that the epoch
// state is the same before and after.  The choice is cached per process by
// (d, precision, sampling form, k, log2 rows, log2 slots, graphs > 1).
// ---------------------------------------------------------------------------
namespace {
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, PackShape> g_tune_cache;

int ilog2(long long v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}
}  // namespace

gempe_status Pack::autotune() {
    const TuneKey key{d, p.precision, block ? 1 : (per_slot ? 2 : 0), k, ilog2(rows), ilog2(std::max<int64_t>(slots, 1)), G > 1};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return set_shape(it->second);
    }
    std::vector<PackShape> cands;
    if (d <= kPackedMaxDim) {
        for (int budget : {64, 128})
            for (int bps : {0, 2}) {
                PackShape s;
                s.unit_pairs = budget;
                s.blocks_per_sm = bps;
                cands.push_back(s);
            }
        for (int chunk : {16, 32, 64}) {   // one lane per vertex
            PackShape s;
            s.kernel = 1;
            s.edge_chunk = chunk;
            cands.push_back(s);
        }
    } else {
        for (int lanes : {d / 8, d / 4})
            for (int chunk : {32, 64, 128}) {
                if (!sweep_lanes_supported(d, lanes)) continue;
                PackShape s;
                s.lanes = lanes;
                s.edge_chunk = chunk;
                cands.push_back(s);
            }
    }
    gempe_status rc = prime();
    if (rc != GEMPE_OK) return rc;
    std::vector<GraphState> saved(G);
    PK(cudaMemcpyAsync(saved.data(), gst, sizeof(GraphState) * G, cudaMemcpyDeviceToHost, stream), "save state");
    // the sweep of the block form consumes the masks of the current epoch
    unsigned long long* mask_copy = nullptr;
    const size_t mask_bytes = sizeof(unsigned long long) * 2 * (size_t)rows;
    const bool sweep_takes_masks = block && !tiles;
    if (sweep_takes_masks) {
        mask_copy = (unsigned long long*)alloc(mask_bytes);
        if (!mask_copy) return pack_fail(GEMPE_E_OOM, "device allocation failed");
        PK(cudaMemcpyAsync(mask_copy, block_mask, mask_bytes, cudaMemcpyDeviceToDevice, stream), "save masks");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PK(cudaEventCreate(&e0), "cudaEventCreate");
    PK(cudaEventCreate(&e1), "cudaEventCreate");
    PackShape best;
    float best_ms = 1e30f;
    cudaError_t err = cudaSuccess;
    for (const PackShape& c : cands) {
        rc = set_shape(c);
        if (rc != GEMPE_OK) break;
        float t_min = 1e30f;
        for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
            if (sweep_takes_masks)
                err = cudaMemcpyAsync(block_mask, mask_copy, mask_bytes, cudaMemcpyDeviceToDevice, stream);
            SweepShape ss;
            ss.grid = sweep_grid;
            ss.lanes = shape.lanes;
            ss.kernel = shape.kernel;
            if (err == cudaSuccess) err = cudaEventRecord(e0, stream);
            if (err == cudaSuccess) err = launch_sweep(args(), ss, stream);
            if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
            if (err == cudaSuccess) err = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)rows * acc_stride, stream);
            if (err == cudaSuccess) err = cudaMemsetAsync(hist, 0, hist_bytes, stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t_min = std::min(t_min, ms);
        }
        if (err != cudaSuccess) break;
        if (t_min < best_ms) {
            best_ms = t_min;
            best = shape;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (sweep_takes_masks && err == cudaSuccess)
        err = cudaMemcpyAsync(block_mask, mask_copy, mask_bytes, cudaMemcpyDeviceToDevice, stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(gst, saved.data(), sizeof(GraphState) * G, cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
    if (mask_copy) release(mask_copy);
    if (err != cudaSuccess) return pack_cuda_fail(err, "autotune");
    if (rc != GEMPE_OK) return rc;
    best.sweep_us = best_ms * 1000.0f;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return set_shape(best);
}

}  // namespace gempe
