// Graph set-up on the device, once per context: the symmetry check of the
// CSR against the graph's edge set, and the degree-oriented CSR of the
// packed sweep (every undirected edge once, in the row of its endpoint with
// the larger (degree, id)).
//
//  k_check_symmetric  one thread per CSR slot: counts the slots above and
//                     below the diagonal and the slots below whose reverse
//                     is not in the edge set (which holds the slots above)
//  k_orient_count     one warp per row: the row's kept slots
//  k_scan_*           exclusive scan of the counts into row offsets
//  k_orient_fill      one warp per row: the kept slots in row order
//  k_add_offset       a graph's column indices shifted to pack rows
#include <cuda_runtime.h>

#include "device_math.cuh"
#include "engine.cuh"

namespace gempe {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

// Local row of CSR slot e of a graph whose offsets are rp[0..n]: the last i
// with rp[i] <= e.
__device__ __forceinline__ int row_of_slot(const int32_t* rp, int n, int64_t e) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(rp + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// counts: {slots above the diagonal, slots below, slots below without their
// reverse in the edge set}.  Rows must be sorted and in range (checked on the
// host); then the graph is symmetric iff above == below and none is missing.
__global__ void k_check_symmetric(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                  int32_t v0, int32_t n, const void* keys, int narrow, unsigned long long key_off,
                                  unsigned long long bucket_mask, unsigned long long* counts) {
    const int32_t* rp = row_ptr + v0;
    const int64_t e0 = __ldg(rp), e1 = __ldg(rp + n);
    unsigned long long above = 0, below = 0, missing = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every lane of a warp runs the same number of iterations (warp sums below)
    const int64_t span = e1 - e0;
    const int64_t iters = span > 0 ? (span + stride - 1) / stride : 0;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t e = start + it * stride;
        if (e < e1) {
            const int i = row_of_slot(rp, n, e);
            const int j = __ldg(col_idx + e) - v0;
            if (j > i) {
                ++above;
            } else if (j < i) {
                ++below;
                if (!edge_set_contains(keys, narrow, key_off, bucket_mask, j, i)) ++missing;
            }
        }
    }
    above = warp_sum(above);
    below = warp_sum(below);
    missing = warp_sum(missing);
    if ((threadIdx.x & 31) == 0) {
        if (above) atomicAdd(counts, above);
        if (below) atomicAdd(counts + 1, below);
        if (missing) atomicAdd(counts + 2, missing);
    }
}

// Slot (r, j) of pack row r is kept in the oriented CSR when
// (deg j, j) < (deg r, r).
__device__ __forceinline__ bool keep_slot(const int32_t* row_ptr, int r, int dr, int j) {
    const int dj = __ldg(row_ptr + j + 1) - __ldg(row_ptr + j);
    return dj < dr || (dj == dr && j < r);
}

__global__ void k_orient_count(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int rows,
                               int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    for (int r = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); r < rows; r += warps) {
        const int e0 = __ldg(row_ptr + r), e1 = __ldg(row_ptr + r + 1), dr = e1 - e0;
        int c = 0;
        for (int b = e0; b < e1; b += 32) {
            const int e = b + lane;
            const bool kept = e < e1 && keep_slot(row_ptr, r, dr, __ldg(col_idx + e));
            c += __popc(__ballot_sync(kFull, kept));
        }
        if (lane == 0) count[r] = c;
    }
}

__global__ void k_orient_fill(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int rows,
                              const int32_t* __restrict__ orow_ptr, int32_t* __restrict__ ocol_idx) {
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    for (int r = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); r < rows; r += warps) {
        const int e0 = __ldg(row_ptr + r), e1 = __ldg(row_ptr + r + 1), dr = e1 - e0;
        int o = __ldg(orow_ptr + r);
        for (int b = e0; b < e1; b += 32) {
            const int e = b + lane;
            const int j = e < e1 ? __ldg(col_idx + e) : 0;
            const bool kept = e < e1 && keep_slot(row_ptr, r, dr, j);
            const unsigned m = __ballot_sync(kFull, kept);
            if (kept) ocol_idx[o + __popc(m & ((1u << lane) - 1u))] = j;
            o += __popc(m);
        }
    }
}

// Exclusive scan, three passes: tiles of kScanTile values (block sums), the
// block sums (one block, in tiles), then the offsets added; out has count + 1
// entries, out[count] = the total.
__device__ __forceinline__ int block_exclusive(int v, int* s_warp, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, xi, o);
            if (lane >= o) xi += t;
        }
        s_warp[lane] = xi - x;   // exclusive warp offsets
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    const int res = s_warp[w] + incl - v;
    total = s_warp[32];
    __syncthreads();   // s_warp is reused by the next call
    return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                             int count, int32_t* __restrict__ tile_sums) {
    __shared__ int s_warp[33];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
    int v[kScanPerThread], sum = 0;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        v[q] = base + q < count ? __ldg(in + base + q) : 0;
        sum += v[q];
    }
    int total;
    int run = block_exclusive(sum, s_warp, total);
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        if (base + q < count) out[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t* __restrict__ tile_sums, int tiles) {
    __shared__ int s_warp[33];
    int carry = 0;
    for (int t0 = 0; t0 < tiles; t0 += kScanThreads) {
        const int t = t0 + threadIdx.x;
        const int v = t < tiles ? tile_sums[t] : 0;
        int total;
        const int ex = block_exclusive(v, s_warp, total);
        if (t < tiles) tile_sums[t] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tile_sums[tiles] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t* __restrict__ out, int count,
                                                           const int32_t* __restrict__ tile_sums, int tiles) {
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
    const int off = tile_sums[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q)
        if (base + q < count) out[base + q] += off;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[count] = tile_sums[tiles];
}

__global__ void k_add_offset(int32_t* __restrict__ v, int64_t count, int32_t off) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
        v[q] += off;
}

int grid_for(long long items, int per_block, int cap) {
    long long g = (items + per_block - 1) / per_block;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_check_symmetric(const int32_t* row_ptr, const int32_t* col_idx, int32_t v0, int32_t n, int64_t nnz,
                                   const void* keys, int narrow, unsigned long long key_off,
                                   unsigned long long bucket_mask, unsigned long long* counts3, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    k_check_symmetric<<<grid_for(nnz, 256, 65535), 256, 0, s>>>(row_ptr, col_idx, v0, n, keys, narrow, key_off,
                                                                 bucket_mask, counts3);
    return cudaGetLastError();
}

cudaError_t launch_add_offset(int32_t* v, int64_t count, int32_t off, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_add_offset<<<grid_for(count, 256, 4096), 256, 0, s>>>(v, count, off);
    return cudaGetLastError();
}

size_t orient_scratch_ints(int rows) { return (size_t)rows + (size_t)(rows / kScanTile + 2); }

cudaError_t launch_orient(const int32_t* row_ptr, const int32_t* col_idx, int rows, int32_t* orow_ptr,
                          int32_t* ocol_idx, int32_t* scratch, int sm_count, cudaStream_t s) {
    int32_t* count = scratch;
    int32_t* tile_sums = scratch + rows;
    const int warp_grid = grid_for((long long)rows, 8, sm_count * 16);
    k_orient_count<<<warp_grid, 256, 0, s>>>(row_ptr, col_idx, rows, count);
    const int tiles = (rows + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<tiles < 1 ? 1 : tiles, kScanThreads, 0, s>>>(count, orow_ptr, rows, tile_sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tile_sums, tiles < 1 ? 1 : tiles);
    k_scan_add<<<tiles < 1 ? 1 : tiles, kScanThreads, 0, s>>>(orow_ptr, rows, tile_sums, tiles < 1 ? 1 : tiles);
    k_orient_fill<<<warp_grid, 256, 0, s>>>(row_ptr, col_idx, rows, orow_ptr, ocol_idx);
    return cudaGetLastError();
}

}  // namespace gempe
