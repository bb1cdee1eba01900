// Exact predictive entropy (Eq. 2) over all n(n-1)/2 pairs, and its
// derivative in the slope, for mid-size graphs.
//
// With N = n(n-1)/2 and every pair first counted as a non-edge,
//   N PE(sigma) = sum_{i<j} dl-(delta_ij) + sum_{(i,j) in E, i<j} [dl+ - dl-](delta_ij),
// so the all-pairs part needs no membership test and the edge part is a
// pass over the CSR.  Both passes also sum, with u = (delta - mu)/sigma,
// g(u) = h(-u) and t = ln sigma,
//   F  = sum over non-edges of u g(u) + over edges of -u h(u)   (sign of dPE/dsigma),
//   F' = dF/dt,
// for the Newton search of the slope that minimises Eq. 2 (mu fixed).
// Per-pair values in FP32, sums in FP64.
//
//  k_exact_pairs  64 x 64 tiles of pairs (i < j), rows staged in shared memory
//  k_exact_edges  one thread per CSR slot with j > i
#include <cuda_runtime.h>

#include "device_math.cuh"
#include "engine.cuh"

namespace gempe {

namespace {

constexpr int kExactTile = 64;
constexpr int kExactThreads = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct PairSums {
    float s, f, fp;
};

// Non-edge (edge = false) or edge terms of one pair at u.
__device__ __forceinline__ void pair_sums(float u, bool edge, const MillsCoef* tab, PairSums& acc) {
    if (edge) {
        float h, T;
        mills(u, h, T, tab);
        const float uh = u * h;
        acc.s += neg_log2_Q(u);
        acc.f -= uh;
        acc.fp += uh * fmaf(u, T, 1.0f);
    } else {
        float g, Tn;
        mills(-u, g, Tn, tab);
        const float ug = u * g;
        acc.s += neg_log2_Q(-u);
        acc.f += ug;
        acc.fp -= ug * fmaf(-u, Tn, 1.0f);
    }
}

__device__ __forceinline__ void block_add3(double a, double b, double c, double* out) {
    __shared__ double s_part[3][kExactThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
        c += __shfl_xor_sync(kFull, c, o);
    }
    if (lane == 0) {
        s_part[0][w] = a;
        s_part[1][w] = b;
        s_part[2][w] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_part[threadIdx.x][q];
        if (t != 0.0) atomicAdd(out + threadIdx.x, t);
    }
}

// Tile pair index -> (I, J), I <= J, in row-major order of the upper triangle
// of a T x T tile grid.
__device__ __forceinline__ void tile_pair(long long idx, int T, int& I, int& J) {
    const double b = 2.0 * T + 1.0;
    int i = (int)floor((b - sqrt(b * b - 8.0 * (double)idx)) * 0.5);
    if (i < 0) i = 0;
    auto start = [&](int r) { return (long long)r * T - (long long)r * (r - 1) / 2; };
    while (i > 0 && start(i) > idx) --i;
    while (i + 1 < T && start(i + 1) <= idx) ++i;
    I = i;
    J = i + (int)(idx - start(i));
}

// D: the dimension; rows of both tiles in shared memory with stride D + 1.
template <int D>
__global__ void __launch_bounds__(kExactThreads) k_exact_pairs(const float* __restrict__ x, int n, float mu,
                                                               float inv_sigma, const MillsCoef* tab, double* out) {
    constexpr int XS = D + 1;
    extern __shared__ float s_x[];   // [2][kExactTile][XS]
    float* xi_s = s_x;
    float* xj_s = s_x + kExactTile * XS;
    const int T = (n + kExactTile - 1) / kExactTile;
    const long long n_pairs = (long long)T * (T + 1) / 2;
    const int r = threadIdx.x >> 2;          // row within tile I
    const int c0 = threadIdx.x & 3;          // columns c0, c0 + 4, ... within tile J
    double ds = 0.0, df = 0.0, dfp = 0.0;
    for (long long idx = blockIdx.x; idx < n_pairs; idx += gridDim.x) {
        int I, J;
        tile_pair(idx, T, I, J);
        __syncthreads();   // the previous tiles are no longer read
        for (int q = threadIdx.x; q < kExactTile * D; q += blockDim.x) {
            const int rr = q / D, cc = q - rr * D;
            const int gi = I * kExactTile + rr, gj = J * kExactTile + rr;
            xi_s[rr * XS + cc] = gi < n ? __ldg(x + (size_t)gi * D + cc) : 0.0f;
            xj_s[rr * XS + cc] = gj < n ? __ldg(x + (size_t)gj * D + cc) : 0.0f;
        }
        __syncthreads();
        const int gi = I * kExactTile + r;
        PairSums acc{0.0f, 0.0f, 0.0f};
        if (gi < n) {
#pragma unroll 4
            for (int q = 0; q < kExactTile / 4; ++q) {
                const int c = c0 + 4 * q;
                const int gj = J * kExactTile + c;
                if (gj >= n || (I == J && c <= r)) continue;
                float ss = 0.0f;
#pragma unroll 8
                for (int k = 0; k < D; ++k) {
                    const float df2 = xi_s[r * XS + k] - xj_s[c * XS + k];
                    ss = fmaf(df2, df2, ss);
                }
                const float u = (sqrtf(ss) - mu) * inv_sigma;
                pair_sums(u, false, tab, acc);
            }
        }
        ds += (double)acc.s;
        df += (double)acc.f;
        dfp += (double)acc.fp;
    }
    block_add3(ds, df, dfp, out);
}

// The edge correction: for each CSR slot (i, j) with j > i, the edge terms
// minus the non-edge terms the all-pairs pass counted for the pair.
__global__ void __launch_bounds__(kExactThreads) k_exact_edges(const int32_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ col_idx,
                                                               const float* __restrict__ x, int n, int d, float mu,
                                                               float inv_sigma, const MillsCoef* tab, double* out) {
    const int64_t nnz = __ldg(row_ptr + n);
    double ds = 0.0, df = 0.0, dfp = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;   // row of slot e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(row_ptr + mid) <= e) lo = mid; else hi = mid - 1;
        }
        const int i = lo, j = __ldg(col_idx + e);
        if (j <= i) continue;
        float ss = 0.0f;
        for (int k = 0; k < d; ++k) {
            const float df2 = __ldg(x + (size_t)i * d + k) - __ldg(x + (size_t)j * d + k);
            ss = fmaf(df2, df2, ss);
        }
        const float u = (sqrtf(ss) - mu) * inv_sigma;
        PairSums pe{0.0f, 0.0f, 0.0f}, pn{0.0f, 0.0f, 0.0f};
        pair_sums(u, true, tab, pe);
        pair_sums(u, false, tab, pn);
        ds += (double)pe.s - (double)pn.s;
        df += (double)pe.f - (double)pn.f;
        dfp += (double)pe.fp - (double)pn.fp;
    }
    block_add3(ds, df, dfp, out);
}

template <int D>
cudaError_t exact_pairs_for(const float* x, int n, float mu, float inv_sigma, const MillsCoef* tab, double* out,
                            int sm_count, cudaStream_t s) {
    const size_t smem = 2 * (size_t)kExactTile * (D + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_exact_pairs<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_exact_pairs<D>, kExactThreads, smem);
    if (e != cudaSuccess) return e;
    const long long T = (n + kExactTile - 1) / kExactTile;
    long long grid = T * (T + 1) / 2;
    const long long cap = (long long)sm_count * (per_sm > 0 ? per_sm : 1);
    if (grid > cap) grid = cap;
    k_exact_pairs<D><<<(int)grid, kExactThreads, smem, s>>>(x, n, mu, inv_sigma, tab, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_exact_pe(const int32_t* row_ptr, const int32_t* col_idx, const float* x, int n, int d, float mu,
                            float sigma, const MillsCoef* tab, double* out3, int sm_count, cudaStream_t s) {
    const float inv_sigma = 1.0f / sigma;
    cudaError_t e = cudaMemsetAsync(out3, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    switch (d) {
#define GEMPE_CASE(D)                                                              \
    case D: e = exact_pairs_for<D>(x, n, mu, inv_sigma, tab, out3, sm_count, s); \
        break;
        GEMPE_CASE(1) GEMPE_CASE(2) GEMPE_CASE(3) GEMPE_CASE(4) GEMPE_CASE(8) GEMPE_CASE(16) GEMPE_CASE(32)
        GEMPE_CASE(64) GEMPE_CASE(128) GEMPE_CASE(256)
#undef GEMPE_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    int grid = sm_count * 4;
    k_exact_edges<<<grid, kExactThreads, 0, s>>>(row_ptr, col_idx, x, n, d, mu, inv_sigma, tab, out3);
    return cudaGetLastError();
}

}  // namespace gempe
