// Host construction of the Mills-ratio interpolation table used by the pair
// term and the slope fit.
//
// h(v) = phi(v) / Q(v) (Q the upper normal tail) and T(v) = h(v) - v are
// evaluated in double precision from erfc at the interval ends; each interval
// of width 1/kMillsStepsPerUnit gets the cubic Hermite interpolant of log2 h
// with the slopes (log2 h)' = T / ln2 (from h' = h (h - v)).  On [-14, 8)
// the interpolant is within 5e-10 of h relative and its slope within 4e-8 of
// T relative (in exact arithmetic), far below FP32 rounding; the device reads
// T from that slope.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "device_math.cuh"
#include "engine.cuh"

namespace gempe {

namespace {

void h_and_T(double v, double& h, double& T) {
    const double phi = std::exp(-0.5 * v * v) / std::sqrt(2.0 * M_PI);
    const double Q = 0.5 * std::erfc(v / std::sqrt(2.0));
    h = phi / Q;
    T = h - v;
}

std::vector<MillsCoef> build_table() {
    const double ln2 = std::log(2.0);
    const double s = 1.0 / kMillsStepsPerUnit;
    std::vector<MillsCoef> tab(kMillsIntervals);
    auto cubic = [&](double fa, double fb, double da, double db) {
        return make_float4((float)fa, (float)(s * da), (float)(3.0 * (fb - fa) - s * (2.0 * da + db)),
                           (float)(2.0 * (fa - fb) + s * (da + db)));
    };
    for (int i = 0; i < kMillsIntervals; ++i) {
        const double va = (double)kMillsV0 + i * s, vb = va + s;
        double ha, Ta, hb, Tb;
        h_and_T(va, ha, Ta);
        h_and_T(vb, hb, Tb);
        tab[i].lh = cubic(std::log2(ha), std::log2(hb), Ta / ln2, Tb / ln2);
    }
    return tab;
}

}  // namespace

cudaError_t ensure_mills_table() {
    static std::mutex mu;
    static std::vector<MillsCoef> table;
    static std::vector<bool> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (table.empty()) table = build_table();
    if ((int)done.size() <= dev) done.resize(dev + 1, false);
    if (done[dev]) return cudaSuccess;
    e = upload_mills_table(table.data(), sizeof(MillsCoef) * table.size());
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

}  // namespace gempe
