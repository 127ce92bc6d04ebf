// Wang-Bovik Q of one 32 x 32 window from exact integer sums, shared by the
// metric passes (metrics.cu) and the fused forward + metrics kernel
// (fuse_metrics.cu).  The quality index (Sec. 4 / Table 3 report QNR without
// defining it):  Q = 4 s_xy mu_x mu_y / ((s_x^2 + s_y^2)(mu_x^2 + mu_y^2)).
#pragma once

#include <cstdint>

namespace dwtfuse {

constexpr int kQWinPx = 32 * 32;  // pixels per window

// Position of band pair (b, c), b < c < nb, among the pair sums (b-major
// order); the band-PAN pairs follow at nb(nb-1)/2 + b.  Loops over pairs run
// b and c over [0, nb) with a `c > b` test, so that both have constant trip
// counts, unroll fully, and the position is a compile-time constant (a
// triangular inner loop stays a loop and its sums go to local memory).
__host__ __device__ constexpr int pair_index(int nb, int b, int c) { return b * nb - b * (b + 1) / 2 + (c - b - 1); }

// Q of one window, given exact integer sums (8-bit data).  ys = scale of y.
__device__ __forceinline__ float q_exact(long long sx, long long sxx, long long sy, long long syy,
                                         long long sxy, int ys) {
    const long long n = kQWinPx;
    const long long vx = n * sxx - sx * sx;                 // n^2 var(x)
    const long long vy = n * syy - sy * sy;                 // ys^2 n^2 var(y)
    const long long cxy = n * sxy - sx * sy;                // ys n^2 cov(x, y)
    const long long ax = sx + 128 * n;                      // n mean(X)
    const long long ay = sy + 128 * n * ys;                 // ys n mean(Y)
    const float inv = 1.0f / (float)ys, inv2 = inv * inv;
    const float fvx = (float)vx, fvy = (float)vy * inv2, fc = (float)cxy * inv;
    const float fax = (float)ax, fay = (float)ay * inv;
    const float den = (fvx + fvy) * (fax * fax + fay * fay);
    if (vx + vy == 0 || (ax == 0 && ay == 0)) {
        // zero denominator: identical windows <=> sum (ys x - y)^2 = 0
        const long long d2 = (long long)ys * ys * sxx - 2LL * ys * sxy + syy;
        return (d2 == 0) ? 1.0f : 0.0f;
    }
    return 4.0f * fc * fax * fay / den;
}

}  // namespace dwtfuse
