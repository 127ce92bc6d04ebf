// Adjoint of the fused forward (vector-Jacobian product for autograd).
//
// Forward, per band:  F_b = P + U(gain * M_b - LL(P))   (see fuse_tile.cuh),
// with LL(X) = L_H X L_W^T and U(C) = sigma^2 L_H^T C L_W, where S = sigma A^T
// is the synthesis of the paper's inverse transform (Eq. 11-16): sigma = 2 for
// the /2 Haar of Eq. 1-2 (its inverse is 2 A^T, not A^T) and 1 for D4.
// Transposing:
//     grad_M_b = gain * sigma^2 * LL(G_b)
//     grad_P   = sum_b (G_b - U(LL(G_b))) = G - U(LL(G)),   G = sum_b G_b.
// Haar: grad_M_b = 2x2 block sum of G_b; grad_P = G - repeat2x2(blockmean(G)).
// D4:   grad_M_b = 2 LL(G_b); grad_P = G - U(LL(G)) with the D4 U of the forward.
//
// Same warp-strip decomposition as the forward.  Bands are a run-time loop:
// the per-band state of a row is consumed before the next band is loaded, so
// any band count runs in one launch.  D4 reads the four PAN-resolution rows
// of each band's low-pass window directly (rows 2m+2, 2m+3 are read again by
// row m+1 from L1/L2, never again from HBM in steady state).
#include "fuse_tile.cuh"
#include "launch.h"

namespace dwtfuse {

constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;

struct BwdArgs {
    const float *g;               // [bands][H][W]
    float *gpan;                  // H x W
    float *gms[kMaxBands];        // (H/2) x (W/2) each
    int64_t H, W;
    int32_t bands;
    float kappa;                  // gain * sigma^2
    int32_t a4;                   // 4-pixel vector path for g / gpan
    int32_t ms2;                  // W/2 even and every gms 8-byte aligned: pair stores
};

__device__ __forceinline__ void store_gms(float *row, const LaneCols &c, bool pair, float a, float b) {
    if (pair) {
        *reinterpret_cast<float2 *>(row + c.nB) = make_float2(a, b);
    } else {
        row[c.nB] = a;
        if (c.two) row[c.nC] = b;
    }
}

__device__ __forceinline__ void store_gpan(float *p, bool a4, bool two, const float *v) {
    if (a4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        if (two) *reinterpret_cast<float2 *>(p + 2) = make_float2(v[2], v[3]);
    }
}

__device__ __forceinline__ void haar_bwd_item(const BwdArgs &s, int64_t x0, int64_t m_s, int64_t m_e,
                                              int lane) {
    const int64_t W = s.W, H = s.H, W2 = W >> 1, HW = H * W;
    const LaneCols c = lane_cols(x0, lane, W);
    const bool a4 = s.a4 != 0, pair = s.ms2 != 0;
    for (int64_t m = m_s; m < m_e; ++m) {
        float g0[4] = {0.f, 0.f, 0.f, 0.f}, g1[4] = {0.f, 0.f, 0.f, 0.f};
        for (int b = 0; b < s.bands; ++b) {
            const float *gb = s.g + (int64_t)b * HW;
            float p0[4], p1[4];
            load_row4(gb + (2 * m) * W, c, a4, p0);
            load_row4(gb + (2 * m + 1) * W, c, a4, p1);
            if (c.active) {
                const float sA = (p0[0] + p0[1]) + (p1[0] + p1[1]);
                const float sB = (p0[2] + p0[3]) + (p1[2] + p1[3]);
                store_gms(s.gms[b] + m * W2, c, pair, s.kappa * 0.25f * sA, s.kappa * 0.25f * sB);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                g0[q] += p0[q];
                g1[q] += p1[q];
            }
        }
        if (!c.active) continue;
        const float mA = ((g0[0] + g0[1]) + (g1[0] + g1[1])) * 0.25f;
        const float mB = ((g0[2] + g0[3]) + (g1[2] + g1[3])) * 0.25f;
        const float v0[4] = {g0[0] - mA, g0[1] - mA, g0[2] - mB, g0[3] - mB};
        const float v1[4] = {g1[0] - mA, g1[1] - mA, g1[2] - mB, g1[3] - mB};
        store_gpan(s.gpan + (2 * m) * W + c.x, a4, c.two, v0);
        store_gpan(s.gpan + (2 * m + 1) * W + c.x, a4, c.two, v1);
    }
}

// D4 low-pass LL(X)(m, n-1..n+1) of one band, and that band's own pixels of
// rows 2m and 2m+1 (columns x..x+3).
__device__ __forceinline__ void d4_ll_window(const float *gb, int64_t m, int64_t H, int64_t W,
                                             const LaneCols &c, bool a4, float *ll, float *own0,
                                             float *own1) {
    constexpr float kh[4] = {kH0, kH1, kH2, kH3};
    ll[0] = ll[1] = ll[2] = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float v[8], r[3];
        load_row8(gb + wrap(2 * m + a, H) * W, c, a4, v);
        d4_rowpass(v, r);
#pragma unroll
        for (int k = 0; k < 3; ++k) ll[k] = fmaf(kh[a], r[k], ll[k]);
        if (a == 0) { own0[0] = v[2]; own0[1] = v[3]; own0[2] = v[4]; own0[3] = v[5]; }
        if (a == 1) { own1[0] = v[2]; own1[1] = v[3]; own1[2] = v[4]; own1[3] = v[5]; }
    }
}

__device__ __forceinline__ void d4_bwd_item(const BwdArgs &s, int64_t x0, int64_t m_s, int64_t m_e,
                                            int lane) {
    const int64_t W = s.W, H = s.H, W2 = W >> 1, H2 = H >> 1, HW = H * W;
    const LaneCols c = lane_cols(x0, lane, W);
    const bool a4 = s.a4 != 0, pair = s.ms2 != 0;
    // Row synthesis of LL(G) for MS row m-1 (vertical pipeline of U).
    float hprev[4];
    {
        const int64_t mp = wrap(m_s - 1, H2);
        float llg[3] = {0.f, 0.f, 0.f};
        for (int b = 0; b < s.bands; ++b) {
            float ll[3], o0[4], o1[4];
            d4_ll_window(s.g + (int64_t)b * HW, mp, H, W, c, a4, ll, o0, o1);
#pragma unroll
            for (int k = 0; k < 3; ++k) llg[k] += ll[k];
        }
        hprev[0] = fmaf(kH2, llg[0], kH0 * llg[1]);
        hprev[1] = fmaf(kH3, llg[0], kH1 * llg[1]);
        hprev[2] = fmaf(kH2, llg[1], kH0 * llg[2]);
        hprev[3] = fmaf(kH3, llg[1], kH1 * llg[2]);
    }
    for (int64_t m = m_s; m < m_e; ++m) {
        float llg[3] = {0.f, 0.f, 0.f};
        float g0[4] = {0.f, 0.f, 0.f, 0.f}, g1[4] = {0.f, 0.f, 0.f, 0.f};
        for (int b = 0; b < s.bands; ++b) {
            float ll[3], o0[4], o1[4];
            d4_ll_window(s.g + (int64_t)b * HW, m, H, W, c, a4, ll, o0, o1);
            if (c.active) store_gms(s.gms[b] + m * W2, c, pair, s.kappa * ll[1], s.kappa * ll[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) llg[k] += ll[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                g0[q] += o0[q];
                g1[q] += o1[q];
            }
        }
        float hc[4];
        hc[0] = fmaf(kH2, llg[0], kH0 * llg[1]);
        hc[1] = fmaf(kH3, llg[0], kH1 * llg[1]);
        hc[2] = fmaf(kH2, llg[1], kH0 * llg[2]);
        hc[3] = fmaf(kH3, llg[1], kH1 * llg[2]);
        float v0[4], v1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v0[q] = g0[q] - fmaf(kH2, hprev[q], kH0 * hc[q]);
            v1[q] = g1[q] - fmaf(kH3, hprev[q], kH1 * hc[q]);
            hprev[q] = hc[q];
        }
        if (c.active) {
            store_gpan(s.gpan + (2 * m) * W + c.x, a4, c.two, v0);
            store_gpan(s.gpan + (2 * m + 1) * W + c.x, a4, c.two, v1);
        }
    }
}

template <int WAV>
__global__ void __launch_bounds__(kBwdThreads)
fuse_bwd_kernel(const __grid_constant__ BwdArgs s, int64_t strips_x, int64_t items, int R) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kBwdWarps;
    for (int64_t it = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5); it < items; it += nwarps) {
        const int64_t sx = it % strips_x, sy = it / strips_x;
        const int64_t m_s = sy * R;
        const int64_t m_e = min(m_s + (int64_t)R, s.H >> 1);
        if (WAV == 0)
            haar_bwd_item(s, sx * kWarpCols, m_s, m_e, lane);
        else
            d4_bwd_item(s, sx * kWarpCols, m_s, m_e, lane);
    }
}

cudaError_t launch_fuse_backward(const float *g, int bands, int64_t H, int64_t W, int wavelet,
                                 float *gpan, float *const *gms, int R, cudaStream_t stream) {
    BwdArgs s{};
    s.g = g;
    s.gpan = gpan;
    bool ms2 = ((W >> 1) % 2) == 0;
    for (int b = 0; b < bands; ++b) {
        s.gms[b] = gms[b];
        ms2 = ms2 && (reinterpret_cast<uintptr_t>(gms[b]) % 8 == 0);
    }
    s.H = H;
    s.W = W;
    s.bands = bands;
    s.kappa = wavelet == 0 ? 4.0f : 2.0f;  // gain * sigma^2: 1 * 4 (Haar), 2 * 1 (D4)
    s.a4 = (W % 4 == 0) && (reinterpret_cast<uintptr_t>(g) % 16 == 0) &&
           (reinterpret_cast<uintptr_t>(gpan) % 16 == 0);
    s.ms2 = ms2;
    const ItemGrid ig = item_grid(H, W, R);
    const void *fn = wavelet == 0 ? reinterpret_cast<const void *>(&fuse_bwd_kernel<0>)
                                  : reinterpret_cast<const void *>(&fuse_bwd_kernel<1>);
    int occ = 0, sms = 0;
    cudaError_t e = resident_blocks(fn, kBwdThreads, &occ);
    if (e != cudaSuccess) return e;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    const int64_t need = (ig.items + kBwdWarps - 1) / kBwdWarps;
    const int64_t cap = (int64_t)sms * occ;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    if (grid == 0) return cudaSuccess;
    int64_t strips_x = ig.strips_x, items = ig.items;
    void *args[] = {&s, &strips_x, &items, &R};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBwdThreads), args, 0, stream);
}

}  // namespace dwtfuse
