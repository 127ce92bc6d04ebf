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
// Same warp-strip decomposition as the forward: a lane owns PAN columns
// x..x+3 and walks down R MS rows.  Every band's two new PAN rows are loaded
// together in groups (D4: groups of 2 bands, or of 4 for 5-8 bands on
// unshifted rows; measured fastest), and D4 keeps, per band, the row
// low-pass of the two previous rows (a sliding vertical window), plus the
// same for G, in registers.  Up to 8 bands per launch: chunks of 1-4 bands
// run 256-thread CTAs (two per SM, 128 registers), chunks of 5-8 bands
// 384-thread CTAs (one per SM, 168 registers); further launches over the
// remaining bands add their G - U(LL(G)) into grad_P.
#include <cstring>

#include "fuse_tile.cuh"
#include "launch.h"

namespace dwtfuse {

constexpr int kBwdThreads = 256;      // chunks of 1-4 bands
constexpr int kBwdWideThreads = 384;  // chunks of 5-8 bands
constexpr int kBwdChunk = 8;          // bands per launch
constexpr int kBwdGroup = 4;          // Haar: bands whose rows of a step are loaded together

// D4: bands whose rows of a step are loaded together.  Fewer registers in
// flight leave the compiler room to overlap the groups: groups of 2 beat all
// bands at once for 3-4 bands (16384^2 x 4: 1.14 -> 1.00 ms) and for 5-8
// bands on shifted rows (16384 x 16382 x 8: 2.81 -> 2.26 ms); 5-8 bands on
// unshifted rows are fastest in groups of 4 (2.36 ms against 2.99).
template <int NB, bool ALT>
struct D4Group {
    static constexpr int value = NB <= 2 ? NB : (NB <= 4 || ALT ? 2 : 4);
};

struct BwdArgs {
    const float *g;               // [bands][H][W]
    float *gpan;                  // H x W
    float *gms[kMaxBands];        // (H/2) x (W/2) each
    int64_t H, W;
    int32_t bands;
    float kappa;                  // gain * sigma^2
    int32_t a4;                   // 4-pixel vector path for g / gpan
    int32_t ms2;                  // W/2 even and every gms 8-byte aligned: pair stores
    int32_t alt;                  // W % 4 == 2 with 16-byte aligned g / gpan: shifted odd rows
    int32_t wavelet;              // 0 Haar, 1 D4
    int32_t b0;                   // first band of the chunk (batched tables)
    int32_t nbc;                  // bands of the chunk (batched tables)
};

// Scene table of one launch of the batched backward (band chunk b0 of n scenes).
struct BwdBatchTable {
    int32_t n;
    int32_t R;
    int64_t item_start[kMaxScenes + 1];
    int64_t strips_x[kMaxScenes];
    BwdArgs scenes[kMaxScenes];
};
static_assert(sizeof(BwdBatchTable) + 16 <= 32764, "batched backward table exceeds the parameter limit");

__device__ __forceinline__ void store_gms(float *row, const LaneCols &c, bool pair, float a, float b) {
    if (pair) {
        *reinterpret_cast<float2 *>(row + c.nB) = make_float2(a, b);
    } else {
        row[c.nB] = a;
        if (c.two) row[c.nC] = b;
    }
}

// grad_P pixels (y, x..x+3): written, or added to what an earlier chunk wrote.
__device__ __forceinline__ void store_gpan(float *p, bool a4, bool two, bool acc, const float *v) {
    float w[4] = {v[0], v[1], v[2], v[3]};
    if (acc) {
        if (a4) {
            const float4 o = *reinterpret_cast<const float4 *>(p);
            w[0] += o.x; w[1] += o.y; w[2] += o.z; w[3] += o.w;
        } else {
            const float2 o = *reinterpret_cast<const float2 *>(p);
            w[0] += o.x; w[1] += o.y;
            if (two) {
                const float2 u = *reinterpret_cast<const float2 *>(p + 2);
                w[2] += u.x; w[3] += u.y;
            }
        }
    }
    if (a4) {
        *reinterpret_cast<float4 *>(p) = make_float4(w[0], w[1], w[2], w[3]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(w[0], w[1]);
        if (two) *reinterpret_cast<float2 *>(p + 2) = make_float2(w[2], w[3]);
    }
}

// grad_P pixels (y, x..x+3) of a row that starts 2 pixels past a 16-byte
// boundary (W = 2 mod 4, odd rows): every lane but the first writes (or adds
// to) the aligned vector x-2..x+1 with its left neighbour's last two values;
// lane 0 writes x, x+1 and the last lane of the strip also x+2, x+3.  Every
// lane of the warp must call it (warp shuffles); `active` masks the stores.
__device__ __forceinline__ void store_gpan_shifted(float *p, int lane, bool active, bool two, bool last,
                                                   bool acc, const float *v) {
    const float l2 = __shfl_up_sync(0xffffffffu, v[2], 1);
    const float l3 = __shfl_up_sync(0xffffffffu, v[3], 1);
    if (!active) return;
    if (lane > 0) {
        float4 w = make_float4(l2, l3, v[0], v[1]);
        if (acc) {
            const float4 o = *reinterpret_cast<const float4 *>(p - 2);
            w.x += o.x; w.y += o.y; w.z += o.z; w.w += o.w;
        }
        *reinterpret_cast<float4 *>(p - 2) = w;
    } else {
        float2 w = make_float2(v[0], v[1]);
        if (acc) {
            const float2 o = *reinterpret_cast<const float2 *>(p);
            w.x += o.x; w.y += o.y;
        }
        *reinterpret_cast<float2 *>(p) = w;
    }
    if (two && last) {
        float2 w = make_float2(v[2], v[3]);
        if (acc) {
            const float2 o = *reinterpret_cast<const float2 *>(p + 2);
            w.x += o.x; w.y += o.y;
        }
        *reinterpret_cast<float2 *>(p + 2) = w;
    }
}

// Rows 2m, 2m+1 of grad_P.  ALT: the W % 4 == 2 instance (even rows as
// vectors but for the lane at x = W-2, odd rows shifted; all lanes call).
template <bool ALT>
__device__ __forceinline__ void store_gpan_rows(const BwdArgs &s, const LaneCols &c, int lane, int64_t m, bool acc,
                                                const float *o0, const float *o1) {
    float *r0 = s.gpan + (2 * m) * s.W + c.x, *r1 = r0 + s.W;
    if constexpr (ALT) {
        if (s.alt) {
            if (c.active) store_gpan(r0, c.two, c.two, acc, o0);
            store_gpan_shifted(r1, lane, c.active, c.two, c.last, acc, o1);
            return;
        }
    }
    if (c.active) {
        store_gpan(r0, s.a4 != 0, c.two, acc, o0);
        store_gpan(r1, s.a4 != 0, c.two, acc, o1);
    }
}

template <int NB, bool ALT>
__device__ __forceinline__ void haar_bwd_item(const BwdArgs &s, int64_t x0, int64_t m_s, int64_t m_e,
                                              int b0, bool acc, int lane) {
    const int64_t W = s.W, H = s.H, W2 = W >> 1, HW = H * W;
    const LaneCols c = lane_cols(x0, lane, W);
    const bool a4 = s.a4 != 0, pair = s.ms2 != 0;
    const bool lde = a4 || (ALT && s.alt != 0 && c.two);  // 4-pixel loads on even rows
    for (int64_t m = m_s; m < m_e; ++m) {
        float g0[4] = {0.f, 0.f, 0.f, 0.f}, g1[4] = {0.f, 0.f, 0.f, 0.f};
        // A group's two rows of every band in flight together.
#pragma unroll
        for (int gs = 0; gs < NB; gs += kBwdGroup) {
            constexpr int G = NB < kBwdGroup ? NB : kBwdGroup;
            float p0[G][4], p1[G][4];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (gs + j < NB) {
                    const float *gb = s.g + (int64_t)(b0 + gs + j) * HW;
                    load_row4(gb + (2 * m) * W, c, lde, p0[j]);
                    load_row4(gb + (2 * m + 1) * W, c, a4, p1[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int b = gs + j;
                if (b >= NB) continue;
                const float sA = (p0[j][0] + p0[j][1]) + (p1[j][0] + p1[j][1]);
                const float sB = (p0[j][2] + p0[j][3]) + (p1[j][2] + p1[j][3]);
                if (c.active)
                    store_gms(s.gms[b0 + b] + m * W2, c, pair, s.kappa * 0.25f * sA, s.kappa * 0.25f * sB);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    g0[q] += p0[j][q];
                    g1[q] += p1[j][q];
                }
            }
        }
        if (!ALT && !c.active) continue;
        const float mA = ((g0[0] + g0[1]) + (g1[0] + g1[1])) * 0.25f;
        const float mB = ((g0[2] + g0[3]) + (g1[2] + g1[3])) * 0.25f;
        const float v0[4] = {g0[0] - mA, g0[1] - mA, g0[2] - mB, g0[3] - mB};
        const float v1[4] = {g1[0] - mA, g1[1] - mA, g1[2] - mB, g1[3] - mB};
        store_gpan_rows<ALT>(s, c, lane, m, acc, v0, v1);
    }
}

// Row low-pass at MS columns n and n+1 from the 8 pixels x-2..x+5 (v[2..7]).
__device__ __forceinline__ void d4_rowpass2(const float *v, float *r) {
    r[0] = fmaf(kH3, v[5], fmaf(kH2, v[4], fmaf(kH1, v[3], kH0 * v[2])));
    r[1] = fmaf(kH3, v[7], fmaf(kH2, v[6], fmaf(kH1, v[5], kH0 * v[4])));
}

// G: bands whose rows of a step are loaded together (the grouping changes
// only the load schedule, not the arithmetic).
template <int NB, bool ALT, int G = D4Group<NB, ALT>::value>
__device__ __forceinline__ void d4_bwd_item(const BwdArgs &s, int64_t x0, int64_t m_s, int64_t m_e,
                                            int b0, bool acc, int lane) {
    const int64_t W = s.W, H = s.H, W2 = W >> 1, H2 = H >> 1, HW = H * W;
    const LaneCols c = lane_cols(x0, lane, W);
    const bool a4 = s.a4 != 0, pair = s.ms2 != 0;
    const bool lde = a4 || (ALT && s.alt != 0 && c.two);  // 4-pixel loads on even rows
    const float *g = s.g + (int64_t)b0 * HW;

    // Prologue: PAN rows 2mp .. 2mp+3 of every band, mp = m_s - 1 (periodic).
    const int64_t mp = wrap(m_s - 1, H2);
    float rb[NB][2][2];      // per band: row low-pass of rows 2m, 2m+1 at MS columns n, n+1
    float rg0[3], rg1[3];    // G: row low-pass of rows 2m, 2m+1 at n-1, n, n+1
    float go0[4], go1[4];    // G pixels of rows 2m, 2m+1 (this lane's 4 columns)
    float hprev[4];          // row synthesis of LL(G)(m-1)
    {
        // rows 2mp, 2mp+1: only their band sum G is needed
        float r0[3], r1[3];
        {
            float ga[2][8];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int k = 0; k < 8; ++k) ga[r][k] = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    float v[8];
                    load_row8(g + (int64_t)b * HW + wrap(2 * mp + r, H) * W, c, r == 0 ? lde : a4, v);
#pragma unroll
                    for (int k = 0; k < 8; ++k) ga[r][k] += v[k];
                }
            }
            d4_rowpass(ga[0], r0);
            d4_rowpass(ga[1], r1);
        }
        // rows 2mp+2, 2mp+3 (= 2m_s, 2m_s+1): per band low-pass state and G
        float ga[2][8];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) ga[r][k] = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float v[8];
                load_row8(g + (int64_t)b * HW + wrap(2 * mp + 2 + r, H) * W, c, r == 0 ? lde : a4, v);
#pragma unroll
                for (int k = 0; k < 8; ++k) ga[r][k] += v[k];
                d4_rowpass2(v, rb[b][r]);
            }
        }
        d4_rowpass(ga[0], rg0);
        d4_rowpass(ga[1], rg1);
        float llg[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) llg[k] = fmaf(kH3, rg1[k], fmaf(kH2, rg0[k], fmaf(kH1, r1[k], kH0 * r0[k])));
        hprev[0] = fmaf(kH2, llg[0], kH0 * llg[1]);
        hprev[1] = fmaf(kH3, llg[0], kH1 * llg[1]);
        hprev[2] = fmaf(kH2, llg[1], kH0 * llg[2]);
        hprev[3] = fmaf(kH3, llg[1], kH1 * llg[2]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            go0[q] = ga[0][q + 2];
            go1[q] = ga[1][q + 2];
        }
    }

    for (int64_t m = m_s; m < m_e; ++m) {
        float ga[2][8];
        // A group's PAN rows 2m+2 and 2m+3 of every band in flight together.
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += G) {
            float v[G][2][8];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (g0 + j < NB) {
                    const float *gb = g + (int64_t)(g0 + j) * HW;
                    load_row8(gb + wrap(2 * m + 2, H) * W, c, lde, v[j][0]);
                    load_row8(gb + wrap(2 * m + 3, H) * W, c, a4, v[j][1]);
                }
            }
            if (g0 == 0) {
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int k = 0; k < 8; ++k) ga[r][k] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int b = g0 + j;
                if (b >= NB) continue;
                float n0[2], n1[2];
                d4_rowpass2(v[j][0], n0);
                d4_rowpass2(v[j][1], n1);
                // LL(G_b)(m, n), (m, n+1): column low-pass over rows 2m .. 2m+3
                const float llA = fmaf(kH3, n1[0], fmaf(kH2, n0[0], fmaf(kH1, rb[b][1][0], kH0 * rb[b][0][0])));
                const float llB = fmaf(kH3, n1[1], fmaf(kH2, n0[1], fmaf(kH1, rb[b][1][1], kH0 * rb[b][0][1])));
                if (c.active) store_gms(s.gms[b0 + b] + m * W2, c, pair, s.kappa * llA, s.kappa * llB);
                rb[b][0][0] = n0[0]; rb[b][0][1] = n0[1];
                rb[b][1][0] = n1[0]; rb[b][1][1] = n1[1];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    ga[0][k] += v[j][0][k];
                    ga[1][k] += v[j][1][k];
                }
            }
        }
        float rn0[3], rn1[3], llg[3];
        d4_rowpass(ga[0], rn0);
        d4_rowpass(ga[1], rn1);
#pragma unroll
        for (int k = 0; k < 3; ++k) llg[k] = fmaf(kH3, rn1[k], fmaf(kH2, rn0[k], fmaf(kH1, rg1[k], kH0 * rg0[k])));
        float hc[4];
        hc[0] = fmaf(kH2, llg[0], kH0 * llg[1]);
        hc[1] = fmaf(kH3, llg[0], kH1 * llg[1]);
        hc[2] = fmaf(kH2, llg[1], kH0 * llg[2]);
        hc[3] = fmaf(kH3, llg[1], kH1 * llg[2]);
        float o0[4], o1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            o0[q] = go0[q] - fmaf(kH2, hprev[q], kH0 * hc[q]);
            o1[q] = go1[q] - fmaf(kH3, hprev[q], kH1 * hc[q]);
            hprev[q] = hc[q];
        }
        store_gpan_rows<ALT>(s, c, lane, m, acc, o0, o1);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            rg0[k] = rn0[k];
            rg1[k] = rn1[k];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            go0[q] = ga[0][q + 2];
            go1[q] = ga[1][q + 2];
        }
    }
}

// Threads per CTA and CTAs per SM of a chunk's kernel (see above).
template <int NB>
struct BwdShape {
    static constexpr int kThreads = NB <= 4 ? kBwdThreads : kBwdWideThreads;
    static constexpr int kMinBlocks = NB <= 4 ? 2 : 1;
    static constexpr int kWarps = kThreads / 32;
};

template <int WAV, int NB, bool ALT>
__global__ void __launch_bounds__(BwdShape<NB>::kThreads, BwdShape<NB>::kMinBlocks)
fuse_bwd_kernel(const __grid_constant__ BwdArgs s, int b0, int acc, int64_t strips_x, int64_t items, int R) {
    constexpr int kWarps = BwdShape<NB>::kWarps;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t it = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); it < items; it += nwarps) {
        const int64_t sx = it % strips_x, sy = it / strips_x;
        const int64_t m_s = sy * R;
        const int64_t m_e = min(m_s + (int64_t)R, s.H >> 1);
        if (WAV == 0)
            haar_bwd_item<NB, ALT>(s, sx * kWarpCols, m_s, m_e, b0, acc != 0, lane);
        else
            d4_bwd_item<NB, ALT>(s, sx * kWarpCols, m_s, m_e, b0, acc != 0, lane);
    }
}

// Batched: a launch covers one band chunk of the scenes in its table of one
// wavelet whose chunk has 1-4 bands (WIDE = false) or 5-8 bands (WIDE = true);
// item ranges by prefix sums, an atomic queue as in the batched forward.
// Chunks after the first add into grad_P, so they run as later launches.
template <bool WIDE, int WAV>
__global__ void __launch_bounds__(WIDE ? kBwdWideThreads : kBwdThreads, WIDE ? 1 : 2)
fuse_bwd_batched_kernel(const __grid_constant__ BwdBatchTable t, unsigned long long *queue) {
    const int lane = threadIdx.x & 31;
    const unsigned long long total = (unsigned long long)t.item_start[t.n];
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(queue, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        int lo = 0, hi = t.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)t.item_start[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const BwdArgs &s = t.scenes[lo];
        const int64_t local = (int64_t)(it - (unsigned long long)t.item_start[lo]);
        const int64_t sx = local % t.strips_x[lo], sy = local / t.strips_x[lo];
        const int64_t m_s = sy * t.R;
        const int64_t m_e = min(m_s + (int64_t)t.R, s.H >> 1);
        // the table holds a scene here only if its chunk has 1-4 (5-8 when WIDE) bands
        const int b0 = s.b0, nb = s.nbc;
        const bool acc = b0 > 0, alt = s.alt != 0;
        const int64_t x0 = sx * kWarpCols;
#define DWTFUSE_BWD_CASE(NBV)                                                                 \
    case NBV:                                                                                 \
        if constexpr (WAV == 0) {                                                             \
            if (alt) haar_bwd_item<NBV, true>(s, x0, m_s, m_e, b0, acc, lane);                 \
            else haar_bwd_item<NBV, false>(s, x0, m_s, m_e, b0, acc, lane);                    \
        } else {                                                                              \
            if (alt) d4_bwd_item<NBV, true, WIDE ? D4Group<NBV, true>::value : NBV>(           \
                s, x0, m_s, m_e, b0, acc, lane);                                              \
            else d4_bwd_item<NBV, false, WIDE ? D4Group<NBV, false>::value : NBV>(             \
                s, x0, m_s, m_e, b0, acc, lane);                                              \
        }                                                                                     \
        break;
        // 1-4 bands: D4 loads every band's rows at once in this kernel (groups of
        // 2, the per-scene kernel's choice, ran 13 % slower here: 0.625 against
        // 0.551 ms for 8 x 4096^2 x 4).
        if constexpr (WIDE) {
            switch (nb) {
                DWTFUSE_BWD_CASE(5) DWTFUSE_BWD_CASE(6) DWTFUSE_BWD_CASE(7) DWTFUSE_BWD_CASE(8)
                default: break;
            }
        } else {
            switch (nb) {
                DWTFUSE_BWD_CASE(1) DWTFUSE_BWD_CASE(2) DWTFUSE_BWD_CASE(3) DWTFUSE_BWD_CASE(4)
                default: break;
            }
        }
#undef DWTFUSE_BWD_CASE
    }
}

namespace {

template <int WAV, int NB>
const void *bwd_fn(bool alt) {
    return alt ? reinterpret_cast<const void *>(&fuse_bwd_kernel<WAV, NB, true>)
               : reinterpret_cast<const void *>(&fuse_bwd_kernel<WAV, NB, false>);
}

template <int WAV>
const void *bwd_fn_nb(int nb, bool alt) {
    switch (nb) {
        case 1: return bwd_fn<WAV, 1>(alt);
        case 2: return bwd_fn<WAV, 2>(alt);
        case 3: return bwd_fn<WAV, 3>(alt);
        case 4: return bwd_fn<WAV, 4>(alt);
        case 5: return bwd_fn<WAV, 5>(alt);
        case 6: return bwd_fn<WAV, 6>(alt);
        case 7: return bwd_fn<WAV, 7>(alt);
        default: return bwd_fn<WAV, 8>(alt);
    }
}

// Threads per CTA of a chunk of nb bands.
int bwd_threads(int nb) { return nb <= 4 ? kBwdThreads : kBwdWideThreads; }

}  // namespace

BwdArgs make_bwd_args(const float *g, int bands, int64_t H, int64_t W, int wavelet, float *gpan,
                      float *const *gms) {
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
    s.wavelet = wavelet;
    const bool al16 = (reinterpret_cast<uintptr_t>(g) % 16 == 0) && (reinterpret_cast<uintptr_t>(gpan) % 16 == 0);
    s.a4 = (W % 4 == 0) && al16;
    s.alt = (W % 4 == 2) && al16;
    s.ms2 = ms2;
    return s;
}

cudaError_t launch_fuse_backward_batched(const dwtfuse_grad_scene *in, int n, unsigned long long *queue,
                                         cudaStream_t stream) {
    static thread_local BwdBatchTable t;  // ~28 KB: kept off the stack
    static thread_local BwdArgs scenes[kMaxScenes];
    // Band chunk: 8, or the autotuner's band-chunk knob; rows per item: the
    // default, or the rows knob.
    const int knob = bwd_band_chunk();
    const int cw = knob > 0 && knob < kBwdChunk ? knob : kBwdChunk;
    const int rows = rows_per_item();
    int max_chunks = 0;
    for (int i = 0; i < n; ++i) {
        scenes[i] = make_bwd_args(in[i].grad_out, in[i].bands, in[i].H, in[i].W, in[i].wavelet, in[i].grad_pan,
                                  in[i].grad_ms);
        const int nc = (scenes[i].bands + cw - 1) / cw;
        max_chunks = nc > max_chunks ? nc : max_chunks;
    }
    int sms = 0;
    cudaError_t e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    for (int chunk = 0; chunk < max_chunks; ++chunk) {
        for (int kind = 0; kind < 4; ++kind) {  // (1-4 bands, 5-8 bands) x (Haar, D4)
            const int wide = kind >> 1, wav = kind & 1;
            std::memset(&t, 0, sizeof t);
            t.R = rows > 0 ? rows : kDefaultRows;
            int64_t acc = 0;
            int k = 0;
            for (int i = 0; i < n; ++i) {
                const int b0 = chunk * cw;
                const int rest = scenes[i].bands - b0;
                const int nb = rest < cw ? rest : cw;
                if (nb <= 0 || (nb > 4) != (wide != 0) || scenes[i].wavelet != wav) continue;
                const ItemGrid g = item_grid(scenes[i].H, scenes[i].W, t.R);
                t.scenes[k] = scenes[i];
                t.scenes[k].b0 = b0;
                t.scenes[k].nbc = nb;
                t.item_start[k] = acc;
                t.strips_x[k] = g.strips_x;
                acc += g.items;
                ++k;
            }
            if (k == 0) continue;
            t.n = k;
            t.item_start[k] = acc;
            const void *fns[4] = {reinterpret_cast<const void *>(&fuse_bwd_batched_kernel<false, 0>),
                                  reinterpret_cast<const void *>(&fuse_bwd_batched_kernel<false, 1>),
                                  reinterpret_cast<const void *>(&fuse_bwd_batched_kernel<true, 0>),
                                  reinterpret_cast<const void *>(&fuse_bwd_batched_kernel<true, 1>)};
            const void *fn = fns[kind];
            const int threads = wide ? kBwdWideThreads : kBwdThreads;
            int occ = 0;
            e = resident_blocks(fn, threads, &occ);
            if (e != cudaSuccess) return e;
            const int64_t cap = (int64_t)sms * occ;
            const int64_t need = (acc + threads / 32 - 1) / (threads / 32);
            const unsigned grid = (unsigned)(need < cap ? need : cap);
            if (grid == 0) continue;
            e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream);
            if (e != cudaSuccess) return e;
            unsigned long long *q = queue;
            void *args[] = {&t, &q};
            e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, stream);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_fuse_backward(const float *g, int bands, int64_t H, int64_t W, int wavelet,
                                 float *gpan, float *const *gms, int R, cudaStream_t stream) {
    BwdArgs s = make_bwd_args(g, bands, H, W, wavelet, gpan, gms);
    int sms = 0;
    cudaError_t e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    const int knob = bwd_band_chunk();
    const int cw = knob > 0 && knob < kBwdChunk ? knob : kBwdChunk;
    for (int b0 = 0; b0 < bands; b0 += cw) {
        const int nb = bands - b0 < cw ? bands - b0 : cw;
        const void *fn = wavelet == 0 ? bwd_fn_nb<0>(nb, s.alt != 0) : bwd_fn_nb<1>(nb, s.alt != 0);
        const int threads = bwd_threads(nb), warps = threads / 32;
        int occ = 0;
        e = resident_blocks(fn, threads, &occ);
        if (e != cudaSuccess) return e;
        const int64_t cap = (int64_t)sms * occ;
        int Rl = R > 0 ? R : balanced_rows(H, W, cap * warps);
        const ItemGrid ig = item_grid(H, W, Rl);
        const int64_t need = (ig.items + warps - 1) / warps;
        const unsigned grid = (unsigned)(need < cap ? need : cap);
        if (grid == 0) return cudaSuccess;
        int acc = b0 > 0;
        int64_t strips_x = ig.strips_x, items = ig.items;
        void *args[] = {&s, &b0, &acc, &strips_x, &items, &Rl};
        e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dwtfuse
