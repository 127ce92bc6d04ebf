// Standalone one-level 2D DWT and inverse (the transforms either side of the
// LL replacement, Sec. 2): forward = 1D transform of every row, then of every
// column (Haar Eq. 1-2, D4 Eq. 3-10 with periodic wrap); inverse = columns,
// then rows (Haar Eq. 11-12, D4 Eq. 13-16).  The coefficient image Z is H x W
// float in the paper's in-place layout: with A / D the row approximation /
// detail and a column pass of low-pass (h) then high-pass (g),
//     Z(m, j)           = sum_a h_a A(2m+a, j)    (LL, top-left)
//     Z(m, W/2 + j)     = sum_a h_a D(2m+a, j)    (top-right)
//     Z(H/2 + m, j)     = sum_a g_a A(2m+a, j)    (bottom-left)
//     Z(H/2 + m, W/2+j) = sum_a g_a D(2m+a, j)    (bottom-right)
// D4: h of Eq. 7-8, g = (h3, -h2, h1, -h0) (the quadrature mirror; Eq. 9-10
// as printed do not invert).  The D4 synthesis is the transpose of the
// analysis; the /2 Haar synthesis is twice its transpose.
//
// Same warp strips as the fused kernels: a lane owns image columns x..x+3
// (coefficient columns n, n+1 of each half) and walks down R coefficient rows
// with a sliding window of image rows (forward) or coefficient rows (inverse).
// Haar loads two coefficient rows' inputs per step (16384^2: forward 0.32 ->
// 0.23 ms, inverse 0.37 -> 0.35 ms; the forward only with streaming stores,
// with plain stores the two-row body came out slower, 0.46 ms); the same for
// D4 measured slower (forward 0.29 -> 0.37 ms), so D4 keeps one row per step
// and instead loads the next step's rows one step ahead.  Both D4 passes were
// latency-bound (ncu at 8192^2: long-scoreboard stalls 7 and 11 per issue,
// DRAM 48 % and 55 % of peak): with the prefetch and four CTAs per SM for the
// forward (60 registers, uint8 rows kept as raw words) and three for the
// inverse (80 registers, 32 bytes of spill), 16384^2 runs at forward 0.29 ->
// 0.27 ms and inverse 0.45 -> 0.39 ms (two CTAs per SM: 0.44 ms).
#include "fuse_tile.cuh"
#include "launch.h"

namespace dwtfuse {

constexpr int kDwtThreads = 256;
constexpr int kDwtWarps = kDwtThreads / 32;
// Detail filter g = (h3, -h2, h1, -h0).
constexpr float kG0 = kH3, kG1 = -kH2, kG2 = kH1, kG3 = -kH0;

struct DwtArgs {
    const void *src;  // image (forward, u8 or f32) or coefficients (inverse, f32)
    float *dst_f32;   // coefficients (forward) or image (inverse)
    uint8_t *dst_u8;  // image (inverse only), optional
    int64_t H, W;
    int32_t a4;       // W % 4 == 0 and aligned for 4-pixel image vectors
    int32_t pairs;    // W/2 even: coefficient pairs are 8-byte aligned in both halves
};

// Two coefficients (columns n, n+1) of one coefficient row; n+1 only if `two`.
__device__ __forceinline__ void store_pair(float *p, bool pair, bool two, float a, float b) {
    if (pair) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(a, b));
    } else {
        __stcs(p, a);
        if (two) __stcs(p + 1, b);
    }
}

// Row analysis of one image row at coefficient columns n, n+1 (pixels x..x+5 = v[2..7]).
__device__ __forceinline__ void d4_row_ad(const float *v, float *ra, float *rd) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float *s = v + 2 + 2 * j;
        ra[j] = fmaf(kH3, s[3], fmaf(kH2, s[2], fmaf(kH1, s[1], kH0 * s[0])));
        rd[j] = fmaf(kG3, s[3], fmaf(kG2, s[2], fmaf(kG1, s[1], kG0 * s[0])));
    }
}

// Raw uint8 words of one image row for a lane's D4 taps (pixels x-2..x+5,
// periodic): the pair at x-2, the 4 pixels at x (one word on the vector path,
// else two pairs), the pair at x+4.
struct Raw8 {
    uint32_t l, m0, m1, r;
};

template <typename T>
__device__ __forceinline__ Raw8 load_raw8(const T *row, const LaneCols &c, bool a4) {
    const uint8_t *p = reinterpret_cast<const uint8_t *>(row);
    Raw8 w;
    w.l = __ldg(reinterpret_cast<const unsigned short *>(p + c.cm));
    if (a4) {
        w.m0 = __ldg(reinterpret_cast<const unsigned int *>(p + c.x));
        w.m1 = 0;
    } else {
        w.m0 = __ldg(reinterpret_cast<const unsigned short *>(p + c.x));
        w.m1 = __ldg(reinterpret_cast<const unsigned short *>(p + c.c2));
    }
    w.r = __ldg(reinterpret_cast<const unsigned short *>(p + c.c4));
    return w;
}

__device__ __forceinline__ void unpack_raw8(const Raw8 &w, bool a4, float *v) {
    v[0] = byte_f(w.l, 0);
    v[1] = byte_f(w.l, 1);
    const uint32_t mid = a4 ? w.m0 : (w.m0 | (w.m1 << 16));
    v[2] = byte_f(mid, 0);
    v[3] = byte_f(mid, 1);
    v[4] = byte_f(mid, 2);
    v[5] = byte_f(mid, 3);
    v[6] = byte_f(w.r, 0);
    v[7] = byte_f(w.r, 1);
}

// ------------------------------------------------------------------ output sinks
//
// The item bodies below hand their outputs to a sink: a coefficient pair of
// quadrant q (0 LL, 1 HL, 2 LH, 3 HH) of coefficient row m + r (forward), or
// 4 image pixels of image row 2m + r (inverse), then call step_end once per
// step of the walk (every lane, active or not).
//
// Direct sinks store from the lanes.  The staged forward sink (large images
// with W % 8 == 0 and a 16-byte-aligned coefficient plane) puts the step's
// quadrant rows of the CTA's 1024-image-column strip (4 segments of 512
// coefficients per coefficient row) into one of two shared-memory slots; at
// step_end the CTA meets at one barrier and one thread per segment writes it
// with cp.async.bulk (shared::cta -> global).  The slots alternate with a row
// count carried across work items; the issuing threads wait for their
// previous copies' reads before the barrier, so the slot a step overwrites is
// free (the scheme of the staged fused forward).  At 16384^2 D4 it measured
// 0.269 -> 0.258 ms (ncu at 8192^2: 72.7 -> 69.0 us, issue active 72 %, top
// stalls long scoreboard 2.5 and barrier 2.3 per issue); the same staging of
// the inverse's image rows ran slower (0.388 -> 0.401 ms), so the inverse
// keeps direct stores.
constexpr int kDwtCols = kDwtWarps * kWarpCols;  // image columns of a staged CTA strip

__device__ __forceinline__ unsigned dwt_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_row(float *dst, const float *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(dwt_smem(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

struct FwdDirect {
    static constexpr bool kStaged = false;
    float *Z;
    int64_t W, W2, H2;
    const LaneCols &c;
    bool pair;
    __device__ __forceinline__ void quad(int64_t m, int r, int q, float a, float b) const {
        float *p = Z + ((q < 2 ? m : H2 + m) + r) * W + ((q & 1) ? W2 : 0) + c.nB;
        store_pair(p, pair, c.two, a, b);
    }
    __device__ __forceinline__ void step_end(int64_t, bool) const {}
};

// RS coefficient rows per step (2 Haar, 1 D4): 4 RS segments of 512 floats.
template <int RS>
struct FwdStaged {
    static constexpr bool kStaged = true;
    static constexpr int kSegs = 4 * RS, kSeg = kDwtCols / 2;
    float *Z;
    int64_t W, W2, H2;
    const LaneCols &c;
    float *buf;
    int *rowc;
    int64_t n0;  // first coefficient column of the strip (X0 / 2)
    int ncoef;   // coefficient columns of the strip inside the image (a multiple of 4)
    __device__ __forceinline__ float *slot() const { return buf + (*rowc & 1) * kSegs * kSeg; }
    __device__ __forceinline__ void quad(int64_t, int r, int q, float a, float b) const {
        if (!c.active) return;
        *reinterpret_cast<float2 *>(slot() + (r * 4 + q) * kSeg + (c.nB - n0)) = make_float2(a, b);
    }
    __device__ __forceinline__ void step_end(int64_t m, bool second) const {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int t = threadIdx.x;
        if (t < kSegs) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
        __syncthreads();
        if (t < (second ? kSegs : 4)) {
            const int r = t >> 2, q = t & 3;
            float *dst = Z + ((q < 2 ? m : H2 + m) + r) * W + ((q & 1) ? W2 : 0) + n0;
            bulk_row(dst, slot() + t * kSeg, (unsigned)ncoef * 4u);
        }
        ++*rowc;
    }
};

struct InvDirect {
    static constexpr bool kStaged = false;
    OutPtrs o;
    int64_t W;
    const LaneCols &c;
    bool a4;
    __device__ __forceinline__ void img(int64_t m, int r, const float *v) const {
        store4(o, (2 * m + r) * W + c.x, a4, c.two, v);
    }
    __device__ __forceinline__ void step_end(int64_t, bool) const {}
};

template <typename T, int WAV, class Sink>
__device__ __forceinline__ void dwt2_item(const DwtArgs &s, int64_t x0, int64_t m_s, int64_t m_e, int lane,
                                          const Sink &sink) {
    const int64_t W = s.W, H = s.H;
    const LaneCols c = lane_cols(x0, lane, W);
    const bool a4 = s.a4 != 0;
    const T *img = static_cast<const T *>(s.src);
    if (WAV == 0) {
        auto emit = [&](int64_t m, int r, const float *p0, const float *p1) {
            float A0[2], D0[2], A1[2], D1[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // Eq. 1-2 along the rows
                A0[j] = (p0[2 * j] + p0[2 * j + 1]) * 0.5f;
                D0[j] = (p0[2 * j] - p0[2 * j + 1]) * 0.5f;
                A1[j] = (p1[2 * j] + p1[2 * j + 1]) * 0.5f;
                D1[j] = (p1[2 * j] - p1[2 * j + 1]) * 0.5f;
            }
            // Eq. 1-2 along the columns
            sink.quad(m, r, 0, (A0[0] + A1[0]) * 0.5f, (A0[1] + A1[1]) * 0.5f);
            sink.quad(m, r, 1, (D0[0] + D1[0]) * 0.5f, (D0[1] + D1[1]) * 0.5f);
            sink.quad(m, r, 2, (A0[0] - A1[0]) * 0.5f, (A0[1] - A1[1]) * 0.5f);
            sink.quad(m, r, 3, (D0[0] - D1[0]) * 0.5f, (D0[1] - D1[1]) * 0.5f);
        };
        for (int64_t m = m_s; m < m_e; m += 2) {  // two coefficient rows' image rows in flight
            const bool second = m + 1 < m_e;
            float p0[4], p1[4], p2[4], p3[4];
            load_row4(img + (2 * m) * W, c, a4, p0);
            load_row4(img + (2 * m + 1) * W, c, a4, p1);
            if (second) {
                load_row4(img + (2 * m + 2) * W, c, a4, p2);
                load_row4(img + (2 * m + 3) * W, c, a4, p3);
            }
            if (c.active) {
                emit(m, 0, p0, p1);
                if (second) emit(m, 1, p2, p3);
            }
            sink.step_end(m, second);
        }
        return;
    }
    // D4: rows 2m .. 2m+3 (periodic) feed coefficient row m.
    float a0[2], d0[2], a1[2], d1[2];
    {
        float v[8];
        load_row8(img + (2 * m_s) * W, c, a4, v);
        d4_row_ad(v, a0, d0);
        load_row8(img + (2 * m_s + 1) * W, c, a4, v);
        d4_row_ad(v, a1, d1);
    }
    // uint8 images: the raw words of the next step's two rows are loaded one
    // step ahead (a few registers), so a warp's loads overlap its arithmetic.
    constexpr bool kPrefetch = sizeof(T) == 1;
    Raw8 na, nb;
    if constexpr (kPrefetch) {
        na = load_raw8(img + wrap(2 * m_s + 2, H) * W, c, a4);
        nb = load_raw8(img + wrap(2 * m_s + 3, H) * W, c, a4);
    }
    for (int64_t m = m_s; m < m_e; ++m) {
        float va[8], vb[8];
        if constexpr (kPrefetch) {
            const Raw8 ra = na, rb = nb;
            if (m + 1 < m_e) {
                na = load_raw8(img + wrap(2 * m + 4, H) * W, c, a4);
                nb = load_raw8(img + wrap(2 * m + 5, H) * W, c, a4);
            }
            unpack_raw8(ra, a4, va);
            unpack_raw8(rb, a4, vb);
        } else {
            load_row8(img + wrap(2 * m + 2, H) * W, c, a4, va);
            load_row8(img + wrap(2 * m + 3, H) * W, c, a4, vb);
        }
        float a2[2], d2[2], a3[2], d3[2];
        d4_row_ad(va, a2, d2);
        d4_row_ad(vb, a3, d3);
        if (c.active) {
            float ll[2], lh[2], hl[2], hh[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                ll[j] = fmaf(kH3, a3[j], fmaf(kH2, a2[j], fmaf(kH1, a1[j], kH0 * a0[j])));
                lh[j] = fmaf(kG3, a3[j], fmaf(kG2, a2[j], fmaf(kG1, a1[j], kG0 * a0[j])));
                hl[j] = fmaf(kH3, d3[j], fmaf(kH2, d2[j], fmaf(kH1, d1[j], kH0 * d0[j])));
                hh[j] = fmaf(kG3, d3[j], fmaf(kG2, d2[j], fmaf(kG1, d1[j], kG0 * d0[j])));
            }
            sink.quad(m, 0, 0, ll[0], ll[1]);
            sink.quad(m, 0, 1, hl[0], hl[1]);
            sink.quad(m, 0, 2, lh[0], lh[1]);
            sink.quad(m, 0, 3, hh[0], hh[1]);
        }
        sink.step_end(m, false);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            a0[j] = a2[j]; d0[j] = d2[j];
            a1[j] = a3[j]; d1[j] = d3[j];
        }
    }
}

// Inverse.  Per coefficient row i the lane forms, at its 4 image columns,
//   RA(i, .) = row synthesis of (LL, top-right) and RB(i, .) = of (bottom-left, HH),
// then column synthesis mixes rows i = m and m-1 (D4) or row m alone (Haar).
__device__ __forceinline__ void load_coef3(const float *row, const LaneCols &c, float *v) {
    v[0] = __ldg(row + c.nA);
    v[1] = __ldg(row + c.nB);
    v[2] = __ldg(row + c.nC);
}

// D4 row synthesis at image columns x..x+3 of a low-pass half L (h taps) and
// high-pass half G (g taps), each given at coefficient columns n-1, n, n+1.
__device__ __forceinline__ void d4_row_syn(const float *L, const float *G, float *r) {
    r[0] = fmaf(kG0, G[1], fmaf(kG2, G[0], fmaf(kH0, L[1], kH2 * L[0])));
    r[1] = fmaf(kG1, G[1], fmaf(kG3, G[0], fmaf(kH1, L[1], kH3 * L[0])));
    r[2] = fmaf(kG0, G[2], fmaf(kG2, G[1], fmaf(kH0, L[2], kH2 * L[1])));
    r[3] = fmaf(kG1, G[2], fmaf(kG3, G[1], fmaf(kH1, L[2], kH3 * L[1])));
}

template <int WAV, class Sink>
__device__ __forceinline__ void idwt2_item(const DwtArgs &s, int64_t x0, int64_t m_s, int64_t m_e, int lane,
                                           const Sink &sink) {
    const int64_t W = s.W, W2 = W >> 1, H2 = s.H >> 1;
    const LaneCols c = lane_cols(x0, lane, W);
    const float *Z = static_cast<const float *>(s.src);
    if (WAV == 0) {
        auto ld = [&](int64_t m, float *ll, float *hl, float *lh, float *hh) {
            ll[0] = __ldg(Z + m * W + c.nB);              ll[1] = __ldg(Z + m * W + c.nC);
            hl[0] = __ldg(Z + m * W + W2 + c.nB);         hl[1] = __ldg(Z + m * W + W2 + c.nC);
            lh[0] = __ldg(Z + (H2 + m) * W + c.nB);       lh[1] = __ldg(Z + (H2 + m) * W + c.nC);
            hh[0] = __ldg(Z + (H2 + m) * W + W2 + c.nB);  hh[1] = __ldg(Z + (H2 + m) * W + W2 + c.nC);
        };
        auto emit = [&](int64_t m, int r, const float *ll, const float *hl, const float *lh, const float *hh) {
            // Eq. 11-12 on the columns, then on the rows
            float v0[4], v1[4];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float ua = ll[j] + lh[j], ub = ll[j] - lh[j];  // rows 2m, 2m+1, approx column
                const float da = hl[j] + hh[j], db = hl[j] - hh[j];  // rows 2m, 2m+1, detail column
                v0[2 * j] = ua + da;
                v0[2 * j + 1] = ua - da;
                v1[2 * j] = ub + db;
                v1[2 * j + 1] = ub - db;
            }
            sink.img(m, 2 * r, v0);
            sink.img(m, 2 * r + 1, v1);
        };
        for (int64_t m = m_s; m < m_e; m += 2) {  // two coefficient rows in flight
            const bool second = m + 1 < m_e;
            float ll[2], hl[2], lh[2], hh[2], ll2[2], hl2[2], lh2[2], hh2[2];
            ld(m, ll, hl, lh, hh);
            if (second) ld(m + 1, ll2, hl2, lh2, hh2);
            if (c.active) {
                emit(m, 0, ll, hl, lh, hh);
                if (second) emit(m, 1, ll2, hl2, lh2, hh2);
            }
            sink.step_end(m, second);
        }
        return;
    }
    float rap[4], rbp[4];  // RA, RB of coefficient row m-1
    {
        const int64_t mp = wrap(m_s - 1, H2);
        float L[3], G[3];
        load_coef3(Z + mp * W, c, L);
        load_coef3(Z + mp * W + W2, c, G);
        d4_row_syn(L, G, rap);
        load_coef3(Z + (H2 + mp) * W, c, L);
        load_coef3(Z + (H2 + mp) * W + W2, c, G);
        d4_row_syn(L, G, rbp);
    }
    // The next row's 12 coefficients are loaded one step ahead (the kernel
    // runs two CTAs per SM at its register count either way), so a warp's
    // loads overlap its arithmetic.
    float nL0[3], nG0[3], nL1[3], nG1[3];
    load_coef3(Z + m_s * W, c, nL0);
    load_coef3(Z + m_s * W + W2, c, nG0);
    load_coef3(Z + (H2 + m_s) * W, c, nL1);
    load_coef3(Z + (H2 + m_s) * W + W2, c, nG1);
    for (int64_t m = m_s; m < m_e; ++m) {
        float L0[3], G0[3], L1[3], G1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            L0[k] = nL0[k]; G0[k] = nG0[k]; L1[k] = nL1[k]; G1[k] = nG1[k];
        }
        if (m + 1 < m_e) {
            load_coef3(Z + (m + 1) * W, c, nL0);
            load_coef3(Z + (m + 1) * W + W2, c, nG0);
            load_coef3(Z + (H2 + m + 1) * W, c, nL1);
            load_coef3(Z + (H2 + m + 1) * W + W2, c, nG1);
        }
        float ra[4], rb[4];
        d4_row_syn(L0, G0, ra);
        d4_row_syn(L1, G1, rb);
        float v0[4], v1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // image row 2m: h0 RA(m) + h2 RA(m-1) + g0 RB(m) + g2 RB(m-1); row 2m+1: h1, h3, g1, g3
            v0[q] = fmaf(kG2, rbp[q], fmaf(kG0, rb[q], fmaf(kH2, rap[q], kH0 * ra[q])));
            v1[q] = fmaf(kG3, rbp[q], fmaf(kG1, rb[q], fmaf(kH3, rap[q], kH1 * ra[q])));
            rap[q] = ra[q];
            rbp[q] = rb[q];
        }
        if (c.active) {
            sink.img(m, 0, v0);
            sink.img(m, 1, v1);
        }
        sink.step_end(m, false);
    }
}

// Forward instances run four CTAs per SM (at most 64 registers), the
// inverse three (at most 85).
template <typename T, int WAV, bool INV>
__global__ void __launch_bounds__(kDwtThreads, INV ? 3 : 4)
dwt2_kernel(const __grid_constant__ DwtArgs s, int64_t strips_x, int64_t items, int R) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kDwtWarps;
    for (int64_t it = (int64_t)blockIdx.x * kDwtWarps + (threadIdx.x >> 5); it < items; it += nwarps) {
        const int64_t sx = it % strips_x, sy = it / strips_x;
        const int64_t m_s = sy * R;
        const int64_t m_e = min(m_s + (int64_t)R, s.H >> 1);
        const int64_t x0 = sx * kWarpCols;
        const LaneCols c = lane_cols(x0, lane, s.W);
        if (INV) {
            const InvDirect sink{OutPtrs{s.dst_f32, s.dst_u8}, s.W, c, s.a4 != 0};
            idwt2_item<WAV>(s, x0, m_s, m_e, lane, sink);
        } else {
            const FwdDirect sink{s.dst_f32, s.W, s.W >> 1, s.H >> 1, c, s.pairs != 0};
            dwt2_item<T, WAV>(s, x0, m_s, m_e, lane, sink);
        }
    }
}

// Staged forward: CTA items of 1024 image columns x R coefficient rows, it =
// blockIdx.x, + gridDim.x, ...; two shared-memory slots of the step's rows.
template <typename T, int WAV>
__global__ void __launch_bounds__(kDwtThreads, 4)
dwt2_staged_kernel(const __grid_constant__ DwtArgs s, int64_t strips_cta, int64_t items, int R) {
    extern __shared__ __align__(128) float dwt_buf[];
    constexpr int RS = WAV == 0 ? 2 : 1;  // coefficient rows per step
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int rowc = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t sx = it % strips_cta, sy = it / strips_cta;
        const int64_t X0 = sx * kDwtCols, x0 = X0 + (int64_t)warp * kWarpCols;
        const int64_t m_s = sy * R;
        const int64_t m_e = min(m_s + (int64_t)R, s.H >> 1);
        const LaneCols c = lane_cols(x0, lane, s.W);  // warps past W: idle lanes
        const int ncols = (int)min((int64_t)kDwtCols, s.W - X0);
        const FwdStaged<RS> sink{s.dst_f32, s.W, s.W >> 1, s.H >> 1, c, dwt_buf, &rowc, X0 >> 1, ncols >> 1};
        dwt2_item<T, WAV>(s, x0, m_s, m_e, lane, sink);
    }
    if (threadIdx.x < FwdStaged<RS>::kSegs) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

namespace {

const void *dwt_fn(bool inv, bool f32, int wav) {
    if (inv) return wav ? reinterpret_cast<const void *>(&dwt2_kernel<float, 1, true>)
                        : reinterpret_cast<const void *>(&dwt2_kernel<float, 0, true>);
    if (f32) return wav ? reinterpret_cast<const void *>(&dwt2_kernel<float, 1, false>)
                        : reinterpret_cast<const void *>(&dwt2_kernel<float, 0, false>);
    return wav ? reinterpret_cast<const void *>(&dwt2_kernel<uint8_t, 1, false>)
               : reinterpret_cast<const void *>(&dwt2_kernel<uint8_t, 0, false>);
}

const void *dwt_staged_fn(bool f32) {
    return f32 ? reinterpret_cast<const void *>(&dwt2_staged_kernel<float, 1>)
               : reinterpret_cast<const void *>(&dwt2_staged_kernel<uint8_t, 1>);
}

// The staged forward: D4 (Haar's forward, two coefficient rows a step with
// little arithmetic, measured slower staged: 16384^2 0.84 -> 0.74 of the copy
// peak), coefficient rows on the 16-byte grid (the right quadrants start W/2
// columns in, so W % 8 == 0) in a 16-byte-aligned plane, and a last
// 1024-column strip at least 7/8 full (idle warps would wait at every step's
// barrier).
bool dwt_staged_applies(const DwtLaunch &d) {
    if (d.inverse || d.wavelet != DWTFUSE_D4 || d.W % 8 != 0 || (reinterpret_cast<uintptr_t>(d.dst_f32) & 15) != 0)
        return false;
    const int64_t strips = (d.W + kDwtCols - 1) / kDwtCols;
    return (strips * kDwtCols - d.W) * 8 <= strips * kDwtCols;
}

cudaError_t launch_dwt2_staged(const DwtArgs &s, const DwtLaunch &d, cudaStream_t stream) {
    const void *fn = dwt_staged_fn(d.in_f32 != 0);
    const int segs = 4;  // quadrant rows of a step's coefficient row
    const int seg = kDwtCols / 2;
    const int smem = 2 * segs * seg * (int)sizeof(float);
    int occ = 0, sms = 0;
    cudaError_t e = resident_blocks_smem(fn, kDwtThreads, smem, &occ);
    if (e != cudaSuccess) return e;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    const int64_t cap = (int64_t)sms * occ, rows = d.H / 2;
    const int64_t strips = (d.W + kDwtCols - 1) / kDwtCols;
    int R = d.rows;
    if (R <= 0) {  // coefficient rows per CTA item that fill the last wave (+1: the D4 prologue)
        double best = 1e300;
        for (int r = 16; r <= 128; ++r) {
            const int64_t n = strips * ((rows + r - 1) / r);
            const double cost = (double)((n + cap - 1) / cap) * (r + 1);
            if (cost <= best) {
                best = cost;
                R = r;
            }
        }
    }
    const int64_t items = strips * ((rows + R - 1) / R);
    const unsigned grid = (unsigned)(items < cap ? items : cap);
    if (grid == 0) return cudaSuccess;
    DwtArgs sa = s;
    int64_t sv = strips, iv = items;
    void *args[] = {&sa, &sv, &iv, &R};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kDwtThreads), args, (size_t)smem, stream);
}

}  // namespace

cudaError_t launch_dwt2(const DwtLaunch &d, cudaStream_t stream) {
    DwtArgs s{};
    s.src = d.src;
    s.dst_f32 = d.dst_f32;
    s.dst_u8 = d.dst_u8;
    s.H = d.H;
    s.W = d.W;
    s.a4 = d.a4;
    s.pairs = d.pairs;
    if (dwt_staged_applies(d)) return launch_dwt2_staged(s, d, stream);
    const void *fn = dwt_fn(d.inverse != 0, d.in_f32 != 0, d.wavelet);
    int occ = 0, sms = 0;
    cudaError_t e = resident_blocks(fn, kDwtThreads, &occ);
    if (e != cudaSuccess) return e;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    const int64_t cap = (int64_t)sms * occ;
    int R = d.rows > 0 ? d.rows : balanced_rows(d.H, d.W, cap * kDwtWarps);
    const ItemGrid g = item_grid(d.H, d.W, R);
    const int64_t need = (g.items + kDwtWarps - 1) / kDwtWarps;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    if (grid == 0) return cudaSuccess;
    int64_t strips_x = g.strips_x, items = g.items;
    void *args[] = {&s, &strips_x, &items, &R};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kDwtThreads), args, 0, stream);
}

}  // namespace dwtfuse
