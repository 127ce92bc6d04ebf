// Warp-strip tile machinery of the fused DWT pansharpening forward pass.
//
// Method (arXiv:1803.00737 Sec. 2): F_b = IDWT2(DWT2(P) with LL <- gain * M_b).
// The map is linear, so with L the low-pass half of the analysis matrix and U
// the synthesis of an LL-only coefficient image,
//     F_b = P + U(E_b),   E_b = gain * M_b - LL(P),   LL(P) = L_H P L_W^T.
// The detail subbands (HL, LH, HH) are never formed: they pass through
// unchanged, and the identity above is what remains of them.  LL(P) is
// computed once per tile and reused for every band.
//
//  Haar (Eq. 1-2, 11-12):  LL(i,j) = mean of the 2x2 block (i,j)  (rows, then
//                          columns, as the paper orders them), U = repeat 2x2.
//  D4   (Eq. 3-8, 13-16):  LL(i,j) = sum_{a,b} h_a h_b P(2i+a, 2j+b)   (mod H, W)
//                          U(E)(2m+r, 2n+q) = sum_{a,b in 0,1} h_{r+2a} h_{q+2b} E(m-a, n-b)
//
// Work unit: one warp owns a strip of 128 PAN columns (4 per lane: x..x+3,
// MS columns n = x/2 and n+1) and walks down R MS rows.  Everything stays in
// registers: D4 needs, per lane and PAN row, the 8 PAN columns x-2..x+5
// (periodic wrap at the image edges, Eq. 5-6 and 13-14), and a vertical
// pipeline keeps the row-synthesised values of MS row m-1 for row m.  Loads
// use the read-only path; fused rows are written with streaming stores.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dwtfuse {

constexpr int kWarpCols = 128;  // PAN columns per warp strip
constexpr int kMaxBands = 16;

// Daubechies-4 low-pass h of Eq. 7-8: (1+sqrt3, 3+sqrt3, 3-sqrt3, 1-sqrt3) / (4 sqrt2).
constexpr float kH0 = 0.48296291314453414f;
constexpr float kH1 = 0.83651630373780794f;
constexpr float kH2 = 0.22414386804201339f;
constexpr float kH3 = -0.12940952255126037f;

// ------------------------------------------------------------------ scalar helpers

// Exact uint8 -> float: place the byte in the mantissa of 2^23 and subtract.
__device__ __forceinline__ float byte_f(uint32_t word, int k) {
    return __int_as_float(__byte_perm(word, 0x4B000000u, 0x7440u | (uint32_t)k)) - 8388608.0f;
}

// float -> uint8: clamp to [0, 255], round half to even (cvt saturates).
__device__ __forceinline__ uint32_t f2u8(float v) {
    uint32_t r;
    asm("cvt.rni.sat.u8.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ uint32_t pack4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    return __byte_perm(__byte_perm(a, b, 0x0040u), __byte_perm(c, d, 0x0040u), 0x5410u);
}

__device__ __forceinline__ int64_t wrap(int64_t i, int64_t n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// ------------------------------------------------------------------ loads

// Two consecutive pixels starting at an even column (always in bounds).
__device__ __forceinline__ void ld2(const uint8_t *p, float &a, float &b) {
    const uint32_t w = __ldg(reinterpret_cast<const unsigned short *>(p));
    a = byte_f(w, 0);
    b = byte_f(w, 1);
}
__device__ __forceinline__ void ld2(const float *p, float &a, float &b) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    a = v.x;
    b = v.y;
}
// Four consecutive pixels starting at a column that is a multiple of 4 (aligned path).
__device__ __forceinline__ void ld4(const uint8_t *p, float *v) {
    const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(p));
    v[0] = byte_f(w, 0);
    v[1] = byte_f(w, 1);
    v[2] = byte_f(w, 2);
    v[3] = byte_f(w, 3);
}
__device__ __forceinline__ void ld4(const float *p, float *v) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ float ld1(const uint8_t *p) { return (float)__ldg(p); }
__device__ __forceinline__ float ld1(const float *p) { return __ldg(p); }

// ------------------------------------------------------------------ stores

struct OutPtrs {
    float *f32;   // band plane base or nullptr
    uint8_t *u8;  // band plane base or nullptr
};

// Writes the 4 fused pixels (y, x..x+3) of one band.  `two` = x+2 < W.
__device__ __forceinline__ void store4(const OutPtrs &o, int64_t off, bool a4, bool two,
                                       const float *v) {
    if (o.f32) {
        float *p = o.f32 + off;
        if (a4) {
            __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
        } else {
            __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
            if (two) __stcs(reinterpret_cast<float2 *>(p + 2), make_float2(v[2], v[3]));
        }
    }
    if (o.u8) {
        const uint32_t q0 = f2u8(v[0]), q1 = f2u8(v[1]), q2 = f2u8(v[2]), q3 = f2u8(v[3]);
        uint8_t *p = o.u8 + off;
        if (a4) {
            __stcs(reinterpret_cast<unsigned int *>(p), pack4(q0, q1, q2, q3));
        } else {
            __stcs(reinterpret_cast<unsigned short *>(p), (unsigned short)(q0 | (q1 << 8)));
            if (two) __stcs(reinterpret_cast<unsigned short *>(p + 2), (unsigned short)(q2 | (q3 << 8)));
        }
    }
}

// Writes the 4 fused pixels (y, x..x+3) of one band on a row whose start is 2
// pixels past a 16-byte boundary (W = 2 mod 4, odd rows): every lane but the
// first writes the aligned vector (y, x-2..x+1), taking pixels x-2, x-1 from
// its left neighbour; lane 0 writes (x, x+1) and the last lane of the strip
// (x + 4 >= W or lane 31) also writes (x+2, x+3).  Every lane of the warp must
// call it (warp shuffles); `active` masks the stores.
__device__ __forceinline__ void store4_shifted(const OutPtrs &o, int64_t off, int lane, bool active,
                                               bool two, bool last, const float *v) {
    if (o.f32) {
        const float p2 = __shfl_up_sync(0xffffffffu, v[2], 1);
        const float p3 = __shfl_up_sync(0xffffffffu, v[3], 1);
        if (active) {
            float *p = o.f32 + off;
            if (lane > 0)
                __stcs(reinterpret_cast<float4 *>(p - 2), make_float4(p2, p3, v[0], v[1]));
            else
                __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
            if (two && last) __stcs(reinterpret_cast<float2 *>(p + 2), make_float2(v[2], v[3]));
        }
    }
    if (o.u8) {
        const uint32_t q0 = f2u8(v[0]), q1 = f2u8(v[1]), q2 = f2u8(v[2]), q3 = f2u8(v[3]);
        const uint32_t w = pack4(q0, q1, q2, q3);
        const uint32_t pw = __shfl_up_sync(0xffffffffu, w, 1);
        if (active) {
            uint8_t *p = o.u8 + off;
            if (lane > 0)
                __stcs(reinterpret_cast<unsigned int *>(p - 2), __byte_perm(pw, w, 0x5432u));
            else
                __stcs(reinterpret_cast<unsigned short *>(p), (unsigned short)(w & 0xffffu));
            if (two && last) __stcs(reinterpret_cast<unsigned short *>(p + 2), (unsigned short)(w >> 16));
        }
    }
}

// ------------------------------------------------------------------ scene

// Everything a warp needs about one scene.  Band pointers are typed by the
// kernel template (TIn); the plane stride of the outputs is out_plane.
struct SceneArgs {
    const void *pan;
    const void *ms[kMaxBands];
    float *out_f32;
    uint8_t *out_u8;
    int64_t H, W;
    int32_t bands;
    int32_t wavelet;   // 0 Haar, 1 D4
    int32_t in_f32;    // inputs are float (else uint8)
    float gain;
    int32_t a4;        // W % 4 == 0 and PAN/outputs aligned for 4-pixel vectors
    int32_t alt;       // W % 4 == 2 with aligned planes: even rows aligned, odd rows 2 px past
    int64_t out_plane; // elements between output band planes (H * W for a whole scene)
    int32_t m_lo;      // MS rows [m_lo, m_hi) are fused; output row 0 belongs to MS row m_lo
    int32_t m_hi;      // (0 and H/2 for a whole scene; a row band's slab starts past its halo)
};

// Column bookkeeping of one lane for one strip (sides are < 2^20, so 32 bits).
struct LaneCols {
    int32_t x;           // first PAN column (even); clamped to 0 for idle lanes
    int32_t cm, c2, c4;  // wrapped starts of the pixel pairs x-2, x+2, x+4
    int32_t nA, nB, nC;  // MS columns n-1 (wrapped), n, n+1 (wrapped)
    bool active;         // x < W
    bool two;            // x + 2 < W (second MS column exists)
    bool last;           // last active lane of the strip (x + 4 >= W or lane 31)
};

__device__ __forceinline__ int32_t wrap32(int32_t i, int32_t n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

__device__ __forceinline__ LaneCols lane_cols(int64_t x0, int lane, int64_t W64) {
    LaneCols c;
    const int32_t W = (int32_t)W64;
    int32_t x = (int32_t)x0 + 4 * lane;
    c.active = x < W;
    if (!c.active) x = 0;
    c.x = x;
    c.two = x + 2 < W;
    c.last = lane == 31 || x + 4 >= W;
    c.cm = wrap32(x - 2, W);
    c.c2 = wrap32(x + 2, W);
    c.c4 = wrap32(x + 4, W);
    c.c4 = c.c4 >= W ? c.c4 - W : c.c4;
    const int32_t W2 = W >> 1, n = x >> 1;
    c.nA = wrap32(n - 1, W2);
    c.nB = n;
    c.nC = wrap32(n + 1, W2);
    return c;
}

// PAN row y: the 8 pixels x-2..x+5 (D4) with periodic wrap.
template <typename T>
__device__ __forceinline__ void load_row8(const T *row, const LaneCols &c, bool a4, float *v) {
    ld2(row + c.cm, v[0], v[1]);
    if (a4) {
        ld4(row + c.x, v + 2);
    } else {
        ld2(row + c.x, v[2], v[3]);
        ld2(row + c.c2, v[4], v[5]);
    }
    ld2(row + c.c4, v[6], v[7]);
}

// PAN row y: the 4 pixels x..x+3 (Haar; columns past W read column 0, unused).
template <typename T>
__device__ __forceinline__ void load_row4(const T *row, const LaneCols &c, bool a4, float *v) {
    if (a4) {
        ld4(row + c.x, v);
    } else {
        ld2(row + c.x, v[0], v[1]);
        ld2(row + c.c2, v[2], v[3]);
    }
}

// D4 row low-pass R(y, n') = sum_b h_b P(y, 2n'+b) for n' = n-1, n, n+1.
__device__ __forceinline__ void d4_rowpass(const float *v, float *r) {
    r[0] = fmaf(kH3, v[3], fmaf(kH2, v[2], fmaf(kH1, v[1], kH0 * v[0])));
    r[1] = fmaf(kH3, v[5], fmaf(kH2, v[4], fmaf(kH1, v[3], kH0 * v[2])));
    r[2] = fmaf(kH3, v[7], fmaf(kH2, v[6], fmaf(kH1, v[5], kH0 * v[4])));
}

// ------------------------------------------------------------------ row walkers
//
// A walker takes one lane's columns (LaneCols) down MS rows [m_s, m_e) and
// hands every band's two fused PAN rows 2m, 2m+1 (4 pixels per lane) to an
// emitter: out.band(b, m, v0, v1, mn, mn1) per band, with the band's MS values
// at MS columns n = x/2 and n+1 (the ones the lane's pixels were made from),
// then out.row_end(m, pan0, pan1) once per MS row with the lane's PAN pixels
// of rows 2m and 2m+1.  Emit::kAllLanes: the emitter needs every lane (warp
// shuffles), so idle lanes compute on column 0 and call it too.  ld_even /
// ld_odd select the 4-pixel PAN loads on even / odd rows.

// Haar (Eq. 1-2, 11-12).
template <typename T, int NB, class Emit>
__device__ __forceinline__ void haar_rows(const SceneArgs &s, const LaneCols &c, bool ld_even, bool ld_odd,
                                          int64_t m_s, int64_t m_e, int b0, int nb, Emit &out) {
    const int64_t W = s.W, W2 = W >> 1;
    const T *pan = static_cast<const T *>(s.pan);
    for (int64_t m = m_s; m < m_e; ++m) {
        float p0[4], p1[4];
        load_row4(pan + (2 * m) * W, c, ld_even, p0);
        load_row4(pan + (2 * m + 1) * W, c, ld_odd, p1);
        float mv[NB][2];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < nb) {
                const T *ms = static_cast<const T *>(s.ms[b0 + b]) + m * W2;
                mv[b][0] = ld1(ms + c.nB);
                mv[b][1] = ld1(ms + c.nC);
            }
        }
        if (!Emit::kAllLanes && !c.active) continue;
        // Eq. 1 along the rows, then along the columns: LL = 2x2 mean (exact in FP32 for 8-bit input).
        const float ll0 = ((p0[0] + p0[1]) * 0.5f + (p1[0] + p1[1]) * 0.5f) * 0.5f;
        const float ll1 = ((p0[2] + p0[3]) * 0.5f + (p1[2] + p1[3]) * 0.5f) * 0.5f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < nb) {
                // Eq. 11-12 on an LL-only image repeat each coefficient over its 2x2 block.
                const float e0 = fmaf(s.gain, mv[b][0], -ll0);
                const float e1 = fmaf(s.gain, mv[b][1], -ll1);
                float v[4] = {p0[0] + e0, p0[1] + e0, p0[2] + e1, p0[3] + e1};
                float w[4] = {p1[0] + e0, p1[1] + e0, p1[2] + e1, p1[3] + e1};
                out.band(b, m, v, w, mv[b][0], mv[b][1]);
            }
        }
        out.row_end(m, p0, p1);
    }
}

// D4 (Eq. 3-10, 13-16).
template <typename T, int NB, class Emit>
__device__ __forceinline__ void d4_rows(const SceneArgs &s, const LaneCols &c, bool ld_even, bool ld_odd,
                                        int64_t m_s, int64_t m_e, int b0, int nb, Emit &out) {
    const int64_t W = s.W, H = s.H, W2 = W >> 1, H2 = H >> 1;
    const T *pan = static_cast<const T *>(s.pan);
    const float gain = s.gain;

    // Prologue: MS row mp = m_s - 1 (periodic) needs PAN rows 2mp .. 2mp+3.
    const int64_t mp = wrap(m_s - 1, H2);
    float r0[3], r1[3], r2[3], r3[3];
    float pc[4], pd[4];  // own PAN pixels of rows 2m, 2m+1 for the current m
    {
        float v[8];
        load_row8(pan + (2 * mp) * W, c, ld_even, v);
        d4_rowpass(v, r0);
        load_row8(pan + (2 * mp + 1) * W, c, ld_odd, v);
        d4_rowpass(v, r1);
        load_row8(pan + wrap(2 * mp + 2, H) * W, c, ld_even, v);
        d4_rowpass(v, r2);
        pc[0] = v[2]; pc[1] = v[3]; pc[2] = v[4]; pc[3] = v[5];
        load_row8(pan + wrap(2 * mp + 3, H) * W, c, ld_odd, v);
        d4_rowpass(v, r3);
        pd[0] = v[2]; pd[1] = v[3]; pd[2] = v[4]; pd[3] = v[5];
    }
    // hprev[b][q]: row synthesis of E_b(m-1, .) at PAN column x+q.
    float hprev[NB][4];
    {
        float ll[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            ll[k] = fmaf(kH3, r3[k], fmaf(kH2, r2[k], fmaf(kH1, r1[k], kH0 * r0[k])));
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < nb) {
                const T *ms = static_cast<const T *>(s.ms[b0 + b]) + mp * W2;
                const float eA = fmaf(gain, ld1(ms + c.nA), -ll[0]);
                const float eB = fmaf(gain, ld1(ms + c.nB), -ll[1]);
                const float eC = fmaf(gain, ld1(ms + c.nC), -ll[2]);
                hprev[b][0] = fmaf(kH2, eA, kH0 * eB);
                hprev[b][1] = fmaf(kH3, eA, kH1 * eB);
                hprev[b][2] = fmaf(kH2, eB, kH0 * eC);
                hprev[b][3] = fmaf(kH3, eB, kH1 * eC);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) { r0[k] = r2[k]; r1[k] = r3[k]; }

    for (int64_t m = m_s; m < m_e; ++m) {
        // Loads first (PAN rows 2m+2, 2m+3 and every band's MS row m), so their
        // latencies overlap.
        float va[8], vb[8];
        load_row8(pan + wrap(2 * m + 2, H) * W, c, ld_even, va);
        load_row8(pan + wrap(2 * m + 3, H) * W, c, ld_odd, vb);
        float mv[NB][3];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < nb) {
                const T *ms = static_cast<const T *>(s.ms[b0 + b]) + m * W2;
                mv[b][0] = ld1(ms + c.nA);
                mv[b][1] = ld1(ms + c.nB);
                mv[b][2] = ld1(ms + c.nC);
            }
        }
        d4_rowpass(va, r2);
        d4_rowpass(vb, r3);
        float ll[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            ll[k] = fmaf(kH3, r3[k], fmaf(kH2, r2[k], fmaf(kH1, r1[k], kH0 * r0[k])));
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b < nb) {
                const float eA = fmaf(gain, mv[b][0], -ll[0]);
                const float eB = fmaf(gain, mv[b][1], -ll[1]);
                const float eC = fmaf(gain, mv[b][2], -ll[2]);
                // Row synthesis (Eq. 15-16 on an LL-only row, wrap of Eq. 13-14 via nA).
                float hc[4];
                hc[0] = fmaf(kH2, eA, kH0 * eB);
                hc[1] = fmaf(kH3, eA, kH1 * eB);
                hc[2] = fmaf(kH2, eB, kH0 * eC);
                hc[3] = fmaf(kH3, eB, kH1 * eC);
                // Column synthesis: row 2m takes h0 (row m) and h2 (row m-1), row 2m+1 takes h1 and h3.
                float v0[4], v1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v0[q] = fmaf(kH2, hprev[b][q], fmaf(kH0, hc[q], pc[q]));
                    v1[q] = fmaf(kH3, hprev[b][q], fmaf(kH1, hc[q], pd[q]));
                    hprev[b][q] = hc[q];
                }
                out.band(b, m, v0, v1, mv[b][1], mv[b][2]);
            }
        }
        out.row_end(m, pc, pd);
#pragma unroll
        for (int k = 0; k < 3; ++k) { r0[k] = r2[k]; r1[k] = r3[k]; }
        pc[0] = va[2]; pc[1] = va[3]; pc[2] = va[4]; pc[3] = va[5];
        pd[0] = vb[2]; pd[1] = vb[3]; pd[2] = vb[4]; pd[3] = vb[5];
    }
}

// ------------------------------------------------------------------ direct emitter

// Every lane writes its own 4 pixels to global memory.  ALT: the W % 4 == 2
// instance (even rows vectorised, odd rows through store4_shifted).
template <bool ALT>
struct DirectEmit {
    static constexpr bool kAllLanes = ALT;
    const SceneArgs &s;
    const LaneCols &c;
    int b0, lane;
    bool a4, a4e, alt;

    __device__ __forceinline__ void band(int b, int64_t m, const float *v0, const float *v1, float, float) const {
        const int64_t W = s.W, HW = s.out_plane, y = 2 * (m - s.m_lo);
        if constexpr (ALT) {
            OutPtrs o{s.out_f32 ? s.out_f32 + (int64_t)(b0 + b) * HW : nullptr,
                      s.out_u8 ? s.out_u8 + (int64_t)(b0 + b) * HW : nullptr};
            if (c.active) store4(o, y * W + c.x, a4e, c.two, v0);
            if (alt)
                store4_shifted(o, (y + 1) * W + c.x, lane, c.active, c.two, c.last, v1);
            else if (c.active)
                store4(o, (y + 1) * W + c.x, a4, c.two, v1);
        } else if (c.active) {
            OutPtrs o{s.out_f32 ? s.out_f32 + (int64_t)(b0 + b) * HW : nullptr,
                      s.out_u8 ? s.out_u8 + (int64_t)(b0 + b) * HW : nullptr};
            store4(o, y * W + c.x, a4, c.two, v0);
            store4(o, (y + 1) * W + c.x, a4, c.two, v1);
        }
    }
    __device__ __forceinline__ void row_end(int64_t, const float *, const float *) const {}
};

// One warp strip: 128 PAN columns from x0, MS rows [m_s, m_e), bands
// [b0, b0 + NB) (nb of them live), written directly.
template <typename T, int WAV, int NB, bool ALT>
__device__ __forceinline__ void direct_item(const SceneArgs &s, int64_t x0, int64_t m_s, int64_t m_e,
                                            int b0, int nb, int lane) {
    const LaneCols c = lane_cols(x0, lane, s.W);
    const bool a4 = s.a4 != 0;
    const bool alt = ALT && !a4 && s.alt != 0;  // even rows aligned, odd rows 2 pixels past
    // Vector path on even rows; the last lane (x = W-2) keeps the wrapped pair loads
    // and 2-pixel stores there.
    const bool a4e = a4 || (alt && c.two);
    DirectEmit<ALT> out{s, c, b0, lane, a4, a4e, alt};
    if (WAV == 0)
        haar_rows<T, NB>(s, c, a4e, a4, m_s, m_e, b0, nb, out);
    else
        d4_rows<T, NB>(s, c, a4e, a4, m_s, m_e, b0, nb, out);
}

// Geometry of a scene's work items: strips of 128 PAN columns times runs of R MS rows.
struct ItemGrid {
    int64_t strips_x, strips_y, items;
};

__host__ __device__ inline ItemGrid item_grid(int64_t H, int64_t W, int R) {
    ItemGrid g;
    g.strips_x = (W + kWarpCols - 1) / kWarpCols;
    g.strips_y = ((H >> 1) + R - 1) / R;
    g.items = g.strips_x * g.strips_y;
    return g;
}

// Runs work item `item` of a scene: WAV < 0 selects the wavelet at run time
// (batched kernel), 0 / 1 fixes Haar / D4 at compile time.  ALT compiles the
// shifted-row store path of widths W % 4 == 2 (taken when s.alt is set);
// without it such scenes use the scalar edge path.
template <typename T, int WAV, int NB, bool ALT = false>
__device__ __forceinline__ void run_item(const SceneArgs &s, int64_t item, int64_t strips_x, int R,
                                         int b0, int nb, int lane) {
    const int64_t sx = item % strips_x, sy = item / strips_x;
    const int64_t x0 = sx * kWarpCols;
    const int64_t m_s = s.m_lo + sy * R;
    const int64_t m_e = min(m_s + (int64_t)R, (int64_t)s.m_hi);
    if (WAV == 0 || (WAV < 0 && s.wavelet == 0))
        direct_item<T, 0, NB, ALT>(s, x0, m_s, m_e, b0, nb, lane);
    else
        direct_item<T, 1, NB, ALT>(s, x0, m_s, m_e, b0, nb, lane);
}

}  // namespace dwtfuse
