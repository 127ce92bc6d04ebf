// Quality metrics of the fused product (the paper reports ERGAS and QNR,
// Sec. 4 / Table 3, without defining them; definitions used here):
//   ERGAS = 100 * (1/2) * sqrt( (1/B) sum_b RMSE_b^2 / mu_b^2 ), reference MS_b
//           repeated 2x2 to PAN size, mu_b its mean, RMSE over all H x W pixels.
//   Q     = Wang-Bovik index 4 s_xy mu_x mu_y / ((s_x^2 + s_y^2)(mu_x^2 + mu_y^2))
//           on non-overlapping 32 x 32 windows at each image's own resolution
//           (ragged right/bottom edge dropped), averaged over windows; a zero
//           denominator gives 1 for identical windows, 0 otherwise.
//   D_lambda = mean over ordered band pairs |Q(F_l, F_r) - Q(MS_l, MS_r)|,
//   D_s      = mean over bands |Q(F_l, PAN) - Q(MS_l, PAN~)|, PAN~ = 2x2 block mean,
//   QNR      = (1 - D_lambda)(1 - D_s).
//
// Two passes over strips of 128 columns x 32 rows (four windows side by side,
// one warp each): the PAN-resolution pass reads the fused bands, PAN and MS
// (ERGAS squared errors, window sums of F_l, F_l^2, F_l F_r, F_l PAN); the
// MS-resolution pass reads MS and PAN (window sums against PAN~, and the MS
// means).  Every lane keeps all bands of its 4 pixels in registers, so the
// O(B^2) cross sums are register FMAs.
//
// Precision without FP64 in the pixel loop (FP64 is a narrow pipe on this
// GPU): values are shifted by 128.  For 8-bit data every window sum is an
// exact integer (FP32 up to 2^24 in the PAN pass; int32 in the MS pass, where
// PAN~ is carried as 4 * PAN~, an integer), the numerators n*Sxy - Sx*Sy and
// n*Sxx - Sx^2 are formed exactly in int64, and only the final ratio is FP32
// (relative error ~5e-7 per window).  Float data sum in FP32 and form the
// numerators in FP64.  Per-window Q values are accumulated in FP64 in shared
// memory; per-CTA partials go to the caller's workspace and a one-CTA kernel
// reduces them in a fixed order (deterministic).
#include <type_traits>

#include "fuse_tile.cuh"
#include "launch.h"
#include "metric_q.cuh"

namespace dwtfuse {

namespace {

constexpr int kMThreads = 256;
constexpr int kMWarps = kMThreads / 32;
constexpr int kWin = 32;
constexpr float kShift = 128.0f;

template <int NB>
struct Pairs {
    static constexpr int K = NB + 1;                 // images: NB bands + the PAN image
    static constexpr int P = NB * (NB - 1) / 2 + NB;  // band-band pairs, then band-PAN pairs
};

__device__ __forceinline__ void load4f(const uint8_t *p, bool a4, bool two, float *v) {
    if (a4) {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(p));
        v[0] = byte_f(w, 0); v[1] = byte_f(w, 1); v[2] = byte_f(w, 2); v[3] = byte_f(w, 3);
    } else {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned short *>(p));
        v[0] = byte_f(w, 0); v[1] = byte_f(w, 1);
        if (two) {
            const uint32_t u = __ldg(reinterpret_cast<const unsigned short *>(p + 2));
            v[2] = byte_f(u, 0); v[3] = byte_f(u, 1);
        } else {
            v[2] = v[3] = 0.f;
        }
    }
}
__device__ __forceinline__ void load4f(const float *p, bool a4, bool two, float *v) {
    if (a4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = q.x; v[1] = q.y;
        if (two) {
            const float2 u = __ldg(reinterpret_cast<const float2 *>(p + 2));
            v[2] = u.x; v[3] = u.y;
        } else {
            v[2] = v[3] = 0.f;
        }
    }
}
__device__ __forceinline__ float load1f(const uint8_t *p) { return (float)__ldg(p); }
__device__ __forceinline__ float load1f(const float *p) { return __ldg(p); }

constexpr int kN = kWin * kWin;  // pixels per window

__device__ __forceinline__ float xor_sum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}
__device__ __forceinline__ int xor_sum8(int v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

// Window sums of one image pair: x and y are the shifted values (x = X - 128),
// y carried as sy_scale * y (1, or 4 for PAN~ in the MS pass).
struct WinSums {
    double sx, sxx, sy, syy, sxy;
};

// Q of one window from float sums (float data): numerators in FP64.
__device__ __forceinline__ float q_float(float sx, float sxx, float sy, float syy, float sxy) {
    const double n = kN;
    const double vx = n * (double)sxx - (double)sx * (double)sx;
    const double vy = n * (double)syy - (double)sy * (double)sy;
    const double cxy = n * (double)sxy - (double)sx * (double)sy;
    const double ax = (double)sx + 128.0 * n, ay = (double)sy + 128.0 * n;
    const float den = (float)(vx + vy) * ((float)ax * (float)ax + (float)ay * (float)ay);
    if (den == 0.0f) {
        const double d2 = (double)sxx - 2.0 * (double)sxy + (double)syy;
        return (d2 == 0.0 && sx == sy) ? 1.0f : 0.0f;
    }
    return 4.0f * (float)cxy * (float)ax * (float)ay / den;
}

// Cross sums of one pixel: band-band pairs (b < c), then band-PAN pairs.
template <int NB, typename A>
__device__ __forceinline__ void accumulate_pixel(const A *v, A *s1, A *s2, A *sxy) {
#pragma unroll
    for (int k = 0; k <= NB; ++k) {
        s1[k] += v[k];
        s2[k] += v[k] * v[k];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c > b) sxy[pair_index(NB, b, c)] += v[b] * v[c];
#pragma unroll
    for (int b = 0; b < NB; ++b) sxy[NB * (NB - 1) / 2 + b] += v[b] * v[NB];
}

// After a strip: window sums over the 8 lanes of each window (every lane of
// the warp takes part), Q per pair on every lane, and the first lane of each
// full window adds its Q values to its shared slot.  `exact`: sums are exact
// integers; ys: scale of the last image (PAN or 4 * PAN~).
template <int NB, typename A>
__device__ __forceinline__ void finish_strip(const A *s1, const A *s2, const A *sxy, bool exact,
                                             int ys, bool leader, double *slot) {
    constexpr int K = NB + 1;
    A S1[K], S2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        S1[k] = xor_sum8(s1[k]);
        S2[k] = xor_sum8(s2[k]);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            // pairs in the order of accumulate_pixel: band-band first, then band-PAN
            if (c <= b) continue;
            const int p = pair_index(NB, b, c);
            const A Sxy = xor_sum8(sxy[p]);
            const float q = exact ? q_exact((long long)S1[b], (long long)S2[b], (long long)S1[c],
                                            (long long)S2[c], (long long)Sxy, 1)
                                  : q_float((float)S1[b], (float)S2[b], (float)S1[c], (float)S2[c], (float)Sxy);
            if (leader) slot[p] += (double)q;
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int idx = NB * (NB - 1) / 2 + b;
        const A Sxy = xor_sum8(sxy[idx]);
        const float q = exact ? q_exact((long long)S1[b], (long long)S2[b], (long long)S1[NB],
                                        (long long)S2[NB], (long long)Sxy, ys)
                              : q_float((float)S1[b], (float)S2[b], (float)S1[NB], (float)S2[NB], (float)Sxy);
        if (leader) slot[idx] += (double)q;
    }
}

struct MetricArgs {
    const void *fused;             // [B][H][W], TF
    const void *ms[kMaxBands];     // (H/2) x (W/2), TI
    const void *pan;               // H x W, TI (may be null when want_q == 0)
    double *partial;               // [gridDim][stride] per pass
    int64_t H, W;
    int32_t bands;
    int32_t want_q;
    int32_t a4_fused, a4_in;       // 4-pixel vector path allowed
    int32_t stride;                // doubles per CTA partial row
    int32_t wait_test;             // PAN pass, unaligned rows: warp 0 of CTA 0 posts 16 bytes never sent
};

// --------------------------------------------------------------- PAN-resolution pass

template <typename TF, typename TI, int NB>
__global__ void __launch_bounds__(kMThreads, 2)
metrics_pan_kernel(const __grid_constant__ MetricArgs a) {
    constexpr int K = Pairs<NB>::K, P = Pairs<NB>::P;
    // 8-bit data: shifted values are integers and every per-lane (<= 2^21) and
    // window (<= 2^24) sum is exact in FP32.
    constexpr bool kExact = std::is_same<TF, uint8_t>::value && std::is_same<TI, uint8_t>::value;
    __shared__ double sq[kMWarps][4][P];  // one slot per window of each warp's strip
    __shared__ double sse[kMWarps][NB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t H = a.H, W = a.W, W2 = W >> 1, HW = H * W;
    for (int k = lane; k < 4 * P; k += 32) sq[warp][k / P][k % P] = 0.0;
    double se_tot[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) se_tot[b] = 0.0;
    const TF *F = static_cast<const TF *>(a.fused);
    const TI *pan = static_cast<const TI *>(a.pan);
    const int64_t sx_n = (W + kWarpCols - 1) / kWarpCols, sy_n = (H + kWin - 1) / kWin;
    const int64_t items = sx_n * sy_n;
    const int64_t nw = (int64_t)gridDim.x * kMWarps;
    for (int64_t it = (int64_t)blockIdx.x * kMWarps + warp; it < items; it += nw) {
        const int64_t x = (it % sx_n) * kWarpCols + 4 * lane;
        const int64_t y0 = (it / sx_n) * kWin;
        const bool act = x < W, two = x + 2 < W;
        const int64_t xl = act ? x : 0;
        const int64_t xwin = x - 4 * (lane & 7);  // first column of this lane's window
        const bool full = a.want_q && (y0 + kWin <= H) && (xwin + kWin <= W);
        const int64_t y1 = min(y0 + (int64_t)kWin, H);
        float s1[K], s2[K], sxy[P], se[NB];
#pragma unroll
        for (int k = 0; k < K; ++k) s1[k] = s2[k] = 0.f;
#pragma unroll
        for (int k = 0; k < P; ++k) sxy[k] = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) se[b] = 0.f;
        for (int64_t y = y0; y < y1; ++y) {
            float f[NB][4], m[NB][2];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                load4f(F + (int64_t)b * HW + y * W + xl, a.a4_fused != 0, two, f[b]);
                const TI *mr = static_cast<const TI *>(a.ms[b]) + (y >> 1) * W2 + (xl >> 1);
                m[b][0] = load1f(mr);
                m[b][1] = two ? load1f(mr + 1) : 0.f;
            }
            float p[4];
            if (full) load4f(pan + y * W + xl, a.a4_in != 0, true, p);
            if (!act) continue;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float d = (q < 2 || two) ? f[b][q] - m[b][q >> 1] : 0.f;
                    se[b] = fmaf(d, d, se[b]);
                }
            }
            if (full) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v[K];
#pragma unroll
                    for (int b = 0; b < NB; ++b) v[b] = f[b][q] - kShift;
                    v[NB] = p[q] - kShift;
                    accumulate_pixel<NB>(v, s1, s2, sxy);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) se_tot[b] += (double)se[b];
        if (!__any_sync(0xffffffffu, full)) continue;
        finish_strip<NB, float>(s1, s2, sxy, kExact, 1, full && (lane & 7) == 0, sq[warp][lane >> 3]);
    }
    // Per-warp squared errors, then the CTA's partial row.
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double v = se_tot[b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sse[warp][b] = v;
    }
    __syncthreads();
    double *out = a.partial + (int64_t)blockIdx.x * a.stride;
    for (int k = threadIdx.x; k < P + NB; k += kMThreads) {
        double acc = 0.0;
        for (int w = 0; w < kMWarps; ++w)
            acc += k < P ? ((sq[w][0][k] + sq[w][1][k]) + (sq[w][2][k] + sq[w][3][k])) : sse[w][k - P];
        out[k] = acc;
    }
}

// --------------------------------------------------------------- 8-bit fast paths

// Programmatic dependent launch (sm_90+): a primary lets its dependent be
// scheduled; a dependent waits for its primary grid's completion and memory.
// Both are no-ops without the launch attribute.
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_primary() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Asynchronous global -> shared copy of one 16-byte chunk; bytes past
// `valid` are zero-filled (the source is not read there).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, unsigned valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Rows of unaligned planes (any width, any plane alignment) are staged with
// the bulk copy engine: the lane that owns a plane copies the 16-byte chunks of
// its row segment that lie inside the plane with one cp.async.bulk, which
// completes on the ring slot's mbarrier, so byte i of the segment lands at
// dst[(a0 & 15) + i].  The at most 15 bytes at either plane end that no
// in-plane chunk covers are copied with plain loads (bytes outside the plane
// are never read).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits (the whole warp) for the phase of `bar` with parity `parity`; gives up
// after about a second (the copies of one row take microseconds) and returns
// false, the same answer on every lane.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, unsigned parity) {
    bool done = mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (!done) done = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        unsigned late = global_ns() - t0 > 1000000000ull;
        if (__any_sync(0xffffffffu, late)) return false;
    }
}
static __device__ __noinline__ void stage_bytes(unsigned char *dst, uintptr_t c0, uintptr_t from, uintptr_t to) {
    for (uintptr_t p = from; p < to; ++p) dst[p - c0] = __ldg(reinterpret_cast<const uint8_t *>(p));
}
__device__ __forceinline__ void stage_row(unsigned char *dst, const uint8_t *a0, int len, const uint8_t *lo,
                                          const uint8_t *hi, uint64_t *bar) {
    const uintptr_t ua = reinterpret_cast<uintptr_t>(a0), c0 = ua & ~(uintptr_t)15, ue = ua + (uintptr_t)len;
    const uintptr_t ulo = reinterpret_cast<uintptr_t>(lo), uhi = reinterpret_cast<uintptr_t>(hi);
    uintptr_t bs = c0, be = (ue + 15) & ~(uintptr_t)15;
    if (bs < ulo) bs = (ulo + 15) & ~(uintptr_t)15;
    if (be > uhi) be = uhi & ~(uintptr_t)15;
    if (be > bs) {
        const unsigned n = (unsigned)(be - bs);
        mbar_expect_tx(bar, n);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                         smem_u32(dst + (bs - c0))),
                     "l"(reinterpret_cast<const void *>(bs)), "r"(n), "r"(smem_u32(bar))
                     : "memory");
        if (ua < bs) stage_bytes(dst, c0, ua, bs);
        if (be < ue) stage_bytes(dst, c0, be, ue);
    } else {
        stage_bytes(dst, c0, ua, ue);
    }
}

// Per-warp ring of row slots for the unaligned path: slot k's mbarrier
// completes when every bulk copy of the row staged there has landed (the one
// arrival is lane 0's, after all lanes have posted their byte counts).
template <int S>
struct BulkRing {
    uint64_t *bar;
    unsigned phase = 0;  // bit k: parity of slot k's next phase
    int issue_slot = 0, wait_slot = 0, pending = 0;
    __device__ __forceinline__ void init(uint64_t *bars, int lane) {
        bar = bars;
        if (lane == 0)
            for (int k = 0; k < S; ++k) mbar_init(bar + k);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        __syncwarp();
    }
    // after this lane staged its plane's row into slot issue_slot
    __device__ __forceinline__ void commit(int lane) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar + issue_slot);
        issue_slot = issue_slot + 1 == S ? 0 : issue_slot + 1;
        ++pending;
    }
    __device__ __forceinline__ bool wait() {
        const bool ok = mbar_wait_warp(bar + wait_slot, (phase >> wait_slot) & 1u);
        if (ok) {
            phase ^= 1u << wait_slot;
            wait_slot = wait_slot + 1 == S ? 0 : wait_slot + 1;
            --pending;
        }
        __syncwarp();
        return ok;
    }
    // After a wait gave up: wait (again bounded) for the other rows in flight.
    __device__ __forceinline__ void drain() {
        while (pending > 0) {
            mbar_wait_warp(bar + wait_slot, (phase >> wait_slot) & 1u);
            phase ^= 1u << wait_slot;
            wait_slot = wait_slot + 1 == S ? 0 : wait_slot + 1;
            --pending;
        }
    }
};

// NW 32-bit words of a staged row starting at byte offset off (one offset per
// image row, the same for every lane, so the branches are uniform).  Lanes
// sit 4 NW bytes apart.  An unaligned row is read as the NW + 1 words that
// cover it (NW <= 4), or as the aligned 16-byte pieces that cover it (NW = 8,
// where word loads would conflict 8 ways), and the words are shifted into
// place with funnel shifts.
template <int NW>
__device__ __forceinline__ void read_words(const unsigned char *base, int off, uint32_t *w) {
    if (NW % 4 == 0 && (off & 15) == 0) {
#pragma unroll
        for (int k = 0; k < NW / 4; ++k) {
            const uint4 q = *reinterpret_cast<const uint4 *>(base + off + 16 * k);
            w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
        }
        return;
    }
    if (NW == 2 && (off & 7) == 0) {
        const uint2 q = *reinterpret_cast<const uint2 *>(base + off);
        w[0] = q.x;
        w[1] = q.y;
        return;
    }
    const int sh = (off & 3) * 8;
    if constexpr (NW <= 4) {
        // lanes 4 NW bytes apart: word loads (2-way or 4-way bank conflicts)
        // and funnel shifts cost fewer instructions than selecting words out of
        // aligned vector loads
        const uint32_t *a = reinterpret_cast<const uint32_t *>(base + (off & ~3));
        uint32_t r[NW + 1];
#pragma unroll
        for (int k = 0; k <= NW; ++k) r[k] = a[k];
#pragma unroll
        for (int k = 0; k < NW; ++k) w[k] = __funnelshift_r(r[k], r[k + 1], sh);  // sh = 0: r[k]
    } else {
        static_assert(NW % 4 == 0, "read_words: NW is 2, 4 or a multiple of 4");
        const unsigned char *a = base + (off & ~15);
        const int s = off & 15;
        uint32_t r[NW + 4];
#pragma unroll
        for (int c = 0; c <= NW / 4; ++c) {
            const uint4 q = *reinterpret_cast<const uint4 *>(a + 16 * c);
            r[4 * c] = q.x; r[4 * c + 1] = q.y; r[4 * c + 2] = q.z; r[4 * c + 3] = q.w;
        }
        uint32_t t[NW + 3];
#pragma unroll
        for (int k = 0; k < NW + 3; ++k) t[k] = (s & 4) ? r[k + 1] : r[k];
#pragma unroll
        for (int k = 0; k <= NW; ++k) t[k] = (s & 8) ? t[k + 2] : t[k];
#pragma unroll
        for (int k = 0; k < NW; ++k) w[k] = __funnelshift_r(t[k], t[k + 1], sh);  // sh = 0: t[k]
    }
}

// Byte mask keeping the first `v` bytes of word q of a lane (v may exceed 4q+3).
__device__ __forceinline__ uint32_t keep_mask(int v, int q) {
    const int n = v - 4 * q;
    return n >= 4 ? 0xffffffffu : (n <= 0 ? 0u : (0xffffffffu >> (32 - 8 * n)));
}

// 8-bit product and inputs, any even width and plane alignment.  A lane owns
// 16 consecutive pixels of a row, a window is two lanes, a warp strip is 512
// columns (16 windows) x 32 rows.  Each warp streams its strip's rows through
// a ring of kStages rows in shared memory with cp.async, so several rows of
// every band are in flight without holding registers.  Shifted values are
// signed bytes (X ^ 0x80 = X - 128) and every sum is a dp4a over 4 pixels,
// exact in int32.
constexpr int kLanePx = 16;
constexpr int kStrip = 32 * kLanePx;
constexpr int kWinPerStrip = kStrip / kWin;
constexpr int kImgRow = kStrip + 32;       // staged bytes per image row (alignment slack, 16-aligned)
constexpr int kMsRow = kStrip / 2 + 32;    // staged bytes per MS row in the PAN pass
constexpr int kGenWarps = 12;              // warps per CTA, unaligned path, 7-8 bands

// Warps per CTA and ring depth: up to 6 bands, 16 warps with a 2-row ring
// (more warps hide the row-shifting work of unaligned widths and the state
// fits 128 registers); 7-8 bands, 8 warps with a 3-row ring, or on the
// unaligned path (kGenWarps) more warps with a 2-row ring.
template <int NB, bool GEN>
struct FastPan {
    static constexpr int K = NB + 1, P = NB * (NB - 1) / 2 + NB;
    static constexpr int kWarps = NB <= 6 ? 16 : (GEN ? kGenWarps : 8);
    static constexpr int kFastWarps = kWarps;
    static constexpr int kStages = NB <= 6 || GEN ? 2 : 3;
    static constexpr int kRowBytes = K * kImgRow + NB * kMsRow;
    static constexpr int kBarOffset = kFastWarps * kStages * kRowBytes + kFastWarps * kWinPerStrip * P * 4 +
                                      kFastWarps * NB * 8;
    static constexpr int kSmem = kBarOffset + kFastWarps * kStages * 8;  // with the mbarriers (GEN)
};

// GEN = false: rows of every plane start on 16-byte boundaries (W % 16 == 0,
// aligned planes): one cp.async chunk per lane and image, read back by the
// same lane.  GEN = true: any width and alignment; lane p stages plane p's row
// (fused bands, PAN, then the MS bands) with one bulk copy, and every lane
// shifts its words into place when it reads them.  A bulk-copy wait that gives
// up (about a second) stops the warp and is reported in the CTA's partial row
// (entry P + NB), which turns the figures into NaN.
template <int NB, bool GEN>
__global__ void __launch_bounds__(FastPan<NB, GEN>::kWarps * 32, 1)
metrics_pan_u8_kernel(const __grid_constant__ MetricArgs a) {
    allow_dependents();
    using C = FastPan<NB, GEN>;
    constexpr int kFastWarps = C::kWarps;
    constexpr int K = C::K, P = C::P, S = C::kStages, RB = C::kRowBytes;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *ring = smem + warp * S * RB;
    float *sq = reinterpret_cast<float *>(smem + kFastWarps * S * RB) + warp * kWinPerStrip * P;
    double *sse = reinterpret_cast<double *>(smem + kFastWarps * S * RB + kFastWarps * kWinPerStrip * P * 4);
    for (int k = lane; k < kWinPerStrip * P; k += 32) sq[k] = 0.f;
    double se_tot[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) se_tot[b] = 0.0;
    const int64_t H = a.H, W = a.W, W2 = W >> 1, H2 = H >> 1, HW = H * W;
    const uint8_t *F = static_cast<const uint8_t *>(a.fused);
    const uint8_t *pan = static_cast<const uint8_t *>(a.pan);
    const int64_t sx_n = (W + kStrip - 1) / kStrip, sy_n = (H + kWin - 1) / kWin;
    const int64_t items = sx_n * sy_n;
    const int64_t nw = (int64_t)gridDim.x * kFastWarps;
    // GEN: this lane's plane -- fused band `lane`, PAN (lane NB, when Q is
    // wanted), MS band lane - NB - 1 -- and where its rows go in a slot.
    BulkRing<S> br;
    const uint8_t *pl = nullptr;
    int64_t pl_n = 0;
    int kind = 0, dst_off = 0;  // kind 1: PAN-resolution row, 2: MS row
    bool err = false;
    bool stall = GEN && a.wait_test && blockIdx.x == 0 && warp == 0;  // test hook, first slot only
    if (GEN) {
        br.init(reinterpret_cast<uint64_t *>(smem + C::kBarOffset) + warp * S, lane);
        if (lane < NB) {
            pl = F + (int64_t)lane * HW; pl_n = HW; kind = 1; dst_off = lane * kImgRow;
        } else if (lane == NB) {
            if (a.want_q) { pl = pan; pl_n = HW; kind = 1; dst_off = NB * kImgRow; }
        } else if (lane <= 2 * NB) {
            const int b = lane - NB - 1;
            pl = static_cast<const uint8_t *>(a.ms[b]); pl_n = H2 * W2; kind = 2; dst_off = K * kImgRow + b * kMsRow;
        }
    }
    for (int64_t it = (int64_t)blockIdx.x * kFastWarps + warp; it < items; it += nw) {
        const int64_t x0 = (it % sx_n) * kStrip;
        const int64_t x = x0 + kLanePx * lane;
        const int64_t y0 = (it / sx_n) * kWin;
        const bool act = x < W;
        const int nval = act ? (int)min((int64_t)kLanePx, W - x) : 0;  // valid pixels of this lane
        const int64_t xwin = x - kLanePx * (lane & 1);
        const bool full = a.want_q && (y0 + kWin <= H) && (xwin + kWin <= W);
        const int nrows = (int)min((int64_t)kWin, H - y0);
        const int span = (int)min((int64_t)kStrip, W - x0);
        // Row r of this strip into the next ring slot (r % S on the aligned path).
        auto issue = [&](int r) {
            if (GEN) {
                if (r < nrows) {
                    unsigned char *slot = ring + br.issue_slot * RB;
                    const int64_t y = y0 + r;
                    if (kind == 1)
                        stage_row(slot + dst_off, pl + y * W + x0, span, pl, pl + pl_n, br.bar + br.issue_slot);
                    else if (kind == 2)
                        stage_row(slot + dst_off, pl + (y >> 1) * W2 + (x0 >> 1), span / 2, pl, pl + pl_n,
                                  br.bar + br.issue_slot);
                    if (stall) {
                        if (lane == 0) mbar_expect_tx(br.bar + br.issue_slot, 16u);
                        stall = false;
                    }
                    br.commit(lane);
                }
                return;
            }
            if (r < nrows) {
                unsigned char *slot = ring + (r % S) * RB;
                const int64_t y = y0 + r;
                if (act) {
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        cp_async16(slot + b * kImgRow + lane * 16, F + (int64_t)b * HW + y * W + x, 16u);
                    if (a.want_q) cp_async16(slot + NB * kImgRow + lane * 16, pan + y * W + x, 16u);
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        cp_async8(slot + K * kImgRow + b * kMsRow + lane * 8,
                                  static_cast<const uint8_t *>(a.ms[b]) + (y >> 1) * W2 + (x >> 1));
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int r = 0; r < S - 1; ++r) issue(r);
        int s1[K], s2[K], sxy[P], se[NB];
#pragma unroll
        for (int k = 0; k < K; ++k) s1[k] = s2[k] = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) sxy[k] = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) se[b] = 0;
        for (int r = 0; r < nrows; ++r) {
            const unsigned char *slot;
            const int64_t y = y0 + r;
            int my_o = 0;  // GEN: offset of this lane's plane row in its staged slot
            if (GEN) {
                __syncwarp();  // every lane is done with the slot refilled next
                issue(r + S - 1);
                const int rs = br.wait_slot;
                if (!br.wait()) {
                    err = true;
                    break;
                }
                slot = ring + rs * RB;
                const unsigned rowbase = kind == 2 ? (unsigned)(y >> 1) * (unsigned)W2 + (unsigned)(x0 >> 1)
                                                   : (unsigned)y * (unsigned)W + (unsigned)x0;
                my_o = (int)(((unsigned)reinterpret_cast<uintptr_t>(pl) + rowbase) & 15u);
            } else {
                issue(r + S - 1);
                cp_async_wait<S - 1>();
                slot = ring + (r % S) * RB;
            }
            int o_f[NB], o_m[NB], o_p = 0;
            if (GEN) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    o_f[b] = __shfl_sync(0xffffffffu, my_o, b);
                    o_m[b] = __shfl_sync(0xffffffffu, my_o, NB + 1 + b);
                }
                o_p = __shfl_sync(0xffffffffu, my_o, NB);
            }
            if (!act) continue;
            uint32_t f[NB][4], m[NB][2];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (GEN) {
                    read_words<4>(slot + b * kImgRow, o_f[b] + kLanePx * lane, f[b]);
                    read_words<2>(slot + K * kImgRow + b * kMsRow, o_m[b] + (kLanePx / 2) * lane, m[b]);
                } else {
                    const uint4 q4 = *reinterpret_cast<const uint4 *>(slot + b * kImgRow + lane * 16);
                    f[b][0] = q4.x; f[b][1] = q4.y; f[b][2] = q4.z; f[b][3] = q4.w;
                    const uint2 q2 = *reinterpret_cast<const uint2 *>(slot + K * kImgRow + b * kMsRow + lane * 8);
                    m[b][0] = q2.x; m[b][1] = q2.y;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t keep = GEN ? keep_mask(nval, q) : 0xffffffffu;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    // MS pixels 2q, 2q+1 of this lane, each repeated twice
                    const uint32_t rep = __byte_perm(m[b][q >> 1], 0u, (q & 1) ? 0x3322u : 0x1100u);
                    const uint32_t d = __vabsdiffu4(f[b][q], rep) & keep;
                    se[b] = (int)__dp4a(d, d, (unsigned)se[b]);
                }
            }
            if (full) {
                uint32_t pw[4];
                if (GEN) {
                    read_words<4>(slot + NB * kImgRow, o_p + kLanePx * lane, pw);
                } else {
                    const uint4 q4 = *reinterpret_cast<const uint4 *>(slot + NB * kImgRow + lane * 16);
                    pw[0] = q4.x; pw[1] = q4.y; pw[2] = q4.z; pw[3] = q4.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int v[K];
#pragma unroll
                    for (int b = 0; b < NB; ++b) v[b] = (int)(f[b][q] ^ 0x80808080u);
                    v[NB] = (int)(pw[q] ^ 0x80808080u);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        s1[k] = __dp4a(v[k], 0x01010101, s1[k]);
                        s2[k] = __dp4a(v[k], v[k], s2[k]);
                    }
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int c = 0; c < NB; ++c)
                            if (c > b) {
                                const int idx = pair_index(NB, b, c);
                                sxy[idx] = __dp4a(v[b], v[c], sxy[idx]);
                            }
#pragma unroll
                    for (int b = 0; b < NB; ++b) {
                        const int idx = NB * (NB - 1) / 2 + b;
                        sxy[idx] = __dp4a(v[b], v[NB], sxy[idx]);
                    }
                }
            }
        }
        if (GEN && err) {
            br.drain();
            break;
        }
        if (!GEN) cp_async_wait<0>();
#pragma unroll
        for (int b = 0; b < NB; ++b) se_tot[b] += (double)(unsigned)se[b];
        if (!__any_sync(0xffffffffu, full)) continue;
        // Window sums over the lane pair, Q per pair on every lane; the even
        // lane of a full window adds its Q values to its slot.
        int S1[K], S2[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            S1[k] = s1[k] + __shfl_xor_sync(0xffffffffu, s1[k], 1);
            S2[k] = s2[k] + __shfl_xor_sync(0xffffffffu, s2[k], 1);
        }
        const bool leader = full && (lane & 1) == 0;
        float *slotq = sq + (lane >> 1) * P;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c <= b) continue;
                const int idx = pair_index(NB, b, c);
                const int Sxy = sxy[idx] + __shfl_xor_sync(0xffffffffu, sxy[idx], 1);
                const float qv = q_exact(S1[b], S2[b], S1[c], S2[c], Sxy, 1);
                if (leader) slotq[idx] += qv;
            }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int idx = NB * (NB - 1) / 2 + b;
            const int Sxy = sxy[idx] + __shfl_xor_sync(0xffffffffu, sxy[idx], 1);
            const float qv = q_exact(S1[b], S2[b], S1[NB], S2[NB], Sxy, 1);
            if (leader) slotq[idx] += qv;
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double v = se_tot[b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sse[warp * NB + b] = v;
    }
    const int any_err = __syncthreads_or(err);
    const float *sq0 = reinterpret_cast<const float *>(smem + kFastWarps * S * RB);
    double *out = a.partial + (int64_t)blockIdx.x * a.stride;
    if (GEN && threadIdx.x == 0) out[P + NB] = any_err ? 1.0 : 0.0;
    for (int k = threadIdx.x; k < P + NB; k += kFastWarps * 32) {
        double acc = 0.0;
        for (int w = 0; w < kFastWarps; ++w) {
            if (k < P) {
                for (int s = 0; s < kWinPerStrip; ++s) acc += (double)sq0[(w * kWinPerStrip + s) * P + k];
            } else {
                acc += sse[w * NB + k - P];
            }
        }
        out[k] = acc;
    }
}

// MS-resolution pass: up to 6 bands, 8-warp CTAs, two per SM.  Against
// 16-warp CTAs, one per SM: faster alone (bench.py --case score_finish,
// 16384^2 x 6 0.155 -> 0.151 ms, 8192^2 0.076 -> 0.068 ms), and as a
// programmatic dependent of a primary with two CTAs per SM it can start when
// either of them has finished (step 1.687 -> 1.650 ms when the fused forward
// ran 8-warp CTAs; its 16-warp TMEM CTAs free whole SMs only).
template <int NB, bool GEN>
struct FastMs {
    static constexpr int K = NB + 1, P = NB * (NB - 1) / 2 + NB;
    static constexpr int kWarps = NB <= 6 ? 8 : (GEN ? kGenWarps : 8);
    static constexpr int kMinBlocks = NB <= 6 ? 2 : 1;
    static constexpr int kFastWarps = kWarps;
    static constexpr int kStages = NB <= 6 || GEN ? 2 : 3;
    static constexpr int kPanRow = 2 * kStrip + 32;  // 32 PAN pixels per lane
    static constexpr int kRowBytes = NB * kImgRow + 2 * kPanRow;
    static constexpr int kBarOffset = kFastWarps * kStages * kRowBytes + kFastWarps * kWinPerStrip * P * 4 +
                                      kFastWarps * NB * 8;
    static constexpr int kSmem = kBarOffset + kFastWarps * kStages * 8;  // with the mbarriers (GEN)
};

// Signed bytes of a times unsigned bytes of b, summed into c.
__device__ __forceinline__ int dp4a_su(int a, uint32_t b, int c) {
    int d;
    asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// MS-resolution pass, 8-bit: a lane owns 16 MS pixels of an MS row (and the
// 2 x 32 PAN pixels above them).  MS values are signed bytes (dp4a); PAN~ is
// carried as Z = 4 PAN~ - 512 (the 2x2 sum, exact).  The MS x PAN~ sums are
// taken as sum v (P_tl + P_tr + P_bl + P_br) by four mixed-sign dp4a over the
// words of the blocks' four corner pixels, and the -512 sum v term is
// subtracted from the window totals (sum v is the band's s1).
// GEN as for the PAN pass (aligned: W % 32 == 0, 16-byte aligned MS and PAN);
// on the GEN path lane b stages MS band b's row and lanes NB, NB + 1 the two
// PAN rows above it.
template <int NB, bool GEN>
__global__ void __launch_bounds__(FastMs<NB, GEN>::kWarps * 32, FastMs<NB, GEN>::kMinBlocks)
metrics_ms_u8_kernel(const __grid_constant__ MetricArgs a) {
    using C = FastMs<NB, GEN>;
    constexpr int kFastWarps = C::kWarps;
    constexpr int K = C::K, P = C::P, S = C::kStages, RB = C::kRowBytes, PR = C::kPanRow;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *ring = smem + warp * S * RB;
    float *sq = reinterpret_cast<float *>(smem + kFastWarps * S * RB) + warp * kWinPerStrip * P;
    double *ssum = reinterpret_cast<double *>(smem + kFastWarps * S * RB + kFastWarps * kWinPerStrip * P * 4);
    for (int k = lane; k < kWinPerStrip * P; k += 32) sq[k] = 0.f;
    double sum_tot[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) sum_tot[b] = 0.0;
    const int64_t H2 = a.H >> 1, W2 = a.W >> 1, W = a.W, HW = a.H * a.W;
    const uint8_t *pan = static_cast<const uint8_t *>(a.pan);
    const int64_t sx_n = (W2 + kStrip - 1) / kStrip, sy_n = (H2 + kWin - 1) / kWin;
    const int64_t items = sx_n * sy_n;
    const int64_t nw = (int64_t)gridDim.x * kFastWarps;
    BulkRing<S> br;
    const uint8_t *pl = nullptr;
    int64_t pl_n = 0;
    int kind = 0, dst_off = 0;  // kind 1: MS row, 2: PAN row 2i + (lane - NB)
    bool err = false;
    if (GEN) {
        br.init(reinterpret_cast<uint64_t *>(smem + C::kBarOffset) + warp * S, lane);
        if (lane < NB) {
            pl = static_cast<const uint8_t *>(a.ms[lane]); pl_n = H2 * W2; kind = 1; dst_off = lane * kImgRow;
        } else if (lane < NB + 2) {
            pl = pan; pl_n = HW; kind = 2; dst_off = NB * kImgRow + (lane - NB) * PR;
        }
    }
    for (int64_t it = (int64_t)warp * gridDim.x + blockIdx.x; it < items; it += nw) {  // items round the CTAs first
        const int64_t j0 = (it % sx_n) * kStrip;
        const int64_t j = j0 + kLanePx * lane;  // MS column
        const int64_t i0 = (it / sx_n) * kWin;
        const bool act = j < W2;
        const int nval = act ? (int)min((int64_t)kLanePx, W2 - j) : 0;
        const int64_t jwin = j - kLanePx * (lane & 1);
        const bool full = a.want_q && (i0 + kWin <= H2) && (jwin + kWin <= W2);
        const bool any_full = __any_sync(0xffffffffu, full);
        const int nrows = (int)min((int64_t)kWin, H2 - i0);
        const int span = (int)min((int64_t)kStrip, W2 - j0);
        auto issue = [&](int r) {
            if (GEN) {
                if (r < nrows) {
                    unsigned char *slot = ring + br.issue_slot * RB;
                    const int64_t i = i0 + r;
                    if (kind == 1)
                        stage_row(slot + dst_off, pl + i * W2 + j0, span, pl, pl + pl_n, br.bar + br.issue_slot);
                    else if (kind == 2 && any_full)
                        stage_row(slot + dst_off, pl + (2 * i + (lane - NB)) * W + 2 * j0, 2 * span, pl, pl + pl_n,
                                  br.bar + br.issue_slot);
                    br.commit(lane);
                }
                return;
            }
            if (r < nrows) {
                unsigned char *slot = ring + (r % S) * RB;
                const int64_t i = i0 + r;
                if (act) {
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        cp_async16(slot + b * kImgRow + lane * 16, static_cast<const uint8_t *>(a.ms[b]) + i * W2 + j, 16u);
                    if (full) {
                        const uint8_t *p0 = pan + (2 * i) * W + 2 * j;
                        cp_async16(slot + NB * kImgRow + lane * 32, p0, 16u);
                        cp_async16(slot + NB * kImgRow + lane * 32 + 16, p0 + 16, 16u);
                        cp_async16(slot + NB * kImgRow + PR + lane * 32, p0 + W, 16u);
                        cp_async16(slot + NB * kImgRow + PR + lane * 32 + 16, p0 + W + 16, 16u);
                    }
                }
            }
            cp_async_commit();
        };
#pragma unroll
        for (int r = 0; r < S - 1; ++r) issue(r);
        int s1[K], s2[K], sxy[P], sm[NB];
#pragma unroll
        for (int k = 0; k < K; ++k) s1[k] = s2[k] = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) sxy[k] = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) sm[b] = 0;
        for (int r = 0; r < nrows; ++r) {
            const unsigned char *slot;
            const int64_t i = i0 + r;
            int my_o = 0;  // GEN: offset of this lane's plane row in its staged slot
            if (GEN) {
                __syncwarp();  // every lane is done with the slot refilled next
                issue(r + S - 1);
                const int rs = br.wait_slot;
                if (!br.wait()) {
                    err = true;
                    break;
                }
                slot = ring + rs * RB;
                const unsigned rowbase = kind == 2 ? (unsigned)(2 * i + (lane - NB)) * (unsigned)W + (unsigned)(2 * j0)
                                                   : (unsigned)i * (unsigned)W2 + (unsigned)j0;
                my_o = (int)(((unsigned)reinterpret_cast<uintptr_t>(pl) + rowbase) & 15u);
            } else {
                issue(r + S - 1);
                cp_async_wait<S - 1>();
                slot = ring + (r % S) * RB;
            }
            int o_m[NB], o_p0 = 0, o_p1 = 0;
            if (GEN) {
#pragma unroll
                for (int b = 0; b < NB; ++b) o_m[b] = __shfl_sync(0xffffffffu, my_o, b);
                o_p0 = __shfl_sync(0xffffffffu, my_o, NB);
                o_p1 = __shfl_sync(0xffffffffu, my_o, NB + 1);
            }
            if (!act) continue;
            uint32_t mv[NB][4];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (GEN) {
                    read_words<4>(slot + b * kImgRow, o_m[b] + kLanePx * lane, mv[b]);
                } else {
                    const uint4 q4 = *reinterpret_cast<const uint4 *>(slot + b * kImgRow + lane * 16);
                    mv[b][0] = q4.x; mv[b][1] = q4.y; mv[b][2] = q4.z; mv[b][3] = q4.w;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    sm[b] = (int)__dp4a(GEN ? (mv[b][q] & keep_mask(nval, q)) : mv[b][q], 0x01010101u, (unsigned)sm[b]);
            }
            if (!full) continue;
            uint32_t r0[8], r1[8];
            if (GEN) {
                read_words<8>(slot + NB * kImgRow, o_p0 + 2 * kLanePx * lane, r0);
                read_words<8>(slot + NB * kImgRow + PR, o_p1 + 2 * kLanePx * lane, r1);
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(slot + NB * kImgRow + lane * 32 + 16 * k);
                    const uint4 v = *reinterpret_cast<const uint4 *>(slot + NB * kImgRow + PR + lane * 32 + 16 * k);
                    r0[4 * k] = u.x; r0[4 * k + 1] = u.y; r0[4 * k + 2] = u.z; r0[4 * k + 3] = u.w;
                    r1[4 * k] = v.x; r1[4 * k + 1] = v.y; r1[4 * k + 2] = v.z; r1[4 * k + 3] = v.w;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // PAN words of rows 2i, 2i+1 covering MS pixels 4q .. 4q+3
                const uint32_t ua = r0[2 * q], ub = r0[2 * q + 1], la = r1[2 * q], lb = r1[2 * q + 1];
                // the four corner pixels of MS pixels 4q .. 4q+3's PAN blocks
                const uint32_t ptl = __byte_perm(ua, ub, 0x6420u), ptr = __byte_perm(ua, ub, 0x7531u);
                const uint32_t pbl = __byte_perm(la, lb, 0x6420u), pbr = __byte_perm(la, lb, 0x7531u);
                int z[4];
                z[0] = (int)__dp4a(__byte_perm(ua, la, 0x5410u), 0x01010101u, 0u) - 512;
                z[1] = (int)__dp4a(__byte_perm(ua, la, 0x7632u), 0x01010101u, 0u) - 512;
                z[2] = (int)__dp4a(__byte_perm(ub, lb, 0x5410u), 0x01010101u, 0u) - 512;
                z[3] = (int)__dp4a(__byte_perm(ub, lb, 0x7632u), 0x01010101u, 0u) - 512;
                int v[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) v[b] = (int)(mv[b][q] ^ 0x80808080u);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    s1[b] = __dp4a(v[b], 0x01010101, s1[b]);
                    s2[b] = __dp4a(v[b], v[b], s2[b]);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    s1[NB] += z[t];
                    s2[NB] += z[t] * z[t];
                }
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int c = 0; c < NB; ++c)
                        if (c > b) {
                            const int idx = pair_index(NB, b, c);
                            sxy[idx] = __dp4a(v[b], v[c], sxy[idx]);
                        }
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int idx = NB * (NB - 1) / 2 + b;
                    // signed bytes of v[b] times the 2x2 PAN sums (the -512 part at the window total)
                    sxy[idx] = dp4a_su(v[b], pbr, dp4a_su(v[b], pbl, dp4a_su(v[b], ptr, dp4a_su(v[b], ptl, sxy[idx]))));
                }
            }
        }
        if (GEN && err) {
            br.drain();
            break;
        }
        if (!GEN) cp_async_wait<0>();
#pragma unroll
        for (int b = 0; b < NB; ++b) sum_tot[b] += (double)(unsigned)sm[b];
        if (!any_full) continue;
        int S1[K], S2[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            S1[k] = s1[k] + __shfl_xor_sync(0xffffffffu, s1[k], 1);
            S2[k] = s2[k] + __shfl_xor_sync(0xffffffffu, s2[k], 1);
        }
        const bool leader = full && (lane & 1) == 0;
        float *slotq = sq + (lane >> 1) * P;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c <= b) continue;
                const int idx = pair_index(NB, b, c);
                const int Sxy = sxy[idx] + __shfl_xor_sync(0xffffffffu, sxy[idx], 1);
                const float qv = q_exact(S1[b], S2[b], S1[c], S2[c], Sxy, 1);
                if (leader) slotq[idx] += qv;
            }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int idx = NB * (NB - 1) / 2 + b;
            const int Sxy = sxy[idx] + __shfl_xor_sync(0xffffffffu, sxy[idx], 1) - 512 * S1[b];
            const float qv = q_exact(S1[b], S2[b], S1[NB], S2[NB], Sxy, 4);
            if (leader) slotq[idx] += qv;
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double v = sum_tot[b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) ssum[warp * NB + b] = v;
    }
    const int any_err = __syncthreads_or(err);
    const float *sq0 = reinterpret_cast<const float *>(smem + kFastWarps * S * RB);
    double *out = a.partial + (int64_t)blockIdx.x * a.stride;
    if (GEN && threadIdx.x == 0) out[P + NB] = any_err ? 1.0 : 0.0;
    for (int k = threadIdx.x; k < P + NB; k += kFastWarps * 32) {
        double acc = 0.0;
        for (int w = 0; w < kFastWarps; ++w) {
            if (k < P) {
                for (int s = 0; s < kWinPerStrip; ++s) acc += (double)sq0[(w * kWinPerStrip + s) * P + k];
            } else {
                acc += ssum[w * NB + k - P];
            }
        }
        out[k] = acc;
    }
    wait_primary();  // a programmatic dependent completes only after its primary grid
}

// --------------------------------------------------------------- MS-resolution pass

template <typename TI, int NB>
__global__ void __launch_bounds__(kMThreads, 2)
metrics_ms_kernel(const __grid_constant__ MetricArgs a) {
    constexpr int K = Pairs<NB>::K, P = Pairs<NB>::P;
    // 8-bit data: integer accumulation, PAN~ carried as 4 * (PAN~ - 128).
    constexpr bool kExact = std::is_same<TI, uint8_t>::value;
    using Acc = typename std::conditional<kExact, int, float>::type;
    __shared__ double sq[kMWarps][4][P];
    __shared__ double ssum[kMWarps][NB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t H2 = a.H >> 1, W2 = a.W >> 1, W = a.W;
    for (int k = lane; k < 4 * P; k += 32) sq[warp][k / P][k % P] = 0.0;
    double sum_tot[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) sum_tot[b] = 0.0;
    const TI *pan = static_cast<const TI *>(a.pan);
    const int64_t sx_n = (W2 + kWarpCols - 1) / kWarpCols, sy_n = (H2 + kWin - 1) / kWin;
    const int64_t items = sx_n * sy_n;
    const int64_t nw = (int64_t)gridDim.x * kMWarps;
    for (int64_t it = (int64_t)blockIdx.x * kMWarps + warp; it < items; it += nw) {
        const int64_t j = (it % sx_n) * kWarpCols + 4 * lane;  // MS column
        const int64_t i0 = (it / sx_n) * kWin;
        const int64_t jwin = j - 4 * (lane & 7);
        const bool full = a.want_q && (i0 + kWin <= H2) && (jwin + kWin <= W2);
        const int64_t i1 = min(i0 + (int64_t)kWin, H2);
        Acc s1[K], s2[K], sxy[P];
        float sm[NB];
#pragma unroll
        for (int k = 0; k < K; ++k) s1[k] = s2[k] = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) sxy[k] = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) sm[b] = 0.f;
        for (int64_t i = i0; i < i1; ++i) {
            float v4[NB][4];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const TI *mr = static_cast<const TI *>(a.ms[b]) + i * W2;
#pragma unroll
                for (int q = 0; q < 4; ++q) v4[b][q] = (j + q < W2) ? load1f(mr + j + q) : 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) sm[b] += v4[b][q];
            }
            if (full) {
                // PAN~ from PAN rows 2i, 2i+1, columns 2j .. 2j+7.
                float r0[8], r1[8];
                load4f(pan + (2 * i) * W + 2 * j, a.a4_in != 0, true, r0);
                load4f(pan + (2 * i) * W + 2 * j + 4, a.a4_in != 0, true, r0 + 4);
                load4f(pan + (2 * i + 1) * W + 2 * j, a.a4_in != 0, true, r1);
                load4f(pan + (2 * i + 1) * W + 2 * j + 4, a.a4_in != 0, true, r1 + 4);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float s4 = (r0[2 * q] + r0[2 * q + 1]) + (r1[2 * q] + r1[2 * q + 1]);
                    Acc v[K];
                    if (kExact) {
#pragma unroll
                        for (int b = 0; b < NB; ++b) v[b] = (Acc)(v4[b][q] - kShift);
                        v[NB] = (Acc)(s4 - 4.0f * kShift);  // 4 * (PAN~ - 128), exact
                    } else {
#pragma unroll
                        for (int b = 0; b < NB; ++b) v[b] = (Acc)(v4[b][q] - kShift);
                        v[NB] = (Acc)(s4 * 0.25f - kShift);
                    }
                    accumulate_pixel<NB, Acc>(v, s1, s2, sxy);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) sum_tot[b] += (double)sm[b];
        if (!__any_sync(0xffffffffu, full)) continue;
        finish_strip<NB, Acc>(s1, s2, sxy, kExact, kExact ? 4 : 1, full && (lane & 7) == 0,
                              sq[warp][lane >> 3]);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double v = sum_tot[b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) ssum[warp][b] = v;
    }
    __syncthreads();
    double *out = a.partial + (int64_t)blockIdx.x * a.stride;
    for (int k = threadIdx.x; k < P + NB; k += kMThreads) {
        double acc = 0.0;
        for (int w = 0; w < kMWarps; ++w)
            acc += k < P ? ((sq[w][0][k] + sq[w][1][k]) + (sq[w][2][k] + sq[w][3][k])) : ssum[w][k - P];
        out[k] = acc;
    }
}

// --------------------------------------------------------------- finalize

// One CTA: sums the per-CTA partial rows and writes out[0..3] = ERGAS, QNR,
// D_lambda, D_s (QNR terms NaN when not requested or when no full window
// exists at either resolution; all four NaN when a pass flagged in
// `status_mask` (bit 0 PAN-resolution, bit 1 MS) reported a wait that gave up
// in entry P + nb of a partial row).  Each warp reduces one column of partials:
// lanes stride over the CTAs, then a xor butterfly (a fixed order, so the
// result is the same on every run).  The lane loop is unrolled so that its
// loads are in flight together: the partials sit in L2 and each round trip
// is a few hundred cycles.
constexpr int kFinalizeThreads = 1024;
__global__ void __launch_bounds__(kFinalizeThreads)
metrics_finalize_kernel(const double *pan_part, const double *ms_part, int ctas_pan, const int *ctas_pan_dev,
                        int ctas_ms, int stride, int nb, int want_q, int64_t H, int64_t W, int64_t nwin_pan,
                        int64_t nwin_ms, int status_mask, double *out) {
    if (ctas_pan_dev) ctas_pan = *ctas_pan_dev;
    __shared__ double tot_pan[64 + kMaxBands];
    __shared__ double tot_ms[64 + kMaxBands];
    const int P = nb * (nb - 1) / 2 + nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = warp; k < 2 * (P + nb + 1); k += nwarps) {
        const bool ms = k >= P + nb + 1;
        const int kk = ms ? k - (P + nb + 1) : k;
        const double *part = ms ? ms_part : pan_part;
        const int ctas = (kk < P + nb || ((status_mask >> (ms ? 1 : 0)) & 1)) ? (ms ? ctas_ms : ctas_pan) : 0;
        double a = 0.0;
#pragma unroll 8
        for (int c = lane; c < ctas; c += 32) a += part[(int64_t)c * stride + kk];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) (ms ? tot_ms : tot_pan)[kk] = a;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    // The FP64 divisions of the figures run one per lane (the FP64 pipe is
    // narrow; in one thread they would take most of this kernel's time), then
    // fixed butterflies sum them (the same order on every run).
    const int NBB = nb * (nb - 1) / 2;
    const bool q_ok = want_q && nwin_pan >= 1 && nwin_ms >= 1;
    double e = 0.0, dl = 0.0, ds = 0.0;
    if (lane < nb) {
        const double mse = tot_pan[P + lane] / ((double)H * (double)W);
        const double mu = tot_ms[P + lane] / ((double)(H / 2) * (double)(W / 2));
        e = mse / (mu * mu);
    }
    if (q_ok) {
        for (int k = lane; k < P; k += 32) {  // up to 36 pairs (8 bands)
            const double d = fabs(tot_pan[k] / (double)nwin_pan - tot_ms[k] / (double)nwin_ms);
            if (k < NBB) dl += d; else ds += d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        dl += __shfl_xor_sync(0xffffffffu, dl, o);
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
    }
    if (lane != 0) return;
    int *status = reinterpret_cast<int *>(out + kMetricStatusSlot);
    if (tot_pan[P + nb] + tot_ms[P + nb] > 0.0) {
        out[0] = out[1] = out[2] = out[3] = __longlong_as_double(0x7ff8000000000000ll);
        *status = DWTFUSE_ETIMEOUT;
        return;
    }
    *status = DWTFUSE_OK;
    out[0] = 100.0 * 0.5 * sqrt(e / nb);
    if (!q_ok) {
        out[1] = out[2] = out[3] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    dl = nb > 1 ? 2.0 * dl / (nb * (nb - 1)) : 0.0;
    ds /= nb;
    out[1] = (1.0 - dl) * (1.0 - ds);
    out[2] = dl;
    out[3] = ds;
}

template <typename TF, typename TI, int NB>
const void *pan_fn() { return reinterpret_cast<const void *>(&metrics_pan_kernel<TF, TI, NB>); }
template <typename TI, int NB>
const void *ms_fn() { return reinterpret_cast<const void *>(&metrics_ms_kernel<TI, NB>); }

template <typename TF, typename TI>
const void *pan_fn_nb(int nb) {
    switch (nb) {
        case 1: return pan_fn<TF, TI, 1>();
        case 2: return pan_fn<TF, TI, 2>();
        case 3: return pan_fn<TF, TI, 3>();
        case 4: return pan_fn<TF, TI, 4>();
        case 5: return pan_fn<TF, TI, 5>();
        case 6: return pan_fn<TF, TI, 6>();
        case 7: return pan_fn<TF, TI, 7>();
        default: return pan_fn<TF, TI, 8>();
    }
}
struct FastFn {
    const void *fn;
    int smem;
    int warps;
};
template <int NB, bool GEN>
FastFn pan_u8_fn() {
    return {reinterpret_cast<const void *>(&metrics_pan_u8_kernel<NB, GEN>),
            GEN ? FastPan<NB, GEN>::kSmem : FastPan<NB, GEN>::kBarOffset, FastPan<NB, GEN>::kWarps};
}
template <int NB, bool GEN>
FastFn ms_u8_fn() {
    return {reinterpret_cast<const void *>(&metrics_ms_u8_kernel<NB, GEN>),
            GEN ? FastMs<NB, GEN>::kSmem : FastMs<NB, GEN>::kBarOffset, FastMs<NB, GEN>::kWarps};
}
template <bool GEN>
FastFn fast_fn_g(bool ms_pass, int nb) {
    switch (nb) {
        case 1: return ms_pass ? ms_u8_fn<1, GEN>() : pan_u8_fn<1, GEN>();
        case 2: return ms_pass ? ms_u8_fn<2, GEN>() : pan_u8_fn<2, GEN>();
        case 3: return ms_pass ? ms_u8_fn<3, GEN>() : pan_u8_fn<3, GEN>();
        case 4: return ms_pass ? ms_u8_fn<4, GEN>() : pan_u8_fn<4, GEN>();
        case 5: return ms_pass ? ms_u8_fn<5, GEN>() : pan_u8_fn<5, GEN>();
        case 6: return ms_pass ? ms_u8_fn<6, GEN>() : pan_u8_fn<6, GEN>();
        case 7: return ms_pass ? ms_u8_fn<7, GEN>() : pan_u8_fn<7, GEN>();
        default: return ms_pass ? ms_u8_fn<8, GEN>() : pan_u8_fn<8, GEN>();
    }
}
FastFn fast_fn(bool ms_pass, int nb, bool aligned) {
    return aligned ? fast_fn_g<false>(ms_pass, nb) : fast_fn_g<true>(ms_pass, nb);
}

// Grid of a fast-path kernel: the resident CTAs (the row rings use most of
// shared memory), at most kMetricMaxCtas, fewer with fewer items.  spread:
// the kernel takes its items round the CTAs first and gets one CTA per item up
// to that cap, so a scene with fewer items than warps still reaches every SM
// (the MS-resolution pass: 8190^2 x 8 0.135 -> 0.119 ms, 16382^2 x 8 0.307 ->
// 0.270 ms; the PAN-resolution pass, whose CTAs each end with a wide partial
// row, ran slower that way and keeps items / warps CTAs).
cudaError_t fast_grid(const FastFn &f, int64_t items, int *grid, bool spread = false) {
    static_assert(kMetricMaxCtas >= 1, "");
    int occ = 0, sms = 0;
    cudaError_t e = resident_blocks_smem(f.fn, f.warps * 32, f.smem, &occ);
    if (e != cudaSuccess) return e;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    int64_t g = spread ? items : (items + f.warps - 1) / f.warps;
    const int64_t cap = (int64_t)sms * occ;
    if (g > cap) g = cap;
    if (g > kMetricMaxCtas) g = kMetricMaxCtas;
    if (g < 1) g = 1;
    *grid = (int)g;
    return cudaSuccess;
}

template <typename TI>
const void *ms_fn_nb(int nb) {
    switch (nb) {
        case 1: return ms_fn<TI, 1>();
        case 2: return ms_fn<TI, 2>();
        case 3: return ms_fn<TI, 3>();
        case 4: return ms_fn<TI, 4>();
        case 5: return ms_fn<TI, 5>();
        case 6: return ms_fn<TI, 6>();
        case 7: return ms_fn<TI, 7>();
        default: return ms_fn<TI, 8>();
    }
}

cudaError_t grid_for(const void *fn, int64_t items, int *grid) {
    int occ = 0, sms = 0;
    cudaError_t e = resident_blocks(fn, kMThreads, &occ);
    if (e != cudaSuccess) return e;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    int64_t g = (items + kMWarps - 1) / kMWarps;
    const int64_t cap = (int64_t)sms * occ;
    if (g > cap) g = cap;
    if (g > kMetricMaxCtas) g = kMetricMaxCtas;
    if (g < 1) g = 1;
    *grid = (int)g;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_metrics(const MetricLaunch &m, cudaStream_t stream) {
    MetricArgs a{};
    a.fused = m.fused;
    for (int b = 0; b < m.bands; ++b) a.ms[b] = m.ms[b];
    a.pan = m.pan;
    a.H = m.H;
    a.W = m.W;
    a.bands = m.bands;
    a.want_q = m.want_q;
    a.a4_fused = m.a4_fused;
    a.a4_in = m.a4_in;
    a.stride = kMetricStride;
    a.wait_test = m.wait_test;
    const bool fast = !m.fused_f32 && !m.in_f32;
    double *out = m.workspace;
    double *pan_part = m.workspace + kMetricPanPartialOffset;
    double *ms_part = pan_part + (int64_t)kMetricMaxCtas * kMetricStride;
    int gp = 0, gm = 0, status_mask = 0;
    cudaError_t e;
    // PAN-resolution pass (unless the fused forward + metrics kernel wrote it)
    if (m.pan_done) {
        e = cudaSuccess;
    } else if (fast) {
        const FastFn fp = fast_fn(false, m.bands, m.a16 != 0);
        if (!m.a16) status_mask |= 1;
        const int64_t items = ((m.W + kStrip - 1) / kStrip) * ((m.H + kWin - 1) / kWin);
        e = fast_grid(fp, items, &gp);
        if (e != cudaSuccess) return e;
        a.partial = pan_part;
        void *args[] = {&a};
        e = cudaLaunchKernel(fp.fn, dim3(gp), dim3(fp.warps * 32), args, fp.smem, stream);
    } else {
        const void *fp = m.fused_f32 ? (m.in_f32 ? pan_fn_nb<float, float>(m.bands) : pan_fn_nb<float, uint8_t>(m.bands))
                                     : (m.in_f32 ? pan_fn_nb<uint8_t, float>(m.bands) : pan_fn_nb<uint8_t, uint8_t>(m.bands));
        const int64_t items = ((m.W + kWarpCols - 1) / kWarpCols) * ((m.H + kWin - 1) / kWin);
        e = grid_for(fp, items, &gp);
        if (e != cudaSuccess) return e;
        a.partial = pan_part;
        void *args[] = {&a};
        e = cudaLaunchKernel(fp, dim3(gp), dim3(kMThreads), args, 0, stream);
    }
    if (e != cudaSuccess) return e;
    // MS-resolution pass
    MetricLaunch ml = m;
    if (!m.pan_done) ml.ms_early = 1;  // right after our own PAN-resolution pass
    MetricArgs b = a;
    b.partial = ms_part;
    void *args2[] = {&b};
    if (!m.in_f32) {
        const FastFn fm = fast_fn(true, m.bands, m.a32_ms != 0);
        if (!m.a32_ms) status_mask |= 2;
        const int64_t items = ((m.W / 2 + kStrip - 1) / kStrip) * ((m.H / 2 + kWin - 1) / kWin);
        e = fast_grid(fm, items, &gm, true);
        if (e != cudaSuccess) return e;
        // The MS pass reads only MS and PAN.  When the kernel before it on the
    // stream is the PAN-resolution pass or the fused forward + metrics kernel
    // (ms_early), it is launched as that kernel's programmatic dependent: its
    // CTAs start on SMs the primary has drained (the primary's last wave
    // leaves SMs idle), and it waits for the primary grid only before it
    // exits, so work after it still sees the primary's results.
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(gm);
        cfg.blockDim = dim3(fm.warps * 32);
        cfg.dynamicSmemBytes = (size_t)fm.smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = ml.ms_early ? 1 : 0;
        e = cudaLaunchKernelExC(&cfg, fm.fn, args2);
    } else {
        const void *fm = m.in_f32 ? ms_fn_nb<float>(m.bands) : ms_fn_nb<uint8_t>(m.bands);
        const int64_t items = ((m.W / 2 + kWarpCols - 1) / kWarpCols) * ((m.H / 2 + kWin - 1) / kWin);
        e = grid_for(fm, items, &gm);
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernel(fm, dim3(gm), dim3(kMThreads), args2, 0, stream);
    }
    if (e != cudaSuccess) return e;
    const int64_t nwp = (m.H / kWin) * (m.W / kWin), nwm = (m.H / 2 / kWin) * (m.W / 2 / kWin);
    const int *gp_dev = m.pan_done ? reinterpret_cast<const int *>(m.workspace + kMetricPanCtasSlot) : nullptr;
    metrics_finalize_kernel<<<1, kFinalizeThreads, 0, stream>>>(pan_part, ms_part, gp, gp_dev, gm, kMetricStride,
                                                                m.bands, m.want_q, m.H, m.W, nwp, nwm, status_mask,
                                                                out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (m.result && m.result != out)
        e = cudaMemcpyAsync(m.result, out, 4 * sizeof(double), cudaMemcpyDeviceToDevice, stream);
    return e;
}

}  // namespace dwtfuse
