// Fused forward with the PAN-resolution half of the quality metrics in the
// same kernel.  The forward (Sec. 2, Eq. 1-16) is the one of fuse_fwd.cu; the
// metrics are those of metrics.cu (ERGAS squared errors against MS repeated
// 2x2, window sums of Q(F_l, F_r) and Q(F_l, PAN) over 32 x 32 windows, the
// paper's Sec. 4 / Table 3 scores).  Scoring the uint8 product while it is
// still on chip saves the metric pass's read of every fused band, of PAN and
// of MS (about a quarter of a benchmark step's HBM traffic).
//
// Work item: a warp strip of 128 PAN columns (four windows side by side, 8
// lanes each) over R MS rows, R a multiple of 16 and items starting on window
// rows.  Every SR MS rows (4 for up to 6 bands, else 2) the warp parks its
// uint8 pixels, the matching PAN pixels and the MS reference values in a
// per-warp shared tile (a private spill area: each lane reads back only its
// own words, so the fusion's registers are free again) and adds their terms
// to its running sums over the current window row (S1, S2 of every image,
// S_xy of every pair, squared errors: signed-byte dp4a sums, exact in int32).
// The running sums live in the lane's own cells of tensor memory (TMEM,
// tcgen05.ld / tcgen05.st): read, added to and written back without
// shared-memory traffic (7-8 bands in two or three passes over the parked
// words, fewer cells live at once).  At the end of a window row the 8 lanes of
// each window add their sums into the window's shared-memory sums, lane j of
// the window computes Q for pairs j, j + 8, ... (integer numerators, FP32
// ratio), and the value goes to a per-warp float slot of that window
// position; squared errors go to per-lane int64 slots.  The CTA writes one
// partial row in the layout of the separate PAN-resolution pass, so the
// MS-resolution pass and the finalize kernel of metrics.cu complete the
// figures unchanged.
//
// A CTA that holds TMEM runs alone on its SM: up to 7 bands a CTA is 16 warps
// (the SM's 64 K registers at 128 per thread), 8 bands 12 warps at up to 168
// registers (at 128 the 8-band walker spills).  Against per-lane
// shared-memory slots for the sums (8-warp CTAs, two per SM): 16384^2 x 6
// 1.525 -> 1.493 ms, 16384^2 x 7 2.212 -> 2.057 ms, 16382^2 x 8 2.805 ->
// 2.554 ms.
#include "fuse_tile.cuh"
#include "launch.h"
#include "metric_q.cuh"
#include "tmem.cuh"

namespace dwtfuse {

namespace {

constexpr int kFmWinMs = 16;  // MS rows per 32-row window row

constexpr int fm_pow2_at_least(int n, int lo) { return n <= lo ? lo : 2 * fm_pow2_at_least((n + 1) / 2, lo); }

// Bands b < c of band-band pair p (p < NB(NB-1)/2), in the order of the pair sums.
template <int NB>
__device__ __forceinline__ void pair_bands(int p, int &b, int &c) {
    b = 0;
    while (p >= NB - 1 - b) {
        p -= NB - 1 - b;
        ++b;
    }
    c = b + 1 + p;
}

// Band b of MS row m: parks its uint8 words of PAN rows 2m, 2m+1 in tile slot
// r (of SR) and its MS reference word, and writes the fused pixels.
template <int NB, int SR>
__device__ __forceinline__ void metric_band(const SceneArgs &s, const LaneCols &c, uint32_t *tile, uint32_t *rep,
                                            int lane, int r, bool a4, bool alt, int b, int64_t m,
                                            const float *v0, const float *v1, float mn, float mn1) {
    const uint32_t w0 = pack4(f2u8(v0[0]), f2u8(v0[1]), f2u8(v0[2]), f2u8(v0[3]));
    const uint32_t w1 = pack4(f2u8(v1[0]), f2u8(v1[1]), f2u8(v1[2]), f2u8(v1[3]));
    tile[(b * 2 * SR + 2 * r) * 32 + lane] = w0;
    tile[(b * 2 * SR + 2 * r + 1) * 32 + lane] = w1;
    // ERGAS reference: MS(m, n), MS(m, n+1) each repeated over 2 PAN columns.
    rep[(b * SR + r) * 32 + lane] = __byte_perm(f2u8(mn), f2u8(mn1), 0x4400u);
    const int64_t HW = s.H * s.W;
    const int64_t o0 = (int64_t)b * HW + (2 * m) * s.W + c.x, o1 = o0 + s.W;
    if (alt) {
        // Even row on the 16-byte grid (the lane at x = W-2 writes pairs),
        // odd row 2 pixels past it: every lane takes part in the shuffles.
        OutPtrs o{s.out_f32 ? s.out_f32 + (int64_t)b * HW : nullptr, s.out_u8 + (int64_t)b * HW};
        if (c.active) store4(o, (2 * m) * s.W + c.x, c.two, c.two, v0);
        store4_shifted(o, (2 * m + 1) * s.W + c.x, lane, c.active, c.two, c.last, v1);
        return;
    }
    if (!c.active) return;
    if (s.out_f32) {
        float *p0 = s.out_f32 + o0, *p1 = s.out_f32 + o1;
        if (a4) {
            __stcs(reinterpret_cast<float4 *>(p0), make_float4(v0[0], v0[1], v0[2], v0[3]));
            __stcs(reinterpret_cast<float4 *>(p1), make_float4(v1[0], v1[1], v1[2], v1[3]));
        } else {
            __stcs(reinterpret_cast<float2 *>(p0), make_float2(v0[0], v0[1]));
            __stcs(reinterpret_cast<float2 *>(p1), make_float2(v1[0], v1[1]));
            if (c.two) {
                __stcs(reinterpret_cast<float2 *>(p0 + 2), make_float2(v0[2], v0[3]));
                __stcs(reinterpret_cast<float2 *>(p1 + 2), make_float2(v1[2], v1[3]));
            }
        }
    }
    uint8_t *q0 = s.out_u8 + o0, *q1 = s.out_u8 + o1;
    if (a4) {
        __stcs(reinterpret_cast<unsigned int *>(q0), w0);
        __stcs(reinterpret_cast<unsigned int *>(q1), w1);
    } else {
        __stcs(reinterpret_cast<unsigned short *>(q0), (unsigned short)(w0 & 0xffffu));
        __stcs(reinterpret_cast<unsigned short *>(q1), (unsigned short)(w1 & 0xffffu));
        if (c.two) {
            __stcs(reinterpret_cast<unsigned short *>(q0 + 2), (unsigned short)(w0 >> 16));
            __stcs(reinterpret_cast<unsigned short *>(q1 + 2), (unsigned short)(w1 >> 16));
        }
    }
}

// PAN rows 2m, 2m+1 of the lane into tile slot r.
template <int NB, int SR>
__device__ __forceinline__ void metric_pan(uint32_t *tile, int lane, int r, const float *pan0, const float *pan1) {
    tile[(NB * 2 * SR + 2 * r) * 32 + lane] = pack4(f2u8(pan0[0]), f2u8(pan0[1]), f2u8(pan0[2]), f2u8(pan0[3]));
    tile[(NB * 2 * SR + 2 * r + 1) * 32 + lane] = pack4(f2u8(pan1[0]), f2u8(pan1[1]), f2u8(pan1[2]), f2u8(pan1[3]));
}

template <int NB>
struct FmLayout {
    static constexpr int K = NB + 1;                  // images: NB bands, then PAN
    static constexpr int P = NB * (NB - 1) / 2 + NB;  // band-band pairs (b < c), then band-PAN pairs
    static constexpr int NS = 2 * K + P;              // window sums per lane: S1[K], S2[K], Sxy[P]
    static constexpr int NT = NS + NB;                // TMEM cells per lane: window sums, squared errors
    // MS rows parked before they are scored (divides 16): 4 rows of 6 bands
    // take 12.4 KB of shared memory per warp; 7-8 bands park 2.
    static constexpr int SR = NB <= 6 ? 4 : 2;
    // One CTA per SM (it holds TMEM): 16 warps at up to 128 registers, 8
    // bands 12 warps at up to 168 (the 8-band walker spills at 128).
    static constexpr int kThreads = NB <= 7 ? 512 : 384;
    static constexpr int kWarps = kThreads / 32;
    // Per-warp shared memory (32-bit words, lane-minor so that lane accesses are conflict-free).
    static constexpr int kTile = K * 2 * SR * 32;     // uint8 words of 2 SR PAN rows: bands, PAN
    static constexpr int kRep = NB * SR * 32;         // MS reference words of SR MS rows
    static constexpr int kGsum = 4 * NS;              // window sums of the warp's 4 windows
    static constexpr int kQ = 4 * P;                  // float Q sums per window position
    static constexpr int kWords = (kTile + kRep + kGsum + kQ + 1) & ~1;
    static constexpr int kWarpBytes = kWords * 4 + NB * 32 * 8;  // + int64 squared errors per lane
    static constexpr int kSmem = kWarps * kWarpBytes + 16;     // + the TMEM base address
    // TMEM: warps w, w + 4, w + 8, ... share a quarter of the lanes, side by side.
    static constexpr int kWarpTmem = fm_pow2_at_least(NT, 16);
    static constexpr int kTmemCols = fm_pow2_at_least((kWarps + 3) / 4 * kWarpTmem, 32);
    static_assert(NT <= 64 && kTmemCols <= 512, "TMEM columns of an SM");
};

template <int NB>
struct MetricEmit {
    using L = FmLayout<NB>;
    static constexpr bool kAllLanes = true;
    static constexpr int K = L::K, P = L::P, NS = L::NS, SR = L::SR;
    const SceneArgs &s;
    const LaneCols &c;
    uint32_t *tile, *rep;
    int *gsum;
    float *qs;
    long long *se64;
    uint32_t taddr;  // this warp's TMEM cells
    int64_t x0, m_s, m_e;
    int lane;
    bool a4;
    bool alt;       // W % 4 == 2 with vector-aligned planes: even rows vectorised, odd rows shifted
    uint32_t keep;  // bytes of this lane's 4-pixel words inside the image
    bool fresh;     // the lane's TMEM sums start over (item start, after a window row)

    __device__ __forceinline__ void band(int b, int64_t m, const float *v0, const float *v1, float mn,
                                         float mn1) const {
        metric_band<NB, SR>(s, c, tile, rep, lane, (int)((m - m_s) & (SR - 1)), a4, alt, b, m, v0, v1, mn, mn1);
    }

    // Terms of the tile's first `nr` PAN rows for the cells [LO, HI) into
    // a[0, HI - LO), and with SE the squared errors into a[HI - LO, + NB).
    // Cells: S1[k] at k, S2[k] at K + k, Sxy[p] at 2K + p.
    template <int LO, int HI, bool SE>
    __device__ __forceinline__ void add_terms(uint32_t *a, int nr) const {
        for (int r = 0; r < nr; ++r) {
            uint32_t f[K];
#pragma unroll
            for (int k = 0; k < K; ++k) f[k] = tile[(k * 2 * SR + r) * 32 + lane];
            if constexpr (SE) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const uint32_t d = __vabsdiffu4(f[b], rep[(b * SR + (r >> 1)) * 32 + lane]) & keep;
                    a[HI - LO + b] = __dp4a(d, d, a[HI - LO + b]);
                }
            }
            int v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = (int)(f[k] ^ 0x80808080u);  // signed bytes X - 128
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k >= LO && k < HI) a[k - LO] = (uint32_t)__dp4a(v[k], 0x01010101, (int)a[k - LO]);
                if (K + k >= LO && K + k < HI) a[K + k - LO] = (uint32_t)__dp4a(v[k], v[k], (int)a[K + k - LO]);
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c2 = 0; c2 < NB; ++c2) {
                    const int q = 2 * K + pair_index(NB, b, c2);
                    if (c2 > b && q >= LO && q < HI) a[q - LO] = (uint32_t)__dp4a(v[b], v[c2], (int)a[q - LO]);
                }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int q = 2 * K + NB * (NB - 1) / 2 + b;
                if (q >= LO && q < HI) a[q - LO] = (uint32_t)__dp4a(v[b], v[NB], (int)a[q - LO]);
            }
        }
    }

    // The lane's cells [LO, HI) (and with SE its squared errors, cells
    // NS .. NS + NB): TMEM -> add the tile's terms -> TMEM; at the end of a
    // window row (fl) they go to the window's shared-memory sums (win_in: the
    // window lies inside the image) and the squared errors to int64 instead.
    template <int LO, int HI, bool SE>
    __device__ __forceinline__ void score_cells(int nr, bool fl, bool win_in) const {
        constexpr int N = HI - LO, NE = SE ? NB : 0;
        uint32_t a[N + NE];
        tm_wait_st();  // this lane's earlier stores to these cells are done (read or overwritten next)
        if (fresh) {
#pragma unroll
            for (int k = 0; k < N + NE; ++k) a[k] = 0;
        } else {
            tm_issue<N>(taddr + LO, a);
            if constexpr (SE) tm_issue<NB>(taddr + NS, a + N);
            tm_wait_ld<N + NE>(a);
        }
        add_terms<LO, HI, SE>(a, nr);
        if (!fl) {
            tm_store<N>(taddr + LO, a);
            if constexpr (SE) tm_store<NB>(taddr + NS, a + N);
            return;
        }
        if (win_in) {
            int *gs = gsum + (lane >> 3) * NS + LO;
#pragma unroll
            for (int k = 0; k < N; ++k) atomicAdd(gs + k, (int)a[k]);  // 8 lanes per window: exact in any order
        }
        if constexpr (SE) {
#pragma unroll
            for (int b = 0; b < NB; ++b) se64[b * 32 + lane] += (long long)a[N + b];
        }
    }

    // End of a window row: lane j of each window inside the image computes Q
    // for pairs j, j + 8, ... from the window's sums; the sums are cleared.
    __device__ __forceinline__ void finish_window(bool row_full) const {
        const int g = lane >> 3, j = lane & 7;
        __syncwarp();
        if (row_full && x0 + 32 * (g + 1) <= s.W) {
            const int *gs = gsum + g * NS;
            for (int p = j; p < P; p += 8) {
                int b, c2;
                if (p < P - NB) {
                    pair_bands<NB>(p, b, c2);
                } else {
                    b = p - (P - NB);
                    c2 = NB;
                }
                qs[g * P + p] += q_exact(gs[b], gs[K + b], gs[c2], gs[K + c2], gs[2 * K + p], 1);
            }
        }
        __syncwarp();
        for (int k = lane; k < 4 * NS; k += 32) gsum[k] = 0;
        __syncwarp();
    }

    __device__ __forceinline__ void row_end(int64_t m, const float *pan0, const float *pan1) {
        const int r = (int)((m - m_s) & (SR - 1));
        metric_pan<NB, SR>(tile, lane, r, pan0, pan1);
        const bool last = m + 1 == m_e;
        if (r != SR - 1 && !last) return;
        // Rows 2m' .. 2m+1 of the window row starting at PAN row y_win.
        const bool fl = (m - m_s + 1) % kFmWinMs == 0 || last;
        const int64_t y_win = ((2 * m) / 32) * 32;
        const bool row_full = y_win + 32 <= s.H;
        const bool win_in = row_full && x0 + 32 * ((lane >> 3) + 1) <= s.W;
        if constexpr (NB <= 6) {
            score_cells<0, NS, true>(2 * (r + 1), fl, win_in);
        } else if constexpr (NB == 7) {  // 7 bands: three passes over the parked words, fewer cells live at once
            constexpr int A = 2 * K, B = 2 * K + P / 2;
            score_cells<0, A, true>(2 * (r + 1), fl, win_in);
            score_cells<A, B, false>(2 * (r + 1), fl, win_in);
            score_cells<B, NS, false>(2 * (r + 1), fl, win_in);
        } else {
            constexpr int B = 2 * K + P / 2;
            score_cells<0, B, true>(2 * (r + 1), fl, win_in);
            score_cells<B, NS, false>(2 * (r + 1), fl, win_in);
        }
        fresh = fl;
        if (fl) finish_window(row_full);
    }
};

template <typename T, int WAV, int NB>
__global__ void __launch_bounds__(FmLayout<NB>::kThreads, 1)
fuse_metrics_kernel(const __grid_constant__ SceneArgs s, double *partial, int stride, int *ctas_out,
                    int64_t strips_x, int64_t items, int R) {
    using L = FmLayout<NB>;
    extern __shared__ __align__(16) unsigned char fm_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wb = fm_smem + warp * L::kWarpBytes;
    uint32_t *tile = reinterpret_cast<uint32_t *>(wb);
    uint32_t *rep = tile + L::kTile;
    int *gsum = reinterpret_cast<int *>(rep + L::kRep);
    float *qs = reinterpret_cast<float *>(gsum + L::kGsum);
    long long *se64 = reinterpret_cast<long long *>(wb + L::kWords * 4);
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(fm_smem + L::kWarps * L::kWarpBytes);
    // Let a programmatic dependent (the MS-resolution pass) be scheduled as
    // this grid drains (no-op without one).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctas_out = (int)gridDim.x;  // partial rows, for the finalize
    if (warp == 0) tmem_alloc(tmem_base, L::kTmemCols);
    for (int k = lane; k < L::kGsum; k += 32) gsum[k] = 0;
    for (int k = lane; k < L::kQ; k += 32) qs[k] = 0.f;
    for (int b = 0; b < NB; ++b) se64[b * 32 + lane] = 0;
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t taddr =
        *tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * L::kWarpTmem);

    // Items go round the CTAs first (warp w of CTA b starts at item w G + b,
    // G CTAs), so a scene with fewer items than warps still spreads over every SM.
    const int64_t nwarps = (int64_t)gridDim.x * L::kWarps;
    for (int64_t it = (int64_t)warp * gridDim.x + blockIdx.x; it < items; it += nwarps) {
        const int64_t sx = it % strips_x, sy = it / strips_x;
        const int64_t x0 = sx * kWarpCols;
        const int64_t m_s = sy * R;
        const int64_t m_e = min(m_s + (int64_t)R, s.H >> 1);
        const LaneCols c = lane_cols(x0, lane, s.W);
        const int64_t x = x0 + 4 * lane;
        const uint32_t keep = x + 4 <= s.W ? 0xffffffffu : (x + 2 <= s.W ? 0x0000ffffu : 0u);
        const bool a4 = s.a4 != 0, alt = !a4 && s.alt != 0;
        const bool lde = a4 || (alt && c.two);  // 4-pixel PAN loads on even rows
        MetricEmit<NB> out{s, c, tile, rep, gsum, qs, se64, taddr, x0, m_s, m_e, lane, a4, alt, keep, true};
        if (WAV == 0)
            haar_rows<T, NB>(s, c, lde, a4, m_s, m_e, 0, NB, out);
        else
            d4_rows<T, NB>(s, c, lde, a4, m_s, m_e, 0, NB, out);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(*tmem_base, L::kTmemCols);

    // One partial row per CTA, in the layout of the PAN-resolution pass:
    // Q sums of the P pairs, then the NB squared-error sums (fixed order).
    double *outp = partial + (int64_t)blockIdx.x * stride;
    for (int k = threadIdx.x; k < L::P + NB; k += L::kThreads) {
        double acc = 0.0;
        for (int w = 0; w < L::kWarps; ++w) {
            const unsigned char *wbw = fm_smem + w * L::kWarpBytes;
            if (k < L::P) {
                const float *qw = reinterpret_cast<const float *>(wbw) + L::kTile + L::kRep + L::kGsum;
                for (int g = 0; g < 4; ++g) acc += (double)qw[g * L::P + k];
            } else {
                const long long *sw = reinterpret_cast<const long long *>(wbw + L::kWords * 4);
                long long t = 0;
                for (int l = 0; l < 32; ++l) t += sw[(k - L::P) * 32 + l];
                acc += (double)t;
            }
        }
        outp[k] = acc;
    }
}

// ---------------------------------------------------------------- launch

struct FmKernel {
    void *fn;
    int threads, smem, tmem_cols;
};

template <int WAV, int NB>
FmKernel fm_of() {
    return {reinterpret_cast<void *>(&fuse_metrics_kernel<uint8_t, WAV, NB>), FmLayout<NB>::kThreads,
            FmLayout<NB>::kSmem, FmLayout<NB>::kTmemCols};
}

FmKernel fm_kernel(int wav, int nb) {
    switch (nb) {
#define DWTFUSE_FM(NBV) \
    case NBV:           \
        return wav ? fm_of<1, NBV>() : fm_of<0, NBV>();
        DWTFUSE_FM(1) DWTFUSE_FM(2) DWTFUSE_FM(3) DWTFUSE_FM(4) DWTFUSE_FM(5) DWTFUSE_FM(6)
        DWTFUSE_FM(7) DWTFUSE_FM(8)
#undef DWTFUSE_FM
        default: return {nullptr, 0, 0, 0};
    }
}

}  // namespace

bool fuse_metrics_supported(const SceneArgs &s) {
    return !s.in_f32 && s.out_u8 != nullptr && s.bands >= 1 && s.bands <= kFuseMetricsMaxBands;
}

cudaError_t launch_fuse_metrics(const SceneArgs &s, double *pan_partial, int stride, int *ctas_dev,
                                cudaStream_t stream) {
    const FmKernel k = fm_kernel(s.wavelet, s.bands);
    if (k.fn == nullptr || s.in_f32 || s.out_u8 == nullptr) return cudaErrorInvalidValue;
    int occ = 0, sms = 0;
    cudaError_t e = resident_blocks_smem(k.fn, k.threads, k.smem, &occ);
    if (e != cudaSuccess) return e;
    if (occ < 1 || occ * k.tmem_cols > 512) return cudaErrorInvalidConfiguration;  // TMEM columns of an SM
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    const int warps = k.threads / 32;
    const int64_t cap = (int64_t)sms * occ, wcap = cap * warps;
    // Rows per item: a multiple of the 16 MS rows of a window row, balancing the last wave.
    int R = kFmWinMs;
    double best = 1e300;
    for (int r = kFmWinMs; r <= 4 * kFmWinMs; r += kFmWinMs) {
        const ItemGrid g = item_grid(s.H, s.W, r);
        const double cost = (double)((g.items + wcap - 1) / wcap) * (r + 1);
        if (cost <= best) {
            best = cost;
            R = r;
        }
    }
    const ItemGrid g = item_grid(s.H, s.W, R);
    int64_t grid = g.items;  // every resident CTA, unless there are fewer items
    if (grid > cap) grid = cap;
    if (grid > kMetricMaxCtas) grid = kMetricMaxCtas;
    if (grid < 1) grid = 1;
    SceneArgs sa = s;
    int64_t strips_x = g.strips_x, items = g.items;
    int strd = stride, Rv = R;
    void *args[] = {&sa, &pan_partial, &strd, &ctas_dev, &strips_x, &items, &Rv};
    return cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(k.threads), args, (size_t)k.smem, stream);
}

}  // namespace dwtfuse
