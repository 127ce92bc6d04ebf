// Fused forward with the float output rows written by the bulk copy engine.
//
// The arithmetic is that of fuse_fwd.cu (Sec. 2, Eq. 1-16, through the warp
// walkers of fuse_tile.cuh); what changes is how the float rows reach HBM.
// A CTA of 8 warps owns a strip of 1024 PAN columns (its warps' 128-column
// strips side by side) and walks down its MS rows in step: for every MS row
// the lanes put their 4 float pixels of both PAN rows of every band into a
// shared-memory slot, the CTA meets at one barrier, and 2 NB threads each
// issue one cp.async.bulk (shared::cta -> global) of a 4 KB row segment.  The
// CTA's rows alternate between two slots (a count carried across work items,
// so consecutive rows never share one); the issuing threads wait
// (cp.async.bulk.wait_group.read) for their previous copies before the
// barrier of the next row, when those reads are long done, so the slot a row
// overwrites is free.  uint8 outputs keep the per-lane stores.
//
// Why: a warp's 16-byte-per-lane stores send a row segment to L2 as 4 line
// requests (5 when the row starts off the 128-byte line grid, with the
// segment's end sectors shared between two warps' requests); the bulk copy
// moves 4 KB per request stream and leaves only the CTA strip ends partial.
// Measured (16384 rows, 6 bands, float32 + uint8, CUDA events): W = 16384
// 6168 -> 6538 GB/s, W = 16380 5117 -> 6261, W = 16376 5729 -> 6307,
// W = 4092 5364 -> 6137.  A single slot with a second barrier per row (wait
// for the copies' reads, then release the slot) ran 5180-5330 GB/s on every
// width.
//
// Used for single scenes (fuse_staged_applies) with rows on the 16-byte grid
// (W % 4 == 0 with 16-byte-aligned float planes: every bulk copy starts on a
// 16-byte boundary and moves a multiple of 16 bytes) and at most
// kStagedMaxBands bands (two slots of 6 bands x 2 rows x 4 KB = 96 KB, two
// CTAs per SM); the band-chunk knob splits them further.
#include "fuse_tile.cuh"
#include "launch.h"

namespace dwtfuse {

namespace {

constexpr int kStThreads = 256;
constexpr int kStWarps = kStThreads / 32;
constexpr int kStCols = kStWarps * kWarpCols;  // 1024 PAN columns per CTA strip

__device__ __forceinline__ unsigned st_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// The issuing threads' bulk copies have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

template <int NB>
struct StagedEmit {
    static constexpr bool kAllLanes = true;  // every lane reaches the row barrier
    const SceneArgs &s;
    const LaneCols &c;
    float *buf;    // two slots of [NB][2][kStCols] floats
    int64_t X0;    // first column of the CTA strip
    int ncols;     // columns of the strip inside the image (a multiple of 4)
    int b0;        // first band of the launch's chunk
    int *rowc;     // the CTA's row count: row k fills slot k & 1

    __device__ __forceinline__ float *slot() const { return buf + (*rowc & 1) * (NB * 2 * kStCols); }

    __device__ __forceinline__ void band(int b, int64_t m, const float *v0, const float *v1, float, float) const {
        if (!c.active) return;
        const int col = c.x - (int)X0;
        float *row = slot() + b * 2 * kStCols + col;
        *reinterpret_cast<float4 *>(row) = make_float4(v0[0], v0[1], v0[2], v0[3]);
        *reinterpret_cast<float4 *>(row + kStCols) = make_float4(v1[0], v1[1], v1[2], v1[3]);
        if (s.out_u8) {
            const int64_t W = s.W, y = 2 * (m - s.m_lo);
            OutPtrs o{nullptr, s.out_u8 + (int64_t)(b0 + b) * s.out_plane};
            store4(o, y * W + c.x, true, c.two, v0);
            store4(o, (y + 1) * W + c.x, true, c.two, v1);
        }
    }

    __device__ __forceinline__ void row_end(int64_t m, const float *, const float *) const {
        // Make this thread's shared-memory writes visible to the bulk copy engine.
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int t = threadIdx.x;
        if (t < 2 * NB) bulk_wait_read();  // row m-1's copies: the slot row m+1 will fill
        __syncthreads();
        if (t < 2 * NB) {
            const int b = t >> 1, r = t & 1;
            const int64_t y = 2 * (m - s.m_lo) + r;
            float *dst = s.out_f32 + (int64_t)(b0 + b) * s.out_plane + y * s.W + X0;
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst),
                         "r"(st_smem(slot() + (b * 2 + r) * kStCols)), "r"((unsigned)ncols * 4u)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        }
        ++*rowc;
    }
};

// One CTA item: columns [X0, X0 + 1024), MS rows [m_s, m_e), bands
// [b0, b0 + NB).  Every thread of the CTA calls it, with the same row count.
template <typename T, int WAV, int NB>
__device__ __forceinline__ void staged_item(const SceneArgs &s, float *buf, int64_t X0, int64_t m_s, int64_t m_e,
                                            int b0, int *rowc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LaneCols c = lane_cols(X0 + (int64_t)warp * kWarpCols, lane, s.W);  // warps past W: idle lanes
    const int ncols = (int)min((int64_t)kStCols, s.W - X0);
    StagedEmit<NB> out{s, c, buf, X0, ncols, b0, rowc};
    if (WAV == 0)
        haar_rows<T, NB>(s, c, true, true, m_s, m_e, b0, NB, out);
    else
        d4_rows<T, NB>(s, c, true, true, m_s, m_e, b0, NB, out);
}

__device__ __forceinline__ void bulk_drain() {
    if (threadIdx.x < 2 * kStagedMaxBands) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

}  // namespace

// Single scene, bands [b0, b0 + NB); CTA items it = blockIdx.x, + gridDim.x, ...
template <typename T, int WAV, int NB>
__global__ void __launch_bounds__(kStThreads, 2)
fuse_staged_kernel(const __grid_constant__ SceneArgs s, int b0, int64_t strips_cta, int64_t items, int R) {
    extern __shared__ __align__(128) float st_buf[];
    int rowc = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t sx = it % strips_cta, sy = it / strips_cta;
        const int64_t m_s = s.m_lo + sy * R;
        staged_item<T, WAV, NB>(s, st_buf, sx * kStCols, m_s, min(m_s + (int64_t)R, (int64_t)s.m_hi), b0, &rowc);
    }
    bulk_drain();
}

namespace {

template <typename T, int WAV>
void *st_fn(int nb) {
    switch (nb) {
        case 1: return reinterpret_cast<void *>(&fuse_staged_kernel<T, WAV, 1>);
        case 2: return reinterpret_cast<void *>(&fuse_staged_kernel<T, WAV, 2>);
        case 3: return reinterpret_cast<void *>(&fuse_staged_kernel<T, WAV, 3>);
        case 4: return reinterpret_cast<void *>(&fuse_staged_kernel<T, WAV, 4>);
        case 5: return reinterpret_cast<void *>(&fuse_staged_kernel<T, WAV, 5>);
        case 6: return reinterpret_cast<void *>(&fuse_staged_kernel<T, WAV, 6>);
        default: return nullptr;
    }
}

constexpr int staged_smem(int nb) { return 2 * nb * 2 * kStCols * (int)sizeof(float); }

}  // namespace

// The staged kernel pays where a CTA's 8 warps, which meet at a barrier every
// MS row, rarely wait for one another: whole 1024-column strips (idle warps
// in a ragged last strip are lost time), and at most kStagedMaxBands bands
// (8 bands would run as two 4-band launches reading PAN twice, slower than
// the warp kernel's one).  Measured against the warp kernel (float32 out,
// bench.py --case fuse and single scenes of the 96-scene workload): 16384^2 x
// 6 6168 -> 6538 GB/s, 16384 x 4092 x 6 5364 -> 6137, 4958 x 7932 x 6 5728 ->
// 5728, 6408 x 2256 x 8 4875 -> 3804 (8 bands, a 3/4-empty last strip).  The
// same CTA items in the batched launch ran slower than its warp items on
// every scene class tried (46 scenes on the grid: 5356 -> 4651 GB/s; with the
// next item fetched during the current one and 64-row items: 4644), so the
// batched launch keeps warp items.
bool fuse_staged_applies(const SceneArgs &s) {
    if (s.a4 == 0 || s.out_f32 == nullptr || s.bands > kStagedMaxBands) return false;
    const int64_t strips = (s.W + kStCols - 1) / kStCols;
    return (strips * kStCols - s.W) * 8 <= strips * kStCols;
}

static int64_t staged_strips(int64_t W) { return (W + kStCols - 1) / kStCols; }

cudaError_t launch_fuse_staged(const SceneArgs &s, int R, cudaStream_t stream) {
    int cap = kStagedMaxBands;
    const int knob = fwd_band_chunk();
    if (knob > 0 && knob < cap) cap = knob;
    const int nchunks = (s.bands + cap - 1) / cap;
    const int chunk = (s.bands + nchunks - 1) / nchunks;  // balanced
    int sms = 0;
    cudaError_t e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    for (int b0 = 0; b0 < s.bands; b0 += chunk) {
        const int nb = s.bands - b0 < chunk ? s.bands - b0 : chunk;
        void *fn = s.in_f32 ? (s.wavelet ? st_fn<float, 1>(nb) : st_fn<float, 0>(nb))
                            : (s.wavelet ? st_fn<uint8_t, 1>(nb) : st_fn<uint8_t, 0>(nb));
        if (fn == nullptr) return cudaErrorInvalidValue;
        const int smem = staged_smem(nb);
        int occ = 0;
        e = resident_blocks_smem(fn, kStThreads, smem, &occ);
        if (e != cudaSuccess) return e;
        const int64_t capc = (int64_t)sms * occ;
        const int64_t rows = (int64_t)(s.m_hi - s.m_lo);
        const int64_t strips = staged_strips(s.W);
        int Rl = R;
        if (Rl <= 0) {  // MS rows per CTA item that fill the last wave (+1: the D4 prologue row)
            double best = 1e300;
            for (int r = 16; r <= 128; ++r) {
                const int64_t n = strips * ((rows + r - 1) / r);
                const double cost = (double)((n + capc - 1) / capc) * (r + 1);
                if (cost <= best) {
                    best = cost;
                    Rl = r;
                }
            }
        }
        const int64_t items = strips * ((rows + Rl - 1) / Rl);
        const unsigned grid = (unsigned)(items < capc ? items : capc);
        if (grid == 0) continue;
        SceneArgs sa = s;
        int b0v = b0;
        int64_t sv = strips, iv = items;
        void *args[] = {&sa, &b0v, &sv, &iv, &Rl};
        e = cudaLaunchKernel(fn, dim3(grid), dim3(kStThreads), args, (size_t)smem, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dwtfuse
