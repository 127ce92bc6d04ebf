// Fused forward kernels: the single-scene grid-stride kernel and the batched
// persistent kernel fed by a device-side work queue.
#include "fuse_tile.cuh"
#include "launch.h"

namespace dwtfuse {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kAltMaxBands = 6;  // widest band chunk of the shifted-row instance
constexpr int kBatchNarrowBands = 4;     // batched instance for tables of at most 4 bands per entry
constexpr int kBatchNarrowThreads = 320;  // ... and its CTA size (two per SM)

// Single scene, bands [b0, b0 + NB).  Each warp takes work items
// warp, warp + total_warps, ... (grid sized to the resident capacity).
// ALT: the instance for widths W % 4 == 2 with vector-aligned planes.
template <typename T, int WAV, int NB, bool ALT>
__global__ void __launch_bounds__(kThreads, 2)
fuse_fwd_kernel(const __grid_constant__ SceneArgs s, int b0, int64_t strips_x, int64_t items, int R) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t it = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); it < items; it += nwarps)
        run_item<T, WAV, NB, ALT>(s, it, strips_x, R, b0, NB, lane);
}

// Batched: every warp pulls the next item index from `queue[0]`; item ranges
// of the scenes are given by the prefix sums item_start[].  A warp whose
// scene table entry fails its checks records DWTFUSE_EDEVICE in status[0].
// MAXB: the most bands of a table entry the instance handles; its registers
// are those of its widest body, so a table of at most 4 bands per entry runs
// an instance of 4 with 320-thread CTAs (20 warps per SM at up to 96
// registers instead of 16 at 128).
template <int MAXB, int THREADS>
__global__ void __launch_bounds__(THREADS, 2)
fuse_batched_kernel(const __grid_constant__ BatchTable t, unsigned long long *queue, int *status) {
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
        const SceneArgs &s = t.scenes[lo];
        if (s.bands < 1 || s.bands > MAXB) {
            if (lane == 0) atomicCAS(status, 0, 7);
            continue;
        }
        const int64_t local = (int64_t)(it - (unsigned long long)t.item_start[lo]);
        const int64_t sx = t.strips_x[lo];
        // Exact band count: the same specialised item code as the single-scene
        // kernel (one of 32 bodies: wavelet x input type x 1..8 bands).
        const int nb = s.bands;
#define DWTFUSE_CASE(NBV)                                                                    \
    case NBV:                                                                                \
        if constexpr (NBV > MAXB) break;                                                     \
        if constexpr (NBV <= kBatchAltMaxBands) {                                            \
            if (s.alt && !s.a4) {                                                            \
                if (s.in_f32) {                                                              \
                    if (s.wavelet) run_item<float, 1, NBV, true>(s, local, sx, t.R, 0, NBV, lane);   \
                    else run_item<float, 0, NBV, true>(s, local, sx, t.R, 0, NBV, lane);             \
                } else {                                                                     \
                    if (s.wavelet) run_item<uint8_t, 1, NBV, true>(s, local, sx, t.R, 0, NBV, lane); \
                    else run_item<uint8_t, 0, NBV, true>(s, local, sx, t.R, 0, NBV, lane);           \
                }                                                                            \
                break;                                                                       \
            }                                                                                \
        }                                                                                    \
        if (s.in_f32) {                                                                      \
            if (s.wavelet) run_item<float, 1, NBV>(s, local, sx, t.R, 0, NBV, lane);         \
            else run_item<float, 0, NBV>(s, local, sx, t.R, 0, NBV, lane);                   \
        } else {                                                                             \
            if (s.wavelet) run_item<uint8_t, 1, NBV>(s, local, sx, t.R, 0, NBV, lane);       \
            else run_item<uint8_t, 0, NBV>(s, local, sx, t.R, 0, NBV, lane);                 \
        }                                                                                    \
        break;
        switch (nb) {
            DWTFUSE_CASE(1) DWTFUSE_CASE(2) DWTFUSE_CASE(3) DWTFUSE_CASE(4)
            DWTFUSE_CASE(5) DWTFUSE_CASE(6) DWTFUSE_CASE(7) DWTFUSE_CASE(8)
            default: break;
        }
#undef DWTFUSE_CASE
    }
}

// ------------------------------------------------------------------ host side

namespace {

template <typename T, int WAV, int NB>
void *fwd_fn(bool alt) {
    if constexpr (NB <= kAltMaxBands)
        if (alt) return reinterpret_cast<void *>(&fuse_fwd_kernel<T, WAV, NB, true>);
    return alt ? nullptr : reinterpret_cast<void *>(&fuse_fwd_kernel<T, WAV, NB, false>);
}

template <typename T, int WAV>
void *fwd_fn_nb(int nb, bool alt) {
    switch (nb) {
        case 1: return fwd_fn<T, WAV, 1>(alt);
        case 2: return fwd_fn<T, WAV, 2>(alt);
        case 3: return fwd_fn<T, WAV, 3>(alt);
        case 4: return fwd_fn<T, WAV, 4>(alt);
        case 5: return fwd_fn<T, WAV, 5>(alt);
        case 6: return fwd_fn<T, WAV, 6>(alt);
        case 7: return fwd_fn<T, WAV, 7>(alt);
        case 8: return fwd_fn<T, WAV, 8>(alt);
        default: return nullptr;
    }
}

void *fwd_kernel_ptr(bool f32, int wav, int nb, bool alt) {
    if (f32) return wav ? fwd_fn_nb<float, 1>(nb, alt) : fwd_fn_nb<float, 0>(nb, alt);
    return wav ? fwd_fn_nb<uint8_t, 1>(nb, alt) : fwd_fn_nb<uint8_t, 0>(nb, alt);
}

}  // namespace

cudaError_t launch_fuse(const SceneArgs &s, int R, int blocks_per_sm, cudaStream_t stream) {
    // Large scenes whose rows lie on the 16-byte grid with a float output: the
    // staged kernel (its float rows go out as bulk copies).
    if (fuse_staging() && fuse_staged_applies(s)) return launch_fuse_staged(s, R, stream);
    // Bands go in chunks of up to 8; the shifted-row instance (W % 4 == 2)
    // holds more live registers per band and takes balanced chunks of <= 6;
    // a band-chunk knob (autotuner) caps both, in balanced chunks.
    const bool alt = s.alt != 0 && s.a4 == 0;
    const int knob = fwd_band_chunk();
    int cap = alt ? kAltMaxBands : kChunkBands;
    if (knob > 0 && knob < cap) cap = knob;
    const int nchunks = (s.bands + cap - 1) / cap;
    const int chunk = (alt || knob > 0) ? (s.bands + nchunks - 1) / nchunks : kChunkBands;
    for (int b0 = 0; b0 < s.bands; b0 += chunk) {
        const int nb = s.bands - b0 < chunk ? s.bands - b0 : chunk;
        void *fn = fwd_kernel_ptr(s.in_f32 != 0, s.wavelet, nb, alt);
        if (fn == nullptr) return cudaErrorInvalidValue;
        int occ = 0;
        cudaError_t e = resident_blocks(fn, kThreads, &occ);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
        int sms = 0;
        e = sm_count(&sms);
        if (e != cudaSuccess) return e;
        const int64_t cap = (int64_t)sms * occ;
        // Items cover the MS rows [m_lo, m_hi) (all of them for a whole scene).
        const int64_t rows2 = 2 * (int64_t)(s.m_hi - s.m_lo);
        int Rl = R > 0 ? R : balanced_rows(rows2, s.W, cap * kWarps);
        const ItemGrid g = item_grid(rows2, s.W, Rl);
        const int64_t need = (g.items + kWarps - 1) / kWarps;
        const unsigned grid = (unsigned)(need < cap ? need : cap);
        if (grid == 0) continue;
        SceneArgs sa = s;
        int64_t strips_x = g.strips_x, items = g.items;
        void *args[] = {&sa, (void *)&b0, &strips_x, &items, &Rl};
        e = cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, 0, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

// One launch over table t: the narrow instance when every entry has at most
// kBatchNarrowBands bands.  clear: bytes of the queue word(s) to zero first
// (the queue counter and status word, or only the counter so that a status an
// earlier launch of the same call recorded survives).
cudaError_t launch_table(const BatchTable &t, unsigned long long *queue, int *status, int blocks_per_sm,
                         size_t clear, cudaStream_t stream) {
    int maxb = 0;
    for (int i = 0; i < t.n; ++i) maxb = t.scenes[i].bands > maxb ? t.scenes[i].bands : maxb;
    const bool narrow = maxb <= kBatchNarrowBands;
    const int threads = narrow ? kBatchNarrowThreads : kThreads;
    void *fn = narrow ? reinterpret_cast<void *>(&fuse_batched_kernel<kBatchNarrowBands, kBatchNarrowThreads>)
                      : reinterpret_cast<void *>(&fuse_batched_kernel<kBatchMaxBands, kThreads>);
    int occ = 0;
    cudaError_t e = resident_blocks(fn, threads, &occ);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
    int sms = 0;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(queue, 0, clear, stream);
    if (e != cudaSuccess) return e;
    const int64_t total = t.item_start[t.n];
    const int64_t need = (total + threads / 32 - 1) / (threads / 32);
    const int64_t cap = (int64_t)sms * occ;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    if (grid == 0) return cudaSuccess;
    void *args[] = {const_cast<BatchTable *>(&t), &queue, &status};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, stream);
}

// The entries of t with (narrow) or without at most kBatchNarrowBands bands.
void split_table(const BatchTable &t, bool narrow, BatchTable *o) {
    o->n = 0;
    o->R = t.R;
    o->item_start[0] = 0;
    for (int i = 0; i < t.n; ++i) {
        if ((t.scenes[i].bands <= kBatchNarrowBands) != narrow) continue;
        o->scenes[o->n] = t.scenes[i];
        o->strips_x[o->n] = t.strips_x[i];
        o->item_start[o->n + 1] = o->item_start[o->n] + (t.item_start[i + 1] - t.item_start[i]);
        ++o->n;
    }
}

}  // namespace

// A table mixing entries of at most kBatchNarrowBands bands with wider ones
// runs as two launches: the narrow entries on the narrow instance, the rest on
// the 8-band one.
cudaError_t launch_fuse_batched(const BatchTable &t, unsigned long long *queue, int *status,
                                int blocks_per_sm, cudaStream_t stream) {
    int nn = 0;
    for (int i = 0; i < t.n; ++i) nn += t.scenes[i].bands <= kBatchNarrowBands;
    if (nn == 0 || nn == t.n) return launch_table(t, queue, status, blocks_per_sm, kQueueBytes, stream);
    static thread_local BatchTable part;
    split_table(t, false, &part);
    cudaError_t e = launch_table(part, queue, status, blocks_per_sm, kQueueBytes, stream);
    if (e != cudaSuccess) return e;
    split_table(t, true, &part);
    return launch_table(part, queue, status, blocks_per_sm, sizeof(unsigned long long), stream);
}

}  // namespace dwtfuse
