// C ABI of libdwtfuse: argument validation, launch-shape selection and
// dispatch to the kernels.  Declarations and the contract are in dwtfuse.h.
#include <atomic>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <map>
#include <unordered_map>

#include "dwtfuse.h"
#include "launch.h"

namespace dwtfuse {

// Defined in fuse_static.cu.
int noalloc_device_status(cudaStream_t stream);

namespace {
std::mutex g_mu;
std::unordered_map<const void *, int> g_occ;
std::map<std::pair<int, const void *>, int> g_occ_smem;
std::unordered_map<int, int> g_sms;
std::atomic<int> g_rows{0};  // 0: balanced_rows() per launch
std::atomic<int> g_fwd_chunk{0};  // dwtfuse_set_band_chunks (0: library default)
std::atomic<int> g_bwd_chunk{0};
std::atomic<int> g_metric_wait_test{0};  // dwtfuse_set_metric_wait_test
std::atomic<int> g_staging{1};           // dwtfuse_set_fuse_staging
thread_local cudaError_t g_last_cuda = cudaSuccess;
}  // namespace

cudaError_t resident_blocks(const void *fn, int threads, int *out) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_occ.find(fn);
        if (it != g_occ.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    std::lock_guard<std::mutex> lk(g_mu);
    g_occ[fn] = occ;
    *out = occ;
    return cudaSuccess;
}

cudaError_t resident_blocks_smem(const void *fn, int threads, int smem, int *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const std::pair<int, const void *> key{dev, fn};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_occ_smem.find(key);
        if (it != g_occ_smem.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    std::lock_guard<std::mutex> lk(g_mu);
    g_occ_smem[key] = occ;
    *out = occ;
    return cudaSuccess;
}

cudaError_t sm_count(int *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_sms.find(dev);
        if (it != g_sms.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    g_sms[dev] = n;
    *out = n;
    return cudaSuccess;
}

int rows_per_item() { return g_rows.load(std::memory_order_relaxed); }
int fwd_band_chunk() { return g_fwd_chunk.load(std::memory_order_relaxed); }
int bwd_band_chunk() { return g_bwd_chunk.load(std::memory_order_relaxed); }
int fuse_staging() { return g_staging.load(std::memory_order_relaxed); }

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DWTFUSE_OK;
    g_last_cuda = e;
    return DWTFUSE_ECUDA;
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

constexpr int64_t kMaxSide = int64_t(1) << 20;  // 1 Mi px per side

int check_shape(int64_t H, int64_t W, int wavelet) {
    if (wavelet != DWTFUSE_HAAR && wavelet != DWTFUSE_D4) return DWTFUSE_EINVAL;
    const int64_t lo = wavelet == DWTFUSE_D4 ? 4 : 2;
    if (H < lo || W < lo || (H & 1) || (W & 1) || H > kMaxSide || W > kMaxSide)
        return DWTFUSE_ESHAPE;
    return DWTFUSE_OK;
}

// Validates one scene and fills its kernel arguments.
int make_scene(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
               int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, int max_bands,
               SceneArgs *s) {
    if (!pan || !ms || (!out_f32 && !out_u8)) return DWTFUSE_EINVAL;
    if (in_dtype != DWTFUSE_U8 && in_dtype != DWTFUSE_F32) return DWTFUSE_EINVAL;
    const int st = check_shape(H, W, wavelet);
    if (st != DWTFUSE_OK) return st;
    if (bands < 1) return DWTFUSE_EINVAL;
    if (bands > max_bands) return DWTFUSE_ESHAPE;
    const uintptr_t es = in_dtype == DWTFUSE_F32 ? 4 : 1;
    // PAN is read as pixel pairs and outputs are written as pixel pairs.
    if (!aligned(pan, 2 * es) || (out_f32 && !aligned(out_f32, 8)) || (out_u8 && !aligned(out_u8, 2)))
        return DWTFUSE_EALIGN;
    std::memset(s, 0, sizeof *s);
    for (int b = 0; b < bands; ++b) {
        if (!ms[b]) return DWTFUSE_EINVAL;
        if (!aligned(ms[b], es)) return DWTFUSE_EALIGN;
        s->ms[b] = ms[b];
    }
    s->pan = pan;
    s->out_f32 = out_f32;
    s->out_u8 = out_u8;
    s->H = H;
    s->W = W;
    s->bands = bands;
    s->wavelet = wavelet;
    s->in_f32 = in_dtype == DWTFUSE_F32;
    s->gain = wavelet == DWTFUSE_D4 ? 2.0f : 1.0f;
    const bool vec_ok = aligned(pan, 4 * es) && (!out_f32 || aligned(out_f32, 16)) &&
                        (!out_u8 || aligned(out_u8, 4));
    s->a4 = (W % 4 == 0) && vec_ok;
    s->alt = (W % 4 == 2) && vec_ok;
    s->out_plane = H * W;
    s->m_lo = 0;
    s->m_hi = (int32_t)(H / 2);
    return DWTFUSE_OK;
}

// Scene table of a batched launch.  A scene whose rows are 2 pixels off the
// 16-byte grid on every other row (W % 4 == 2, aligned planes) is run by the
// shifted-row item body, which holds at most kBatchAltMaxBands bands: with
// more, its bands are split over two table entries (the same PAN read twice)
// while the table has room, else it takes the plain pixel-pair body.
int build_batch_table(const dwtfuse_scene *scenes, int n, int rows_per_item, BatchTable *t) {
    std::memset(t, 0, sizeof *t);
    t->R = rows_per_item > 0 ? rows_per_item : kDefaultRows;
    const int knob = fwd_band_chunk();
    int64_t acc = 0;
    int k = 0;
    for (int i = 0; i < n; ++i) {
        const dwtfuse_scene &d = scenes[i];
        if (d.reserved != 0) return DWTFUSE_EINVAL;
        SceneArgs sa;
        const int st = make_scene(d.pan, d.ms, d.bands, d.H, d.W, d.wavelet, d.in_dtype, d.out_f32, d.out_u8,
                                  kBatchMaxBands, &sa);
        if (st != DWTFUSE_OK) return st;
        const ItemGrid g = item_grid(d.H, d.W, t->R);
        const bool alt = sa.alt && !sa.a4;
        // Band groups per entry: at most kBatchAltMaxBands on shifted rows, at
        // most the band-chunk knob when it is set; balanced groups.
        int cap = alt ? kBatchAltMaxBands : kBatchMaxBands;
        if (knob > 0 && knob < cap) cap = knob;
        int parts = (sa.bands + cap - 1) / cap;
        if (parts > 1 && (n - i - 1) + k + parts > kMaxScenes) {
            // no room in the table: one entry (shifted rows then take the pair body)
            parts = 1;
            if (alt && sa.bands > kBatchAltMaxBands) sa.alt = 0;
        }
        const int per = (sa.bands + parts - 1) / parts;
        const int64_t HW = d.H * d.W;
        for (int p = 0; p < parts; ++p) {
            SceneArgs e = sa;
            if (parts > 1) {
                const int b0 = p * per;
                const int nb = sa.bands - b0 < per ? sa.bands - b0 : per;
                for (int b = 0; b < kMaxBands; ++b) e.ms[b] = b < nb ? sa.ms[b0 + b] : nullptr;
                e.bands = nb;
                if (e.out_f32) e.out_f32 += (int64_t)b0 * HW;
                if (e.out_u8) e.out_u8 += (int64_t)b0 * HW;
            }
            t->scenes[k] = e;
            t->item_start[k] = acc;
            t->strips_x[k] = g.strips_x;
            acc += g.items;
            ++k;
        }
    }
    t->n = k;
    t->item_start[k] = acc;
    return DWTFUSE_OK;
}

}  // namespace dwtfuse

using namespace dwtfuse;

extern "C" {

const char *dwtfuse_status_string(int status) {
    switch (status) {
        case DWTFUSE_OK: return "ok";
        case DWTFUSE_EINVAL: return "invalid argument (NULL pointer, bad enum or count)";
        case DWTFUSE_ESHAPE: return "unsupported shape (H, W must be even, >= 2 Haar / >= 4 D4; band count)";
        case DWTFUSE_EALIGN: return "misaligned pointer";
        case DWTFUSE_ENOMEM: return "workspace too small";
        case DWTFUSE_ECUDA: return "CUDA runtime error";
        case DWTFUSE_ETIMEOUT: return "bounded device wait timed out";
        case DWTFUSE_EDEVICE: return "device-side check failed";
        default: return "unknown status";
    }
}

int dwtfuse_version(void) { return 100; }

int dwtfuse_last_cuda_error(void) { return (int)g_last_cuda; }

int dwtfuse_set_metric_wait_test(int on) {
    if (on != 0 && on != 1) return DWTFUSE_EINVAL;
    g_metric_wait_test.store(on, std::memory_order_relaxed);
    return DWTFUSE_OK;
}

int dwtfuse_set_rows_per_item(int rows) {
    if (rows < 0 || rows > 4096) return DWTFUSE_EINVAL;
    g_rows.store(rows, std::memory_order_relaxed);
    return DWTFUSE_OK;
}

int dwtfuse_set_band_chunks(int fwd, int bwd) {
    if (fwd < 0 || fwd > kChunkBands || bwd < 0 || bwd > kChunkBands) return DWTFUSE_EINVAL;
    g_fwd_chunk.store(fwd, std::memory_order_relaxed);
    g_bwd_chunk.store(bwd, std::memory_order_relaxed);
    return DWTFUSE_OK;
}

int dwtfuse_set_fuse_staging(int on) {
    if (on != 0 && on != 1) return DWTFUSE_EINVAL;
    g_staging.store(on, std::memory_order_relaxed);
    return DWTFUSE_OK;
}

int dwtfuse_fuse(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                 int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *stream) {
    SceneArgs s;
    const int st = make_scene(pan, ms, bands, H, W, wavelet, in_dtype, out_f32, out_u8, kMaxBands, &s);
    if (st != DWTFUSE_OK) return st;
    return cuda_status(launch_fuse(s, rows_per_item(), 0, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_fuse_ex(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                    int wavelet, int in_dtype, float ll_gain, float *out_f32, uint8_t *out_u8,
                    void *stream) {
    if (!(ll_gain == ll_gain) || ll_gain > 3.4e38f || ll_gain < -3.4e38f) return DWTFUSE_EINVAL;
    SceneArgs s;
    const int st = make_scene(pan, ms, bands, H, W, wavelet, in_dtype, out_f32, out_u8, kMaxBands, &s);
    if (st != DWTFUSE_OK) return st;
    s.gain = ll_gain;
    return cuda_status(launch_fuse(s, rows_per_item(), 0, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_fuse_rows(const void *pan_slab, const void *const *ms_slab, int bands, int64_t H, int64_t W,
                      int64_t y0, int64_t y1, int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8,
                      void *stream) {
    int st = check_shape(H, W, wavelet);
    if (st != DWTFUSE_OK) return st;
    if ((y0 & 1) || (y1 & 1) || y0 < 0 || y1 > H || y1 <= y0) return DWTFUSE_ESHAPE;
    // The slab is a scene of its own whose MS rows [m_lo, m_hi) are the band's:
    // D4 reads PAN rows 2m-2 .. 2m+3 and MS rows m-1, m for MS row m, so with
    // 2 PAN rows and 1 MS row of halo above and 2 PAN rows below, no read of
    // the band wraps inside the slab; the whole image's wrap is in the halo.
    const int64_t halo = wavelet == DWTFUSE_D4 ? 2 : 0;
    const int64_t Hs = (y1 - y0) + 2 * halo;
    SceneArgs s;
    st = make_scene(pan_slab, ms_slab, bands, Hs, W, wavelet, in_dtype, out_f32, out_u8, kMaxBands, &s);
    if (st != DWTFUSE_OK) return st;
    s.out_plane = (y1 - y0) * W;
    s.m_lo = (int32_t)(halo / 2);
    s.m_hi = (int32_t)(halo / 2 + (y1 - y0) / 2);
    return cuda_status(launch_fuse(s, rows_per_item(), 0, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_dwt2(const void *img, int in_dtype, int64_t H, int64_t W, int wavelet, float *coeffs,
                 void *stream) {
    if (!img || !coeffs) return DWTFUSE_EINVAL;
    if (in_dtype != DWTFUSE_U8 && in_dtype != DWTFUSE_F32) return DWTFUSE_EINVAL;
    const int st = check_shape(H, W, wavelet);
    if (st != DWTFUSE_OK) return st;
    const uintptr_t es = in_dtype == DWTFUSE_F32 ? 4 : 1;
    if (!aligned(img, 2 * es) || !aligned(coeffs, 8)) return DWTFUSE_EALIGN;
    DwtLaunch d{};
    d.src = img;
    d.dst_f32 = coeffs;
    d.H = H;
    d.W = W;
    d.wavelet = wavelet;
    d.in_f32 = in_dtype == DWTFUSE_F32;
    d.a4 = (W % 4 == 0) && aligned(img, 4 * es);
    d.pairs = ((W / 2) % 2) == 0;
    d.rows = rows_per_item();
    return cuda_status(launch_dwt2(d, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_idwt2(const float *coeffs, int64_t H, int64_t W, int wavelet, float *out_f32,
                  uint8_t *out_u8, void *stream) {
    if (!coeffs || (!out_f32 && !out_u8)) return DWTFUSE_EINVAL;
    const int st = check_shape(H, W, wavelet);
    if (st != DWTFUSE_OK) return st;
    if (!aligned(coeffs, 4) || (out_f32 && !aligned(out_f32, 8)) || (out_u8 && !aligned(out_u8, 2)))
        return DWTFUSE_EALIGN;
    DwtLaunch d{};
    d.src = coeffs;
    d.dst_f32 = out_f32;
    d.dst_u8 = out_u8;
    d.H = H;
    d.W = W;
    d.wavelet = wavelet;
    d.inverse = 1;
    d.a4 = (W % 4 == 0) && (!out_f32 || aligned(out_f32, 16)) && (!out_u8 || aligned(out_u8, 4));
    d.rows = rows_per_item();
    return cuda_status(launch_dwt2(d, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_fuse_backward(const float *grad_out, int bands, int64_t H, int64_t W, int wavelet,
                          float *grad_pan, float *const *grad_ms, void *stream) {
    if (!grad_out || !grad_pan || !grad_ms) return DWTFUSE_EINVAL;
    const int st = check_shape(H, W, wavelet);
    if (st != DWTFUSE_OK) return st;
    if (bands < 1) return DWTFUSE_EINVAL;
    if (bands > kMaxBands) return DWTFUSE_ESHAPE;
    if (!aligned(grad_out, 8) || !aligned(grad_pan, 8)) return DWTFUSE_EALIGN;
    for (int b = 0; b < bands; ++b) {
        if (!grad_ms[b]) return DWTFUSE_EINVAL;
        if (!aligned(grad_ms[b], 4)) return DWTFUSE_EALIGN;
    }
    return cuda_status(launch_fuse_backward(grad_out, bands, H, W, wavelet, grad_pan, grad_ms,
                                            rows_per_item(), static_cast<cudaStream_t>(stream)));
}

// The Python binding mirrors this layout field by field.
static_assert(sizeof(dwtfuse_grad_scene) == 168 && offsetof(dwtfuse_grad_scene, H) == 144,
              "dwtfuse_grad_scene layout");

int dwtfuse_fuse_backward_batched(const dwtfuse_grad_scene *scenes, int n, void *workspace, size_t ws_bytes,
                                  void *stream) {
    if (!scenes || n < 1 || !workspace) return DWTFUSE_EINVAL;
    if (n > kMaxScenes) return DWTFUSE_ESHAPE;
    if (ws_bytes < dwtfuse_batched_workspace_size()) return DWTFUSE_ENOMEM;
    if (!aligned(workspace, 16)) return DWTFUSE_EALIGN;
    for (int i = 0; i < n; ++i) {
        const dwtfuse_grad_scene &d = scenes[i];
        if (!d.grad_out || !d.grad_pan) return DWTFUSE_EINVAL;
        const int st = check_shape(d.H, d.W, d.wavelet);
        if (st != DWTFUSE_OK) return st;
        if (d.bands < 1) return DWTFUSE_EINVAL;
        if (d.bands > kMaxBands) return DWTFUSE_ESHAPE;
        if (!aligned(d.grad_out, 8) || !aligned(d.grad_pan, 8)) return DWTFUSE_EALIGN;
        for (int b = 0; b < d.bands; ++b) {
            if (!d.grad_ms[b]) return DWTFUSE_EINVAL;
            if (!aligned(d.grad_ms[b], 4)) return DWTFUSE_EALIGN;
        }
    }
    return cuda_status(launch_fuse_backward_batched(scenes, n, static_cast<unsigned long long *>(workspace),
                                                    static_cast<cudaStream_t>(stream)));
}

size_t dwtfuse_metrics_workspace_size(void) { return kMetricWorkspaceBytes; }

static int make_metrics(const void *fused, int fused_dtype, const void *const *ms, const void *pan,
                        int in_dtype, int bands, int64_t H, int64_t W, int window, bool want_q,
                        void *workspace, size_t ws_bytes, MetricLaunch *m) {
    if (!fused || !ms || !workspace || (want_q && !pan)) return DWTFUSE_EINVAL;
    if ((fused_dtype != DWTFUSE_U8 && fused_dtype != DWTFUSE_F32) ||
        (in_dtype != DWTFUSE_U8 && in_dtype != DWTFUSE_F32))
        return DWTFUSE_EINVAL;
    if (bands < 1) return DWTFUSE_EINVAL;
    if (bands > kMetricMaxBands) return DWTFUSE_ESHAPE;
    if (H < 2 || W < 2 || (H & 1) || (W & 1) || H > kMaxSide || W > kMaxSide) return DWTFUSE_ESHAPE;
    if (want_q && (window != kMetricWindow || H / 2 < window || W / 2 < window)) return DWTFUSE_ESHAPE;
    if (ws_bytes < kMetricWorkspaceBytes) return DWTFUSE_ENOMEM;
    const uintptr_t fe = fused_dtype == DWTFUSE_F32 ? 4 : 1, ie = in_dtype == DWTFUSE_F32 ? 4 : 1;
    if (!aligned(workspace, 8) || !aligned(fused, 2 * fe) || (pan && !aligned(pan, 2 * ie)))
        return DWTFUSE_EALIGN;
    std::memset(m, 0, sizeof *m);
    for (int b = 0; b < bands; ++b) {
        if (!ms[b]) return DWTFUSE_EINVAL;
        if (!aligned(ms[b], ie)) return DWTFUSE_EALIGN;
        m->ms[b] = ms[b];
    }
    m->fused = fused;
    m->pan = pan;
    m->H = H;
    m->W = W;
    m->bands = bands;
    m->want_q = want_q;
    m->fused_f32 = fused_dtype == DWTFUSE_F32;
    m->in_f32 = in_dtype == DWTFUSE_F32;
    m->a4_fused = (W % 4 == 0) && aligned(fused, 4 * fe);
    m->a4_in = (W % 4 == 0) && (!pan || aligned(pan, 4 * ie));
    bool a16 = (W % 16 == 0) && aligned(fused, 16) && (!pan || aligned(pan, 16));
    bool a32 = (W % 32 == 0) && (!pan || aligned(pan, 16));
    for (int b = 0; b < bands; ++b) {
        a16 = a16 && aligned(ms[b], 8);
        a32 = a32 && aligned(ms[b], 16);
    }
    m->a16 = a16;
    m->a32_ms = a32;
    m->workspace = static_cast<double *>(workspace);
    m->wait_test = g_metric_wait_test.load(std::memory_order_relaxed);
    return DWTFUSE_OK;
}

int dwtfuse_metrics(const void *fused, int fused_dtype, const void *const *ms, const void *pan,
                    int in_dtype, int bands, int64_t H, int64_t W, int window, void *workspace,
                    size_t ws_bytes, double *out_device, void *stream) {
    if (!out_device) return DWTFUSE_EINVAL;
    if (!aligned(out_device, 8)) return DWTFUSE_EALIGN;
    MetricLaunch m;
    const int st = make_metrics(fused, fused_dtype, ms, pan, in_dtype, bands, H, W, window, true,
                                workspace, ws_bytes, &m);
    if (st != DWTFUSE_OK) return st;
    m.result = out_device;
    return cuda_status(launch_metrics(m, static_cast<cudaStream_t>(stream)));
}

// Validates a fused forward + metrics call (the two halves share it).
static int make_fuse_score(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                           int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *workspace,
                           size_t ws_bytes, SceneArgs *s, MetricLaunch *m) {
    if (!out_u8) return DWTFUSE_EINVAL;
    int st = make_scene(pan, ms, bands, H, W, wavelet, in_dtype, out_f32, out_u8, kMaxBands, s);
    if (st != DWTFUSE_OK) return st;
    return make_metrics(out_u8, DWTFUSE_U8, ms, pan, in_dtype, bands, H, W, kMetricWindow, true, workspace,
                        ws_bytes, m);
}

int dwtfuse_fuse_and_score(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                           int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *workspace,
                           size_t ws_bytes, void *stream) {
    SceneArgs s;
    MetricLaunch m;
    const int st = make_fuse_score(pan, ms, bands, H, W, wavelet, in_dtype, out_f32, out_u8, workspace,
                                   ws_bytes, &s, &m);
    if (st != DWTFUSE_OK) return st;
    if (!fuse_metrics_supported(s)) return DWTFUSE_ESHAPE;
    return cuda_status(launch_fuse_metrics(s, m.workspace + kMetricPanPartialOffset, kMetricStride,
                                           reinterpret_cast<int *>(m.workspace + kMetricPanCtasSlot),
                                           static_cast<cudaStream_t>(stream)));
}

int dwtfuse_score_finish(const void *const *ms, const void *pan, int in_dtype, int bands, int64_t H,
                         int64_t W, const uint8_t *out_u8, void *workspace, size_t ws_bytes,
                         double *out_device, void *stream) {
    if (!out_device) return DWTFUSE_EINVAL;
    if (!aligned(out_device, 8)) return DWTFUSE_EALIGN;
    MetricLaunch m;
    const int st = make_metrics(out_u8, DWTFUSE_U8, ms, pan, in_dtype, bands, H, W, kMetricWindow, true,
                                workspace, ws_bytes, &m);
    if (st != DWTFUSE_OK) return st;
    if (in_dtype != DWTFUSE_U8 || bands > kFuseMetricsMaxBands) return DWTFUSE_ESHAPE;
    m.result = out_device;
    m.pan_done = 1;
    return cuda_status(launch_metrics(m, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_fuse_metrics(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                         int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *workspace,
                         size_t ws_bytes, double *out_device, void *stream) {
    if (!out_device) return DWTFUSE_EINVAL;
    if (!aligned(out_device, 8)) return DWTFUSE_EALIGN;
    SceneArgs s;
    MetricLaunch m;
    const int st = make_fuse_score(pan, ms, bands, H, W, wavelet, in_dtype, out_f32, out_u8, workspace,
                                   ws_bytes, &s, &m);
    if (st != DWTFUSE_OK) return st;
    m.result = out_device;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (fuse_metrics_supported(s)) {
        e = launch_fuse_metrics(s, m.workspace + kMetricPanPartialOffset, kMetricStride,
                                reinterpret_cast<int *>(m.workspace + kMetricPanCtasSlot), cs);
        m.pan_done = 1;
        m.ms_early = 1;  // the MS pass follows our own fused kernel directly
    } else {
        e = launch_fuse(s, rows_per_item(), 0, cs);
    }
    if (e == cudaSuccess) e = launch_metrics(m, cs);
    return cuda_status(e);
}

static int metrics_to_host(const MetricLaunch &m, void *stream, double *out4) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double r[kMetricStatusSlot + 1];
    cudaError_t e = launch_metrics(m, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, m.workspace, sizeof r, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    for (int k = 0; k < 4; ++k) out4[k] = r[k];
    int status;
    std::memcpy(&status, &r[kMetricStatusSlot], sizeof status);
    return status == DWTFUSE_ETIMEOUT ? DWTFUSE_ETIMEOUT : DWTFUSE_OK;
}

int dwtfuse_ergas(const void *fused, int fused_dtype, const void *const *ms, int in_dtype,
                  int bands, int64_t H, int64_t W, void *workspace, size_t ws_bytes,
                  double *out_ergas, void *stream) {
    if (!out_ergas) return DWTFUSE_EINVAL;
    MetricLaunch m;
    int st = make_metrics(fused, fused_dtype, ms, nullptr, in_dtype, bands, H, W, kMetricWindow,
                          false, workspace, ws_bytes, &m);
    if (st != DWTFUSE_OK) return st;
    double r[4];
    st = metrics_to_host(m, stream, r);
    if (st == DWTFUSE_OK) *out_ergas = r[0];
    return st;
}

int dwtfuse_qnr(const void *fused, int fused_dtype, const void *const *ms, const void *pan,
                int in_dtype, int bands, int64_t H, int64_t W, int window, void *workspace,
                size_t ws_bytes, double *out_qnr, double *out_dlambda, double *out_ds,
                void *stream) {
    if (!out_qnr || !out_dlambda || !out_ds) return DWTFUSE_EINVAL;
    MetricLaunch m;
    int st = make_metrics(fused, fused_dtype, ms, pan, in_dtype, bands, H, W, window, true,
                          workspace, ws_bytes, &m);
    if (st != DWTFUSE_OK) return st;
    double r[4];
    st = metrics_to_host(m, stream, r);
    if (st == DWTFUSE_OK) {
        *out_qnr = r[1];
        *out_dlambda = r[2];
        *out_ds = r[3];
    }
    return st;
}

size_t dwtfuse_batched_workspace_size(void) { return 256; }

int dwtfuse_fuse_batched(const dwtfuse_scene *scenes, int n, void *workspace, size_t ws_bytes,
                         int rows_per_item_, int blocks_per_sm, void *stream) {
    if (!scenes || n < 1 || !workspace || rows_per_item_ < 0 || blocks_per_sm < 0)
        return DWTFUSE_EINVAL;
    if (n > kMaxScenes) return DWTFUSE_ESHAPE;
    if (ws_bytes < dwtfuse_batched_workspace_size()) return DWTFUSE_ENOMEM;
    if (!aligned(workspace, 16)) return DWTFUSE_EALIGN;
    static thread_local BatchTable t;  // ~27 KB: kept off the stack
    const int st = build_batch_table(scenes, n, rows_per_item_, &t);
    if (st != DWTFUSE_OK) return st;
    auto *queue = static_cast<unsigned long long *>(workspace);
    int *status = reinterpret_cast<int *>(static_cast<char *>(workspace) + 8);
    return cuda_status(launch_fuse_batched(t, queue, status, blocks_per_sm, static_cast<cudaStream_t>(stream)));
}

int dwtfuse_get_last_device_status(const void *workspace, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!workspace) return noalloc_device_status(s);  // the no-alloc call's static array
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, static_cast<const char *>(workspace) + 8, sizeof v,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return v;
}

}  // extern "C"
