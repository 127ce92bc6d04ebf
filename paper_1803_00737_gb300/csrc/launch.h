// Internal launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dwtfuse.h"
#include "fuse_tile.cuh"

namespace dwtfuse {

constexpr int kChunkBands = 8;     // bands per single-scene launch (more = several launches)
constexpr int kBatchMaxBands = 8;
constexpr int kBatchAltMaxBands = 6;  // bands of the batched shifted-row (W % 4 == 2) item body  // bands per scene in the batched kernel
constexpr int kMaxScenes = 128;    // scenes per batched launch
constexpr int kDefaultRows = 32;   // MS rows per warp work item (batched default)
constexpr size_t kQueueBytes = 16; // queue counter (8) + status word (4) + pad
constexpr int kStagedMaxBands = 6; // bands per launch of the staged forward (fuse_staged.cu)

// Scene table of a batched launch.  It travels by value in the kernel
// parameter block (< 32 KB), so a captured graph owns its own copy.
struct BatchTable {
    int32_t n;
    int32_t R;
    int64_t item_start[kMaxScenes + 1];
    int64_t strips_x[kMaxScenes];
    SceneArgs scenes[kMaxScenes];
};
static_assert(sizeof(BatchTable) + 16 <= 32764, "batched scene table exceeds the parameter limit");

// Quality metrics (metrics.cu).  Workspace layout, in doubles: 8 result slots
// (ERGAS, QNR, D_lambda, D_s, ...), then kMetricMaxCtas partial rows of
// kMetricStride for the PAN-resolution pass and as many for the MS pass.
constexpr int kMetricMaxCtas = 1024;
constexpr int kMetricStride = 64;    // >= pairs + bands for 8 bands (36 + 8)
constexpr int kMetricMaxBands = 8;
constexpr int kMetricWindow = 32;
constexpr size_t kMetricWorkspaceBytes = sizeof(double) * (8 + 2 * (size_t)kMetricMaxCtas * kMetricStride);

struct MetricLaunch {
    const void *fused;
    const void *ms[kMaxBands];
    const void *pan;
    int64_t H, W;
    int32_t bands;
    int32_t want_q;
    int32_t fused_f32, in_f32;
    int32_t a4_fused, a4_in;
    int32_t a16;        // uint8 PAN-pass fast path: W % 16 == 0, fused/PAN 16-byte, MS 8-byte aligned
    int32_t a32_ms;     // uint8 MS-pass fast path: W % 32 == 0, PAN and MS 16-byte aligned
    double *workspace;  // kMetricWorkspaceBytes, 8-byte aligned
    double *result;     // device pointer for the 4 results, or nullptr
    int32_t pan_done;   // PAN-resolution partial rows already written (fused forward + metrics),
                        // their count at kMetricPanCtasSlot
    int32_t ms_early;   // the kernel just before on the stream is one of ours that writes none of
                        // the MS pass's inputs: the MS pass may start as it drains (see launch_metrics)
    int32_t wait_test;  // dwtfuse_set_metric_wait_test: one warp's first slot waits on bytes never sent
};

// Fused forward + PAN-resolution metrics (fuse_metrics.cu): uint8 inputs, a
// uint8 output, up to this many bands in one launch.
constexpr int kFuseMetricsMaxBands = 8;

// MS rows per work item that balance the last wave of a grid of `warps`
// warps: minimises ceil(items / warps) * (R + 1) over R in [16, 64] (the +1
// is the D4 prologue row of every item); ties go to the taller item.
inline int balanced_rows(int64_t H, int64_t W, int64_t warps) {
    int best = kDefaultRows;
    double best_cost = 1e300;
    for (int R = 16; R <= 64; ++R) {
        const ItemGrid g = item_grid(H, W, R);
        const int64_t waves = (g.items + warps - 1) / warps;
        const double cost = (double)waves * (double)(R + 1);
        if (cost <= best_cost) {
            best_cost = cost;
            best = R;
        }
    }
    return best;
}

// Standalone 2D DWT / inverse (dwt2.cu).
struct DwtLaunch {
    const void *src;   // image (forward) or coefficients (inverse)
    float *dst_f32;    // coefficients (forward) or image (inverse), may be null for inverse
    uint8_t *dst_u8;   // image (inverse), optional
    int64_t H, W;
    int32_t wavelet;
    int32_t in_f32;    // forward: image is float (else uint8)
    int32_t inverse;
    int32_t a4;        // 4-pixel image vectors allowed
    int32_t pairs;     // coefficient pairs 8-byte aligned in both halves
    int32_t rows;      // MS rows per work item (0 = balanced)
};

// Launch-shape knobs (dwtfuse_set_rows_per_item, dwtfuse_set_band_chunks);
// 0 means the library default.
int rows_per_item();
int fwd_band_chunk();
int bwd_band_chunk();
// dwtfuse_set_fuse_staging: 1 (default) lets the single-scene forward take the
// staged kernel where it applies, 0 keeps the warp-item kernels.
int fuse_staging();

// Resident CTAs per SM for a kernel at a block size (cached per kernel).
cudaError_t resident_blocks(const void *fn, int threads, int *out);
// Resident CTAs per SM with `smem` bytes of dynamic shared memory; the first
// call per device and kernel also raises the kernel's dynamic shared memory
// limit to `smem` (cached: later launches make no attribute or occupancy call).
cudaError_t resident_blocks_smem(const void *fn, int threads, int smem, int *out);
// SM count of the current device (cached per device).
cudaError_t sm_count(int *out);

cudaError_t launch_fuse(const SceneArgs &s, int R, int blocks_per_sm, cudaStream_t stream);
// Batched adjoint over validated scenes (fuse_bwd.cu).
cudaError_t launch_fuse_backward_batched(const dwtfuse_grad_scene *scenes, int n, unsigned long long *queue,
                                         cudaStream_t stream);
cudaError_t launch_fuse_backward(const float *g, int bands, int64_t H, int64_t W, int wavelet,
                                 float *gpan, float *const *gms, int R, cudaStream_t stream);
cudaError_t launch_dwt2(const DwtLaunch &d, cudaStream_t stream);
cudaError_t launch_metrics(const MetricLaunch &m, cudaStream_t stream);
bool fuse_metrics_supported(const SceneArgs &s);
// Writes the PAN-resolution partial rows (stride doubles apart) and their
// count (device int at ctas_dev).
cudaError_t launch_fuse_metrics(const SceneArgs &s, double *pan_partial, int stride, int *ctas_dev,
                                cudaStream_t stream);
// Metrics workspace: doubles [0, 4) results, the int at double 4 the count of
// PAN-resolution partial rows written by the fused kernel, rows from double 8.
constexpr int64_t kMetricPanCtasSlot = 4;
constexpr int64_t kMetricStatusSlot = 5;  // int: DWTFUSE_OK, or DWTFUSE_ETIMEOUT when a bounded wait gave up
constexpr int64_t kMetricPanPartialOffset = 8;
cudaError_t launch_fuse_batched(const BatchTable &t, unsigned long long *queue, int *status,
                                int blocks_per_sm, cudaStream_t stream);

// Staged single-scene forward (fuse_staged.cu): taken for rows on the 16-byte
// grid with a float output, at most kStagedMaxBands bands, and a last CTA
// strip at least 7/8 full.
bool fuse_staged_applies(const SceneArgs &s);
cudaError_t launch_fuse_staged(const SceneArgs &s, int R, cudaStream_t stream);

}  // namespace dwtfuse
