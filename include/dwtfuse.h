/*
 * libdwtfuse -- one-level 2D DWT pansharpening on one GPU (sm_103a).
 *
 * The method is that of Al-Oraiqat, Bashkov, Babkov, Titarenko, "Fusion of
 * multispectral satellite imagery using a cluster of graphics processing unit"
 * (arXiv:1803.00737), Sec. 2: forward 2D DWT of the panchromatic image (PAN),
 * replacement of the approximation (LL) subband by a multispectral (MS) band,
 * inverse 2D DWT, once per MS band.  Wavelets: Haar (Eq. 1-2, 11-12) and
 * Daubechies-4 with periodic wrap (Eq. 3-10, 13-16).
 *
 * Conventions shared by every entry point:
 *  - All image pointers are DEVICE pointers owned by the caller; the library
 *    never frees or keeps them.  Arrays of per-band pointers (ms, grad_ms) are
 *    HOST arrays of `bands` device pointers.
 *  - Images are dense row-major.  PAN and fused bands are H x W; MS bands are
 *    (H/2) x (W/2).  Fused outputs and output gradients are planar
 *    [bands][H][W] in one allocation.
 *  - H and W are even; Haar needs H, W >= 2, D4 needs H, W >= 4.  1 <= bands
 *    <= DWTFUSE_MAX_BANDS.  Otherwise DWTFUSE_ESHAPE.
 *  - MS pointers must be aligned to their element size; PAN, output and
 *    gradient-image pointers to twice their element size (they are accessed
 *    as pixel pairs); otherwise DWTFUSE_EALIGN.  W a multiple of 4 with
 *    16-byte-aligned float / 4-byte-aligned uint8 images enables the
 *    4-pixel vector path.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously; the call returns once it is enqueued.
 *  - The arithmetic is FP32.  Inputs are uint8 (DWTFUSE_U8) or float
 *    (DWTFUSE_F32).  uint8 outputs are clamp(round-half-even(v), 0, 255).
 *  - The LL replacement is LL <- gain * MS with gain 1 for Haar (the 2 x 2 mean
 *    is the Haar approximation) and 2 for D4 (its 2D low-pass has DC gain 2).
 *  - Errors are returned as dwtfuse_status codes; nothing aborts the process.
 *    A CUDA failure is DWTFUSE_ECUDA (see dwtfuse_last_cuda_error).  No entry
 *    point allocates device memory.
 */
#ifndef DWTFUSE_H
#define DWTFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DWTFUSE_OK = 0,
    DWTFUSE_EINVAL = 1,   /* NULL pointer, bad enum, bad count                */
    DWTFUSE_ESHAPE = 2,   /* odd or too small H/W, too many bands             */
    DWTFUSE_EALIGN = 3,   /* pointer not aligned to its element size          */
    DWTFUSE_ENOMEM = 4,   /* caller workspace too small                       */
    DWTFUSE_ECUDA = 5,    /* a CUDA runtime call or launch failed             */
    DWTFUSE_ETIMEOUT = 6, /* a bounded device-side wait gave up               */
    DWTFUSE_EDEVICE = 7   /* a device-side check failed (see device status)   */
} dwtfuse_status;

typedef enum { DWTFUSE_HAAR = 0, DWTFUSE_D4 = 1 } dwtfuse_wavelet;
typedef enum { DWTFUSE_U8 = 0, DWTFUSE_F32 = 1 } dwtfuse_dtype;

#define DWTFUSE_MAX_BANDS 16

/* Human-readable name of a status code (static string, never NULL). */
const char *dwtfuse_status_string(int status);

/* Library version as major * 10000 + minor * 100 + patch. */
int dwtfuse_version(void);

/* cudaError_t value behind the last DWTFUSE_ECUDA returned on this thread
 * (0 if none).  The library clears the CUDA error it reports. */
int dwtfuse_last_cuda_error(void);

/*
 * Fused forward (Sec. 2 step list; Eq. 1-16): for each band b,
 *   F_b = IDWT2( DWT2(PAN) with LL <- gain * MS_b ).
 * One pass over HBM: the PAN low-pass is computed once per tile and shared by
 * all bands, and the detail subbands are never materialised (by linearity,
 * F_b = PAN + U(gain * MS_b - LL(PAN)), U = synthesis of an LL-only image).
 *   pan      H x W, in_dtype
 *   ms       host array of `bands` device pointers, each (H/2) x (W/2), in_dtype
 *   out_f32  [bands][H][W] float, or NULL
 *   out_u8   [bands][H][W] uint8 (clamped, rounded half to even), or NULL
 * At least one of out_f32 / out_u8 must be non-NULL; both are written in the
 * same pass when both are given.  Outputs must not overlap inputs.
 */
int dwtfuse_fuse(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                 int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *stream);

/*
 * dwtfuse_fuse with an explicit LL replacement gain: LL <- ll_gain * MS_b.
 * The paper (Sec. 2) does not state the gain; dwtfuse_fuse uses the DC gain
 * of the 2D low-pass (1 Haar, 2 D4).  ll_gain = 1 for D4 replaces the
 * approximation by the raw MS values, one reading of the paper's weak D4
 * quality figures (Table 3).  ll_gain must be finite, else DWTFUSE_EINVAL.
 */
int dwtfuse_fuse_ex(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                    int wavelet, int in_dtype, float ll_gain, float *out_f32, uint8_t *out_u8,
                    void *stream);

/*
 * Fused forward of one band of PAN rows [y0, y1) of an H x W scene, from a
 * slab that carries the band's halo rows (Sec. 3 splits the source image
 * into parts for the nodes of a cluster; with the periodic wrap of Eq. 5-6
 * and 13-14 a D4 part needs its neighbours' rows, which the paper's merge of
 * separately fused parts leaves out).  The result equals rows [y0, y1) of
 * dwtfuse_fuse on the whole scene bit for bit, for any split.  With
 * h = 2 PAN rows and hm = 1 MS row for D4 (0 and 0 for Haar):
 *   pan_slab  PAN rows y0 - h .. y1 + h - 1, each taken mod H (the first and
 *             last parts carry the rows of the image's other end), W columns
 *   ms_slab   host array of `bands` device pointers, each holding MS rows
 *             y0/2 - hm .. y1/2 - 1 (mod H/2), W/2 columns
 *   out_f32   [bands][y1 - y0][W] float, or NULL
 *   out_u8    [bands][y1 - y0][W] uint8, or NULL
 * y0, y1 even, 0 <= y0 < y1 <= H, else DWTFUSE_ESHAPE; H, W, bands, dtypes,
 * alignment and errors as for dwtfuse_fuse.  Serves a scene split across
 * devices (each fuses its own rows after receiving its halo rows) and scenes
 * processed in row bands to bound device memory.
 */
int dwtfuse_fuse_rows(const void *pan_slab, const void *const *ms_slab, int bands, int64_t H, int64_t W,
                      int64_t y0, int64_t y1, int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8,
                      void *stream);

/*
 * One-level 2D DWT of an image (Sec. 2: 1D transform of every row, then of
 * every column; Haar Eq. 1-2, Daubechies-4 Eq. 3-10 with periodic wrap), the
 * transform the fusion applies before the LL replacement.
 *   img     H x W, in_dtype (uint8 or float)
 *   coeffs  H x W float, the paper's in-place layout: with A / D the row
 *           approximation / detail and a column pass of low-pass then
 *           high-pass, top-left = LL (low-pass of A), top-right = low-pass of D,
 *           bottom-left = high-pass of A, bottom-right = high-pass of D.
 * The D4 detail filter is the quadrature mirror (h3, -h2, h1, -h0) of Eq. 7-8's h
 * (Eq. 9-10 as printed do not invert).  coeffs must be 8-byte aligned.
 */
int dwtfuse_dwt2(const void *img, int in_dtype, int64_t H, int64_t W, int wavelet, float *coeffs,
                 void *stream);

/*
 * Inverse one-level 2D DWT (Sec. 2: columns, then rows; Haar Eq. 11-12, D4
 * Eq. 13-16) of a coefficient image in the layout of dwtfuse_dwt2, into a float
 * image and/or a uint8 image (clamped, rounded half to even); at least one
 * output.  dwtfuse_idwt2(dwtfuse_dwt2(x)) = x up to rounding.
 */
int dwtfuse_idwt2(const float *coeffs, int64_t H, int64_t W, int wavelet, float *out_f32,
                  uint8_t *out_u8, void *stream);

/*
 * Adjoint (vector-Jacobian product) of dwtfuse_fuse with respect to PAN and
 * every MS band, for float images.  With U and LL as above and S the
 * synthesis matrix (S = A^T for D4, S = 2 A^T for the /2 Haar of Eq. 1-2, so
 * the transpose is not the inverse):
 *   grad_ms_b = gain * sigma^2 * LL(grad_out_b)
 *   grad_pan  = G - U(LL(G)),  G = sum_b grad_out_b
 * (sigma = 2 for Haar, 1 for D4).
 *   grad_out  [bands][H][W] float
 *   grad_pan  H x W float (overwritten)
 *   grad_ms   host array of `bands` device pointers, each (H/2) x (W/2) float
 *             (overwritten)
 */
int dwtfuse_fuse_backward(const float *grad_out, int bands, int64_t H, int64_t W, int wavelet,
                          float *grad_pan, float *const *grad_ms, void *stream);

/*
 * Quality metrics of a fused product.  The paper reports ERGAS and QNR
 * (Sec. 4, Table 3) without defining them; the definitions used are:
 *   ERGAS    = 100 * (1/2) * sqrt( (1/B) sum_b RMSE_b^2 / mu_b^2 ), RMSE_b over
 *              all H x W pixels against MS_b repeated 2 x 2, mu_b = mean of MS_b;
 *   Q        = Wang-Bovik index on non-overlapping 32 x 32 windows at each
 *              image's own resolution, averaged (ragged edge dropped; a zero
 *              denominator gives 1 for identical windows, else 0);
 *   D_lambda = mean over ordered band pairs |Q(F_l, F_r) - Q(MS_l, MS_r)|;
 *   D_s      = mean over bands |Q(F_l, PAN) - Q(MS_l, PAN~)|, PAN~ = 2 x 2 block
 *              mean of PAN;  QNR = (1 - D_lambda)(1 - D_s).
 *   fused     [bands][H][W], fused_dtype (uint8 or float)
 *   ms        host array of `bands` device pointers, (H/2) x (W/2), in_dtype
 *   pan       H x W, in_dtype
 *   window    must be DWTFUSE_QNR_WINDOW (32)
 *   workspace dwtfuse_metrics_workspace_size() bytes of device memory, 8-byte
 *             aligned; its contents are scratch between calls
 * bands <= DWTFUSE_METRIC_MAX_BANDS (8).  QNR needs H/2, W/2 >= window.
 * Results are deterministic (fixed reduction order).
 */
#define DWTFUSE_QNR_WINDOW 32
#define DWTFUSE_METRIC_MAX_BANDS 8

size_t dwtfuse_metrics_workspace_size(void);

/* Asynchronous on `stream`: writes four doubles to DEVICE memory out_device:
 * ERGAS, QNR, D_lambda, D_s.  Capturable in a CUDA graph.  On rows off the
 * 16-byte grid the passes wait on their own bulk copies; a wait that gives up
 * (about a second; not seen in normal operation) makes all four figures NaN,
 * and the synchronous dwtfuse_ergas / dwtfuse_qnr return DWTFUSE_ETIMEOUT. */
int dwtfuse_metrics(const void *fused, int fused_dtype, const void *const *ms, const void *pan,
                    int in_dtype, int bands, int64_t H, int64_t W, int window, void *workspace,
                    size_t ws_bytes, double *out_device, void *stream);

/* ERGAS only (pan not needed); waits for the stream and writes the HOST double. */
int dwtfuse_ergas(const void *fused, int fused_dtype, const void *const *ms, int in_dtype,
                  int bands, int64_t H, int64_t W, void *workspace, size_t ws_bytes,
                  double *out_ergas, void *stream);

/* QNR, D_lambda and D_s; waits for the stream and writes HOST doubles. */
int dwtfuse_qnr(const void *fused, int fused_dtype, const void *const *ms, const void *pan,
                int in_dtype, int bands, int64_t H, int64_t W, int window, void *workspace,
                size_t ws_bytes, double *out_qnr, double *out_dlambda, double *out_ds,
                void *stream);

/*
 * Fused forward followed by the metrics of its uint8 product, in one call:
 * the same outputs as dwtfuse_fuse(pan, ms, ..., out_f32, out_u8) and then
 * dwtfuse_metrics(out_u8, DWTFUSE_U8, ms, pan, in_dtype, ...) into
 * out_device (ERGAS, QNR, D_lambda, D_s as four device doubles).  With uint8
 * inputs (up to 8 bands, as the metrics) the forward scores its product on chip (the
 * PAN-resolution half of the metrics needs no read of the fused bands, PAN or
 * MS); otherwise the two calls run one after the other.  Arguments and errors
 * are those of the two calls; out_u8 is required, out_f32 optional; the
 * workspace is the metrics workspace.  Asynchronous on `stream`, capturable
 * in a CUDA graph.  The ERGAS value equals the separate calls' exactly; Q
 * sums are accumulated in another order (agreement to ~1e-6).
 * The on-chip scoring keeps each lane's running sums in tensor memory (TMEM):
 * every CTA of that kernel allocates 64-256 of its SM's 512 TMEM columns at
 * start and frees them at exit, and runs alone on its SM.  A kernel of another
 * library that holds TMEM on the same SM at the same time (another stream)
 * makes those CTAs wait for free columns until it releases them.
 */
int dwtfuse_fuse_metrics(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                         int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *workspace,
                         size_t ws_bytes, double *out_device, void *stream);

/*
 * dwtfuse_fuse_metrics in two calls on the same workspace, for callers that
 * schedule or time the halves apart.  dwtfuse_fuse_and_score launches only
 * the fused forward that scores its product (uint8 inputs, <= 8 bands; else
 * DWTFUSE_ESHAPE) and leaves the partial scores in the workspace;
 * dwtfuse_score_finish then runs the MS-resolution pass and the reduction
 * into out_device.  The second call must follow the first on the same
 * stream (or after it), with the same ms, pan, bands, H, W and out_u8, and no
 * other metrics call on that workspace in between.
 */
int dwtfuse_fuse_and_score(const void *pan, const void *const *ms, int bands, int64_t H, int64_t W,
                           int wavelet, int in_dtype, float *out_f32, uint8_t *out_u8, void *workspace,
                           size_t ws_bytes, void *stream);
int dwtfuse_score_finish(const void *const *ms, const void *pan, int in_dtype, int bands, int64_t H,
                         int64_t W, const uint8_t *out_u8, void *workspace, size_t ws_bytes,
                         double *out_device, void *stream);

/* One scene of a batched call (all pointers on the device, as above). */
typedef struct {
    const void *pan;
    const void *ms[DWTFUSE_MAX_BANDS];
    float *out_f32;   /* [bands][H][W] or NULL */
    uint8_t *out_u8;  /* [bands][H][W] or NULL */
    int64_t H, W;
    int32_t bands;
    int32_t wavelet;  /* dwtfuse_wavelet */
    int32_t in_dtype; /* dwtfuse_dtype   */
    int32_t reserved; /* must be 0       */
} dwtfuse_scene;

#define DWTFUSE_MAX_SCENES 128

/* One scene of a batched backward (all pointers on the device, as for
 * dwtfuse_fuse_backward). */
typedef struct {
    const float *grad_out;             /* [bands][H][W] */
    float *grad_pan;                   /* H x W (overwritten) */
    float *grad_ms[DWTFUSE_MAX_BANDS]; /* bands planes (H/2) x (W/2) (overwritten) */
    int64_t H, W;
    int32_t bands;
    int32_t wavelet;  /* dwtfuse_wavelet */
} dwtfuse_grad_scene;

/*
 * Batched adjoint: dwtfuse_fuse_backward (the transpose of the Sec. 2 fusion,
 * formulas above) for up to DWTFUSE_MAX_SCENES scenes of any legal sizes,
 * band counts and wavelets.  Per chunk of 8 bands, one persistent launch for
 * each wavelet and chunk width present (1-4 or 5-8 bands); the second and
 * later chunks add into grad_pan, so they follow in order.  Results equal
 * dwtfuse_fuse_backward per scene bit for bit.  Arguments, layouts and errors
 * per scene as dwtfuse_fuse_backward; more than DWTFUSE_MAX_SCENES scenes is
 * DWTFUSE_ESHAPE.  The workspace is dwtfuse_batched_workspace_size() bytes of
 * device memory, 16-byte aligned, scratch between calls (calls sharing it must
 * not overlap).  Asynchronous on `stream`, capturable in a CUDA graph; the
 * scene array is read before the call returns.
 */
int dwtfuse_fuse_backward_batched(const dwtfuse_grad_scene *scenes, int n, void *workspace,
                                  size_t ws_bytes, void *stream);

/* Bytes of device workspace dwtfuse_fuse_batched needs (queue counter and
 * device status word). */
size_t dwtfuse_batched_workspace_size(void);

/*
 * Batched fused forward: up to DWTFUSE_MAX_SCENES scenes of any legal sizes,
 * band counts (<= 8 per scene), wavelets and input types in one persistent
 * launch (two when the table mixes entries of at most 4 bands with wider
 * ones: each set runs the kernel instance sized for it).  Warps pull (scene,
 * tile) work items from a device-side queue whose counter lives in
 * `workspace`; the scene table travels in the kernel's parameter block, so the
 * call is capturable in a CUDA graph (the capture records memsets of the
 * counter and the kernels; the host array `scenes` may be freed after the
 * call).  Results equal dwtfuse_fuse per scene.
 *   rows_per_item  MS rows per work item (0 = library default)
 *   blocks_per_sm  resident CTAs per SM for the persistent grid (0 = max)
 */
int dwtfuse_fuse_batched(const dwtfuse_scene *scenes, int n, void *workspace, size_t ws_bytes,
                         int rows_per_item, int blocks_per_sm, void *stream);

/*
 * Reads (synchronously, on `stream`) the device status word of a batched
 * workspace: DWTFUSE_OK, or the first device-side error recorded.  With
 * workspace = NULL it reads the status word of the last
 * dwtfuse_fuse_batched_noalloc call on the current device (DWTFUSE_OK if
 * there was none); that read allocates nothing either.
 */
int dwtfuse_get_last_device_status(const void *workspace, void *stream);

/*
 * Batched fused forward that needs no device memory from the caller and
 * allocates none itself.  The paper has no counterpart; this is a library
 * convenience.
 *
 * It serves callers that cannot allocate device memory when they call:
 * applications that reserve all of the GPU's memory up front in their own
 * pool (a new allocation would fail or fragment it), plug-in hosts that hand
 * the library only image pointers, and real-time processing chains whose
 * memory footprint must be fixed at start-up.  dwtfuse_fuse_batched needs a
 * caller workspace for its work-queue counter; this variant keeps that counter
 * and the device status word in a DWTFUSE_STATIC_SCRATCH_BYTES-byte array in
 * the library's device code, which every GPU that loads the library holds
 * until the process exits.
 *
 * Arguments and results are those of dwtfuse_fuse_batched without the
 * workspace.  More than DWTFUSE_MAX_SCENES scenes is DWTFUSE_ESHAPE (the
 * queue's 16 bytes fit the array for every legal call).
 * The first call on each device looks up the array's device address (with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture.  cudaDeviceReset on a device makes
 * the kept address stale: do not call this entry point on that device again.
 * Every call shares the one array, which keeps the last call's contents; each
 * call clears the counter and status word on its stream before its kernel.
 * Calls that overlap on the GPU (unordered streams) race on the counter, so
 * order them.  The device status word (DWTFUSE_EDEVICE when a scene-table
 * entry failed its device-side check, the scene's outputs then unwritten) is
 * read by dwtfuse_get_last_device_status(NULL, stream).
 */
#define DWTFUSE_STATIC_SCRATCH_BYTES 256
int dwtfuse_fuse_batched_noalloc(const dwtfuse_scene *scenes, int n, int rows_per_item,
                                 int blocks_per_sm, void *stream);

/*
 * Launch-shape knob of dwtfuse_fuse and dwtfuse_fuse_backward for the
 * autotuner: MS rows per warp work item.  0 (the default) picks, per launch,
 * the height in [16, 64] that fills the last wave of the persistent grid.
 * Process-wide.
 */
int dwtfuse_set_rows_per_item(int rows);

/*
 * Launch-shape knobs for the autotuner: the most bands one launch (or one
 * batched table entry) of the forward handles (fwd) and of the adjoint
 * (bwd).  A scene with more bands is run in balanced chunks of at most that
 * many (the forward reads PAN once per chunk; later adjoint chunks add into
 * grad_pan).  0 (the default) keeps the library's choice: 8 bands, 6 on rows
 * off the 16-byte grid.  With a bwd knob set, or a rows knob
 * (dwtfuse_set_rows_per_item), the batched adjoint uses it too.  Fused values
 * do not depend on the forward knob; grad_pan sums its chunks in order, so
 * the adjoint knob can change its last bits.  Process-wide; values outside
 * [0, 8] are DWTFUSE_EINVAL.
 */
int dwtfuse_set_band_chunks(int fwd, int bwd);

/*
 * Store-path knob of the single-scene forward (a launch-shape choice, no
 * counterpart in the paper): with on = 1 (the default) dwtfuse_fuse takes the
 * staged kernel where it applies (rows on the 16-byte grid, a float output, at
 * most 6 bands per launch, whole 1024-column CTA strips, the last one at least
 * 7/8 full), which writes the float rows through shared memory and bulk
 * copies; with on = 0 it runs the warp-strip kernels everywhere.  The outputs
 * are the same bits either way.  Process-wide; other values are
 * DWTFUSE_EINVAL.
 */
int dwtfuse_set_fuse_staging(int on);

/*
 * Test hook for the metric passes' bounded waits (no counterpart in the
 * paper).  With on = 1, every later metrics call whose PAN-resolution pass
 * stages unaligned rows (W % 16 != 0, uint8 data) makes one warp post 16 bytes
 * to its first ring slot that no copy delivers, so that warp's wait gives up
 * after about a second: the call's figures are NaN and dwtfuse_ergas /
 * dwtfuse_qnr return DWTFUSE_ETIMEOUT; the context stays usable.  on = 0
 * (the default) turns it off.  Process-wide; anything else is DWTFUSE_EINVAL.
 */
int dwtfuse_set_metric_wait_test(int on);

#ifdef __cplusplus
}
#endif

#endif /* DWTFUSE_H */
