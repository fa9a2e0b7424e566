/*
 * gs.h -- C ABI of libgs: tile-binned 3D Gaussian Splatting rasterisation that
 * also emits the analytic screen-space derivatives of each pixel colour, and the
 * gradient-aware bicubic Hermite upscale built on them (Niedermayr, Neuhauser,
 * Westermann, "Lightweight Gradient-Aware Upscaling of 3D Gaussian Splatting
 * Images", ICCV 2025).  Hand-written CUDA for sm_103a (GB300).
 *
 * Conventions shared by every call
 * --------------------------------
 * Pointers.  Unless a parameter says "host", every array pointer is a DEVICE
 *   pointer (cudaMalloc / torch CUDA memory on the context's device) owned by the
 *   caller.  The library never frees caller memory and never keeps a caller
 *   pointer beyond the call that received it.  All arrays are dense, row-major,
 *   fp32 unless stated.
 * Context.  A gs_ctx owns only scratch memory (per-Gaussian records, sort
 *   buffers, per-tile ranges, per-pixel blend state) and a CUDA stream handle.
 *   One context must not be used from two host threads at once.
 * Streams.  Work is enqueued on the context's stream and is asynchronous,
 *   except where a call says it synchronises.  gs_project (and the render calls
 *   that include it) read the number of (tile, Gaussian) pairs back to the host
 *   once per call, which synchronises the context's stream.
 * Errors.  Every call returns a gs_status; nothing throws across the ABI.
 *   GS_ERR_INVALID_ARG: a NULL pointer where one is required, a negative count,
 *     an image side < 1 (< 2 for the upscale input), an unsupported option.
 *   GS_ERR_CUDA: a CUDA runtime error (gs_last_error() has the text).
 *   GS_ERR_OOM: scratch could not be allocated.
 *   GS_ERR_CAPACITY: the pair count exceeds gs_options.max_pairs (or 2^30 - 1);
 *     nothing is written out of bounds.
 *   GS_ERR_TIMEOUT / GS_ERR_DEVICE_CHECK: a kernel's bounded wait expired or a
 *     device-side check failed; the outputs of that call are undefined, the
 *     context stays usable.
 * Image layout.  Planar: channel-major [3][H][W] colour, derivative stacks
 *   [3 (d/dx, d/dy, d2/dxdy)][3][H][W].  Pixel (i, j) (column i, row j) is the
 *   continuous image point (i, j); x grows with the column, y with the row.
 */
#ifndef GS_H
#define GS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,
    GS_ERR_CUDA = 2,
    GS_ERR_OOM = 3,
    GS_ERR_CAPACITY = 4,
    GS_ERR_TIMEOUT = 5,
    GS_ERR_DEVICE_CHECK = 6,
    GS_ERR_NOT_READY = 7
} gs_status;

/* Blend modes.  GS_MODE_3DGS: alpha = min(0.99, sigma e^g), pairs with
 * alpha < 1/255 are skipped, a pixel stops before the Gaussian that would take
 * its transmittance below 1e-4, tile sets are the rects of radius
 * ceil(3 sqrt(lambda_max)).  GS_MODE_EXACT: none of these cut-offs, every visible
 * Gaussian is binned into every tile (a smooth image; meant for small scenes). */
#define GS_MODE_3DGS 0
#define GS_MODE_EXACT 1

typedef struct gs_ctx gs_ctx;

/* A set of 3D Gaussians (Sec. 4: centre mu, covariance Sigma = R S S^T R^T from a
 * scale and a rotation, opacity sigma, spherical-harmonics colour).  Device
 * pointers, structure-of-arrays:
 *   means          [n][3]                world-space centre
 *   log_scales     [n][3]                log of the per-axis standard deviation
 *   quats          [n][4]                rotation quaternion (w, x, y, z); normalised here
 *   opacity_logits [n]                   sigma = 1 / (1 + e^-logit)
 *   sh             [n][(deg+1)^2][3]     real SH coefficients, index l^2 + l + m,
 *                                        colour = max(0, sum_k sh_k Y_k(dir) + 1/2),
 *                                        dir from the camera centre to mu; or NULL
 *   rgb            [n][3]                direct colour, used when sh == NULL */
typedef struct gs_gaussians {
    int64_t n;
    int32_t sh_degree;            /* 0..3, ignored when sh == NULL */
    int32_t reserved;
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity_logits;
    const float* sh;
    const float* rgb;
} gs_gaussians;

/* Gradients of a scalar loss with respect to the inputs of gs_gaussians
 * (caller-owned device fp32 arrays of the same shapes; overwritten).  sh is
 * written when the projected Gaussians used SH, rgb when they used direct
 * colours; either may be NULL to skip it. */
typedef struct gs_gaussian_grads {
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logits;
    float* sh;
    float* rgb;
} gs_gaussian_grads;

/* Pinhole camera, passed by value from the host.  viewmat: row-major 4x4
 * world->camera (x right, y down, z forward); pixel = (fx x/z + cx, fy y/z + cy);
 * Gaussians with view depth z <= znear are culled. */
typedef struct gs_camera {
    float viewmat[16];
    float fx, fy, cx, cy;
    float znear;
} gs_camera;

typedef struct gs_options {
    int32_t tile;        /* tile side in pixels; 16 is the only supported value */
    int32_t mode;        /* GS_MODE_3DGS or GS_MODE_EXACT */
    float bg[3];         /* background colour composited behind the Gaussians */
    int32_t flags;       /* GS_FLAG_* bits; 0 = default */
    int64_t max_pairs;   /* upper bound on (tile, Gaussian) pairs; 0 = 2^30 - 1 */
} gs_options;

/* gs_options.flags: frames without a host wait.  gs_project then never waits
 * for the pair count: the pair totals stay on the device, the pair buffers are
 * those reserved with gs_reserve (no call allocates), and a frame whose pairs
 * exceed them (or max_pairs) renders as background only, with
 * GS_ERR_CAPACITY reported by the next gs_synchronize (gs_pair_count then
 * gives the pairs the frame needed).  Requires gs_reserve first.  With it the
 * project -> render -> upscale sequence makes no host-blocking call, so it can
 * be captured in a CUDA graph. */
#define GS_FLAG_NO_HOST_WAIT 1

/* gs_options.flags: the recompute variant of the blend's adjoint
 * (gs_render_backward, gs_backward).  Instead of recovering the blend state of
 * each step by inverting the forward's update from the stored final state
 * through the whole list (the supplement's inversion trick), the adjoint first
 * re-runs each tile's forward walk (the transmittance state only, every
 * decision taken on the same FP32 values) and checkpoints the exact state at
 * the start of each round of 256 candidates in context scratch (8 per tile,
 * thinned to every second, fourth, ... round on longer lists); walking back,
 * every round starts from the exact state at its end.  Needs the projection
 * only (not the forward's stored state); costs a second walk of each tile. */
#define GS_FLAG_BWD_RECOMPUTE 2

/* Human-readable name of a status code (static string). */
const char* gs_status_string(gs_status status);

/* Text of the last error recorded on ctx (static per context; "" if none). */
const char* gs_last_error(const gs_ctx* ctx);

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL =
 * the legacy default stream).  opt may be NULL (tile 16, 3DGS mode, black
 * background, no pair limit).  *out receives the context; free it with
 * gs_destroy.  The projection's depth sort runs, up to about 10k Gaussians per
 * SM, as one cooperative grid of one block per SM that expects the GPU to
 * itself: do not run the frames of two contexts concurrently on different
 * streams (their bounded grid barriers would report GS_ERR_TIMEOUT). */
gs_status gs_create(gs_ctx** out, void* stream, const gs_options* opt);

/* Release the context and its scratch memory (synchronises its stream). */
gs_status gs_destroy(gs_ctx* ctx);

/* Change the stream later calls enqueue on. */
gs_status gs_set_stream(gs_ctx* ctx, void* stream);

/* Change blend mode / background / pair limit / flags for later calls. */
gs_status gs_set_options(gs_ctx* ctx, const gs_options* opt);

/* Allocate every scratch buffer for frames of up to n Gaussians, W x H pixels
 * and super_pairs (super-tile, Gaussian) pairs, and fix those
 * capacities.  Needed before frames with GS_FLAG_NO_HOST_WAIT; afterwards no
 * call of this context allocates: a frame beyond n, W or H returns
 * GS_ERR_CAPACITY at once, one beyond super_pairs as described for the flag.
 * Synchronises the stream.  W x H <= 4096 super-tiles (e.g. 4096 x 4096). */
gs_status gs_reserve(gs_ctx* ctx, int64_t n, int32_t W, int32_t H, int64_t super_pairs);

/* gs_reserve plus the per-view buffers of gs_render_views and
 * gs_render_views_scenes for up to V views (1 <= V <= 32), each of up to n
 * Gaussians (for a batch over several Gaussian sets: the largest set); W, H
 * and super_pairs (the capacity of each view's pair buffers) bound every
 * view. */
gs_status gs_reserve_views(gs_ctx* ctx, int64_t n, int32_t V, int32_t W, int32_t H, int64_t super_pairs);

/* Several views of one Gaussian set in one batch (e.g. the stereo pairs of a
 * VR headset, which the paper names as a use of cheap upscaling; Sec. 1):
 * one launch projects every view (each Gaussian's inputs, SH coefficients
 * included, are read once for all views), one sort puts every view's
 * Gaussians in depth order (the view as the top digit), one launch emits
 * every view's pairs into buffers of its own, one launch per pass sorts every
 * view's pairs; one launch blends every tile of every view with derivatives
 * into out_C[v] [3][H_v][W_v] and out_grads[v] [3][3][H_v][W_v] (launch shape
 * from gs_views_config / gs_autotune_views), and one launch upscales, where
 * out_up != NULL and out_up[v] != NULL, by factors[v] into out_up[v].  View v
 * uses cams[v], Ws[v] x Hs[v]; each view equals a single-view
 * gs_render_with_grads of the same camera bit for bit.  Requires
 * GS_FLAG_NO_HOST_WAIT and gs_reserve_views; makes no host-blocking call
 * (capturable in a CUDA graph); a view beyond the reserved pairs renders as
 * background with GS_ERR_CAPACITY at the next gs_synchronize (gs_pair_count /
 * gs_super_pair_count then give the batch's sums).  Host arrays of V entries
 * (cams, Ws, Hs, factors) and of V device pointers (out_C, out_grads,
 * out_up).  The context's single-view results (gs_render_binned, gs_read_*,
 * gs_backward) are invalid afterwards. */
gs_status gs_render_views(gs_ctx* ctx, const gs_gaussians* g, int32_t V, const gs_camera* cams, const int32_t* Ws,
                          const int32_t* Hs, float* const* out_C, float* const* out_grads, const int32_t* factors,
                          float* const* out_up);

/* gs_render_views over several Gaussian sets of uneven size in one batch
 * (e.g. views of different scenes, or of one scene at several levels of
 * detail): scenes is a host array of S (1 <= S <= 32) sets, view v renders
 * scenes[scene_of_view[v]] (host int32[V], each in 0..S-1).  One projection
 * launch per set (over the views that use it); everything after it runs as in
 * gs_render_views, and each view equals a single-view gs_render_with_grads of
 * its set bit for bit.  Every set must fit the reservation's n. */
gs_status gs_render_views_scenes(gs_ctx* ctx, const gs_gaussians* scenes, int32_t S, const int32_t* scene_of_view,
                                 int32_t V, const gs_camera* cams, const int32_t* Ws, const int32_t* Hs,
                                 float* const* out_C, float* const* out_grads, const int32_t* factors,
                                 float* const* out_up);

/* Tuning of the batched views (the binning and launch shapes; the images do
 * not depend on them, bit for bit).  warp_map: the pixels of each warp of a
 * 16 x 16 tile, 0 = an 8 x 4 block, 1 = a 16 x 2 strip.  schedule: 0 = one
 * block per tile in tile order, 1 = one block per tile, the heaviest tiles of
 * the previous batch first, 2 = resident blocks taking tiles from a counter,
 * 3 = one block per tile, the views in order and each view's heaviest tiles of
 * the previous batch first (each view's Gaussian records stay in L2 while its
 * tiles run).  super_side: the super-tile side of every view's binning, 0 = per
 * view by the single-frame rule (gs_super_pair_count), 4 = 4 x 4 tiles
 * (fewer pairs, longer lists per blend block).  Default (0, 1, 0). */
#define GS_VIEWS_CONFIGS 16   /* configuration k: warp_map = k % 2, schedule = (k / 2) % 4, super_side = 4 if k >= 8 */
gs_status gs_views_config(gs_ctx* ctx, int32_t warp_map, int32_t schedule, int32_t super_side);

/* Autotuner: renders the batch of gs_render_views (same arguments) once
 * untimed and `reps` times timed (CUDA events on the context's stream) in each
 * of the GS_VIEWS_CONFIGS configurations, keeps the fastest in the context and
 * returns the mean milliseconds per batch of each configuration in ms[k] (host
 * float[GS_VIEWS_CONFIGS], may be NULL) and the chosen k in *best (may be
 * NULL).  Synchronises; not for use inside a CUDA graph capture. */
gs_status gs_autotune_views(gs_ctx* ctx, const gs_gaussians* g, int32_t V, const gs_camera* cams, const int32_t* Ws,
                            const int32_t* Hs, float* const* out_C, float* const* out_grads, const int32_t* factors,
                            float* const* out_up, int32_t reps, float* ms, int32_t* best);

/* The autotuner on a gs_render_views_scenes batch (same arguments). */
gs_status gs_autotune_views_scenes(gs_ctx* ctx, const gs_gaussians* scenes, int32_t S, const int32_t* scene_of_view,
                                   int32_t V, const gs_camera* cams, const int32_t* Ws, const int32_t* Hs,
                                   float* const* out_C, float* const* out_grads, const int32_t* factors,
                                   float* const* out_up, int32_t reps, float* ms, int32_t* best);

/* Projection and tile binning for a W x H image (Sec. 4: EWA projection
 * Sigma' = J W Sigma W^T J^T + 0.3 I, front-to-back order).  Per Gaussian: view
 * depth, 2D mean, conic Sigma'^-1, colour, opacity, radius ceil(3 sqrt(lambda_max))
 * and the tiles whose pixel centres fall in the square of that half-width; then
 * every (tile, Gaussian) pair is ordered by tile, FP32 depth bits, id.  Results
 * stay in ctx for gs_render_binned / gs_read_projected / gs_read_bins.
 * Waits once for the pair count (to size the pair buffers), unless
 * GS_FLAG_NO_HOST_WAIT is set. */
gs_status gs_project(gs_ctx* ctx, const gs_gaussians* g, const gs_camera* cam, int32_t W, int32_t H);

/* Blend the scene binned by the last gs_project.  Per pixel, front to back
 * (Sec. 4 blend; Sec. 5 and supplement "Forward pass" recurrences):
 *   C = sum_i T_i alpha_i c_i + T_N bg, with T_i = 1 - A_{i-1},
 * and, when out_grads != NULL, dC/dx, dC/dy, d2C/dxdy accumulated through the
 * same loop.  out_C [3][H][W] (required); out_grads [3][3][H][W] or NULL (then only
 * the plain colour is computed).  The per-pixel final transmittance state is kept
 * in ctx (gs_read_state). */
gs_status gs_render_binned(gs_ctx* ctx, float* out_C, float* out_grads);

/* gs_project followed by gs_render_binned with derivatives: the low-resolution
 * render of the method (Sec. 5, pipeline figure).  out_C [3][H][W],
 * out_grads [3][3][H][W], both required. */
gs_status gs_render_with_grads(gs_ctx* ctx, const gs_gaussians* g, const gs_camera* cam,
                               int32_t W, int32_t H, float* out_C, float* out_grads);

/* gs_project followed by a plain blend (colour only): the direct
 * full-resolution render the method is compared against (Table 2 "3DGS"). */
gs_status gs_render(gs_ctx* ctx, const gs_gaussians* g, const gs_camera* cam,
                    int32_t W, int32_t H, float* out_C);

/* Gradient-aware bicubic Hermite upscale (Sec. 5 "Spline Interpolation";
 * supplement "Spline Image Interpolation").  For every output pixel (X, Y) of
 * the factor*W x factor*H image: x = (X + 0.5)/factor - 0.5 (likewise y), cell
 * i = clamp(floor(x), 0, W-2), t = x - i; the patch of cell (i, j) matches the
 * four corner values and their d/dx, d/dy, d2/dxdy; border half-cells
 * extrapolate the edge patch.  C [3][H][W], grads [3][3][H][W] (as written by the
 * render), out [3][factor*H][factor*W].  W, H >= 2; 1 <= factor <= 16.
 * Asynchronous. */
gs_status gs_upscale(gs_ctx* ctx, const float* C, const float* grads, int32_t W, int32_t H,
                     int32_t factor, float* out);

/* gs_upscale to any output size W2 x H2 (integer or fractional factors,
 * supplement "Qualitative Results for Different Upsampling Rates"): output
 * pixel X samples x = (X + 0.5) W / W2 - 0.5, likewise for Y.  W, H >= 2;
 * W <= W2 <= 16 W, H <= H2 <= 16 H.  out [3][H2][W2].  Asynchronous.  For
 * W2 = factor W it equals gs_upscale bit for bit. */
gs_status gs_upscale_to(gs_ctx* ctx, const float* C, const float* grads, int32_t W, int32_t H, int32_t W2,
                        int32_t H2, float* out);

/* Classical bicubic upscale, the paper's comparator: cubic convolution of the
 * colour samples C [3][H][W] alone with Keys' kernel of parameter a (a = -0.5:
 * the Hermite patch with central-difference slopes, the finite-difference
 * gradients of Sec. 5; a = -0.75: the bicubic interpolation of PyTorch used in
 * the experiments, Sec. 6), same half-pixel map as gs_upscale_to, sample
 * indices clamped to the image.  W, H >= 1; W <= W2 <= 16 W, H <= H2 <= 16 H;
 * -2 <= a <= 0.  out [3][H2][W2].  Asynchronous. */
gs_status gs_upscale_bicubic(gs_ctx* ctx, const float* C, int32_t W, int32_t H, int32_t W2, int32_t H2, float a,
                             float* out);

/* ---- Learned residual on the spline (an extension beside the paper's method:
 * the paper upscales with the spline alone, Sec. 5, and argues against learned
 * upscalers, Sec. 2).  A per-output-pixel MLP 50 -> 64 -> 64 -> 3 with ReLU
 * reads the 48 values the spline reads -- f[12 k + 3 q + c] = quantity q (C,
 * dC/dx, dC/dy, d2C/dxdy) of channel c at corner k ((i, j), (i+1, j),
 * (i, j+1), (i+1, j+1)) of the pixel's cell -- and f[48] = t, f[49] = u, the
 * local coordinates of its sample point, and adds its output to the spline.
 *
 * params: GS_MLP_PARAMS FP32 values, device memory, row-major in the order
 * W1 [64][50], b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3]; the
 * matrices are used as BF16 (round to nearest even), the biases as FP32, and
 * every product is accumulated in FP32 (tensor cores for the two hidden
 * layers).  Training uses the mean squared error over samples and channels,
 * L = sum (spline + r - target)^2 / (3 M), and Adam. */
#define GS_MLP_IN 50
#define GS_MLP_HIDDEN 64
#define GS_MLP_PARAMS 7619
#define GS_MLP_ROW 64   /* BF16 values per feature row of gs_mlp_samples (50 used) */

/* Spline plus residual at any output size (the sizes of gs_upscale_to), the
 * MLP fused into the upscale pass.  params == NULL: the spline alone
 * (gs_upscale_to).  out [3][H2][W2].  Asynchronous; a bounded device wait that
 * expires is reported by gs_synchronize (GS_ERR_TIMEOUT). */
gs_status gs_upscale_mlp(gs_ctx* ctx, const float* C, const float* grads, int32_t W, int32_t H, int32_t W2,
                         int32_t H2, const float* params, float* out);

/* Training samples of the residual at M output pixels (device int32 [M][2] of
 * (X, Y) in the W2 x H2 output): features [M][GS_MLP_ROW] as BF16 bit
 * patterns (slots 50..63 zero), the spline value base [M][3] and, when
 * target_image [3][H2][W2] and target are given, target [M][3] = the image at
 * the pixel.  All device memory.  A pixel outside the output is written as
 * zeros and reported by gs_synchronize (GS_ERR_DEVICE_CHECK). */
gs_status gs_mlp_samples(gs_ctx* ctx, const float* C, const float* grads, int32_t W, int32_t H, int32_t W2,
                         int32_t H2, const int32_t* pixels, int64_t M, const float* target_image,
                         uint16_t* features, float* base, float* target);

/* Loss and gradient over M samples: grads [GS_MLP_PARAMS] = dL/dparams
 * (overwritten; the gradient of the BF16-rounded matrices, applied to the FP32
 * values), *loss = L (device float, overwritten; may be NULL).  Asynchronous. */
gs_status gs_mlp_gradient(gs_ctx* ctx, const float* params, const uint16_t* features, const float* base,
                          const float* target, int64_t M, float* grads, float* loss);

/* One Adam step (Kingma and Ba, 2015, with bias correction) at step >= 1:
 * m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g^2,
 * params -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps).
 * All arrays device FP32 [GS_MLP_PARAMS]; m and v start at zero. */
gs_status gs_mlp_adam(gs_ctx* ctx, float* params, float* m, float* v, const float* grads, int32_t step, float lr,
                      float beta1, float beta2, float eps);

/* ---- Reverse mode (training with differentiable upscaling; supplement
 * "Backward Pass").  All gradients are of one scalar loss L; upstream arrays
 * hold dL/d(output).  Asynchronous on the context's stream. */

/* Adjoint of gs_upscale (a linear map): dL_dout [3][factor*H][factor*W] ->
 * dL_dC [3][H][W] and dL_dgrads [3 (d/dx, d/dy, d2/dxdy)][3][H][W], overwritten.
 * Each low-res value gathers the output pixels whose cell has it as a corner,
 * weighted by the same Hermite basis; no atomics.  W, H >= 2; 1 <= factor <= 16. */
gs_status gs_upscale_backward(gs_ctx* ctx, const float* dL_dout, int32_t W, int32_t H, int32_t factor,
                              float* dL_dC, float* dL_dgrads);

/* Adjoint of gs_upscale_to: dL_dout [3][H2][W2] (same size rules). */
gs_status gs_upscale_backward_to(gs_ctx* ctx, const float* dL_dout, int32_t W, int32_t H, int32_t W2, int32_t H2,
                                 float* dL_dC, float* dL_dgrads);

/* Adjoint of the last derivative blend (gs_render_with_grads, or
 * gs_render_binned with out_grads, after gs_project): upstream dL_dC [3][H][W]
 * and dL_dgrads [3][3][H][W] (dL_dgrads may be NULL: zero) -> grad2d [n][9],
 * overwritten: dL/d(mean_x, mean_y, conic a, conic b, conic c, opacity, r, g, b)
 * per Gaussian, with g = -1/2 (a dx^2 + 2 b dx dy + c dy^2) (b the off-diagonal
 * entry).  Per pixel the tile list is walked back to front from the last
 * blended Gaussian, with the blend state before each step recovered from the
 * stored final state by inverting T -> T (1 - alpha) (the inversion trick of
 * the supplement, written for T = 1 - A).  GS_ERR_NOT_READY without such a
 * blend since the last projection or option change. */
gs_status gs_render_backward(gs_ctx* ctx, const float* dL_dC, const float* dL_dgrads, float* grad2d);

/* Adjoint of the last gs_project: grad2d [n][9] (the layout above) -> the
 * gradients of the projected Gaussians' inputs.  The arrays passed to that
 * gs_project must still hold the same values.  Culled Gaussians get zeros. */
gs_status gs_project_backward(gs_ctx* ctx, const float* grad2d, const gs_gaussian_grads* out);

/* The whole chain of the last project -> derivative blend -> upscale by
 * factor: gs_upscale_backward into context scratch, gs_render_backward,
 * gs_project_backward.  dL_dout [3][factor*H][factor*W]. */
gs_status gs_backward(gs_ctx* ctx, const float* dL_dout, int32_t factor, const gs_gaussian_grads* out);

/* gs_render_with_grads for callers that cannot allocate device memory (an
 * engine or compositor that owns every device byte, a plugin restricted to
 * the buffers its host provides, a real-time loop that must not stall on an
 * allocation).  The paper has no counterpart; it is a deployment variant of
 * the render above and produces the same outputs.
 *
 * No context: every scratch buffer comes from one file-scope device array of
 * about 6.6 MB that each GPU loading the library holds until the process
 * exits; no cudaMalloc, cudaFree or other allocating call is made.  Limits:
 * g->n <= 16384, W * H <= 65536 with W, H <= 4096, at most 262144
 * (super-tile, Gaussian) pairs; beyond them GS_ERR_CAPACITY and
 * nothing is written.  opt may be NULL (3DGS mode, black background);
 * opt->flags must be 0 (GS_ERR_INVALID_ARG otherwise: the call always waits
 * for its pair count), and opt->max_pairs limits the (tile, Gaussian) pairs
 * as for gs_render_with_grads (GS_ERR_CAPACITY beyond it, nothing written).
 * stream: a cudaStream_t (NULL = legacy default stream).  Inputs and outputs
 * are caller-owned device pointers as for gs_render_with_grads: out_C
 * [3][H][W], out_grads [3][3][H][W].
 *
 * The first call on each device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress; make it before any stream
 * capture.  The call synchronises the stream (pair-count readback and a final
 * error check).  All calls share the array and its contents persist between
 * calls; whatever must start at zero is cleared by each call.  Calls whose
 * work could overlap on the same GPU (other streams, other host threads) race
 * on that GPU's array and must be serialised by the caller.  The host side
 * keeps no per-call state outside the call (the read-backs are locals, the
 * per-device address an atomic word), so calls on different GPUs from
 * different host threads are independent. */
gs_status gs_render_with_grads_noalloc(const gs_gaussians* g, const gs_camera* cam, int32_t W, int32_t H,
                                       const gs_options* opt, void* stream, float* out_C, float* out_grads);

/* Number of (tile, Gaussian) pairs of the last gs_project (host int64).  After
 * a frame with GS_FLAG_NO_HOST_WAIT it waits for the stream and reads the count
 * the frame produced (also when it exceeded the reservation). */
gs_status gs_pair_count(gs_ctx* ctx, int64_t* P);

/* Number of (super-tile, Gaussian) pairs of the last gs_project (a super-tile
 * is ks x ks tiles of 16 x 16 pixels, ks the smallest of 1, 2, 4 for which the
 * frame has at most 256 super-tiles, else 4; 4 in GS_MODE_EXACT):
 * the pair buffers' size (and the super_pairs a gs_reserve for such frames
 * needs).  Waits as gs_pair_count does. */
gs_status gs_super_pair_count(gs_ctx* ctx, int64_t* Ps);

/* Copy the last gs_project's per-Gaussian results to caller device buffers (any
 * may be NULL): mean2d [n][2], conic [n][3] (Sigma'^-1 as a, b, c), rgb [n][3],
 * opacity [n], depth [n], radius [n] (int32, 0 = culled), tiles_touched [n]. */
gs_status gs_read_projected(gs_ctx* ctx, float* mean2d, float* conic, float* rgb, float* opacity,
                            float* depth, int32_t* radius, int32_t* tiles_touched);

/* Copy the last gs_project's sorted pair list and per-tile ranges to caller
 * device buffers: keys [P] (tile << 32 | FP32 depth bits), vals [P] (Gaussian id),
 * ranges [tiles][2] ([start, end) into the list; [0, 0) for an empty tile),
 * tiles = ceil(W/16) * ceil(H/16).  capacity: the length of keys/vals; fails
 * with GS_ERR_CAPACITY if P > capacity.  Any pointer may be NULL. */
gs_status gs_read_bins(gs_ctx* ctx, uint64_t* keys, uint32_t* vals, uint32_t* ranges, int64_t capacity);

/* Copy the per-pixel state of the last blend: state [4][H][W] = transmittance
 * T_N = 1 - A_N and its d/dx, d/dy, d2/dxdy; count [H][W] (int32) = 1 + the list
 * position of the last Gaussian blended (0 = none).  Either may be NULL. */
gs_status gs_read_state(gs_ctx* ctx, float* state, int32_t* count);

/* Duration of each tile's block in the last blend, in units of 16 SM clock
 * cycles: work [tiles_y][tiles_x] (device uint32; the next frame's blend takes
 * the tiles heaviest first by these).  For load-balance inspection. */
gs_status gs_read_tile_work(gs_ctx* ctx, uint32_t* work);

/* Work counts of a blend of the last gs_project's binning (3DGS or exact mode
 * as configured): counts[0] = (pixel, Gaussian) pairs evaluated, counts[1] =
 * pairs blended, summed over the image (host int64[2]).  Runs a counting
 * variant of the blend kernel that writes no image; synchronises. */
gs_status gs_blend_stats(gs_ctx* ctx, int64_t* counts);

/* Number of kernels libgs has launched on behalf of ctx since gs_create (host
 * int64; counts every kernel of every call, e.g. for launch accounting). */
gs_status gs_launch_count(const gs_ctx* ctx, int64_t* count);

/* Fault injection for tests of the error paths (no counterpart in the paper).
 * Nothing injected faults, traps or hangs the GPU:
 *   GS_INJECT_WAIT_EXPIRY, value = polls (1..2^24): the next frame whose depth
 *     sort is the persistent cooperative sort (up to about 10k Gaussians per
 *     SM) first makes one thread wait, with that bound, for a device word that
 *     nothing sets.  The wait runs out, records the expiry in the context's
 *     error word like any bounded wait of the library, and the frame goes on
 *     unchanged; the next gs_synchronize returns GS_ERR_TIMEOUT.
 *   GS_INJECT_ALLOC_FAILURE, value = n >= 0: the scratch allocation after the
 *     next n ones fails as if cudaMalloc had run out of memory (GS_ERR_OOM from
 *     the call that needed it; the context stays usable).
 *   GS_INJECT_NONE: cancel both.
 * Each injection is consumed once. */
#define GS_INJECT_NONE 0
#define GS_INJECT_WAIT_EXPIRY 1
#define GS_INJECT_ALLOC_FAILURE 2
gs_status gs_debug_inject(gs_ctx* ctx, int32_t what, int64_t value);

/* Wait for the context's stream and report any device-side error recorded by
 * its kernels since the last check (GS_ERR_TIMEOUT / GS_ERR_DEVICE_CHECK, or
 * GS_ERR_CAPACITY for a frame beyond its reservation under
 * GS_FLAG_NO_HOST_WAIT). */
gs_status gs_synchronize(gs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
