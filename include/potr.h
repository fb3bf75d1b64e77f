/*
 * potr.h -- C ABI of the GB300 (sm_103a) removal-effect rasterizer.
 *
 * The library computes, for one or many views of a 3D Gaussian splat scene, every splat's
 * removal effect: the change in squared error against a target image when that splat alone
 * is dropped from front-to-back alpha compositing (POTR, arXiv 2601.14821, Section IV-B,
 * Eqs. "pruning difference" and "pixel squared error"), summed over pixels and views into
 * dMSE_k (Section IV-B, last equation), together with the splat importance I_k (Section IV-A).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* and every pointer inside potr_views / potr_frame are DEVICE
 *     pointers owned by the caller.  Pointers named h_* are host pointers.  The library
 *     never allocates or frees memory.  It keeps no device state between calls, with one
 *     exception: potr_bin_sort_static (for callers that cannot allocate) works in a fixed
 *     scratch array of the library's own, held by every GPU that loads it until exit.
 *   - Work is enqueued asynchronously on the caller's stream; no call synchronises the
 *     host with the device, so a sequence of calls can be captured in a CUDA graph.
 *   - Return value: POTR_OK, or an error detected on the host before anything was
 *     enqueued (POTR_ERR_INVALID_ARGUMENT, POTR_ERR_UNSUPPORTED), or POTR_ERR_CUDA when a
 *     launch failed.  Errors found on the device (instance capacity exceeded, a non-finite
 *     splat parameter, a bounded wait that ran out) are written to a caller-provided
 *     potr_device_status, read by the caller after synchronising.
 *   - Planes: "[3][n]" means three contiguous arrays of n floats (structure of arrays).
 *   - Index "vk" = v * n + k for view v and splat k of a frame.
 */
#ifndef POTR_H_
#define POTR_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define POTR_API __attribute__((visibility("default")))
#else
#define POTR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* potr_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef int32_t potr_status;
enum {
  POTR_OK = 0,
  POTR_ERR_INVALID_ARGUMENT = 1,
  POTR_ERR_CUDA = 2,
  POTR_ERR_CAPACITY = 3, /* device: more tile instances than instance_capacity */
  POTR_ERR_TIMEOUT = 4,  /* device: a bounded wait ran out */
  POTR_ERR_NUMERIC = 5,  /* device: a splat parameter is NaN or infinite (potr_preprocess) */
  POTR_ERR_UNSUPPORTED = 6,
  POTR_ERR_TOO_LARGE = 7, /* a size exceeds potr_bin_sort_static's fixed scratch */
  POTR_ERR_CORRUPT = 8    /* device: a malformed codec stream (potr_codec_decode) */
};

/* Device-side status word; zero it before the calls that may write it. */
typedef struct {
  int32_t code;               /* POTR_OK or a POTR_ERR_* code (the first error written wins) */
  int32_t n_nonfinite;        /* splats culled for a non-finite parameter (potr_preprocess) */
  int64_t required_instances; /* instance count needed when code == POTR_ERR_CAPACITY */
} potr_device_status;

/*
 * Splat parameters (Section 3): N splats as SoA planes, all float32 device arrays.
 *   means[3][n]          centre mu
 *   log_scales[3][n]     scale = exp(log_scale) per principal axis
 *   quats[4][n]          rotation quaternion (w, x, y, z), w real; normalised on use
 *   opacity_logits[n]    base opacity o = sigmoid(logit)
 *   sh[16][3][n]         SH coefficients L_i per channel, index i = l(l+1)+m (degree <= 3)
 */
typedef struct {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  int64_t n;
} potr_scene;

/* Pinhole camera: world-to-camera rows [R | t], camera space looks along +z, image y down. */
typedef struct {
  float w2c[12];
  float fx, fy, cx, cy;
  int32_t width, height;
} potr_camera;

/*
 * Rasterizer configuration.  tile_w * tile_h must be 256 (16x16, 8x32 or 32x8); batch must be
 * 128, 256 or 512 and no longer changes anything (the tile kernels size their own staging of
 * records; the field keeps earlier configurations valid).  The remaining
 * fields are the readings of the original 3DGS renderer the paper modifies (Section 3):
 *   near_z     cull when camera-space z <= near_z                         (default 0.2)
 *   lowpass    added to the diagonal of the 2D covariance, pixel^2       (default 0.3)
 *   alpha_min  a pixel skips a splat whose alpha < alpha_min             (default 1/255)
 *   alpha_max  alpha is clamped to alpha_max                              (default 0.99)
 *   t_min      compositing stops before a splat that would take T below t_min (1e-4)
 */
typedef struct {
  int32_t tile_w, tile_h;
  int32_t batch;
  float near_z, lowpass, alpha_min, alpha_max, t_min;
} potr_raster_config;

/* Placement of one view inside a frame (a set of views processed together). */
typedef struct {
  int32_t width, height;
  int32_t tiles_x, tiles_y;
  int64_t tile_base;  /* first global tile index of the view */
  int64_t pixel_base; /* first pixel of the view in packed per-pixel arrays */
} potr_view_info;

/* A frame: views laid out one after another (tiles and pixels in view order). */
typedef struct {
  const potr_camera* cams;     /* device [n_views] */
  const potr_view_info* info;  /* device [n_views], from potr_view_layout */
  int32_t n_views;
  int64_t total_tiles;
  int64_t total_pixels;
} potr_frame;

/*
 * Per-(view, splat) buffers produced by potr_preprocess and potr_bin_sort (device, caller
 * owned).  raster holds 12 floats (48 bytes) per vk, 16-byte aligned (written for the vk with
 * kept tiles):
 *   [0] mean x  [1] mean y  [2] A  [3] B  [4] C  [5] opacity  [6] prefilter  [7] indefinite
 *   [8] r       [9] g       [10] b [11] rectangle bits (x0 | y0 << 11 | width << 22)
 * where log2 G(dx, dy) = A dx^2 + B dx dy + C dy^2 and [7] is 0 when that form is negative
 * definite (decided exactly), 1 otherwise.  cull holds 4 words per vk, 16-byte
 * aligned (written for every vk):
 *   [0] kept-tile mask, low word  [1] high word  [2] rectangle bits (as raster [11])
 *   [3] kept tiles | (1 << 31 if every tile is kept)
 * where mask bit (ty - y0) width + (tx - x0) says whether tile (tx, ty) of the rectangle is
 * kept (rectangles of at most 64 tiles; larger ones keep every tile).  A vk's emission slots
 * start at offsets[vk] (written by potr_bin_sort).
 */
typedef struct {
  float* cov3d;          /* [6][n] activated covariance (xx, xy, xz, yy, yz, zz) */
  float* opacity;        /* [n] */
  float* raster;         /* [V * n][12] */
  float* depth;          /* [V * n] camera-space z, the sort key's low word */
  uint32_t* rect;        /* [V * n][2] (x0 | y0 << 16, x1 | y1 << 16), tiles, half open */
  uint32_t* touched;     /* [V * n] kept tiles, 0 when culled */
  uint32_t* offsets;     /* [V * n] exclusive prefix sum of touched (emission slots) */
  uint32_t* n_instances; /* [1] total instances (potr_bin_sort) */
  uint32_t* cull;        /* [V * n][4] kept-tile mask, rectangle, kept count (see above) */
} potr_views;

/*
 * Measurement hook (no counterpart in the paper).  Arms two CUDA events (cudaEvent_t, passed as
 * void*, created by the caller) for the next tile-pass kernel this host thread launches -- the
 * compositing kernel of potr_render, the removal-effect kernel of potr_removal_effect or the
 * backward tile kernel of potr_render_backward: start is recorded on that call's stream just
 * before the kernel and stop just after it, so the time between them is the kernel's alone
 * (no memsets, no per-splat reductions).  The launch disarms the hook; (NULL, NULL) disarms it
 * without a launch.  INVALID_ARGUMENT when exactly one event is NULL.  Host state only.
 */
POTR_API potr_status potr_time_next_tile_kernel(void* start_event, void* stop_event);

/* Text for a status code (static string). */
POTR_API const char* potr_status_string(potr_status status);

/* Library version, major * 10000 + minor * 100 + patch. */
POTR_API int32_t potr_version(void);

/*
 * Host only.  Fills h_info[n_views] from h_cams and cfg (tiles per view, tile and pixel
 * bases in view order) and the frame totals.  Errors: INVALID_ARGUMENT on a bad tile
 * shape or camera size; UNSUPPORTED when a view has more than 1023 tile columns or 2047
 * tile rows (the raster record packs the rectangle in 32 bits).
 */
POTR_API potr_status potr_view_layout(const potr_camera* h_cams, int32_t n_views, const potr_raster_config* cfg,
                             potr_view_info* h_info, int64_t* total_tiles, int64_t* total_pixels);

/*
 * Section 3 (Eqs. 1-2 and the SH colour equation): activation of every splat (exp of the
 * log-scales, quaternion normalisation, Sigma = R S S^T R^T, o = sigmoid(logit)), then, for
 * every view of the frame, EWA projection (view transform, near cull, clamped Jacobian,
 * Sigma2D = J W Sigma W^T J^T + lowpass I, conic, radius ceil(3 sqrt(lambda_max))), pixel
 * centre, tile rectangle, depth and the SH colour max(0, sum_i L_i Y_i(d) + 0.5) along the
 * camera-to-splat direction d.  A tile of the rectangle is kept only if some pixel centre in
 * it can reach alpha >= alpha_min (the exponent's maximum over the tile's pixel-centre
 * rectangle, on its edges or at the splat centre, plus a rounding margin of 1e-5 x the
 * largest term magnitude + 1e-4, through the same exp2): such tiles hold no pair the
 * compositor takes, so no output changes.  Rectangles of more than 64 tiles keep every tile.
 * Writes views->cov3d, opacity, raster (all but the offset word), depth, rect, touched
 * (kept tiles).  Every quantity that decides the binning or the per-pixel
 * alpha test is computed in binary32 with a fixed operation order (no contraction), with
 * exp taken by a reproducible exp2 (Cody-Waite reduction plus a degree-6 Taylor polynomial).
 * Non-finite parameters (no counterpart in the paper): a splat whose mean, log-scale,
 * quaternion or opacity logit holds a NaN or an infinity -- or one of its 48 SH coefficients,
 * checked where the splat is first visible -- is culled in every view (touched 0: it enters no
 * list, image, removal effect or gradient; its opacity is stored as NaN).  Each such splat adds
 * 1 to d_status->n_nonfinite and the first one writes POTR_ERR_NUMERIC to d_status->code
 * (d_status: device, caller-zeroed, nullable -- then the splats are still culled, silently).
 * cfg->tile_w * cfg->tile_h must be 256 (as for potr_view_layout), else
 * POTR_ERR_INVALID_ARGUMENT.
 */
POTR_API potr_status potr_preprocess(const potr_scene* scene, const potr_frame* frame, const potr_raster_config* cfg,
                            const potr_views* views, potr_device_status* d_status, potr_stream_t stream);

/* Workspace bytes of potr_tile_schedule. */
POTR_API size_t potr_tile_schedule_workspace_size(void);

/*
 * Longest-list-first order of the frame's tiles (no counterpart in the paper: scheduling of
 * the per-tile work of Section 3's compositing).  Tiles are bucketed by the bit length of their
 * list length from d_tile_ranges; d_tile_order[0 .. total_tiles) receives the tiles of the
 * longest bucket first and empty tiles last (order inside a bucket unspecified).  The word at
 * d_tile_order[total_tiles] is left for the work counter of the tile kernels.
 */
POTR_API potr_status potr_tile_schedule(const potr_frame* frame, const uint32_t* d_tile_ranges,
                                        uint32_t* d_tile_order, void* d_ws, size_t ws_bytes, potr_stream_t stream);

/* Workspace bytes potr_bin_sort needs (scan partials, sort double buffers for the V * n depth
 * keys and the instances, histograms): about 16 (V * n) + 8 instance_capacity bytes. */
POTR_API size_t potr_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t total_tiles, int64_t instance_capacity);

/*
 * Binning (Section 3, "ordering these layers according to the splats' approximate depth").
 * Defined result: one instance per kept tile, emitted in vk order and, within a rectangle,
 * row-major, with key (global tile << 32) | bits(depth) and value vk, stably sorted by key;
 * its emission slot is views->offsets[vk] (exclusive scan of touched over vk) plus the tile's
 * rank among the vk's kept tiles.  Outputs: d_tiles[i] = the
 * global tile (the key's high word) and d_vals[i] = vk of sorted instance i, both
 * instance_capacity entries; *views->n_instances; per-global-tile [start, end) ranges into
 * d_tile_ranges[total_tiles][2] (empty tiles get [0, 0)).  Computed as a stable radix sort
 * of the vk by depth bits, emission in that order, and a stable radix partition by tile,
 * which yields the same order.  If the instance count exceeds instance_capacity, d_status
 * gets POTR_ERR_CAPACITY and the required count, and every tile range is left empty.
 * UNSUPPORTED if the frame has 2^32 or more tiles or V * n >= 2^32 - 1.
 */
POTR_API potr_status potr_bin_sort(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                          int64_t n, int64_t instance_capacity, uint32_t* d_tiles, uint32_t* d_vals,
                          uint32_t* d_tile_ranges, potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                          potr_stream_t stream);

/*
 * Render (Section 3, Eqs. 2-4): per pixel, front to back over its tile's sorted list,
 * alpha = min(alpha_max, o G), skip alpha < alpha_min, stop before T (1 - alpha) < t_min,
 * c = sum T_k alpha_k c_k over a black background.  Outputs (device, per frame pixel):
 * d_images planar [3][H][W] per view at offset 3 * pixel_base; d_t_final the final
 * transmittance; d_n_last one past the tile-list position of the last composited splat
 * (0 if none).  Any output may be NULL.  d_tile_order (nullable, [total_tiles + 1]) is a tile
 * order from potr_tile_schedule: with it the kernel's warps take (tile, 8 x 8 pixel block) items
 * in that order (the last word is the work counter, reset by the call); without it they take
 * the items in tile index order.  The order changes scheduling only, never a result.
 */
POTR_API potr_status potr_render(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                 int64_t n, const uint32_t* d_vals, const uint32_t* d_tile_ranges,
                                 uint32_t* d_tile_order, float* d_images, float* d_t_final, uint32_t* d_n_last,
                                 potr_stream_t stream);

/*
 * Removal effect (Section IV-B).  For every pixel: the render above, then a back-to-front
 * pass over the composited splats that forms, with S_{>i} = P_K - P_{i+1} (suffix sum),
 *   PD_i  = alpha_i / (1 - alpha_i) S_{>i} - T_i alpha_i c_i     (Eq. pruning difference)
 *   dSE_i = sum_ch PD_i (PD_i + 2 (c - c_t))                      (Eq. pixel squared error)
 * reduced per (tile, splat) in a fixed order (warp transpose-sums over each 8 x 8 pixel block,
 * then the tile's blocks in order) into
 * d_inst_dse[emission slot] (float, instance_capacity entries, required; the same capacity
 * as potr_bin_sort -- when the frame's instance count exceeded it, nothing is reduced and
 * d_dmse / d_importance / d_dsse_view are left untouched).  Then, per
 * splat, the tile partials are summed in emission order (a compensated binary32 sum, rounded
 * to binary32), giving dSSE_k(v) = sum_x dSE, and
 *   d_dmse[k] += dSSE_k(v) / (3 P_v n_views_total)        (binary64, views added in order)
 * where the term is dSSE_k(v) times the binary32 rounding of 1 / (3 P_v n_views_total),
 * rounded to binary32, so that calls over consecutive view chunks add the same terms in the
 * same order as one call over all of them (zero d_dmse before the first call).
 * With d_inst_imp / d_importance non-NULL the same is done for T_i alpha_i, giving
 * I_k += (sum_x T alpha) / (P_v n_views_total) (Section IV-A).  d_dsse_view (nullable,
 * [n_views][n] binary64) receives dSSE_k(v) itself, and d_imp_view (nullable, [n_views][n]
 * binary64, needs d_inst_imp) the per-view importance I_k(v) = (sum_x T alpha) / P_v (the
 * weights of the SH energy compaction).  d_images (nullable) receives the
 * render.  d_targets: planar [3][H][W] per view at offset 3 * pixel_base.  d_tile_order as in
 * potr_render.  d_ws: potr_removal_workspace_size(instance_capacity, total_tiles, d_inst_imp !=
 * NULL) bytes of device scratch (the per-block sums before they are added per tile: 16 bytes per
 * instance, 32 with importance, and 20 bytes per tile, each part aligned to 256 bytes; 0 for a
 * non-positive size).
 */
POTR_API size_t potr_removal_workspace_size(int64_t instance_capacity, int64_t total_tiles, int32_t with_importance);
POTR_API potr_status potr_removal_effect(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                int64_t n, const uint32_t* d_vals, const uint32_t* d_tile_ranges,
                                uint32_t* d_tile_order, const float* d_targets, int32_t n_views_total,
                                int64_t instance_capacity,
                                float* d_inst_dse,
                                float* d_inst_imp, double* d_dmse, double* d_importance, double* d_dsse_view,
                                double* d_imp_view, float* d_images, void* d_ws, size_t ws_bytes,
                                potr_stream_t stream);

/* Gradients of a scene's parameters: the same SoA planes as potr_scene (device, overwritten). */
typedef struct {
  float* means;          /* [3][n] */
  float* log_scales;     /* [3][n] */
  float* quats;          /* [4][n] */
  float* opacity_logits; /* [n] */
  float* sh;             /* [16][3][n] */
} potr_scene_grads;

/* Workspace bytes of potr_loss_grad (a per-block partial sum when the loss value is wanted). */
POTR_API size_t potr_loss_workspace_size(int64_t total_pixels);

/*
 * Fine-tuning loss of POTR-FT (Section IV-F fine-tunes with the original 3DGS training
 * routine; its SSIM term is replaced by a squared error):
 *   L = (1 - lambda) mean |c - c_t| + lambda mean (c - c_t)^2
 * over every channel of every pixel of the frame (d_images, d_targets packed like
 * potr_render's images).  Writes dL/dc to d_dL_dimages (same layout; the L1 subgradient at
 * c = c_t is 0) and, when d_loss is non-NULL, L as binary64 (summed in a fixed order; needs
 * potr_loss_workspace_size bytes of d_ws).  0 <= lambda <= 1.
 */
POTR_API potr_status potr_loss_grad(const potr_frame* frame, const float* d_images, const float* d_targets,
                                    float lambda, double* d_loss, float* d_dL_dimages, void* d_ws, size_t ws_bytes,
                                    potr_stream_t stream);

/* Workspace bytes of potr_render_backward: 9 floats of partial gradients per instance slot
 * (instance_capacity) and 13 floats per (view, splat) (n_view_splats = n_views * n).  0 for a
 * non-positive argument. */
POTR_API size_t potr_render_backward_workspace_size(int64_t instance_capacity, int64_t n_view_splats);

/*
 * Backward (adjoint) rasterizer, the derivative of potr_render with respect to the scene
 * parameters for a given dL/dc (d_dL_dimages, packed like the images).  Per pixel, back to
 * front over the composited splats with S_{>i} = sum_{j>i} T_j alpha_j c_j:
 *   dL/dc_i     = T_i alpha_i dL/dc
 *   dL/dalpha_i = T_i c_i . dL/dc - S_{>i} . dL/dc / (1 - alpha_i)      (Section 3, Eqs. 2-4)
 * then through alpha = o 2^p (zero where alpha is clamped to alpha_max) to the opacity, the
 * exponent coefficients and the pixel-space centre; per (tile, splat) sums in a fixed order;
 * per splat, the adjoint of the EWA projection, the SH colour (zero where it is clamped at 0)
 * and the activation, summed over the frame's views in order.  Decisions (which splats a pixel
 * composites) are those of the forward pass and carry no gradient.  The depth order and the
 * tile rectangle carry none either.
 * Transmittance: pass the forward render's d_t_final and d_n_last (stored), or NULL for both to
 * recompute them inside the kernel (no per-pixel storage; results are identical).  The same
 * inputs as potr_render plus the scene; writes every plane of *grads.  d_ws:
 * potr_render_backward_workspace_size bytes.  d_tile_order as in potr_render.
 */
POTR_API potr_status potr_render_backward(const potr_scene* scene, const potr_views* views, const potr_frame* frame,
                                          const potr_raster_config* cfg, const uint32_t* d_vals,
                                          const uint32_t* d_tile_ranges, uint32_t* d_tile_order,
                                          const float* d_t_final,
                                          const uint32_t* d_n_last, const float* d_dL_dimages,
                                          int64_t instance_capacity, const potr_scene_grads* grads, void* d_ws,
                                          size_t ws_bytes, potr_stream_t stream);

/*
 * Exact pair counts for throughput and roofline accounting (no counterpart in the paper;
 * the counts define the algorithmic work of Section 3 / IV-B in pairs).  d_counts[5]
 * (device, uint64, overwritten): [0] (pixel, splat) pairs examined by the front-to-back walk,
 * [1] of those passing the opacity prefilter, [2] pairs composited, [3] list positions
 * walked back to front by the removal pass (sum of n_last), [4] of those passing the
 * prefilter.  Same inputs as potr_render.
 */
POTR_API potr_status potr_pair_stats(const potr_views* views, const potr_frame* frame, const potr_raster_config* cfg,
                                     int64_t n, const uint32_t* d_vals, const uint32_t* d_tile_ranges,
                                     uint64_t* d_counts, potr_stream_t stream);

/*
 * potr_bin_sort without a workspace argument, for callers that cannot allocate device
 * memory (no counterpart in the paper).  Same inputs, outputs and device-status behaviour as
 * potr_bin_sort; the scratch it needs lives in a 56 MiB array inside the library, held by
 * every GPU that loads the library until the process exits.  Limits: instance_capacity <=
 * POTR_STATIC_MAX_INSTANCES and n * n_views <= POTR_STATIC_MAX_VIEW_SPLATS, otherwise it
 * returns POTR_ERR_TOO_LARGE and enqueues nothing.  Calls made outside a stream capture look up
 * the array's device address; calls inside a capture use the address the last such call found,
 * so the first call on a device must come before any capture (else POTR_ERR_UNSUPPORTED).
 * Calls share the array: calls that overlap on the GPU race, so serialise them.  It allocates
 * nothing.
 */
#define POTR_STATIC_MAX_INSTANCES 4194304LL
#define POTR_STATIC_MAX_VIEW_SPLATS 1048576LL
POTR_API potr_status potr_bin_sort_static(const potr_views* views, const potr_frame* frame,
                                          const potr_raster_config* cfg, int64_t n, int64_t instance_capacity,
                                          uint32_t* d_tiles, uint32_t* d_vals, uint32_t* d_tile_ranges,
                                          potr_device_status* d_status, potr_stream_t stream);

/*
 * Self-test of the library's bounded device waits (no counterpart in the paper).  The only
 * device-side wait is the sort's decoupled look-back; this runs that wait against a predecessor
 * whose counts are never published, so it must give up after spin_limit polls and write
 * POTR_ERR_TIMEOUT to *d_status (the kernel returns normally; the context stays usable).
 * d_ws: >= 4096 bytes of device scratch.
 */
POTR_API potr_status potr_selftest_wait_timeout(void* d_ws, size_t ws_bytes, int32_t spin_limit,
                                                potr_device_status* d_status, potr_stream_t stream);

/* Workspace bytes of potr_prune_select for n splats (about 16 n). */
POTR_API size_t potr_prune_workspace_size(int64_t n);

/*
 * One iteration of the pruning controller (Section IV-C, "Iterative pruning": the pruning
 * approximation, the budget and mapping-function equations).  Candidates are the splats with
 * d_alive[k] != 0 and d_dmse[k] < dmse_max.  Budget B = floor(sum of q_k over candidates /
 * remaining_iterations) with q_k = floor(d_importance[k] * 2^40) (importance counted in integer
 * units of 2^-40, so the budget test is exact; q_k = 0 when the importance is not >= 0).  The
 * removal set S is the shortest prefix of the candidates in ascending (m(d_dmse[k] / dmse_max),
 * k) order whose q-sum reaches B (empty when B = 0), with m(x) = x for x >= 0 and
 * (sqrt(1 - 2 a x) - 1) / a for x < 0, in binary64 IEEE arithmetic in that order.  Effect:
 * d_alive[k] = 0 for k in S; *d_removed (device, nullable) = |S|.
 * Inputs (device): d_dmse, d_importance [n] binary64 (potr_removal_effect's outputs);
 * d_alive [n] uint8, in/out.  d_ws: potr_prune_workspace_size(n) bytes.  n <= 2^32 - 1,
 * remaining_iterations >= 1, dmse_max > 0, a > 0, else INVALID_ARGUMENT.  Asynchronous; no
 * host synchronisation, graph-capturable.
 */
POTR_API potr_status potr_prune_select(int64_t n, const double* d_dmse, const double* d_importance,
                                       uint8_t* d_alive, double dmse_max, double a, int32_t remaining_iterations,
                                       unsigned long long* d_removed, void* d_ws, size_t ws_bytes,
                                       potr_stream_t stream);

/*
 * Removes the pruned splats from the scene (Section IV-C: the splats of the removal set S leave
 * it): d_opacity_logits[k] = -infinity where d_alive[k] == 0 (opacity 0 after activation: the splat keeps no tile and composites nowhere, so its
 * removal effect and importance are 0 from then on).  Device arrays of n entries.
 */
POTR_API potr_status potr_prune_apply(int64_t n, const uint8_t* d_alive, float* d_opacity_logits,
                                      potr_stream_t stream);

/*
 * Spherical-harmonics energy compaction (Section IV-D: the per-splat linear system, the
 * ridge-regression closed form with the Tikhonov matrix that spares the DC coefficient, and the
 * importance, colour-model, sparsity and two-pass modifications).  For every splat k of the
 * scene and every view s of the frame with I_k(s) = d_imp_view[s * n + k] > 0 (from
 * potr_removal_effect), weighted relative to each other, w_s = I_k(s) / max_s' I_k(s'): rows
 * w_s Y(d_s) of the real SH basis at the direction camera -> splat and
 * colours w_s C(d_s), C = sum_i L_i Y_i(d_s) the splat's linear SH colour (before the +0.5 offset
 * and the clamp) in YCoCg (Y = R/4 + G/2 + B/4, Co = R/2 - B/2, Cg = -R/4 + G/2 - B/4).  Columns
 * are kept in index order unless |cosine| with a kept preceding column exceeds alpha (or the
 * column is all zero); the DC column is always kept.  Pass 1 solves, per YCoCg channel, the
 * ridge system over the kept columns with lambda (Y) or 3 lambda (Co, Cg) on the AC
 * coefficients only; pass 2 repeats it per channel without the AC coefficients x of pass 1 with
 * floor(1/2 + x sf) == 0 (quantised to zero).  A splat no view sees keeps its coefficients.
 * Binary64 throughout.  Outputs (device, nullable): d_sh_out [16][3][n] float, the compacted
 * coefficients back in RGB (must not alias scene->sh); d_sh_ycocg [16][3][n] binary64, in YCoCg;
 * d_kept [4][n] bit masks of the kept columns (after the cosine test, then per channel after
 * pass 2; all 0 for an unseen splat).  Paper values: lambda = 10^-q, alpha = sigmoid(3q),
 * sf = 1 + 100 q.
 */
POTR_API potr_status potr_sh_compact(const potr_scene* scene, const potr_frame* frame, const double* d_imp_view,
                                     double lambda, double alpha, double sf, float* d_sh_out, double* d_sh_ycocg,
                                     uint32_t* d_kept, potr_stream_t stream);

/*
 * One Adam step over every parameter plane of a scene (the optimiser of the fine-tuning loop,
 * Section IV-F: the original 3DGS training routine; Kingma & Ba 2015 in PyTorch's form):
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   p <- p - (lr / (1 - b1^step)) m / (sqrt(v) / sqrt(1 - b2^step) + eps)   (p unchanged if m = 0).
 * params / m / v: device planes in the potr_scene layout, updated in place; grads: the
 * gradients (e.g. from potr_render_backward).  lr[6] (host): means, log_scales, quats,
 * opacity_logits, SH DC (planes 0-2 of sh), SH rest (planes 3-47).  step >= 1, 0 <= beta < 1,
 * eps >= 0, else INVALID_ARGUMENT.
 */
POTR_API potr_status potr_adam_step(const potr_scene_grads* params, const potr_scene_grads* grads,
                                    const potr_scene_grads* m, const potr_scene_grads* v, int64_t n, int64_t step,
                                    const float* lr, float beta1, float beta2, float eps, potr_stream_t stream);

/* The per-step factors potr_adam_step uses (Adam's bias corrections, Kingma & Ba 2015; the
 * optimiser of Section IV-F's fine-tuning), for steps first_step .. first_step + count - 1 (host):
 * out[i][0..5] = lr[g] / (1 - beta1^t) of the six groups, out[i][6] = 1 / sqrt(1 - beta2^t),
 * t = first_step + i, computed in binary64 and rounded to float.  first_step >= 1. */
POTR_API potr_status potr_adam_schedule(int64_t first_step, int64_t count, const float* lr, float beta1,
                                        float beta2, float* out);

/* potr_adam_step (Section IV-F's fine-tuning optimiser) with t taken from the device: the
 * update of step t = *d_step + 1 uses row *d_step of d_sched ([n_sched][7], device, from
 * potr_adam_schedule with first_step 1), then *d_step is incremented on the device; a step past the table changes nothing but the counter.
 * Gives the same bits as potr_adam_step(step = t) and needs no host argument that changes from
 * step to step, so a fine-tuning iteration can be captured in a CUDA graph. */
POTR_API potr_status potr_adam_step_scheduled(const potr_scene_grads* params, const potr_scene_grads* grads,
                                              const potr_scene_grads* m, const potr_scene_grads* v, int64_t n,
                                              const float* d_sched, int64_t n_sched, uint32_t* d_step, float beta1,
                                              float beta2, float eps, potr_stream_t stream);

/* Scale factors and precision parameters of the codec (Section IV-E, hyper-parameter table:
 * SF_scale = 1 + 4000q, SF_rotation = 1 + 400q, SF_opacity = 1 + 200q, SF_SH = 1 + 100q,
 * beta = 1.4e-4 q, gamma = 5 10^(-3-5q)). */
typedef struct {
  double sf_scale, sf_rotation, sf_opacity, sf_sh, beta, gamma;
} potr_codec_params;

/* Workspace bytes of potr_codec_encode for n splats (about 150 n). */
POTR_API size_t potr_codec_workspace_size(int64_t n);

/*
 * The encoder's device part (Section IV-E, quantisation equation and the octree precision
 * criterion ||mu - mu^|| < max(gamma, beta min_s ||mu - mu_s||)).  Root cube: corner = per-axis
 * minimum of the positions, edge = the largest per-axis range (1 if all coincide); depth limit
 * 21; child octant c = (x bit << 2) | (y bit << 1) | z bit.  A cell is split while it holds
 * several splats or its single splat is not within the tolerance of the cell centre (binary64).
 * Outputs (device): d_nodes [<= 22 n] the node bytes in depth-first order -- an internal node
 * its child octant mask, every leaf 0 -- and *d_n_nodes their number; d_dups [n] (room for n/2
 * pairs) the leaves that hold several (coincident) splats, which only a depth-21 leaf can, as
 * (leaf ordinal in depth-first order, splat count - 1) pairs in ascending ordinal, and
 * *d_n_dups their number; d_order [n] the splats in that leaf order (ties by index); d_attrs [55][n]
 * int32, in that order, property after property: floor(1/2 + x SF) of the 3 log-scales, of x,
 * y, z of the normalised quaternion made to have w >= 0, of sigmoid(opacity logit), and of the
 * 48 SH values (coefficient-major; planes 0-2, the DC, as differences from the previous splat);
 * d_cube (nullable) [4] binary64: corner x, y, z and edge.  d_eyes [n_eyes][3] binary64: the
 * camera centres.  d_status as potr_bin_sort (bounded waits).  UNSUPPORTED if 22 n >= 2^31.
 */
POTR_API potr_status potr_codec_encode(const potr_scene* scene, const double* d_eyes, int32_t n_eyes,
                                       const potr_codec_params* params, uint8_t* d_nodes, uint32_t* d_n_nodes,
                                       uint32_t* d_dups, uint32_t* d_n_dups, uint32_t* d_order, int32_t* d_attrs,
                                       double* d_cube, potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                                       potr_stream_t stream);

/* Workspace bytes of potr_codec_decode for a stream of n_nodes node bytes and n splats
 * (about 22 n_nodes + 26 n). */
POTR_API size_t potr_codec_decode_workspace_size(int64_t n_nodes, int64_t n);

/*
 * The decoder's device part: the inverse of potr_codec_encode (Section IV-E; dequantisation
 * x~ = x^ / SF, opacity x~ = (x^ + 1/4) / SF).  Inputs (device): d_nodes [n_nodes] the node
 * bytes, d_dups [2 n_dups] the shared-leaf pairs, d_attrs [55][n] the quantised attributes in
 * stream order; (host) cube [4] corner x, y, z and edge, params (only the four SF are used).
 * Output: the scene in stream order, written to the planes of *out (device, float32): means =
 * the centres of the splats' leaf cells, corner + (cell + 1/2) edge / 2^depth in binary64;
 * log-scales; quaternion (w, x, y, z) with w = sqrt(max(0, 1 - x^2 - y^2 - z^2)); opacity
 * logit log(o / (1 - o)) of the dequantised opacity clamped to [1e-6, 1 - 1e-6]; the 48 SH
 * values, DC as running sums of the stored differences.  A malformed stream (a node sequence
 * that is not one complete tree of depth <= 21, table entries out of order or out of range,
 * leaf and splat counts that disagree with n) writes POTR_ERR_CORRUPT to *d_status (nullable)
 * and leaves the affected outputs unspecified; nothing is read or written out of bounds.
 * INVALID_ARGUMENT for null pointers, n_nodes <= 0, n <= 0, n_dups outside [0, n/2], a scale
 * factor or edge <= 0, or a short workspace; UNSUPPORTED if n_nodes >= 2^31 or 55 n >= 2^31.
 */
POTR_API potr_status potr_codec_decode(const uint8_t* d_nodes, int64_t n_nodes, const uint32_t* d_dups,
                                       int64_t n_dups, const int32_t* d_attrs, int64_t n, const double* cube,
                                       const potr_codec_params* params, const potr_scene_grads* out,
                                       potr_device_status* d_status, void* d_ws, size_t ws_bytes,
                                       potr_stream_t stream);

/* Number of kernels the library has launched in this process (host-side counter). */
POTR_API uint64_t potr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* POTR_H_ */
