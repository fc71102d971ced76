/*
 * bs.h -- C ABI of the GB300 Bezier Splatting rasterizer (libbs.so).
 *
 * The library implements the differentiable splatting rasterizer of
 * "Bezier Splatting for Fast and Differentiable Vector Graphics Rendering"
 * (Liu, Zhou, Zhao, Huang): 2D Gaussians sampled along cubic Bezier curves
 * and inside closed curves (Section 3.3, Eq. 3-8), binned into screen tiles
 * by (tile, depth) keys (Section 3.4), alpha-blended front to back
 * (Eq. 9-12), and the reverse-order backward to the curve parameters.
 *
 * Conventions for every call
 *   - All array pointers are DEVICE pointers owned by the caller, unless a
 *     parameter says "host".  The library never allocates device memory.
 *   - Calls are asynchronous on the given stream (a cudaStream_t; NULL is
 *     the legacy default stream).  The calls that synchronise are
 *     bs_bin_tiles and bs_bin_tiles_static (one read-back of the pair
 *     count), bs_prune_densify (its counts), bs_batch_setup (the copy of the
 *     layout table), and the status reads bs_device_status,
 *     bs_bin_tiles_result, bs_batch_status and bs_sync_status.  Every other
 *     call (bs_bin_tiles_async for the binning) can be captured in a CUDA
 *     graph.
 *   - Every call returns a bs_status.  Arguments are validated on the host
 *     before anything is launched; an invalid argument returns
 *     BS_ERR_INVALID_ARG and launches nothing.  bs_last_error() gives a
 *     thread-local message for the last non-OK status.
 *   - Errors found by a kernel are recorded in device status words and read
 *     later, so that no call waits on them: a count that overflowed in the
 *     binning workspace's word (bs_device_status, bs_bin_tiles_result), a
 *     non-finite Gaussian record or gradient in the library's own word of
 *     each device (bs_sync_status).
 *   - Coordinates are pixels: pixel (x, y) covers [x, x+1) x [y, y+1) and
 *     its centre is (x + 0.5, y + 0.5).  Colours and opacities are the
 *     activated values in [0, 1].
 *   - Images are planar float32 [3][H][W]; per-pixel maps are [H][W].
 *   - Only sm_103a is supported; other devices return BS_ERR_UNSUPPORTED.
 *   - The calls may be made from several host threads.  Per device, the
 *     library raises some kernels' dynamic shared-memory limits once (under
 *     a lock) and keeps a status word and the addresses of its device
 *     arrays; a device reset (cudaDeviceReset) discards all of them, so do
 *     not call the library on a device after resetting it in the same
 *     process.
 */
#ifndef BEZIER_SPLATTING_BS_H
#define BEZIER_SPLATTING_BS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, spelled without the CUDA headers. */
typedef struct CUstream_st *bs_stream;

typedef enum {
  BS_OK = 0,
  BS_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported parameter value */
  BS_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in bs_last_error) */
  BS_ERR_CAPACITY = 3,      /* pair_capacity too small; *n_pairs_out holds the need  */
  BS_ERR_TIMEOUT = 4,       /* a bounded device-side retry loop ran out              */
  BS_ERR_NOT_FINITE = 5,    /* a kernel wrote a non-finite record or gradient (bs_sync_status) */
  BS_ERR_UNSUPPORTED = 6    /* device or configuration the library does not support */
} bs_status;

/*
 * A set of curves (Section 3.2).  Open curves are 3 chained cubic segments
 * (10 control points, the end of one segment is the start of the next) with
 * a stroke width and one opacity per segment (Appendix D); closed curves are
 * 4 chained cubic segments whose 13th point is the first one, stored as 12
 * points, with one colour and one opacity (Appendix D).
 * Curve i < n_open is open curve i; curve n_open + j is closed curve j.
 */
typedef struct {
  int32_t n_open;
  int32_t n_closed;
  const float *open_ctrl;     /* [n_open][10][2] px                                  */
  const float *open_width;    /* [n_open]        px, the y-scale of its Gaussians    */
  const float *open_color;    /* [n_open][3]                                         */
  const float *open_opac;     /* [n_open][3]     one per segment                     */
  const float *closed_ctrl;   /* [n_closed][12][2] px                                */
  const float *closed_color;  /* [n_closed][3]                                       */
  const float *closed_opac;   /* [n_closed]                                          */
  const uint32_t *draw_first; /* [n_open + n_closed] index of each curve's first
                                 Gaussian in the draw-ordered table (bs_curve_order) */
  /* Linear-gradient fills of closed curves (Appendix D), each may be NULL
   * (a uniform fill): the colour / opacity at P6.  Sample k of a row of K
   * takes x = x0 + u (x1 - x0), u = k / (K - 1), from the value x0 at P0
   * (closed_color / closed_opac) to x1 at P6. */
  const float *closed_color2; /* [n_closed][3] or NULL                               */
  const float *closed_opac2;  /* [n_closed] or NULL                                  */
} bs_curves;

/* Gradients in the layout of bs_curves (device, written by the callee). */
typedef struct {
  float *open_ctrl;     /* [n_open][10][2] */
  float *open_width;    /* [n_open]        */
  float *open_color;    /* [n_open][3]     */
  float *open_opac;     /* [n_open][3]     */
  float *closed_ctrl;   /* [n_closed][12][2] */
  float *closed_color;  /* [n_closed][3]   */
  float *closed_opac;   /* [n_closed]      */
  float *closed_color2; /* [n_closed][3], written when the curves have closed_color2 and this is non-NULL */
  float *closed_opac2;  /* [n_closed], likewise                                                          */
} bs_curves_grad;

/* Sampling of Gaussians on curves (Section 3.3, Eq. 3-8). */
typedef struct {
  int32_t g_open;      /* K: samples per open curve, 2..1024                      */
  int32_t rows_closed; /* R + 2: rows of a closed curve incl. both boundaries, >= 2 */
  int32_t k_closed;    /* K: samples per row of a closed curve, >= 2;
                          rows_closed * k_closed <= 3072                           */
  float rho;           /* the density constant of Eq. 7, > 0                      */
  float cov_eps;       /* isotropic covariance floor in px^2 (Sigma += eps I), >= 0 */
  int32_t tangent_mode;/* the Gaussian's rotation (Eq. 8): 0 from the neighbour
                          difference X_{k+1} - X_{k-1} (one-sided at the ends), as
                          the paper; 1 from the derivative B'(t) of the sample's own
                          segment (a closed row's: (1 - tau) A'(t) + tau B'(t)).
                          A zero vector gives theta = 0 either way.               */
} bs_sample_cfg;

/* The canvas and its tiling (Section 3.4). */
typedef struct {
  int32_t width;   /* W px, 1..32768 */
  int32_t height;  /* H px, 1..32768 */
  int32_t tile;    /* tile side in px: 8, 16 or 32 */
  float bg[3];     /* background colour blended with the final transmittance */
} bs_canvas;

/*
 * Gaussian table record: 12 float32 per Gaussian, in draw order (front
 * first), 16-byte aligned rows.  A Gaussian is kept in the eigen-frame of
 * Eq. 11-12: Sigma = R diag(sx^2 + eps, sy^2 + eps) R^T, R = [[ux, -uy], [uy, ux]],
 * so Sigma^-1 = R diag(isx^2, isy^2) R^T.
 *   [0] mx  [1] my              mean (px)
 *   [2] ux  [3] uy              unit tangent: first column of R
 *   [4] isx [5] isy             (sx^2 + eps)^-1/2, (sy^2 + eps)^-1/2
 *   [6] o                       opacity
 *   [7] r   [8] g   [9] b       colour
 *   [10] ext_x [11] ext_y       half extents of the box holding every pixel
 *                               centre with alpha >= 1/255; < 0: never binned
 * Per-Gaussian gradient record: 12 float32,
 * d/d(mx, my, ux, uy, isx, isy, o, r, g, b) in [0..9], [10..11] = 0.
 */
#define BS_GAUSS_FLOATS 12
#define BS_DGAUSS_FLOATS 12

/* Number of Gaussians the curves produce: n_open*g_open + n_closed*rows*k.
 * Host arithmetic only.  Returns -1 on invalid arguments. */
int64_t bs_num_gaussians(int32_t n_open, int32_t n_closed, const bs_sample_cfg *cfg);

/*
 * Draw order (Section 3.3: depth from curve area, small curves in front).
 * The area key is computed in float32 with a fixed operation order: for a
 * closed curve half the absolute shoelace sum of its 12-point control
 * polygon, for an open curve the length of its 10-point control polygon
 * times its width.  Curves are ranked by ascending key, equal keys by index.
 *   rank_out  [n_open + n_closed]  0 = front-most        (device, written)
 *   first_out [n_open + n_closed]  first Gaussian index   (device, written)
 * curves->draw_first is not read.
 */
bs_status bs_curve_order(const bs_curves *curves, const bs_sample_cfg *cfg,
                         uint32_t *rank_out, uint32_t *first_out, bs_stream stream);

/*
 * Sample Gaussians on curves (Section 3.3, Eq. 3-8; covariance Eq. 11-12).
 * Open curve: K samples uniform in u = k/(K-1) over the 3-segment chain;
 * sigma_x = |X_{k+1} - X_k| / rho (last sample: previous pair),
 * sigma_y = width, theta from the central difference (ends: one-sided), or
 * with tangent_mode 1 from the derivative of the sample's segment.
 * Closed curve: rows r = 0..R+1 interpolate the control points of boundary
 * A = P0..P6 and boundary B = P0,P11,...,P7,P6 with weights
 * tau_r = (1 - cos(pi r/(R+1)))/2; K samples per row; sigma_y is the distance
 * to the next row (last row: previous).  Sigma = R S S^T R^T + eps I.
 *   gauss [n_gauss][12]  (device, written; n_gauss = bs_num_gaussians)
 */
bs_status bs_sample_curves(const bs_curves *curves, const bs_sample_cfg *cfg,
                           float *gauss, bs_stream stream);

/*
 * Backward of bs_sample_curves: given dL/d(table record) [n_gauss][12],
 * write dL/d(curve parameters).  Every array of grad is overwritten.
 */
bs_status bs_sample_curves_bwd(const bs_curves *curves, const bs_sample_cfg *cfg,
                               const float *dgauss, const bs_curves_grad *grad,
                               bs_stream stream);

/* Workspace bytes bs_bin_tiles needs for n_gauss Gaussians and up to
 * pair_capacity (tile, Gaussian) pairs.  Host arithmetic only. */
bs_status bs_bin_tiles_workspace(int64_t n_gauss, const bs_canvas *canvas,
                                 int64_t pair_capacity, size_t *bytes);

/*
 * Tile binning (Section 3.4, the tile pipeline of 3D Gaussian splatting).
 * A Gaussian is listed in every tile that holds a pixel whose centre lies in
 * its box [mx - ext_x, mx + ext_x] x [my - ext_y, my + ext_y], decided in
 * float32 as: xlo = (mx - ext_x) - 0.5, xhi = (mx + ext_x) - 0.5,
 * x0 = max(ceil(xlo), 0), x1 = min(floor(xhi), W - 1) (same for y).  Keys are
 *     key = tile_id << gbits | g,  tile_id = ty * tiles_x + tx,
 *     gbits = max(1, bit length of n_gauss - 1),
 * and are put in ascending order, so each tile's list is front to back.
 * With 32-bit keys on a grid of at most 512 x 512 tiles this is a two-level
 * stable counting sort over the Gaussians' tile rectangles (every Gaussian
 * into the list of each tile row it covers, then each row list into its
 * tiles, ranks from per-chunk bit tables); otherwise a hand-written stable
 * LSD radix sort of the tile bits (per pass: digit counts per partition,
 * their scan, a stable scatter).  Both give the same keys.
 * When tile bits + gbits exceed 32 ("wide" keys), the keys are 64-bit
 * (tile << 32 | g) inside the workspace and tile_keys receives only g for
 * each pair, in the same order; the blend calls tell the two apart from
 * n_gauss and the canvas.
 *   ws, ws_bytes    scratch of bs_bin_tiles_workspace bytes (device)
 *   pair_capacity   room in tile_keys and ws
 *   n_pairs_out     (HOST) the number of pairs P; on BS_ERR_CAPACITY the
 *                   number needed (nothing else is valid then)
 *   tile_keys       [pair_capacity] sorted keys, or their g (wide keys)
 *                   (device, written [0, P))
 *   tile_ranges     [n_tiles][2] (start, end) into tile_keys; an empty tile
 *                   has (0, 0) (device, written)
 * Synchronises the stream once to read P.
 */
bs_status bs_bin_tiles(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                       void *ws, size_t ws_bytes, int64_t pair_capacity,
                       int64_t *n_pairs_out, uint32_t *tile_keys, uint32_t *tile_ranges,
                       bs_stream stream);

/*
 * bs_bin_tiles without the read-back (the tile pipeline of Section 3.4, the
 * rules of bs_bin_tiles): every grid of the sort is sized by pair_capacity
 * (>= 1) and the kernels read the pair count P from the workspace, so the
 * call never waits on the host and can be captured in a CUDA graph.
 *   n_pairs_dev  (device int64, may be NULL) receives P, stream-ordered
 *   tile_keys, tile_ranges  as bs_bin_tiles
 * When P > pair_capacity nothing is emitted or sorted, every range is (0, 0)
 * (a blend then draws only the background), and the workspace's status word
 * records BS_ERR_CAPACITY: bs_bin_tiles_result (or bs_device_status) reports
 * it together with P, for a retry with a larger capacity.
 */
bs_status bs_bin_tiles_async(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                             void *ws, size_t ws_bytes, int64_t pair_capacity, int64_t *n_pairs_dev,
                             uint32_t *tile_keys, uint32_t *tile_ranges, bs_stream stream);

/* Synchronise the stream and read the outcome of the last binning in `ws`:
 * *status_out = BS_OK or BS_ERR_CAPACITY (BS_ERR_TIMEOUT is reserved), and
 * *n_pairs_out (HOST, may be NULL) = the pairs that binning found. */
bs_status bs_bin_tiles_result(const void *ws, size_t ws_bytes, int32_t *status_out, int64_t *n_pairs_out,
                              bs_stream stream);

/*
 * bs_bin_tiles for callers that cannot allocate device memory: the same
 * binning, with its scratch in one fixed array of 32 MiB that the library
 * keeps in device memory (every GPU that loads the library holds it until the
 * process exits).  Meant for code that may not call cudaMalloc or a caching
 * allocator, for instance a host that hands this library a fixed memory
 * budget, or a callback that must not allocate.  The caller still provides
 * gauss, tile_keys and tile_ranges.  The paper has no counterpart of this call.
 *   - It always sorts with the radix passes, whose scratch is smaller than
 *     the two-level sort's tables (bs_bin_tiles_workspace reports the
 *     larger of the two where bs_bin_tiles would use the two-level sort).
 *     A request whose scratch would exceed 32 MiB (a pair_capacity above
 *     about 7.1 M for 262,144 Gaussians on a 2048 x 2048 canvas) returns
 *     BS_ERR_INVALID_ARG with the size it needs; nothing is launched.
 *   - No allocation is made: no cudaMalloc, cudaFree or allocating library
 *     routine.  The first call on a device looks up the array's device
 *     address (once per device, safe from several host threads), so make
 *     that first call before any stream capture.  A device reset
 *     (cudaDeviceReset) unloads the array and leaves that address stale: do
 *     not call this entry point on a device after resetting it in the same
 *     process.
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call clears what it needs cleared): calls that overlap on the GPU,
 *     on any streams, race with each other.  bs_device_status does not read it.
 * Arguments, results and the one synchronisation are those of bs_bin_tiles.
 */
bs_status bs_bin_tiles_static(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                              int64_t pair_capacity, int64_t *n_pairs_out,
                              uint32_t *tile_keys, uint32_t *tile_ranges, bs_stream stream);

/*
 * Forward blend (Eq. 9-10).  Per pixel, over its tile's list in order:
 * alpha = min(0.99, o exp(-0.5 d^T Sigma^-1 d)); skipped if alpha < 1/255;
 * the pixel stops at the first Gaussian that would bring its transmittance
 * T below 1e-4 (not blended); C += c alpha T, T *= 1 - alpha; finally
 * C += T bg.
 *   img       [3][H][W]  (device, written)
 *   T_final   [H][W]     final transmittance (device, written)
 *   n_contrib [H][W]     entries of the tile list up to and including the
 *                        last blended Gaussian, 0 if none (device, written)
 */
bs_status bs_render_fwd(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                        const uint32_t *tile_keys, const uint32_t *tile_ranges,
                        float *img, float *T_final, uint32_t *n_contrib, bs_stream stream);

/*
 * bs_render_fwd followed by bs_l2_loss_grad on its image (Eq. 9-10, then the
 * L2 term of Eq. 13 with lambda_1 = 1 over the 3 H W entries), in one pass
 * over the pixels: img, T_final and n_contrib as bs_render_fwd writes them,
 * dL_dimg = 2 (img - target) / (3 H W) bit-identical to bs_l2_loss_grad's,
 * and loss_out = mean((img - target)^2) equal to it up to the order of the
 * summation.
 *   target   [3][H][W]  (device, read)
 *   dL_dimg  [3][H][W]  (device, written)
 *   loss_out            (device double, written)
 */
bs_status bs_render_fwd_l2(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                           const uint32_t *tile_keys, const uint32_t *tile_ranges,
                           const float *target, float *img, float *T_final, uint32_t *n_contrib,
                           float *dL_dimg, double *loss_out, bs_stream stream);

/*
 * bs_render_fwd plus work counters, for measurement: stats_out (device,
 * 4 x uint64, zeroed and written) receives [0] the (pixel, list entry)
 * evaluations performed (after the block culling), [1] the entries blended,
 * [2] the sum over tiles of list length x tile pixels, [3] the sum over
 * pixels of the list entries up to the pixel's stop point (the entry whose
 * blend would bring its transmittance below 1e-4, or the list's end).
 */
bs_status bs_render_stats(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                          const uint32_t *tile_keys, const uint32_t *tile_ranges,
                          float *img, float *T_final, uint32_t *n_contrib,
                          unsigned long long *stats_out, bs_stream stream);

/*
 * L2 term of Eq. 13 with lambda_1 = 1 averaged over the n entries:
 * loss = mean((img - target)^2) (device double, written), and
 * dL_dimg = 2 (img - target) / n (device, written).
 */
bs_status bs_l2_loss_grad(const float *img, const float *target, int64_t n,
                          float *dL_dimg, double *loss_out, bs_stream stream);

/*
 * Backward of bs_render_fwd, then of bs_sample_curves.  Per pixel, walks its
 * tile list from its last blended Gaussian to the front, recovering
 * T_i = T_{i+1} / (1 - alpha_i) from T_final (no per-Gaussian state is
 * stored), and accumulates dL/d(mean, conic, opacity, colour) per Gaussian.
 *   dgauss [n_gauss][12]  per-Gaussian gradients (device, zeroed and written)
 *   curves, cfg, grad     if grad is non-NULL, the curve gradients are
 *                         written as by bs_sample_curves_bwd; if NULL only
 *                         dgauss is produced and curves/cfg may be NULL.
 */
bs_status bs_render_bwd(const float *gauss, int64_t n_gauss, const bs_canvas *canvas,
                        const uint32_t *tile_keys, const uint32_t *tile_ranges,
                        const float *T_final, const uint32_t *n_contrib,
                        const float *dL_dimg, float *dgauss,
                        const bs_curves *curves, const bs_sample_cfg *cfg,
                        const bs_curves_grad *grad, bs_stream stream);

/* Curves that bs_prune_densify edits in place: the arrays of bs_curves,
 * writable (device, same layouts). */
typedef struct {
  int32_t n_open;
  int32_t n_closed;
  float *open_ctrl;     /* [n_open][10][2] px  */
  float *open_width;    /* [n_open]            */
  float *open_color;    /* [n_open][3]         */
  float *open_opac;     /* [n_open][3]         */
  float *closed_ctrl;   /* [n_closed][12][2] px */
  float *closed_color;  /* [n_closed][3]       */
  float *closed_opac;   /* [n_closed]          */
} bs_curves_mut;

/* Parameters of one pruning and densification pass (Section 3.5,
 * Algorithm 1, Appendix B).  Thresholds compare float32 values. */
typedef struct {
  float op_start;     /* opacity threshold at step 0, e.g. 0.2                */
  float op_end;       /* opacity threshold from step t_end on, e.g. 0.02      */
  int32_t step;       /* optimisation step of this pass, >= 0                 */
  int32_t t_end;      /* step where the threshold reaches op_end, >= 1        */
  float area_min;     /* px^2: a curve whose area key is below is pruned      */
  float color_eps;    /* RGB distance below which two curves are similar      */
  float iou_min;      /* box IoU above which a similar curve is redundant     */
  float err_thresh;   /* a pixel is in error when its channel-mean |img - target| exceeds it */
  float split_drop;   /* an open curve whose middle opacity is this far below
                         both end opacities is split                          */
  float new_opacity;  /* opacity of a new curve (every segment), in [0, 1]    */
  float new_width;    /* width of a new open curve, px, > 0                   */
} bs_pd_cfg;

/* What one pass did (host struct, written). */
typedef struct {
  int32_t pruned;        /* curves removed (any criterion)                      */
  int32_t low_opacity;   /* curves below the opacity threshold                  */
  int32_t small_area;    /* curves below the area threshold                     */
  int32_t overlap;       /* curves redundant with a similar curve in front      */
  int32_t split;         /* open curves split                                   */
  int32_t split_placed;  /* second halves written into a freed open slot        */
  int32_t regions;       /* connected error regions found                       */
  int32_t inserted;      /* new curves placed on error regions                  */
  int32_t transparent;   /* freed slots left with opacity 0 (no region left)    */
} bs_pd_stats;

/* Workspace bytes bs_prune_densify needs.  Host arithmetic only. */
bs_status bs_prune_densify_workspace(int32_t n_open, int32_t n_closed, const bs_canvas *canvas,
                                     size_t *bytes);

/*
 * One pass of adaptive pruning and densification (Section 3.5, Algorithm 1;
 * the split rule of Appendix B), in place on `curves`; the number of curves
 * stays the same (the budget is constant).
 * Pruning.  Curve i is removed when
 *   - its opacity (closed: its opacity; open: ((o0 + o1) + o2) / 3) is below
 *     tau = op_start (1 - f) + op_end f, f = min(1, step / t_end);
 *   - its area key (the draw-order key of bs_curve_order) is below area_min;
 *   - a curve j drawn in front of it (lower draw rank) has RGB distance
 *     < color_eps and bounding-box IoU > iou_min.  Boxes are the control
 *     points' box, widened by width / 2 on every side for an open curve.
 * Splitting.  A kept open curve whose middle opacity is more than
 * split_drop below both end opacities keeps its first segment, re-cut into
 * three segments (de Casteljau at 1/3 and 2/3) with opacity o0; its last
 * segment, cut the same way with opacity o2 and the curve's colour and
 * width, goes into the lowest-index freed open slot not yet taken (split
 * curves in index order); without a free open slot it is dropped.
 * Densification.  Error map e = ((|d_r| + |d_g|) + |d_b|) / 3, d = img -
 * target; regions are the 4-connected components of e > err_thresh, ranked
 * by pixel count (descending), equal counts by their first pixel in
 * row-major order.  The freed slots still empty, open ones first then closed
 * ones, each in index order, receive the regions in rank order: control
 * points on the circle around the region's centroid (pixel centres) of
 * radius sqrt(count / pi) at angles 2 pi j / 12 (closed, j = 0..11) or
 * 2 pi j / 11 (open, j = 0..9), colour = the region's mean target colour,
 * opacity new_opacity, width new_width.  Freed slots left over keep their
 * geometry with opacity 0.
 *   img, target  [3][H][W] (device, read); canvas: width and height are used
 *   ws, ws_bytes scratch of bs_prune_densify_workspace bytes (device)
 *   changed_out  [n_open + n_closed] 1 where a curve was pruned, split,
 *                replaced or made transparent, else 0 (device, written;
 *                may be NULL)
 *   stats_out    (HOST, may be NULL) counts of the pass
 * n_open + n_closed <= 65536 (the pair test is quadratic).  The draw order
 * (bs_curve_order) must be recomputed afterwards.  Synchronises the stream
 * once, at the end.  BS_ERR_TIMEOUT if a bounded retry loop of the region
 * labelling ran out (the curves are then unchanged only up to that point).
 */
bs_status bs_prune_densify(const bs_curves_mut *curves, const bs_pd_cfg *cfg,
                           const bs_canvas *canvas, const float *img, const float *target,
                           void *ws, size_t ws_bytes, uint8_t *changed_out,
                           bs_pd_stats *stats_out, bs_stream stream);

/* ------------------------------------------------------------------------
 * Batches: many images of different sizes and curve counts optimised
 * together (the method of Section 3 applied to each image independently).
 * Each image b has its own canvas, curves and sampling; its arrays are
 * concatenated image after image:
 *   curves      bs_curves whose n_open / n_closed are the batch totals; image
 *               b's open curves are rows [open0_b, open0_b + n_open_b) of the
 *               open arrays (open0_b = sum of the earlier images' n_open), its
 *               closed curves likewise in the closed arrays.  Control points
 *               are in the image's own pixel coordinates.
 *   Gaussians   image b's records are rows [gauss0_b, gauss0_b + n_gauss_b)
 *               of the table, in the image's draw order (gauss0_b = sum of
 *               the earlier images' bs_num_gaussians).
 *   pixels      image b's planar image [3][H_b][W_b] starts at float 3 pix0_b
 *               of an image buffer, its per-pixel maps [H_b][W_b] at pix0_b
 *               (pix0_b = sum of the earlier images' W H).
 *   tiles       image b's tiles are numbered tile0_b + ty tiles_x_b + tx
 *               (tile0_b = sum of the earlier images' tile counts).
 * Every batched call takes the same bs_batch descriptor.  Its workspace
 * holds the device table of the layout (written by bs_batch_setup) and the
 * binning scratch.  No batched call synchronises the stream, allocates, or
 * depends on a value read back to the host, so a whole optimisation step
 * (draw order, sampling, binning, blend with loss, backward, bs_adam_step)
 * can be captured in a CUDA graph; bs_batch_status reports a capacity
 * overflow afterwards.
 * ---------------------------------------------------------------------- */

/* One image of a batch (host struct). */
typedef struct {
  int32_t width, height;   /* canvas px, 1..32768                        */
  int32_t n_open, n_closed;/* its curves                                 */
  bs_sample_cfg sample;    /* its sampling (Section 3.3)                 */
  float bg[3];             /* its background colour                      */
} bs_batch_image;

/* A batch: the layout, the tiling, and the workspace. */
typedef struct {
  const bs_batch_image *images;  /* HOST [n_images]                                  */
  int32_t n_images;              /* >= 1                                             */
  int32_t tile;                  /* tile side in px: 8, 16 or 32                     */
  int64_t pair_capacity;         /* room for (tile, Gaussian) pairs, >= 1            */
  void *ws;                      /* device workspace of bs_batch_plan's ws_bytes     */
  size_t ws_bytes;
} bs_batch;

/* Totals of a batch (host struct, written by bs_batch_plan). */
typedef struct {
  int64_t n_open, n_closed;  /* curves of all images                          */
  int64_t n_gauss;           /* rows of the Gaussian table                    */
  int64_t n_pixels;          /* sum of W H; image buffers hold 3 n_pixels floats */
  int64_t n_tiles;           /* rows of tile_ranges                           */
  size_t ws_bytes;           /* workspace bytes                               */
} bs_batch_sizes;

/* Host arithmetic only: the totals of a batch and its workspace size
 * (batch->ws is not read).  Batch keys are 64-bit (tile << 32 | Gaussian),
 * so any batch whose tiles and Gaussians each fit in 32 bits is accepted. */
bs_status bs_batch_plan(const bs_batch *batch, bs_batch_sizes *out);

/* Write the layout's device table into the workspace, and the curve
 * indices grouped by sample count (curves of fewer than 512 samples, then
 * the rest; the batched sampling runs each group in its own launch) (two
 * host-to-device copies, synchronous).  Call once before the other batched calls, and again
 * whenever images, tile or pair_capacity change; every later call must pass
 * the same images, tile and pair_capacity. */
bs_status bs_batch_setup(const bs_batch *batch, bs_stream stream);

/* Draw order of every image (bs_curve_order per image): ranks are within an
 * image, first_out indexes the batch's Gaussian table (gauss0_b + the
 * image's own first index).  rank_out, first_out [n_open + n_closed]
 * (device, written), in the batch's curve numbering (open curves, then
 * closed).  curves->draw_first is not read. */
bs_status bs_batch_curve_order(const bs_batch *batch, const bs_curves *curves, uint32_t *rank_out,
                               uint32_t *first_out, bs_stream stream);

/* bs_sample_curves for every image with its own bs_sample_cfg (Section 3.3,
 * Eq. 3-8, 11-12).  gauss [n_gauss][12] (device, written). */
bs_status bs_batch_sample_curves(const bs_batch *batch, const bs_curves *curves, float *gauss,
                                 bs_stream stream);

/*
 * Tile binning of every image (Section 3.4; the same tile rule as
 * bs_bin_tiles, with each image's own canvas).  Keys (global tile << 32 | g)
 * are emitted in Gaussian order and sorted stably by the tile bits with the
 * library's LSD radix sort; the last pass writes only the Gaussian indices.
 *   tile_vals    [pair_capacity] Gaussian indices, each tile's list front to
 *                back (device, written [0, P))
 *   tile_ranges  [n_tiles][2] (start, end) into tile_vals, (0, 0) when empty
 *                (device, written)
 * Grids are sized by pair_capacity and nothing is read back.  When P exceeds
 * pair_capacity the status word records BS_ERR_CAPACITY, every range is
 * (0, 0) (nothing is blended), and bs_batch_status reports P.
 */
bs_status bs_batch_bin_tiles(const bs_batch *batch, const float *gauss, uint32_t *tile_vals,
                             uint32_t *tile_ranges, bs_stream stream);

/*
 * Forward blend of every image (Eq. 9-10, the rules of bs_render_fwd), by a
 * persistent kernel whose CTAs take (image, tile) work items from an atomic
 * queue.  If target is non-NULL, also the L2 term of Eq. 13 per image:
 * dL_dimg = 2 (img - target) / (3 W_b H_b) and loss_out[b] =
 * mean((img_b - target_b)^2) (otherwise dL_dimg and loss_out are not
 * touched and may be NULL).
 *   target, img, dL_dimg  [3 n_pixels] in the batch's image layout (device)
 *   T_final, n_contrib    [n_pixels]  (device, written)
 *   loss_out              [n_images] double (device, written)
 */
bs_status bs_batch_render_fwd(const bs_batch *batch, const float *gauss, const uint32_t *tile_vals,
                              const uint32_t *tile_ranges, const float *target, float *img, float *T_final,
                              uint32_t *n_contrib, float *dL_dimg, double *loss_out, bs_stream stream);

/*
 * Backward of bs_batch_render_fwd (the reverse walk of bs_render_bwd on
 * every image, persistent, atomic work queue), then of the sampling of every
 * image: dgauss [n_gauss][12] (device, zeroed and written); if grad is
 * non-NULL, the curve gradients in the batch's curve layout.
 */
bs_status bs_batch_render_bwd(const bs_batch *batch, const float *gauss, const uint32_t *tile_vals,
                              const uint32_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                              const float *dL_dimg, float *dgauss, const bs_curves *curves,
                              const bs_curves_grad *grad, bs_stream stream);

/* Synchronise the stream and read the batch workspace's status word:
 * *status_out = BS_OK, BS_ERR_CAPACITY (the last bs_batch_bin_tiles found
 * more pairs than pair_capacity) or BS_ERR_UNSUPPORTED (its pair totals over
 * Gaussians and over tiles disagreed, so nothing was sorted; not expected,
 * bs_last_error has both totals); *n_pairs_out (HOST, may be NULL) = the
 * pairs that call found. */
bs_status bs_batch_status(const bs_batch *batch, int32_t *status_out, int64_t *n_pairs_out, bs_stream stream);

/* ------------------------------------------------------------------------
 * Adam (Kingma and Ba; the optimiser of Section 4.1) over parameter groups,
 * in one launch:  t = *step + 1,
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p = clamp(p - lr_i (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), lo, hi),
 * lr_i = lr * row_scale[i / row_len] (row_scale NULL: lr); then *step = t.
 * The step counter lives in device memory, so a replayed CUDA graph
 * advances it.
 * ---------------------------------------------------------------------- */
typedef struct {
  float *param;            /* [n] device, updated in place                     */
  const float *grad;       /* [n] device                                        */
  float *m, *v;            /* [n] device moments (zero before the first step)   */
  int64_t n;
  float lr;                /* >= 0                                              */
  float lo, hi;            /* the updated value is clamped to [lo, hi]          */
  const float *row_scale;  /* [n / row_len] device lr multipliers, or NULL      */
  int32_t row_len;         /* >= 1                                              */
} bs_adam_group;

typedef struct {
  float beta1, beta2, eps;
} bs_adam_cfg;

#define BS_ADAM_MAX_GROUPS 16

/* groups: HOST [n_groups], 1 <= n_groups <= BS_ADAM_MAX_GROUPS;
 * step: device int32, t before this step (0 before the first). */
bs_status bs_adam_step(const bs_adam_group *groups, int32_t n_groups, const bs_adam_cfg *cfg, int32_t *step,
                       bs_stream stream);

/*
 * The Xing loss of Eq. 13 (the convexity term, as defined by LIVE, which the
 * paper adopts): per cubic segment (A, B, C, D) of every closed curve, with
 * u = B - A, v = C - B, w = D - C, D1 = [u x v >= 0], D2 = (u x w) / (|u| |w|),
 * L_seg = D1 relu(-D2) + (1 - D1) relu(D2) (0 when |u| or |w| is 0).
 *   loss_out          lambda * mean of L_seg over the 4 n_closed segments
 *                     (device double, written)
 *   grad_closed_ctrl  [n_closed][12][2] (device): d(loss_out)/d(control
 *                     points) is ADDED to it; may be NULL
 * Only curves->n_closed and closed_ctrl are read.
 */
bs_status bs_xing_loss(const bs_curves *curves, float lambda, double *loss_out, float *grad_closed_ctrl,
                       bs_stream stream);

/*
 * SVG export (Appendix C, Algorithm 2).  All arrays of `curves` and `rank`
 * are HOST pointers here (pixel coordinates, activated colours).  Curves are
 * written back to front: by descending draw rank when rank is non-NULL
 * (rank 0 is front-most, so it comes last), else in index order.  A closed
 * curve is the path M P0, C P1 P2 P3, C P4 P5 P6, C P7 P8 P9, C P10 P11 P0, Z,
 * filled with rgb(round(255 colour)) at fill-opacity 1 (Algorithm 2), or at
 * its own opacity with flags bit 0; a closed curve with a gradient fill is
 * filled by a linearGradient from P0 to P6 whose stops are its two colours
 * (and, with bit 0, opacities).  An open curve is the unfilled path M P0,
 * C P1 P2 P3, C P4 P5 P6, C P7 P8 P9 stroked with its colour at width
 * 2 width and the mean of its segment opacities.  Numbers carry 9
 * significant digits, so float32 values read back exactly.
 *   buf, buf_bytes  (HOST) receives the NUL-terminated document; may be NULL
 *                   to ask for the size
 *   needed_out      (HOST) bytes the document needs, NUL included
 * Host-only: needs no GPU.
 */
bs_status bs_svg_export(const bs_curves *curves, const uint32_t *rank, int32_t width, int32_t height,
                        int32_t flags, char *buf, size_t buf_bytes, size_t *needed_out);

/* ------------------------------------------------------------------------
 * Learned initialisation (not in the paper: a proposal network for initial
 * curves).  A 5-layer convolutional encoder maps a side x side RGB patch
 * (side a multiple of 32) to one closed curve and one open stroke (the two
 * kinds of Section 3.2) per 32 x 32 cell: five 4 x 4 convolutions of stride
 * 2 and padding 1 with ReLU (channels 8 -> 32 -> 64 -> 128 -> 256 -> 256,
 * the RGB input padded to 8), then a 1 x 1 head (256 -> 64).  The head's
 * outputs o of a cell with centre c give (patch pixels):
 *   closed curve  P_j = c + BS_NET_REACH tanh(o_{2j}, o_{2j+1}) (j = 0..11),
 *                 colour sigmoid(o_24..26), opacity sigmoid(o_27);
 *   open stroke   Q_j = c + BS_NET_REACH tanh(o_{28+2j}, o_{29+2j})
 *                 (j = 0..9), width BS_NET_WIDTH_MAX sigmoid(o_48), colour
 *                 sigmoid(o_49..51), segment opacities sigmoid(o_52..54);
 * outputs 55..63 are unused.  Convolutions run as implicit GEMMs on the
 * bf16 tensor cores with float32 accumulation; activations are bf16.
 * ---------------------------------------------------------------------- */
#define BS_NET_LAYERS 6
#define BS_NET_REACH 24.0f
#define BS_NET_WIDTH_MAX 8.0f

/* Weights of the network (device, caller-owned).  w[l]: float32 master
 * weights of layer l, [Cout][ky][kx][Cin] then the bias [Cout]
 * (bs_net_param_count(l) floats; layer 5 is the head, [64][256] + [64]).
 * w_bf16[l]: bfloat16 copy of the weights (without the bias), written by
 * bs_net_sync_weights. */
typedef struct {
  const float *w[BS_NET_LAYERS];
  uint16_t *w_bf16[BS_NET_LAYERS];
} bs_net;

/* Gradients of the master weights (device, float32, same layouts). */
typedef struct {
  float *g[BS_NET_LAYERS];
} bs_net_grad;

/* Per-cell curves of n patches (device, cells = (side / 32)^2, row-major,
 * patch after patch): the network's proposals, or the targets of a training
 * step (then read only). */
typedef struct {
  float *ctrl;        /* [n][cells][12][2] closed-curve control points, patch px */
  float *color;       /* [n][cells][3]                                            */
  float *opac;        /* [n][cells]                                               */
  float *open_ctrl;   /* [n][cells][10][2] open-stroke control points, patch px   */
  float *open_width;  /* [n][cells]        px, in (0, BS_NET_WIDTH_MAX)           */
  float *open_color;  /* [n][cells][3]                                            */
  float *open_opac;   /* [n][cells][3]     one per segment                        */
} bs_net_curves;

/* Floats of layer `layer`'s master array (weights + bias); -1 if out of range. */
int64_t bs_net_param_count(int32_t layer);

/* Workspace bytes for n patches of side `side` (activations and their
 * gradients, bf16).  Host arithmetic only. */
bs_status bs_net_workspace(int32_t n, int32_t side, size_t *bytes);

/* w_bf16[l] = bf16(w[l]) for every layer (after an update of the master
 * weights). */
bs_status bs_net_sync_weights(const bs_net *net, bs_stream stream);

/*
 * Forward of n patches (planar float32 [n][3][side][side], values in [0,1]).
 * Writes (device, each may be NULL) the head outputs head_out [n][cells][64]
 * and, when curves is non-NULL, the proposals into those of its arrays that
 * are non-NULL.  Synchronises the stream once, at the end, to read how many
 * tensor-core tiles gave up their bounded wait for their MMAs: any such tile
 * left its outputs unwritten, and the call returns BS_ERR_TIMEOUT (never
 * expected; the test hook bs_debug_umma_wait makes it happen).
 */
bs_status bs_net_forward(const bs_net *net, const float *patches, int32_t n, int32_t side, void *ws,
                         size_t ws_bytes, float *head_out, const bs_net_curves *curves, bs_stream stream);

/*
 * One training step's forward and backward against the target curves
 * `target` (device, every array non-NULL): the loss, the mean over cells of
 *   sum_j |P_j - P*_j|^2 / BS_NET_REACH^2 + |colour - colour*|^2
 *   + (opacity - opacity*)^2 + sum_j |Q_j - Q*_j|^2 / BS_NET_REACH^2
 *   + (width - width*)^2 / BS_NET_WIDTH_MAX^2 + |colour' - colour'*|^2
 *   + sum_s (opacity'_s - opacity'*_s)^2
 * (primes: the open stroke), to loss_out (device double), and dL/d(master
 * weights) to grad (zeroed and written).  Synchronises and reports
 * BS_ERR_TIMEOUT as bs_net_forward does.
 */
bs_status bs_net_train_step(const bs_net *net, const float *patches, int32_t n, int32_t side,
                            const bs_net_curves *target, void *ws, size_t ws_bytes, const bs_net_grad *grad,
                            double *loss_out, bs_stream stream);

/* Test hook: the engine of the network's GEMMs for later calls in this
 * process.  1 (the default): the forward convolutions with 64 or more input
 * channels on the TMA-fed tcgen05 kernel (im2col and tiled TMA loads into
 * 128-byte-swizzled stages of an mbarrier ring, 128 x 128 tiles accumulated
 * in tensor memory), the other GEMMs on tcgen05 with thread-gathered
 * operands (128 x 64 tiles) when their reduction per CTA is at least 1024
 * long and on mma.sync (64 x 64 tiles, accumulators in registers) below;
 * 2: as 1, with every other GEMM on the gathered tcgen05 kernel; 3: every
 * GEMM on the gathered tcgen05 kernel; 0: every GEMM on mma.sync.
 * timeouts_out (HOST, may be NULL): how many tcgen05 tiles so far gave up a
 * bounded wait on their MMAs (their results were not stored; 0 expected). */
bs_status bs_debug_gemm_engine(int32_t engine, int64_t *timeouts_out);

/* Test hook: the tries of the tcgen05 GEMM's wait for its last MMA commit
 * before the read-back, for later calls in this process (< 0: the default,
 * 2^24; 0: the wait gives up at once).  A tile whose wait gave up waits
 * again with the full bound before it releases its tensor memory, stores
 * nothing, and makes bs_net_forward / bs_net_train_step return
 * BS_ERR_TIMEOUT.  No wait of the library is unbounded either way. */
bs_status bs_debug_umma_wait(int64_t first_wait);

/* Synchronise the stream and read the device status word of a binning
 * workspace: BS_OK or the first kernel-side error recorded since the
 * workspace's last bs_bin_tiles call. */
bs_status bs_device_status(const void *ws, size_t ws_bytes, int32_t *status_out,
                           bs_stream stream);

/* Test hook for the bounded device-side retry loops.  The only one is the
 * union step of bs_prune_densify's region labelling, which tries again when
 * another thread moved a root under it.  Each union makes at most
 * max_attempts linking attempts (< 0: the default bound, 2^20; 0: a union
 * with anything to link gives up at once); a union that gives up makes that
 * bs_prune_densify call return BS_ERR_TIMEOUT.  Applies to later calls in
 * this process.  No device loop is unbounded either way, and no kernel of
 * the library waits on another thread. */
bs_status bs_debug_retry_limit(int64_t max_attempts);

/* Synchronise the stream and read the library's status word of the current
 * device: *status_out = BS_ERR_NOT_FINITE when, since the word was last
 * cleared, the sampling (bs_sample_curves, bs_batch_sample_curves) wrote a
 * non-finite Gaussian record (mean, direction, inverse scales, opacity or
 * colour; e.g. from NaN control points, or eps = 0 with coincident samples),
 * or a backward (bs_render_bwd, bs_batch_render_bwd, bs_sample_curves_bwd)
 * wrote a non-finite per-Gaussian or curve gradient; else BS_OK.  With
 * clear != 0 the word is reset after the read (stream-ordered).  The word
 * is shared by every stream and caller on the device. */
bs_status bs_sync_status(int32_t clear, int32_t *status_out, bs_stream stream);

/* Message of the last non-OK status on this thread ("" if none). */
const char *bs_last_error(void);

/* Name of a status code. */
const char *bs_status_string(bs_status status);

#ifdef __cplusplus
}
#endif

#endif /* BEZIER_SPLATTING_BS_H */
