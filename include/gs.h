/*
 * gs.h -- C ABI of the GB300 tile-based Gaussian-splatting library (libgs103.so).
 *
 * The operations follow RT-GuIDE (arXiv 2409.18122):
 *   Sec. III "Gaussian Splatting": Gaussians are sorted by increasing depth
 *     relative to the camera pose and splatted onto the image plane with
 *     mu_2D = K R^T (mu - T) / d, d = e3^T R^T (mu - T); pixel colour
 *     C(p) = sum_i c_i f_i(p) prod_{j<i} (1 - f_j(p)); depth by replacing c_i with d_i.
 *   Eq. (2): the map is the minimiser of the rendering loss over the keyframes,
 *     refined by back-propagation (Sec. IV-A).
 *   Eq. (nbv) and Sec. IV-A: information gain of a candidate view scored from the
 *     per-Gaussian uncertainty u_i = |mu_k - mu_{k-1}| of the Gaussians it sees.
 *
 * Conventions shared by every entry point
 *   - All array pointers are DEVICE pointers owned by the caller (e.g. PyTorch
 *     tensors), except where a comment says HOST.  The library never allocates
 *     device memory, never synchronises the stream and never prints; every
 *     entry point only enqueues kernels on `stream` (a cudaStream_t passed as
 *     void*, NULL = legacy default stream), so a sequence of calls can be
 *     captured into a CUDA graph.
 *   - Host-detectable argument errors return immediately with a gs_status code
 *     and enqueue nothing.  Conditions only the device can see (pair or range
 *     capacity exceeded, a camera with no pixels, non-finite Gaussian
 *     parameters) are OR-ed as GS_FLAG_* bits into the caller's device status
 *     word, which gs_read_status reads after the stream has been synchronised.
 *     Outputs of a call whose status carries GS_FLAG_PAIR_OVERFLOW or
 *     GS_FLAG_RANGE_OVERFLOW are incomplete and must be discarded.
 *   - gs_proj.splat ([n][8] floats) must be 32-byte aligned, other float4-typed
 *     arrays ([n][4] floats) 16-byte aligned, [n][2] float and uint16 [n][4]
 *     arrays 8-byte aligned; all other arrays 4-byte aligned; workspaces
 *     256-byte aligned.
 *   - Rendering constants the paper leaves unstated are fields of gs_params.
 */
#ifndef GS103_GS_H
#define GS103_GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef int32_t gs_status;
enum {
  GS_OK = 0,
  GS_ERR_NULL = 1,          /* a required pointer is NULL                          */
  GS_ERR_ALIGN = 2,         /* a pointer violates the alignment stated above        */
  GS_ERR_ARG = 3,           /* a count, size or parameter is out of range           */
  GS_ERR_WORKSPACE = 4,     /* workspace smaller than gs_workspace_size reports     */
  GS_ERR_CUDA = 5,          /* a CUDA runtime call or kernel launch failed          */
  GS_ERR_DEVICE = 6         /* the device status word carries an error flag          */
};

/* device status word bits */
enum {
  GS_FLAG_PAIR_OVERFLOW = 1u << 0,   /* more (tile, Gaussian) pairs than gs_bins.pair_capacity */
  GS_FLAG_RANGE_OVERFLOW = 1u << 1,  /* more tiles over all views than gs_bins.tile_capacity   */
  GS_FLAG_BAD_CAMERA = 1u << 2,      /* a camera has width*height <= 0, a non-positive focal length or an invalid tile size */
  GS_FLAG_NONFINITE = 1u << 3,       /* informational: Gaussians with a non-finite mean, opacity logit,
                                        log-scale or quaternion entry were culled (colours and u are
                                        not checked: they only scale a channel) */
  GS_FLAG_RECORD_OVERFLOW = 1u << 4, /* more visible (Gaussian, view) records than capacity    */
  GS_FLAG_BAD_RECORDS = 1u << 5      /* gs_bin_sort input: records not grouped by increasing view,
                                        a view id >= n_views, or a rectangle outside its view's tiles */
};
#define GS_FLAG_ERROR_MASK \
  (GS_FLAG_PAIR_OVERFLOW | GS_FLAG_RANGE_OVERFLOW | GS_FLAG_BAD_CAMERA | GS_FLAG_RECORD_OVERFLOW | GS_FLAG_BAD_RECORDS)

/* ------------------------------------------------------------------ inputs */

/* Pinhole camera (Sec. III: intrinsics K, pose R_k, T_k in the world frame).
 * R is camera-to-world, row-major; world-to-camera is t = R^T (mu - T).
 * Axes: x right, y down, z forward.  Pixel (u, v) samples (u + 0.5, v + 0.5).
 * tile_w, tile_h: this view's screen tile (same rules as gs_params.tile_w/h);
 * 0, 0 selects gs_params.tile_w, tile_h.  Low-resolution views render faster
 * with smaller tiles (shorter per-tile lists).
 * 80 bytes; arrays of cameras are DEVICE arrays. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
  float R[9];
  float T[3];
  int32_t tile_w, tile_h;
} gs_camera;

/* Gaussian map (Sec. III: colour c, position mu, size, opacity; anisotropic
 * generalisation with three log-scales and a rotation quaternion; Sec. IV-A:
 * uncertainty u).  Four DEVICE float arrays of shape [n][4], 16-byte aligned:
 *   mo  = (mu_x, mu_y, mu_z, opacity logit)   opacity o = 1 / (1 + exp(-logit))
 *   su  = (log s_0, log s_1, log s_2, u)
 *   q   = (w, x, y, z)  rotation quaternion, need not be normalised
 *   rgb = (r, g, b, unused)                                                  */
typedef struct {
  const float* mo;
  const float* su;
  const float* q;
  const float* rgb;
  int64_t n;
} gs_map;

/* Rendering constants (readings where the paper is silent) and two choices of the
 * compositing loops that change speed, never results.
 *   tile_w, tile_h  screen tile in pixels: tile_w in {8, 16, 32, 64}, tile_h a multiple of 8,
 *                   tile_w * tile_h in {64, 128, 256, 512, 1024} (one warp per 8x4 pixel block)
 *   eps2d           added to the diagonal of every 2D covariance (low-pass), px^2, >= 0
 *   near_plane      Gaussians with view depth <= near_plane are culled, > 0
 *   guard           centres with |t_x / t_z| > guard * (W/2) / f_x (same for y) are culled, > 0
 *   alpha_min       a Gaussian whose alpha at a pixel is below this is skipped, in [0, 1)
 *   alpha_max       alpha = min(alpha_max, o * exp(-q/2)), in (0, 1]
 *   T_min           compositing stops before adding a Gaussian that would take T below this, >= 0
 *   ig_batch        chunk depth of the information-gain compositing: how many of a warp's
 *                   staged list entries have their alphas evaluated together before the
 *                   transmittance updates run through them in list order; 4, 8 or 16 (0: 8)
 *   fwd_batch       the same for gs_render_fwd: 1, 2 or 4 (0: 2)
 * The outputs are bit for bit the same for every ig_batch and fwd_batch.
 * Defaults: 16, 16, 0.3, 0.2, 1.3, 1/255, 0.99, 1e-4, 0, 0. */
typedef struct {
  int32_t tile_w, tile_h;
  float eps2d, near_plane, guard, alpha_min, alpha_max, T_min;
  int32_t ig_batch, fwd_batch;
} gs_params;

/* ------------------------------------------------------------- projection */

/* Projected records, one per visible (Gaussian, view).  Order: by (view,
 * Gaussian id), so the records of one view are contiguous.  Gaussians are
 * taken in groups of 32 consecutive ids (group k = ids 32k .. 32k+31); the
 * records of one (view, group) are contiguous too.  DEVICE buffers of
 * `capacity` entries; capacity >= n * n_views never overflows.
 *   count      [1]        number of records written
 *   status     [1]        device status word (GS_FLAG_* bits), OR-ed by every call
 *   view_info  [V+1][4]   per view: (first global tile, first pixel, first warp item,
 *                         tile_w | tile_h << 8 | tiles_x << 16); entry V holds the totals
 *                         of the first three and, in its fourth field, G (below).
 *                         A warp item is one 8x4 pixel block of a tile: view v has
 *                         tiles(v) * tile_w * tile_h / 32 of them.
 *   gid, view  [cap]      Gaussian index and view index of the record.  gid may be NULL (not
 *                         written; the library itself never reads it).  view may be NULL
 *                         (not written): gs_bin_sort then finds each view's records through
 *                         grp_base and G, which holds only for records written by gs_project.
 *   splat      [cap][8]   32 bytes per record, everything compositing reads:
 *                         (mu_2D x, mu_2D y, ext, u, a, b, c, o) -- u the uncertainty of the
 *                         Gaussian, (a, b, c) the inverse 2D covariance with
 *                         q = a dx^2 + 2 b dx dy + c dy^2, o the opacity, and ext the
 *                         support half-widths sqrt(Q Sigma_2D,xx) (low 16 bits) and
 *                         sqrt(Q Sigma_2D,yy) (high 16 bits) as IEEE half floats rounded
 *                         up (a conservative bound used only to skip Gaussians that
 *                         cannot reach a pixel block).  32-byte aligned.
 *   color_d    [cap][4]   (r, g, b, depth t_z); may be NULL for records that are only used to
 *                         score information gain (gs_project then skips the colours;
 *                         gs_render_fwd / gs_render_bwd require it)
 *   rect       [cap][4]   uint16 tile rectangle (x0, y0, x1, y1), ends exclusive
 *   depth_key  [cap]      IEEE-754 bits of the float32 depth (the sort key)
 *   grp_mask   [V*G]      bit i of entry v*G + k = Gaussian 32k+i is visible in view v (G = ceil(n/32))
 *   grp_base   [V*G+1]    index of the first record of (view v, group k) at v*G + k; last entry = count
 * The record of Gaussian g in view v is grp_base[v*G+k] + popcount(grp_mask[v*G+k] & ((1 << i) - 1))
 * with k = g / 32, i = g % 32, if bit i is set. */
typedef struct {
  int64_t capacity;
  uint32_t* count;
  uint32_t* status;
  uint32_t* view_info;
  uint32_t* gid;
  uint32_t* view;
  float* splat;
  float* color_d;
  uint16_t* rect;
  uint32_t* depth_key;
  uint32_t* grp_mask;
  uint32_t* grp_base;
} gs_proj;

/* gs_project -- EWA projection of every Gaussian into every view (Sec. III
 * projection, anisotropic generalisation).  Per Gaussian: normalised quaternion
 * -> rotation, Sigma = R_q diag(exp(2 log s)) R_q^T, o = sigmoid(logit).  Per view:
 * t = R^T (mu - T); cull if t_z <= near_plane, outside the guard band, or o < alpha_min;
 * J = [[fx/t_z, 0, -fx t_x/t_z^2], [0, fy/t_z, -fy t_y/t_z^2]];
 * Sigma_2D = J R^T Sigma R J^T + eps2d I; conic = Sigma_2D^-1 (cull if det <= 0);
 * mu_2D = (fx t_x/t_z + cx, fy t_y/t_z + cy); support box from
 * q <= Q = 2 ln(o / alpha_min): half-widths sqrt(Q Sigma_2D,xx), sqrt(Q Sigma_2D,yy),
 * clipped to the image and converted to tiles (cull if empty).
 * Records are written to `out` in (view, Gaussian) order.
 * ws: DEVICE workspace of gs_workspace_size(GS_OP_PROJECT, ...) bytes.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG (n < 0, n_views < 1,
 * n >= 2^32, bad params), GS_ERR_WORKSPACE, GS_ERR_CUDA; device flags
 * GS_FLAG_BAD_CAMERA, GS_FLAG_NONFINITE, GS_FLAG_RECORD_OVERFLOW. */
gs_status gs_project(const gs_map* map, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                     gs_proj* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------- binning / sort */

/* Tile-sorted pair list.  DEVICE buffers:
 *   count   [1]               number of (tile, record) pairs P (may exceed capacity: overflow flag)
 *   tile    [pair_capacity]   global tile id of each pair, ascending; may be NULL (not written)
 *   rec     [pair_capacity]   record index of each pair
 *   ranges  [tile_capacity][2] per global tile: [start, end) into tile/rec, clipped to pair_capacity
 *   item_order [item_capacity] optional, may be NULL: the batch's warp items (32-pixel blocks
 *           of tiles, tile_w * tile_h / 32 per tile, numbered view by view, tile by tile,
 *           block by block) longest tile list first.  The lists are bucketed by length
 *           (four buckets per doubling); the order inside a bucket is unspecified.
 *           gs_bin_sort writes it when the batch has at most item_capacity items, and
 *           gs_render_fwd / gs_render_bwd then take their items in this order, so that the
 *           longest lists do not start last.  Any order gives the same outputs.
 * Global tile id of tile (x, y) of view v = view_info[v].first_tile + y * tiles_x(v) + x,
 * tiles_x(v) = ceil(W_v / tile_w(v)), tiles_y(v) = ceil(H_v / tile_h(v)) with the
 * view's tile size (its camera's, else gs_params'); a view whose camera is invalid
 * (GS_FLAG_BAD_CAMERA) has no tiles. */
typedef struct {
  int64_t pair_capacity;
  int64_t tile_capacity;
  uint32_t* count;
  uint32_t* tile;
  uint32_t* rec;
  uint32_t* ranges;
  uint32_t* item_order;
  int64_t item_capacity;
} gs_bins;

/* gs_bin_sort -- Sec. III "sorted in increasing order of depth": emits one pair
 * per tile covered by each record's rectangle and orders all pairs by
 * (view, tile, float32 depth, record index) -- bit-exact, deterministic.
 * Input: records grouped by view in increasing view order (as gs_project
 * writes them), rectangles inside their view's tile grid; other input sets
 * GS_FLAG_BAD_RECORDS and leaves the output unspecified (but in bounds).
 * Records without view ids (proj->view NULL) must be those gs_project wrote with
 * this proj's view table, group masks and offsets: each view's first record is then
 * read from grp_base (no check of the record order).
 * Implementation: stable LSD radix sort of the record indices by depth bits and
 * then by view; per-view chunks count their pairs per tile; one exclusive scan
 * over (tile, chunk) gives every tile's range and every chunk's first slot in
 * it; each pair is then written once, straight to its slot.
 * ws: DEVICE workspace of gs_workspace_size(GS_OP_BIN_SORT, ...) bytes.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA;
 * device flags GS_FLAG_PAIR_OVERFLOW, GS_FLAG_RANGE_OVERFLOW, GS_FLAG_BAD_RECORDS. */
gs_status gs_bin_sort(const gs_proj* proj, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                      gs_bins* out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------- compositing */

/* Rendered images of all views, concatenated: view v starts at pixel
 * view_info[v].first_pixel = sum_{u<v} P_u (P_v = W_v H_v pixels, row-major; a
 * negative width or height counts as 0).  A view whose camera is invalid
 * (GS_FLAG_BAD_CAMERA) keeps its P_v pixels in this layout but has no tiles:
 * its pixels are not written.  DEVICE buffers:
 *   rgb   [sum_v 3 P_v]  planar per view: channel c of view v at 3*first_pixel + c*P_v
 *   depth [sum_v P_v]    sum_i w_i t_z,i      (Sec. III, c_i replaced by d_i)
 *   unc   [sum_v P_v]    sum_i w_i u_i        (uncertainty channel)
 *   T     [sum_v P_v]    final transmittance prod_i (1 - alpha_i)
 *   last  [sum_v P_v]    1 + position (within the tile's range) of the last Gaussian added, 0 if none
 *   n_contrib [sum_v P_v] number of Gaussians added (work statistics)
 * Any of rgb/depth/unc/n_contrib may be NULL to skip writing it; T and last
 * are required when the images will be differentiated (gs_render_bwd). */
typedef struct {
  float* rgb;
  float* depth;
  float* unc;
  float* T;
  int32_t* last;
  int32_t* n_contrib;
} gs_image;

/* gs_render_fwd -- Sec. III front-to-back compositing.  For every pixel p and
 * the Gaussians of its tile in depth order: alpha = min(alpha_max, o exp(-q/2)),
 * skip if alpha < alpha_min, stop (without adding) if T (1 - alpha) < T_min,
 * else w = alpha T, accumulate w c (RGB), w t_z (depth), w u (uncertainty) and
 * T <- T (1 - alpha).  Background is zero.  The pixel blocks are taken in
 * bins->item_order when gs_bin_sort wrote it (longest tile list first), else tile by tile;
 * the outputs are the same either way.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_CUDA. */
gs_status gs_render_fwd(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_camera* cams,
                        int32_t n_views, const gs_params* prm, gs_image* out, void* stream);

/* gs_render_small -- the forward render of gs_render_fwd (Sec. III), from the map
 * directly, in one kernel launch and without records, bins or workspace: for maps of
 * up to a few thousand Gaussians, whose tiled render (gs_project + gs_bin_sort +
 * gs_render_fwd, about 35 kernels) is bound by launch latency.  Every CTA takes screen
 * tiles, projects the whole map for the tile's view with gs_project's decision
 * arithmetic, sorts the Gaussians whose tile rectangle covers the tile by depth key
 * (ties by Gaussian id) in shared memory and composites the tile; the outputs are bit
 * for bit those of the tiled path with the same parameters (`last` indexes the tile's
 * list of gs_bin_sort).  Cost grows with map size x tiles: use the tiled path for
 * large maps.
 *   map->n <= GS_SMALL_MAX_GAUSSIANS, n_views <= GS_SMALL_MAX_VIEWS, else GS_ERR_ARG.
 *   A tile covered by more than GS_SMALL_MAX_LIST Gaussians sets GS_FLAG_PAIR_OVERFLOW
 *   and its pixels are not written: render such a view with the tiled path.
 *   status: DEVICE uint32[1] status word (OR-ed): also GS_FLAG_BAD_CAMERA (the view
 *   keeps its pixels in the layout and they are not written), GS_FLAG_NONFINITE (checked
 *   when the views have at least one tile) and GS_FLAG_RANGE_OVERFLOW (more than 2^20
 *   tiles or 2^32 pixels over the views: the views past that bound are not written).
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_CUDA. */
#define GS_SMALL_MAX_GAUSSIANS (1 << 16)
#define GS_SMALL_MAX_VIEWS 64
#define GS_SMALL_MAX_LIST 2048
gs_status gs_render_small(const gs_map* map, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                          gs_image* out, uint32_t* status, void* stream);

/* Image-space gradient dL/d(rgb, depth), same layouts as gs_image.rgb / .depth.
 * Either may be NULL (treated as zero).  The uncertainty channel is not
 * differentiated: u_i is not a learned parameter. */
typedef struct {
  const float* rgb;
  const float* depth;
} gs_image_grad;

/* Gradient with respect to every map parameter, DEVICE [n][4] arrays laid out
 * like gs_map (dmo = (dmu, dlogit), dsu = (dlog s, 0), dq, drgb = (dc, 0)).
 * Overwritten (not accumulated) by gs_render_bwd. */
typedef struct {
  float* dmo;
  float* dsu;
  float* dq;
  float* drgb;
} gs_map_grad;

/* gs_render_bwd -- Eq. (2): the adjoint of gs_render_fwd and gs_project.
 * Each tile is replayed back to front from the saved final transmittance and
 * last index (T_i = T_{i+1} / (1 - alpha_i)), keeping suffix sums
 * S = sum_{j>i} w_j x_j; dL/dalpha_i = sum_ch g_ch (x_i T_i - S_ch / (1 - alpha_i)).
 * Screen-space gradients are reduced per Gaussian with warp shuffles before one
 * atomic add per warp, then mapped through the projection to dmu, dlog s, dq
 * (through the normalisation), dlogit and dc.  Float atomics make the last bits
 * of the result depend on scheduling.
 * ws: DEVICE workspace of gs_workspace_size(GS_OP_RENDER_BWD, ...) bytes.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
gs_status gs_render_bwd(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_image* fwd,
                        const gs_image_grad* grad, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                        gs_map_grad* out, void* ws, size_t ws_bytes, void* stream);

/* gs_render_bwd_noalloc -- gs_render_bwd for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is a deployment variant.
 *
 * Who needs it: a process that reserves all of its device memory once at
 * start-up and must not allocate afterwards (for example a robot's real-time
 * mapping loop), a plugin that only receives the buffers of its host
 * application and has no allocator of its own, or code whose launches a
 * framework is capturing into a CUDA graph and that must not allocate during
 * the capture.  Such callers cannot provide the workspace of gs_render_bwd.
 *
 * What differs: the per-record scratch (48 bytes per record) lives in a fixed
 * array inside the library's device image, sized for GS_NOALLOC_MAX_RECORDS
 * records (12 MiB), which every GPU that loads the library keeps until the
 * process exits.  Inputs and outputs are exactly those of gs_render_bwd (the
 * caller still passes them); no workspace argument; nothing is allocated (no
 * cudaMalloc, no cudaFree, no allocating library call).
 *   - Every argument is checked exactly as gs_render_bwd checks it (same
 *     codes); then proj->capacity above GS_NOALLOC_MAX_RECORDS is rejected
 *     with GS_ERR_WORKSPACE.  Nothing is enqueued on an error.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one array, which keeps the last call's contents;
 *     the call clears the part it uses before accumulating into it.  Calls
 *     whose executions overlap on the GPU (different streams, or different host
 *     threads on one device) race on the array and must be serialised by the
 *     caller.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
#define GS_NOALLOC_MAX_RECORDS (1 << 18)
gs_status gs_render_bwd_noalloc(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_image* fwd,
                                const gs_image_grad* grad, const gs_camera* cams, int32_t n_views,
                                const gs_params* prm, gs_map_grad* out, void* stream);

/* ------------------------------------------------------- information gain */
/* The `mode` argument of gs_info_gain_batch and gs_info_gain_composite selects
 * the score; GS_IG_RENDER_MEAN is the only value accepted (any other returns
 * GS_ERR_ARG).  The argument is kept for further rendered scores.  The paper's
 * own render-free score (xi, Eq. view_util) has its own entry point,
 * gs_view_utility_batch, because it reads the map directly and needs no
 * records, bins or images. */
enum { GS_IG_RENDER_MEAN = 0 };

/* gs_info_gain_batch -- Eq. (nbv) with the Jacobian replaced by the per-pixel
 * blend weights: IG_v = (1 / P_v) sum_p sum_i w_i(p) u_i, the mean of the
 * composited uncertainty channel of view v.  All n_views candidate views (of
 * any mix of resolutions) are projected, sorted and composited together:
 * projection and sort as gs_project / gs_bin_sort over the whole batch, then
 * one persistent compositing kernel that takes (view, tile) work items from a
 * device queue and writes each tile's sum of U to a fixed slot, then a
 * fixed-order per-view reduction.  Same alpha / skip / stop rules as
 * gs_render_fwd.  ig_out: DEVICE float[n_views].
 * status: DEVICE uint32[1] status word (OR-ed).
 * record_capacity / pair_capacity / tile_capacity: capacities used inside ws (see
 * gs_workspace_size, whose rec_capacity is record_capacity); record_capacity 0
 * means n * n_views, which never overflows.  More visible (Gaussian, view)
 * records than record_capacity set GS_FLAG_RECORD_OVERFLOW.
 * Errors: as gs_project and gs_bin_sort. */
gs_status gs_info_gain_batch(const gs_map* map, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                             int32_t mode, float* ig_out, uint32_t* status, int64_t record_capacity,
                             int64_t pair_capacity, int64_t tile_capacity, void* ws, size_t ws_bytes, void* stream);

/* gs_info_gain_composite -- Eq. (nbv), Sec. IV-A: the compositing stage of
 * gs_info_gain_batch on records and bins already produced by gs_project and
 * gs_bin_sort for the candidate views: U-only front-to-back compositing (same alpha / skip / stop
 * rules as gs_render_fwd) by a persistent kernel that takes warp items (8x4
 * pixel blocks of tiles) longest tile list first from a device queue, one slot
 * per item, then a fixed-order per-view reduction IG_v = (1/P_v) sum_p U(p).
 * Exposed so that one projection and binning can be reused, and so the
 * compositing kernel can be timed on its own.  ig_out: DEVICE float[n_views].
 * ws: DEVICE workspace of gs_workspace_size(GS_OP_IG_COMPOSITE, ...) bytes.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
gs_status gs_info_gain_composite(const gs_proj* proj, const gs_bins* bins, const gs_camera* cams, int32_t n_views,
                                 const gs_params* prm, int32_t mode, float* ig_out, void* ws, size_t ws_bytes,
                                 void* stream);

/* --------------------------------------------- render-free view utility (Sec. IV-A/B)
 * The paper scores candidate poses without rendering: per Gaussian, the magnitude
 * of the change of its mean between map updates is its uncertainty u; Gaussians
 * with u above mean(u) + sigma(u)/2 form G_H, below mean(u) - sigma(u)/2 form G_L;
 * a pose's utility is xi = |visible G_H| - lambda |visible G_L| (Eq. view_util).
 * v(x, g) = 1 iff g's mean lies in front of the camera with near < t_z <= range
 * (the sensor's perception range) and projects inside the image; no occlusion
 * test.  The map's u channel is gs_map.su[i].w. */
enum { GS_U_ABS = 0, GS_U_SQ = 1 };        /* u = |mu_k - mu_{k-1}|, or its square (ablation) */
enum { GS_XI = 0, GS_XI_SUM = 1 };         /* Eq. view_util, or sum of u over visible Gaussians (ablation) */

/* Parameters of the view utility.  near_plane > 0, range > near_plane; lambda:
 * lambda_xi (1 in the paper); Gaussians with mu_z < ground_z are left out of the
 * thresholds and of xi (ground-plane removal; -INFINITY keeps every Gaussian). */
typedef struct {
  float near_plane, range, lambda, ground_z;
} gs_utility_params;

/* Cuboid regions: region (ix, iy, iz), 0 <= i < dims, holds the means with
 * floor((mu - origin) / size) = (ix, iy, iz); region index (iz dims[1] + iy) dims[0] + ix. */
typedef struct {
  float origin[3];
  float size;
  int32_t dims[3];
} gs_region_grid;

/* gs_uncertainty_update -- Sec. IV-A: for every Gaussian whose mean changed
 * between mo_prev and mo_cur (DEVICE float[n][4], means in the first three), set
 * su[i][3] = |mu_cur - mu_prev| (GS_U_ABS) or its square (GS_U_SQ); Gaussians whose
 * mean did not change keep their previous value (the paper's bookkeeping).  Each
 * difference, product and sum is rounded separately (IEEE FP32, no fused
 * multiply-add), the root correctly rounded.  su: DEVICE float[n][4].
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN (16-byte arrays), GS_ERR_ARG, GS_ERR_CUDA. */
gs_status gs_uncertainty_update(const float* mo_prev, const float* mo_cur, float* su, int64_t n, int32_t mode,
                                void* stream);

/* gs_uncertainty_thresholds -- Sec. IV-C: G_H and G_L are the Gaussians whose update
 * magnitude u lies more than half a standard deviation above / below its mean (ground
 * Gaussians left out, Sec. IV-C).  Mean and population standard deviation of u over the
 * Gaussians with mu_z >= ground_z (FP64, two passes, fixed summation order), into
 * DEVICE double stats[5] = (mean, sigma, mean + sigma/2, mean - sigma/2, count).
 * ws: DEVICE workspace of gs_workspace_size(GS_OP_THRESHOLDS, ...) bytes.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
gs_status gs_uncertainty_thresholds(const gs_map* map, float ground_z, double* stats, void* ws, size_t ws_bytes,
                                    void* stream);

/* gs_view_utility_batch -- Eq. view_util for n_views poses in one batch:
 * GS_XI: xi_v = |{g in G_H: v(x_v, g)}| - lambda |{g in G_L: v(x_v, g)}| with
 * G_H = {u > stats[2]}, G_L = {u < stats[3]} (stats from gs_uncertainty_thresholds);
 * GS_XI_SUM: xi_v = sum of u over the visible Gaussians (FP32, fixed order).
 * Visibility is decided in FP32: t = R^T (mu - T) with every product and sum
 * rounded separately in the order (R0 dx + R3 dy) + R6 dz (likewise for t_y, t_z),
 * pixel = (fx t_x / t_z + cx, fy t_y / t_z + cy) with correctly rounded division,
 * visible iff near < t_z <= range, 0 <= px < W and 0 <= py < H.
 * xi_out: DEVICE float[n_views]; counts_out: DEVICE uint32[n_views][2] (visible
 * |G_H|, |G_L|) or NULL.  Deterministic.  ws: gs_workspace_size(GS_OP_VIEW_UTILITY).
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
gs_status gs_view_utility_batch(const gs_map* map, const gs_camera* cams, int32_t n_views,
                                const gs_utility_params* prm, int32_t mode, const double* stats, float* xi_out,
                                uint32_t* counts_out, void* ws, size_t ws_bytes, void* stream);

/* gs_trajectory_utility -- Eq. traj_utility: n_traj trajectories of n_states states
 * each (cams[t * n_states + l] is state l of trajectory t); traj_out[t] = sum over l of
 * xi (as gs_view_utility_batch, summed in FP64 in state order), best_out[0] = the first t
 * with the largest sum.  traj_out: DEVICE float[n_traj]; best_out: DEVICE int32[1].
 * ws: gs_workspace_size(GS_OP_TRAJECTORY, ...) with n_views = n_traj * n_states.
 * Errors: as gs_view_utility_batch. */
gs_status gs_trajectory_utility(const gs_map* map, const gs_camera* cams, int32_t n_traj, int32_t n_states,
                                const gs_utility_params* prm, int32_t mode, const double* stats, float* traj_out,
                                int32_t* best_out, void* ws, size_t ws_bytes, void* stream);

/* gs_collision_check -- Sec. IV-B collision checking with all Gaussians: for every
 * test point p_k (DEVICE float[n_points][4], position in the first three),
 * margin_out[k] = min over the Gaussians with mu_z >= ground_z of |p_k - mu_i| - gamma_i,
 * gamma_i = r_robot + lambda_g r_i, r_i = exp(largest log-scale) (the principal axis
 * as the radius); +INFINITY if there is no Gaussian.  collides_out[k] = 1 iff some
 * Gaussian has |p_k - mu_i|^2 < gamma_i^2, decided in FP32 with separately rounded
 * operations: d = p - mu, |d|^2 = (dx dx + dy dy) + dz dz, gamma = r_robot + lambda_g r,
 * gamma^2 = gamma gamma, r from the library's FP32 exp (Cody-Waite).  Deterministic.
 * margin_out: DEVICE float[n_points]; collides_out: DEVICE uint32[n_points].
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_CUDA. */
gs_status gs_collision_check(const gs_map* map, const float* points, int32_t n_points, float r_robot,
                             float lambda_g, float ground_z, float* margin_out, uint32_t* collides_out,
                             void* stream);

/* gs_region_uncertainty -- Sec. IV-B high-level planner: mean uncertainty of each
 * cuboid region, Omega_o = (1/M_o) sum over the region's Gaussians of u (0 if M_o = 0).
 * omega_out: DEVICE float[R], count_out: DEVICE uint32[R] (M_o) or NULL,
 * R = dims[0] dims[1] dims[2].  Sums in FP64 (atomic, so the last bits of a sum
 * may depend on the order).  ws: gs_workspace_size(GS_OP_REGIONS, ...) with R as
 * rec_capacity.  Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
gs_status gs_region_uncertainty(const gs_map* map, const gs_region_grid* grid, float* omega_out, uint32_t* count_out,
                                void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------ mapping loss (Eq. 3)
 * The map is refined by minimising, over the keyframes, a photometric loss of
 * the rendered colour and depth against the observations (Eq. 3):
 *   L = (1/N_p) sum_p (w_d |d(p) - d_ref(p)| + w_c |c(p) - c_ref(p)|_1) + w_s (1 - SSIM(c, c_ref))
 * with the paper's weights w_d = 1, w_c = lambda_1 = 0.4, w_s = lambda_2 = 0.1.  Readings where the
 * paper is silent: N_p is the total pixel count of all views in the call; |.|_1 sums the
 * three channels; SSIM is the mean over the three channels and all pixels of
 *   S(p) = ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
 * C1 = 0.01^2, C2 = 0.03^2, with windowed moments mu = G*x, s_x^2 = G*(x^2) - mu_x^2,
 * s_xy = G*(x y) - mu_x mu_y over an 11 x 11 Gaussian window (sigma 1.5, normalised),
 * the image taken as zero outside its border; each view is its own image. */
typedef struct {
  float w_depth, w_rgb, w_ssim;
} gs_loss_weights;

/* gs_image_loss -- Eq. 3 for n_views rendered views against their references, and its
 * gradient with respect to the rendered images (ready for gs_render_bwd).
 *   sizes      HOST int32[n_views][2]: (width, height) of each view, > 0
 *   rgb, rgb_ref      DEVICE float, the gs_image.rgb layout (views concatenated, planar per view)
 *   depth, depth_ref  DEVICE float, the gs_image.depth layout; may be NULL iff w_depth = 0
 *   loss_out   DEVICE float[4]: (L, mean |d - d_ref|, mean |c - c_ref|_1, SSIM), the sums in FP64
 *              in a fixed order (deterministic)
 *   d_rgb      DEVICE float, dL/d rgb (rgb layout) or NULL; d_depth: dL/d depth or NULL.
 *              The L1 terms use sign(0) = 0.  Overwritten.
 * w_depth, w_rgb, w_ssim >= 0 and finite.  ws: DEVICE workspace of
 * gs_image_loss_workspace_size bytes (the same sizes).
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA. */
gs_status gs_image_loss(const int32_t* sizes, int32_t n_views, const float* rgb, const float* depth,
                        const float* rgb_ref, const float* depth_ref, const gs_loss_weights* w, float* loss_out,
                        float* d_rgb, float* d_depth, void* ws, size_t ws_bytes, void* stream);

/* gs_image_loss_workspace_size -- HOST.  Workspace bytes of gs_image_loss for these view
 * sizes (HOST int32[n_views][2]) into *bytes.  Errors: GS_ERR_NULL, GS_ERR_ARG. */
gs_status gs_image_loss_workspace_size(const int32_t* sizes, int32_t n_views, size_t* bytes);

/* ------------------------------------------------ optimiser of the mapping iterations
 * The map is refined by gradient steps on the rendering loss (Eq. 2, Sec. IV-A); the
 * mapping module uses Adam (Kingma and Ba). */
typedef struct {
  double lr, beta1, beta2, eps;   /* double, so that 1 - beta and beta^t keep their precision */
} gs_adam_params;

enum { GS_ADAM_MAX_TENSORS = 8 };

/* gs_adam_step -- one Adam update of up to GS_ADAM_MAX_TENSORS tensors in place:
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   p <- p - (lr / c1) m / (sqrt(v) / sqrt(c2) + eps),  c1 = 1 - b1^t, c2 = 1 - b2^t,
 * with t = *step + 1; *step is incremented on the device after the update, so a captured
 * graph replays successive steps.
 *   params, grads, m, v  HOST arrays of n_tensors DEVICE float pointers, 16-byte aligned;
 *                        grads[i] == NULL skips tensor i (no gradient)
 *   sizes                HOST int64[n_tensors]: elements of each tensor, a multiple of 4
 *   step                 DEVICE uint32[1]: steps completed so far (0 before the first)
 * lr >= 0, 0 <= beta1, beta2 < 1, eps > 0, all finite.  Deterministic.
 * Errors: GS_ERR_NULL, GS_ERR_ALIGN, GS_ERR_ARG, GS_ERR_CUDA. */
gs_status gs_adam_step(float* const* params, const float* const* grads, float* const* m, float* const* v,
                       const int64_t* sizes, int32_t n_tensors, const gs_adam_params* prm, uint32_t* step,
                       void* stream);

/* ------------------------------------------------------------- utilities */
/* The library's own bookkeeping (workspace sizes, the device status word, status
 * strings, version, launch count): none of these computes a step of the method, so
 * no passage of the paper applies to them. */
enum {
  GS_OP_PROJECT = 0,
  GS_OP_BIN_SORT = 1,
  GS_OP_RENDER_BWD = 2,
  GS_OP_INFO_GAIN = 3,
  GS_OP_IG_COMPOSITE = 4,
  GS_OP_THRESHOLDS = 5,
  GS_OP_VIEW_UTILITY = 6,
  GS_OP_REGIONS = 7,
  GS_OP_TRAJECTORY = 8
};

/* gs_workspace_size -- HOST.  Bytes of workspace `op` needs:
 *   n, n_views      map size and number of views
 *   rec_capacity    record capacity of the gs_proj in use (GS_OP_INFO_GAIN: the record_capacity
 *                   argument, 0 for n * n_views; GS_OP_REGIONS: the number of regions)
 *   pair_capacity   pair capacity of the gs_bins in use
 *   tile_capacity   tile capacity of the gs_bins in use (GS_OP_IG_COMPOSITE: only this is used)
 * GS_OP_THRESHOLDS needs nothing else; GS_OP_VIEW_UTILITY and GS_OP_TRAJECTORY only n_views
 * (for GS_OP_TRAJECTORY: the total number of states).
 * Writes the byte count to *bytes (HOST).  Errors: GS_ERR_NULL, GS_ERR_ARG, GS_ERR_CUDA. */
gs_status gs_workspace_size(int32_t op, int64_t n, int32_t n_views, int64_t rec_capacity, int64_t pair_capacity,
                            int64_t tile_capacity, size_t* bytes);

/* gs_read_status -- copies the device status word to *flags (HOST) with a
 * blocking cudaMemcpy (synchronises with the device).  Returns GS_ERR_DEVICE if
 * any GS_FLAG_ERROR_MASK bit is set, else GS_OK. */
gs_status gs_read_status(const uint32_t* status, uint32_t* flags);

/* Human-readable name of a status code (static string, HOST). */
const char* gs_status_str(gs_status s);

/* Library version, "major.minor.patch" (static string, HOST). */
const char* gs_version(void);

/* Number of kernels this library has enqueued since it was loaded (HOST, all
 * devices and threads).  Kernels replayed from a captured CUDA graph are not
 * re-counted: a graph replay re-runs the kernels counted while capturing. */
uint64_t gs_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* GS103_GS_H */
