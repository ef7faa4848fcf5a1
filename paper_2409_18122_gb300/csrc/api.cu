// api.cu -- the extern "C" entry points declared in include/gs.h: argument
// validation on the host, then the launches of the stage kernels on the
// caller's stream.  Nothing here allocates, synchronises or prints.
#include <stdint.h>

#include <atomic>
#include <cmath>

#include "gs_internal.h"

namespace gs {

static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 64 && cached[dev] > 0) return cached[dev];
  int n = 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  if (dev < 64) cached[dev] = n;
  return n;
}

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

gs_status check_params(const gs_params* p) {
  if (!p) return GS_ERR_NULL;
  const int B = p->tile_w * p->tile_h;
  if ((p->tile_w != 8 && p->tile_w != 16 && p->tile_w != 32 && p->tile_w != 64) || p->tile_h < 8 ||
      p->tile_h % 8 != 0 || (B != 64 && B != 128 && B != 256 && B != 512 && B != 1024))
    return GS_ERR_ARG;
  if (!(p->eps2d >= 0.f) || !(p->near_plane > 0.f) || !(p->guard > 0.f)) return GS_ERR_ARG;
  if (!(p->alpha_min >= 0.f && p->alpha_min < 1.f)) return GS_ERR_ARG;
  if (!(p->alpha_max > 0.f && p->alpha_max <= 1.f)) return GS_ERR_ARG;
  if (!(p->T_min >= 0.f && p->T_min < 1.f)) return GS_ERR_ARG;
  if (p->ig_batch != 0 && p->ig_batch != 4 && p->ig_batch != 8 && p->ig_batch != 16) return GS_ERR_ARG;
  if (p->fwd_batch != 0 && p->fwd_batch != 1 && p->fwd_batch != 2 && p->fwd_batch != 4) return GS_ERR_ARG;
  return GS_OK;
}

gs_status check_map(const gs_map* m) {
  if (!m) return GS_ERR_NULL;
  if (m->n < 0 || m->n >= ((int64_t)1 << 32) - 1) return GS_ERR_ARG;
  if (m->n == 0) return GS_OK;
  if (!m->mo || !m->su || !m->q || !m->rgb) return GS_ERR_NULL;
  if (!aligned(m->mo, 16) || !aligned(m->su, 16) || !aligned(m->q, 16) || !aligned(m->rgb, 16)) return GS_ERR_ALIGN;
  return GS_OK;
}

gs_status check_views(const gs_camera* cams, int32_t n_views) {
  if (n_views < 1 || n_views > (1 << 20)) return GS_ERR_ARG;
  if (!cams) return GS_ERR_NULL;
  if (!aligned(cams, 4)) return GS_ERR_ALIGN;
  return GS_OK;
}

gs_status check_proj(const gs_proj* p) {
  if (!p) return GS_ERR_NULL;
  if (p->capacity < 0 || p->capacity >= ((int64_t)1 << 32) - 1) return GS_ERR_ARG;
  if (!p->count || !p->status || !p->view_info || !p->grp_mask || !p->grp_base) return GS_ERR_NULL;
  if (p->capacity > 0 && (!p->splat || !p->rect || !p->depth_key)) return GS_ERR_NULL;   // view may be NULL
  if (!aligned(p->splat, 32) || !aligned(p->color_d, 16) || !aligned(p->rect, 8) || !aligned(p->gid, 4) ||
      !aligned(p->view, 4) || !aligned(p->depth_key, 4) || !aligned(p->count, 4) || !aligned(p->status, 4) ||
      !aligned(p->view_info, 4) || !aligned(p->grp_mask, 4) || !aligned(p->grp_base, 4))
    return GS_ERR_ALIGN;
  return GS_OK;
}

gs_status check_bins(const gs_bins* b) {
  if (!b) return GS_ERR_NULL;
  if (b->pair_capacity < 1 || b->pair_capacity >= ((int64_t)1 << 32) - 1) return GS_ERR_ARG;
  if (b->tile_capacity < 1 || b->tile_capacity >= ((int64_t)1 << 27)) return GS_ERR_ARG;
  if (!b->count || !b->rec || !b->ranges) return GS_ERR_NULL;   // tile may be NULL
  if (!aligned(b->count, 4) || !aligned(b->tile, 4) || !aligned(b->rec, 4) || !aligned(b->ranges, 8)) return GS_ERR_ALIGN;
  if (b->item_order && (b->item_capacity < 0 || b->item_capacity >= ((int64_t)1 << 32))) return GS_ERR_ARG;
  if (!aligned(b->item_order, 4)) return GS_ERR_ALIGN;
  return GS_OK;
}

gs_status check_image(const gs_image* im) {
  if (!aligned(im->rgb, 4) || !aligned(im->depth, 4) || !aligned(im->unc, 4) || !aligned(im->T, 4) ||
      !aligned(im->last, 4) || !aligned(im->n_contrib, 4))
    return GS_ERR_ALIGN;
  return GS_OK;
}

gs_status check_image_grad(const gs_image_grad* g) {
  return aligned(g->rgb, 4) && aligned(g->depth, 4) ? GS_OK : GS_ERR_ALIGN;
}

gs_status check_ws(void* ws, size_t have, size_t need) {
  if (need == 0) return GS_OK;
  if (!ws) return GS_ERR_NULL;
  if (!aligned(ws, 256)) return GS_ERR_ALIGN;
  if (have < need) return GS_ERR_WORKSPACE;
  return GS_OK;
}

gs_status from_cuda(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

#define GS_TRY(x)                   \
  do {                              \
    gs_status s__ = (x);            \
    if (s__ != GS_OK) return s__;   \
  } while (0)

}  // namespace

gs_status validate_render_bwd(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_image* fwd,
                              const gs_image_grad* grad, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                              const gs_map_grad* out) {
  GS_TRY(check_map(map));
  GS_TRY(check_proj(proj));
  GS_TRY(check_bins(bins));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  if (!fwd || !grad || !out) return GS_ERR_NULL;
  if (!fwd->T || !fwd->last) return GS_ERR_NULL;
  if (proj->capacity > 0 && !proj->color_d) return GS_ERR_NULL;
  if (map->n > 0 && (!out->dmo || !out->dsu || !out->dq || !out->drgb)) return GS_ERR_NULL;
  if (!aligned(out->dmo, 16) || !aligned(out->dsu, 16) || !aligned(out->dq, 16) || !aligned(out->drgb, 16))
    return GS_ERR_ALIGN;
  GS_TRY(check_image(fwd));
  GS_TRY(check_image_grad(grad));
  return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_project(const gs_map* map, const gs_camera* cams, int32_t n_views, const gs_params* prm, gs_proj* out,
                     void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_project");
  GS_TRY(check_map(map));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  GS_TRY(check_proj(out));
  GS_TRY(check_ws(ws, ws_bytes, project_ws_bytes(map->n, n_views)));
  return from_cuda(launch_project(*map, cams, n_views, *prm, *out, ws, (cudaStream_t)stream));
}

gs_status gs_bin_sort(const gs_proj* proj, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                      gs_bins* out, void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_bin_sort");
  GS_TRY(check_proj(proj));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  GS_TRY(check_bins(out));
  GS_TRY(check_ws(ws, ws_bytes, bin_ws_bytes(proj->capacity, out->pair_capacity, out->tile_capacity, n_views)));
  return from_cuda(launch_bin_sort(*proj, cams, n_views, *prm, *out, ws, (cudaStream_t)stream));
}

gs_status gs_render_fwd(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_camera* cams,
                        int32_t n_views, const gs_params* prm, gs_image* out, void* stream) {
  GS_TRACE("gs_render_fwd");
  GS_TRY(check_map(map));
  GS_TRY(check_proj(proj));
  GS_TRY(check_bins(bins));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  if (!out) return GS_ERR_NULL;
  if (proj->capacity > 0 && !proj->color_d) return GS_ERR_NULL;   // colours are needed to render
  GS_TRY(check_image(out));
  return from_cuda(launch_render_fwd(*map, *proj, *bins, cams, n_views, *prm, *out, (cudaStream_t)stream));
}

gs_status gs_render_small(const gs_map* map, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                          gs_image* out, uint32_t* status, void* stream) {
  GS_TRACE("gs_render_small");
  GS_TRY(check_map(map));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  if (map->n > GS_SMALL_MAX_GAUSSIANS || n_views > GS_SMALL_MAX_VIEWS) return GS_ERR_ARG;
  if (!out || !status) return GS_ERR_NULL;
  if (!aligned(status, 4)) return GS_ERR_ALIGN;
  GS_TRY(check_image(out));
  return from_cuda(launch_render_small(*map, cams, n_views, *prm, *out, status, (cudaStream_t)stream));
}

gs_status gs_render_bwd(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_image* fwd,
                        const gs_image_grad* grad, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                        gs_map_grad* out, void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_render_bwd");
  GS_TRY(validate_render_bwd(map, proj, bins, fwd, grad, cams, n_views, prm, out));
  GS_TRY(check_ws(ws, ws_bytes, bwd_ws_bytes(proj->capacity)));
  return from_cuda(
      launch_render_bwd(*map, *proj, *bins, *fwd, *grad, cams, n_views, *prm, *out, ws, (cudaStream_t)stream));
}

gs_status gs_info_gain_batch(const gs_map* map, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                             int32_t mode, float* ig_out, uint32_t* status, int64_t record_capacity,
                             int64_t pair_capacity, int64_t tile_capacity, void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_info_gain_batch");
  GS_TRY(check_map(map));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  if (mode != GS_IG_RENDER_MEAN) return GS_ERR_ARG;
  if (!ig_out || !status) return GS_ERR_NULL;
  if (!aligned(ig_out, 4) || !aligned(status, 4)) return GS_ERR_ALIGN;
  if (pair_capacity < 1 || pair_capacity >= ((int64_t)1 << 32) - 1) return GS_ERR_ARG;
  if (tile_capacity < 1 || tile_capacity >= ((int64_t)1 << 27)) return GS_ERR_ARG;
  if (record_capacity < 0) return GS_ERR_ARG;
  const int64_t rec_cap = record_capacity > 0 ? record_capacity : map->n * (int64_t)n_views;
  if (rec_cap >= ((int64_t)1 << 32) - 1) return GS_ERR_ARG;
  GS_TRY(check_ws(ws, ws_bytes, ig_ws_bytes(map->n, n_views, rec_cap, pair_capacity, tile_capacity)));
  return from_cuda(launch_info_gain(*map, cams, n_views, *prm, ig_out, status, rec_cap, pair_capacity,
                                    tile_capacity, ws, (cudaStream_t)stream));
}

gs_status gs_info_gain_composite(const gs_proj* proj, const gs_bins* bins, const gs_camera* cams, int32_t n_views,
                                 const gs_params* prm, int32_t mode, float* ig_out, void* ws, size_t ws_bytes,
                                 void* stream) {
  GS_TRACE("gs_info_gain_composite");
  GS_TRY(check_proj(proj));
  GS_TRY(check_bins(bins));
  GS_TRY(check_views(cams, n_views));
  GS_TRY(check_params(prm));
  if (mode != GS_IG_RENDER_MEAN) return GS_ERR_ARG;
  if (!ig_out) return GS_ERR_NULL;
  if (!aligned(ig_out, 4)) return GS_ERR_ALIGN;
  GS_TRY(check_ws(ws, ws_bytes, ig_composite_ws_bytes(bins->tile_capacity)));
  return from_cuda(launch_ig_composite(*proj, *bins, cams, n_views, *prm, ig_out, ws, (cudaStream_t)stream));
}

gs_status gs_uncertainty_update(const float* mo_prev, const float* mo_cur, float* su, int64_t n, int32_t mode,
                                void* stream) {
  GS_TRACE("gs_uncertainty_update");
  if (n < 0 || (mode != GS_U_ABS && mode != GS_U_SQ)) return GS_ERR_ARG;
  if (n > 0 && (!mo_prev || !mo_cur || !su)) return GS_ERR_NULL;
  if (!aligned(mo_prev, 16) || !aligned(mo_cur, 16) || !aligned(su, 16)) return GS_ERR_ALIGN;
  return from_cuda(launch_uncertainty_update(mo_prev, mo_cur, su, n, mode == GS_U_SQ, (cudaStream_t)stream));
}

gs_status gs_uncertainty_thresholds(const gs_map* map, float ground_z, double* stats, void* ws, size_t ws_bytes,
                                    void* stream) {
  GS_TRACE("gs_uncertainty_thresholds");
  GS_TRY(check_map(map));
  if (!stats) return GS_ERR_NULL;
  if (!aligned(stats, 8)) return GS_ERR_ALIGN;
  if (ground_z != ground_z) return GS_ERR_ARG;
  GS_TRY(check_ws(ws, ws_bytes, thresholds_ws_bytes()));
  return from_cuda(launch_uncertainty_thresholds(map->mo, map->su, map->n, ground_z, stats, ws, (cudaStream_t)stream));
}

gs_status gs_view_utility_batch(const gs_map* map, const gs_camera* cams, int32_t n_views,
                                const gs_utility_params* prm, int32_t mode, const double* stats, float* xi_out,
                                uint32_t* counts_out, void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_view_utility_batch");
  GS_TRY(check_map(map));
  GS_TRY(check_views(cams, n_views));
  if (!prm || !xi_out) return GS_ERR_NULL;
  if (mode != GS_XI && mode != GS_XI_SUM) return GS_ERR_ARG;
  if (mode == GS_XI && !stats) return GS_ERR_NULL;
  if (!(prm->near_plane > 0.f) || !(prm->range > prm->near_plane) || !(prm->lambda == prm->lambda) ||
      prm->ground_z != prm->ground_z)
    return GS_ERR_ARG;
  if (!aligned(xi_out, 4) || !aligned(counts_out, 4) || !aligned(stats, 8)) return GS_ERR_ALIGN;
  GS_TRY(check_ws(ws, ws_bytes, utility_ws_bytes(n_views)));
  return from_cuda(launch_view_utility(map->mo, map->su, map->n, cams, n_views, *prm, mode, stats, xi_out, counts_out,
                                       ws, (cudaStream_t)stream));
}

gs_status gs_trajectory_utility(const gs_map* map, const gs_camera* cams, int32_t n_traj, int32_t n_states,
                                const gs_utility_params* prm, int32_t mode, const double* stats, float* traj_out,
                                int32_t* best_out, void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_trajectory_utility");
  GS_TRY(check_map(map));
  if (n_traj < 1 || n_states < 1 || (int64_t)n_traj * n_states > (1 << 20)) return GS_ERR_ARG;
  GS_TRY(check_views(cams, n_traj * n_states));
  if (!prm || !traj_out || !best_out) return GS_ERR_NULL;
  if (mode != GS_XI && mode != GS_XI_SUM) return GS_ERR_ARG;
  if (mode == GS_XI && !stats) return GS_ERR_NULL;
  if (!(prm->near_plane > 0.f) || !(prm->range > prm->near_plane) || !(prm->lambda == prm->lambda) ||
      prm->ground_z != prm->ground_z)
    return GS_ERR_ARG;
  if (!aligned(traj_out, 4) || !aligned(best_out, 4) || !aligned(stats, 8)) return GS_ERR_ALIGN;
  GS_TRY(check_ws(ws, ws_bytes, trajectory_ws_bytes(n_traj * n_states)));
  return from_cuda(launch_trajectory_utility(map->mo, map->su, map->n, cams, n_traj, n_states, *prm, mode, stats,
                                             traj_out, best_out, ws, (cudaStream_t)stream));
}

gs_status gs_collision_check(const gs_map* map, const float* points, int32_t n_points, float r_robot,
                             float lambda_g, float ground_z, float* margin_out, uint32_t* collides_out,
                             void* stream) {
  GS_TRACE("gs_collision_check");
  GS_TRY(check_map(map));
  if (n_points < 0 || !(r_robot >= 0.f) || !(lambda_g >= 0.f) || ground_z != ground_z) return GS_ERR_ARG;
  if (n_points > 0 && (!points || !margin_out || !collides_out)) return GS_ERR_NULL;
  if (!aligned(points, 16) || !aligned(margin_out, 4) || !aligned(collides_out, 4)) return GS_ERR_ALIGN;
  return from_cuda(launch_collision_check(map->mo, map->su, map->n, points, n_points, r_robot, lambda_g, ground_z,
                                          margin_out, collides_out, (cudaStream_t)stream));
}

gs_status gs_region_uncertainty(const gs_map* map, const gs_region_grid* grid, float* omega_out, uint32_t* count_out,
                                void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_region_uncertainty");
  GS_TRY(check_map(map));
  if (!grid || !omega_out) return GS_ERR_NULL;
  if (!(grid->size > 0.f) || grid->dims[0] < 1 || grid->dims[1] < 1 || grid->dims[2] < 1) return GS_ERR_ARG;
  const int64_t nr = (int64_t)grid->dims[0] * grid->dims[1] * grid->dims[2];
  if (nr > ((int64_t)1 << 30)) return GS_ERR_ARG;
  if (!aligned(omega_out, 4) || !aligned(count_out, 4)) return GS_ERR_ALIGN;
  GS_TRY(check_ws(ws, ws_bytes, regions_ws_bytes(nr)));
  return from_cuda(launch_regions(map->mo, map->su, map->n, *grid, omega_out, count_out, ws, (cudaStream_t)stream));
}

gs_status gs_image_loss(const int32_t* sizes, int32_t n_views, const float* rgb, const float* depth,
                        const float* rgb_ref, const float* depth_ref, const gs_loss_weights* w, float* loss_out,
                        float* d_rgb, float* d_depth, void* ws, size_t ws_bytes, void* stream) {
  GS_TRACE("gs_image_loss");
  if (!sizes || !w || !rgb || !rgb_ref || !loss_out) return GS_ERR_NULL;
  if (n_views < 1) return GS_ERR_ARG;
  const float wt[3] = {w->w_depth, w->w_rgb, w->w_ssim};
  for (float x : wt)
    if (!(x >= 0.f) || std::isinf(x)) return GS_ERR_ARG;
  if (w->w_depth != 0.f && (!depth || !depth_ref)) return GS_ERR_NULL;
  if ((depth == nullptr) != (depth_ref == nullptr)) return GS_ERR_NULL;
  const size_t need = image_loss_ws_bytes(sizes, n_views);
  if (need == 0) return GS_ERR_ARG;
  if (!aligned(rgb, 4) || !aligned(rgb_ref, 4) || !aligned(depth, 4) || !aligned(depth_ref, 4) ||
      !aligned(loss_out, 4) || !aligned(d_rgb, 4) || !aligned(d_depth, 4))
    return GS_ERR_ALIGN;
  GS_TRY(check_ws(ws, ws_bytes, need));
  return from_cuda(launch_image_loss(sizes, n_views, rgb, depth, rgb_ref, depth_ref, *w, loss_out, d_rgb, d_depth, ws,
                                     (cudaStream_t)stream));
}

gs_status gs_image_loss_workspace_size(const int32_t* sizes, int32_t n_views, size_t* bytes) {
  if (!sizes || !bytes) return GS_ERR_NULL;
  if (n_views < 1) return GS_ERR_ARG;
  const size_t need = image_loss_ws_bytes(sizes, n_views);
  if (need == 0) return GS_ERR_ARG;
  *bytes = need;
  return GS_OK;
}

gs_status gs_adam_step(float* const* params, const float* const* grads, float* const* m, float* const* v,
                       const int64_t* sizes, int32_t n_tensors, const gs_adam_params* prm, uint32_t* step,
                       void* stream) {
  GS_TRACE("gs_adam_step");
  if (!params || !grads || !m || !v || !sizes || !prm || !step) return GS_ERR_NULL;
  if (n_tensors < 1 || n_tensors > GS_ADAM_MAX_TENSORS) return GS_ERR_ARG;
  if (!(prm->lr >= 0.0) || std::isinf(prm->lr) || !(prm->beta1 >= 0.0 && prm->beta1 < 1.0) ||
      !(prm->beta2 >= 0.0 && prm->beta2 < 1.0) || !(prm->eps > 0.0) || std::isinf(prm->eps))
    return GS_ERR_ARG;
  if (!aligned(step, 4)) return GS_ERR_ALIGN;
  for (int i = 0; i < n_tensors; ++i) {
    if (sizes[i] < 0 || sizes[i] % 4 != 0) return GS_ERR_ARG;
    if (sizes[i] > 0 && grads[i] && (!params[i] || !m[i] || !v[i])) return GS_ERR_NULL;
    if (!aligned(params[i], 16) || !aligned(grads[i], 16) || !aligned(m[i], 16) || !aligned(v[i], 16))
      return GS_ERR_ALIGN;
  }
  return from_cuda(launch_adam(params, grads, m, v, sizes, n_tensors, *prm, step, (cudaStream_t)stream));
}

gs_status gs_workspace_size(int32_t op, int64_t n, int32_t n_views, int64_t rec_capacity, int64_t pair_capacity,
                            int64_t tile_capacity, size_t* bytes) {
  if (!bytes) return GS_ERR_NULL;
  if (n < 0 || n_views < 1 || rec_capacity < 0 || pair_capacity < 0 || tile_capacity < 0) return GS_ERR_ARG;
  switch (op) {
    case GS_OP_PROJECT: *bytes = project_ws_bytes(n, n_views); return GS_OK;
    case GS_OP_BIN_SORT: *bytes = bin_ws_bytes(rec_capacity, pair_capacity, tile_capacity, n_views); return GS_OK;
    case GS_OP_RENDER_BWD: *bytes = bwd_ws_bytes(rec_capacity); return GS_OK;
    case GS_OP_INFO_GAIN: *bytes = ig_ws_bytes(n, n_views, rec_capacity, pair_capacity, tile_capacity); return GS_OK;
    case GS_OP_IG_COMPOSITE: *bytes = ig_composite_ws_bytes(tile_capacity); return GS_OK;
    case GS_OP_THRESHOLDS: *bytes = thresholds_ws_bytes(); return GS_OK;
    case GS_OP_VIEW_UTILITY: *bytes = utility_ws_bytes(n_views); return GS_OK;
    case GS_OP_REGIONS: *bytes = regions_ws_bytes(rec_capacity); return GS_OK;
    case GS_OP_TRAJECTORY: *bytes = trajectory_ws_bytes(n_views); return GS_OK;
    default: return GS_ERR_ARG;
  }
}

gs_status gs_read_status(const uint32_t* status, uint32_t* flags) {
  if (!status || !flags) return GS_ERR_NULL;
  if (cudaMemcpy(flags, status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return GS_ERR_CUDA;
  return (*flags & GS_FLAG_ERROR_MASK) ? GS_ERR_DEVICE : GS_OK;
}

const char* gs_status_str(gs_status s) {
  switch (s) {
    case GS_OK: return "GS_OK";
    case GS_ERR_NULL: return "GS_ERR_NULL: a required pointer is NULL";
    case GS_ERR_ALIGN: return "GS_ERR_ALIGN: a pointer is not aligned as required";
    case GS_ERR_ARG: return "GS_ERR_ARG: a count, size or parameter is out of range";
    case GS_ERR_WORKSPACE: return "GS_ERR_WORKSPACE: workspace too small";
    case GS_ERR_CUDA: return "GS_ERR_CUDA: a CUDA call or kernel launch failed";
    case GS_ERR_DEVICE: return "GS_ERR_DEVICE: the device status word carries an error flag";
    default: return "unknown gs_status";
  }
}

const char* gs_version(void) { return "0.1.0"; }

uint64_t gs_kernel_launches(void) { return launch_count(); }

}  // extern "C"
