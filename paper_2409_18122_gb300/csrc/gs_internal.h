// gs_internal.h -- host-side launchers shared between the translation units of
// libgs103.so.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gs.h"

namespace gs {

// NVTX range over one C-ABI call (host side: argument checks and the enqueue of its
// kernels), named after the entry point, so that a profiler's timeline shows which call
// launched which kernels.  With no tool attached a push or pop is one indirect call.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define GS_TRACE(name) ::gs::TraceRange gs_trace_range_(name)

// ------------------------------------------------------------------ helpers
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves consecutive 256-byte aligned sub-buffers out of a workspace.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int device_sm_count();

// Host-side count of kernel launches enqueued by this library (work accounting).
void note_launch();
uint64_t launch_count();

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of n uint32 values into out[0..n]; out[n] = total.
// n = min(*n_dev, n_cap) when n_dev != NULL, else n_cap.  Prefixes saturate at
// 0xFFFFFFFF.  If total_out != NULL, the (saturated) total is also stored there.
size_t scan_temp_bytes(int64_t n_cap);
cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, int64_t n_cap,
                           uint32_t* total_out, void* temp, cudaStream_t st);

// ------------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, value) uint32 pairs on bits [bit_begin, bit_end).
// Input: keys_in, vals_in (nullable: identity 0..n-1).  Buffers a/b are
// ping-pong storage of n_cap entries each; the sorted result ends in a if the
// number of 8-bit passes is even, else in b.  *result_in_a tells which.
// n = min(*n_dev, n_cap).  With seg != NULL and n_seg > 1 (segmented mode) the
// elements [seg[s], seg[s+1]) of every segment s < n_seg (seg non-decreasing,
// seg[n_seg] = n) are sorted among themselves and stay in place.
// sort_temp_bytes(n_cap, n_seg): scratch for either mode (n_seg 0 for plain).
struct SortBufs {
  uint32_t* keys_a;
  uint32_t* vals_a;
  uint32_t* keys_b;
  uint32_t* vals_b;
};
size_t sort_temp_bytes(int64_t n_cap, int n_seg = 0);
// Optional work of the last pass of a sort whose segments are the views of a
// binning batch and whose values are record indices: for the element r written
// to position i, out_rect[i] = rect[r] and out_cnt[i] = its number of tiles (0,
// with an empty out_rect[i], for an empty rectangle or one outside its view's
// tile grid -- the latter also sets GS_FLAG_BAD_RECORDS).  The sorted keys are
// then not written.
struct SortRectEpilogue {
  const ushort4* rect;
  const uint32_t* view_info;
  ushort4* out_rect;
  uint32_t* out_cnt;
  uint32_t* status;
};
int sort_passes(int bit_begin, int bit_end);
cudaError_t radix_sort(const uint32_t* keys_in, const uint32_t* vals_in, SortBufs bufs, const uint32_t* n_dev,
                       int64_t n_cap, int bit_begin, int bit_end, void* temp, cudaStream_t st, bool* result_in_a,
                       const uint32_t* seg = nullptr, int n_seg = 0, const SortRectEpilogue* epi = nullptr);

// ------------------------------------------------------------------ pipeline stages
size_t project_ws_bytes(int64_t n, int n_views);
cudaError_t launch_project(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                           const gs_proj& out, void* ws, cudaStream_t st);

size_t bin_ws_bytes(int64_t rec_cap, int64_t pair_cap, int64_t tile_cap, int n_views);
// proj.view == NULL: records written by launch_project without view ids; the view segments
// come from proj.grp_base and the group count in view_info[V][3].
cudaError_t launch_bin_sort(const gs_proj& proj, const gs_camera* cams, int n_views, const gs_params& p,
                            const gs_bins& out, void* ws, cudaStream_t st);

cudaError_t launch_render_fwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                              int n_views, const gs_params& p, const gs_image& img, cudaStream_t st);

// the one-launch forward render of a small map (small.cu)
cudaError_t launch_render_small(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                                const gs_image& img, uint32_t* status, cudaStream_t st);

size_t bwd_ws_bytes(int64_t rec_cap);
// Every argument check of gs_render_bwd except the workspace's (api.cu); GS_OK if the
// arguments are valid.  Shared by the workspace and the allocation-free entry points.
gs_status validate_render_bwd(const gs_map* map, const gs_proj* proj, const gs_bins* bins, const gs_image* fwd,
                              const gs_image_grad* grad, const gs_camera* cams, int32_t n_views, const gs_params* prm,
                              const gs_map_grad* out);
cudaError_t launch_render_bwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_image& fwd,
                              const gs_image_grad& g, const gs_camera* cams, int n_views, const gs_params& p,
                              const gs_map_grad& out, void* ws, cudaStream_t st);

size_t ig_composite_ws_bytes(int64_t tile_cap);
cudaError_t launch_ig_composite(const gs_proj& proj, const gs_bins& bins, const gs_camera* cams, int n_views,
                                const gs_params& p, float* ig_out, void* ws, cudaStream_t st);

// rec_cap: record capacity of the batch (n * n_views when 0).
size_t ig_ws_bytes(int64_t n, int n_views, int64_t rec_cap, int64_t pair_cap, int64_t tile_cap);
cudaError_t launch_info_gain(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                             float* ig_out, uint32_t* status, int64_t rec_cap, int64_t pair_cap, int64_t tile_cap,
                             void* ws, cudaStream_t st);

// render-free view utility (utility.cu)
cudaError_t launch_uncertainty_update(const float* mo_prev, const float* mo_cur, float* su, int64_t n, int squared,
                                      cudaStream_t st);
size_t thresholds_ws_bytes();
cudaError_t launch_uncertainty_thresholds(const float* mo, const float* su, int64_t n, float ground_z, double* stats,
                                          void* ws, cudaStream_t st);
size_t utility_ws_bytes(int n_views);
cudaError_t launch_view_utility(const float* mo, const float* su, int64_t n, const gs_camera* cams, int n_views,
                                const gs_utility_params& prm, int mode, const double* stats, float* xi,
                                uint32_t* counts, void* ws, cudaStream_t st);
size_t trajectory_ws_bytes(int n_states_total);
cudaError_t launch_trajectory_utility(const float* mo, const float* su, int64_t n, const gs_camera* cams, int n_traj,
                                      int n_states, const gs_utility_params& prm, int mode, const double* stats,
                                      float* traj_out, int32_t* best_out, void* ws, cudaStream_t st);
cudaError_t launch_collision_check(const float* mo, const float* su, int64_t n, const float* pts, int n_pts,
                                   float r_robot, float lambda_g, float ground_z, float* margin_out,
                                   uint32_t* collides_out, cudaStream_t st);
size_t regions_ws_bytes(int64_t n_regions);

// ------------------------------------------------------------------ Adam step
cudaError_t launch_adam(float* const* params, const float* const* grads, float* const* m, float* const* v,
                        const int64_t* sizes, int n_tensors, const gs_adam_params& prm, uint32_t* step,
                        cudaStream_t st);

// ------------------------------------------------------------------ mapping loss (Eq. 3)
// 0 if the sizes are invalid.
size_t image_loss_ws_bytes(const int32_t* sizes, int n_views);
cudaError_t launch_image_loss(const int32_t* sizes, int n_views, const float* rgb, const float* depth,
                              const float* rgb_ref, const float* depth_ref, const gs_loss_weights& w,
                              float* loss_out, float* d_rgb, float* d_depth, void* ws, cudaStream_t st);
cudaError_t launch_regions(const float* mo, const float* su, int64_t n, const gs_region_grid& grid, float* omega,
                           uint32_t* count_out, void* ws, cudaStream_t st);

}  // namespace gs
