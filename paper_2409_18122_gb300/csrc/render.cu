// render.cu -- front-to-back compositing (gs_render_fwd) and the batched
// information-gain pass (gs_info_gain_batch).
//
// Sec. III of RT-GuIDE: C(p) = sum_i c_i f_i(p) prod_{j<i} (1 - f_j(p)), depth with
// d_i in place of c_i; Sec. IV-A: the per-Gaussian uncertainty u_i composited the
// same way gives the rendered information channel, whose per-view mean scores a
// candidate view (Eq. (nbv) with the Jacobian replaced by the blend weights).
//
// One thread block per screen tile (tile_w x tile_h threads, one pixel each).
// The tile's depth-sorted list is walked in chunks of blockDim entries staged
// in shared memory; each thread leaves the inner loop as soon as its pixel is
// saturated, so a warp stops issuing once all its lanes are done, and the
// block stops loading chunks once every pixel is done (__syncthreads_count).
#include "gs_common.cuh"
#include "gs_internal.h"
#include "render_common.cuh"

namespace gs {
namespace {

constexpr int kFwdWarps = 2;   // warps (work items) per CTA: small CTAs free their slot as soon as both finish
constexpr int kIgWarps = 8;    // warps per CTA of the persistent information-gain kernel
constexpr int kPix = 1;        // pixels per lane of the forward and information-gain kernels

__global__ void __launch_bounds__(kFwdWarps * 32) k_render_fwd(gs_map map, gs_proj proj, gs_bins bins,
                                                                const gs_camera* __restrict__ cams, int n_views,
                                                                gs_params p, gs_image img, uint32_t n_items) {
  __shared__ float4 s_stage[kFwdWarps][3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t item = blockIdx.x * kFwdWarps + warp;
  if (item >= n_items) return;
  const int wpt = warps_per_tile<kPix>(p);
  TileInfo ti;
  if (!warp_tile_setup(proj, bins, cams, n_views, p, item / wpt, ti)) return;
  WarpBlock wb;
  warp_block<kPix>(ti, p, (int)(item % wpt), wb);
  float4* sx = s_stage[warp][0];
  float4* sc = s_stage[warp][1];
  float4* sr = s_stage[warp][2];
  const float pxc = (float)wb.px + 0.5f;
  float pyc[kPix];
  bool inside[kPix], done[kPix];
  float T[kPix], cr[kPix], cg[kPix], cb[kPix], cd[kPix], cu[kPix];
  int32_t last[kPix], n_contrib[kPix];
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    pyc[q] = (float)(wb.py + 4 * q) + 0.5f;
    inside[q] = wb.px < ti.W && wb.py + 4 * q < ti.H;
    done[q] = !inside[q];
    T[q] = 1.f;
    cr[q] = cg[q] = cb[q] = cd[q] = cu[q] = 0.f;
    last[q] = n_contrib[q] = 0;
  }
  const uint32_t beg = ti.beg, n = ti.end - ti.beg;
  const float4* rgb = reinterpret_cast<const float4*>(map.rgb);
  // software pipeline over groups of 32 list entries: while group g is
  // composited, the colours of group g+1, the records of group g+2 and the list
  // indices of group g+3 are in flight
  const uint32_t* rl = bins.rec + beg;
  Entry e1, e2;
  float4 c1 = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t gid2 = 0, r3 = 0;
  if ((uint32_t)lane < n) {
    load_entry(proj, bins, beg + lane, e1);
    c1 = __ldg(rgb + __ldg(proj.gid + e1.rec));
  }
  if (32u + lane < n) {
    load_entry(proj, bins, beg + 32 + lane, e2);
    gid2 = __ldg(proj.gid + e2.rec);
  }
  if (64u + lane < n) r3 = __ldg(rl + 64 + lane);
  for (uint32_t g = 0; g < n; g += 32) {
    if (!__any_sync(0xffffffffu, !all_done<kPix>(done))) break;
    const Entry e = e1;
    const float4 ergb = c1;
    const bool ev = g + lane < n;
    e1 = e2;
    if (g + 32 + lane < n) c1 = __ldg(rgb + gid2);
    if (g + 64 + lane < n) {
      load_record(proj, r3, e2);
      gid2 = __ldg(proj.gid + r3);
    }
    if (g + 96 + lane < n) r3 = __ldg(rl + g + 96 + lane);
    const bool ov = ev && box_overlaps(e.xyod, e.ext, wb);
    uint32_t m = __ballot_sync(0xffffffffu, ov);
    if (m == 0) continue;
    if (ov) {
      sx[lane] = e.xyod;
      sc[lane] = e.con;
      sr[lane] = ergb;
    }
    __syncwarp();
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      if (all_done<kPix>(done)) continue;
      const float4 a = sx[b];
      const float4 k = sc[b];
      const float4 c = sr[b];
#pragma unroll
      for (int q = 0; q < kPix; ++q) {
        if (done[q]) continue;
        const float alpha = splat_alpha(a, k, pxc, pyc[q], p.alpha_max);
        if (alpha < p.alpha_min) continue;
        const float Tn = T[q] * (1.f - alpha);
        if (Tn < p.T_min) { done[q] = true; continue; }
        const float w = alpha * T[q];
        cr[q] += w * c.x;
        cg[q] += w * c.y;
        cb[q] += w * c.z;
        cd[q] += w * a.w;
        cu[q] += w * k.w;
        T[q] = Tn;
        last[q] = (int32_t)(g + b + 1);
        ++n_contrib[q];
      }
    }
    __syncwarp();
  }
  const size_t P = (size_t)ti.W * ti.H;
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    if (!inside[q]) continue;
    const size_t pix = (size_t)(wb.py + 4 * q) * ti.W + wb.px;
    const size_t o = (size_t)ti.pix_base + pix;
    if (img.rgb) {
      float* base = img.rgb + 3 * (size_t)ti.pix_base;
      base[pix] = cr[q];
      base[P + pix] = cg[q];
      base[2 * P + pix] = cb[q];
    }
    if (img.depth) img.depth[o] = cd[q];
    if (img.unc) img.unc[o] = cu[q];
    if (img.T) img.T[o] = T[q];
    if (img.last) img.last[o] = last[q];
    if (img.n_contrib) img.n_contrib[o] = n_contrib[q];
  }
}

// Persistent U-only compositing: every warp takes (tile, 8x4 block) work items
// from a device counter until the batch is exhausted and writes the sum of U
// over its 32 pixels to the item's own slot (fixed shuffle tree), never
// accumulating, so the result does not depend on scheduling.
__global__ void __launch_bounds__(kIgWarps * 32) k_ig_items(gs_proj proj, gs_bins bins,
                                                             const gs_camera* __restrict__ cams, int n_views,
                                                             gs_params p, const uint32_t* __restrict__ order,
                                                             float* __restrict__ item_sum,
                                                             uint32_t* __restrict__ work) {
  __shared__ float4 s_stage[kIgWarps][2][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* sx = s_stage[warp][0];
  float4* sc = s_stage[warp][1];
  const int wpt = warps_per_tile<kPix>(p);
  const uint32_t total = proj.view_info[2 * n_views];
  const uint32_t n_tiles = (int64_t)total < bins.tile_capacity ? total : (uint32_t)bins.tile_capacity;
  const uint32_t n_items = n_tiles * (uint32_t)wpt;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(work, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    // items are handed out longest tile list first; the slot keeps the tile's own index
    const uint32_t tile = __ldg(order + item / wpt);
    const uint32_t slot = tile * (uint32_t)wpt + item % wpt;
    TileInfo ti;
    if (!warp_tile_setup(proj, bins, cams, n_views, p, tile, ti)) {
      if (lane == 0) item_sum[slot] = 0.f;
      continue;
    }
    WarpBlock wb;
    warp_block<kPix>(ti, p, (int)(item % wpt), wb);
    const float pxc = (float)wb.px + 0.5f;
    float pyc[kPix], T[kPix], cu[kPix];
    bool done[kPix];
#pragma unroll
    for (int q = 0; q < kPix; ++q) {
      pyc[q] = (float)(wb.py + 4 * q) + 0.5f;
      done[q] = !(wb.px < ti.W && wb.py + 4 * q < ti.H);
      T[q] = 1.f;
      cu[q] = 0.f;
    }
    const uint32_t beg = ti.beg, n = ti.end - ti.beg;
    // three-stage software pipeline over groups of 32 list entries: while group g
    // is composited, the records of groups g+1 and g+2 are in flight and the list
    // indices of group g+3 are being fetched
    Entry e1, e2;
    uint32_t r3 = 0;
    const uint32_t* rl = bins.rec + beg;
    if ((uint32_t)lane < n) load_entry(proj, bins, beg + lane, e1);
    if (32u + lane < n) load_entry(proj, bins, beg + 32 + lane, e2);
    if (64u + lane < n) r3 = __ldg(rl + 64 + lane);
    for (uint32_t g = 0; g < n; g += 32) {
      if (!__any_sync(0xffffffffu, !all_done<kPix>(done))) break;
      const Entry e = e1;
      const bool ev = g + lane < n;
      e1 = e2;
      if (g + 64 + lane < n) load_record(proj, r3, e2);
      if (g + 96 + lane < n) r3 = __ldg(rl + g + 96 + lane);
      const bool ov = ev && box_overlaps(e.xyod, e.ext, wb);
      uint32_t m = __ballot_sync(0xffffffffu, ov);
      if (m == 0) continue;
      if (ov) {
        sx[lane] = e.xyod;
        sc[lane] = e.con;
      }
      __syncwarp();
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        if (all_done<kPix>(done)) continue;
        const float4 a = sx[b];
        const float4 k = sc[b];
#pragma unroll
        for (int q = 0; q < kPix; ++q) {
          if (done[q]) continue;
          const float alpha = splat_alpha(a, k, pxc, pyc[q], p.alpha_max);
          if (alpha < p.alpha_min) continue;
          const float Tn = T[q] * (1.f - alpha);
          if (Tn < p.T_min) { done[q] = true; continue; }
          cu[q] += alpha * T[q] * k.w;
          T[q] = Tn;
        }
      }
      __syncwarp();
    }
    float su = 0.f;
#pragma unroll
    for (int q = 0; q < kPix; ++q) su += cu[q];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) su += __shfl_down_sync(0xffffffffu, su, d);
    if (lane == 0) item_sum[slot] = su;
  }
}

// IG_v = (1 / P_v) * sum over the items of the view's tiles, in a fixed order.
__global__ void __launch_bounds__(256) k_ig_views(const uint32_t* __restrict__ view_info,
                                                   const gs_camera* __restrict__ cams, int n_views, gs_params p,
                                                   const float* __restrict__ item_sum, int64_t tile_cap,
                                                   float* __restrict__ ig) {
  __shared__ float s_red[32];
  const int v = blockIdx.x;
  const uint32_t wpt = (uint32_t)warps_per_tile<kPix>(p);
  uint32_t t1 = view_info[2 * v + 2];
  if ((int64_t)t1 > tile_cap) t1 = (uint32_t)tile_cap;
  const uint32_t i0 = view_info[2 * v] * wpt, i1 = t1 * wpt;
  const int W = cams[v].width, H = cams[v].height;
  float s = 0.f;
  // fixed assignment of items to threads and a fixed reduction tree: deterministic
  for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += item_sum[i];
  s = block_sum_fixed(s, s_red);
  if (threadIdx.x == 0) ig[v] = (W > 0 && H > 0) ? s / ((float)W * (float)H) : 0.f;
}

__global__ void k_zero_words(uint32_t* p, int n) {
  if (threadIdx.x < n) p[threadIdx.x] = 0u;
}

// Sort key of each tile for longest-first scheduling: 0xFFFF - min(list length, 0xFFFF).
__global__ void k_tile_cost(const uint32_t* __restrict__ ranges, const uint32_t* __restrict__ view_info, int n_views,
                            int64_t tile_cap, uint32_t* __restrict__ key) {
  uint32_t n = view_info[2 * n_views];
  if ((int64_t)n > tile_cap) n = (uint32_t)tile_cap;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const uint32_t len = ranges[2 * (size_t)t + 1] - ranges[2 * (size_t)t];
    key[t] = 0xFFFFu - (len < 0xFFFFu ? len : 0xFFFFu);
  }
}

}  // namespace

cudaError_t launch_render_fwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                              int n_views, const gs_params& p, const gs_image& img, cudaStream_t st) {
  const int64_t items = bins.tile_capacity * (int64_t)((p.tile_w * p.tile_h) / (32 * kPix));
  if (items > 0) {
    k_render_fwd<<<(unsigned)((items + kFwdWarps - 1) / kFwdWarps), kFwdWarps * 32, 0, st>>>(
        map, proj, bins, cams, n_views, p, img, (uint32_t)items);
    note_launch();
  }
  return cudaGetLastError();
}

size_t ig_ws_bytes(int64_t n, int n_views, int64_t pair_cap, int64_t tile_cap) {
  const int64_t rec_cap = n * (int64_t)n_views;
  Carver c(nullptr);
  c.take<uint32_t>(1);                                   // record count
  c.take<uint32_t>(2 * (size_t)(n_views + 1));           // view info
  c.take<uint32_t>(rec_cap);                             // gid
  c.take<uint32_t>(rec_cap);                             // view
  c.take<float4>(rec_cap);                               // xyod
  c.take<float4>(rec_cap);                               // conic_u
  c.take<ushort4>(rec_cap);                              // rect
  c.take<uint32_t>(rec_cap);                             // depth key
  c.take<float2>(rec_cap);                               // ext
  const int64_t slots = ((n + 31) / 32) * (int64_t)n_views;
  c.take<uint32_t>(slots);                               // grp_mask
  c.take<uint32_t>(slots + 1);                           // grp_base
  c.take<uint32_t>(1);                                   // pair count
  c.take<uint32_t>(pair_cap);                            // tile
  c.take<uint32_t>(pair_cap);                            // rec
  c.take<uint32_t>(2 * tile_cap);                        // ranges
  c.take<float>(32 * tile_cap);                          // per work-item sums (<= 32 items per tile)
  c.take<uint32_t>(4);                                   // work counter
  size_t a = project_ws_bytes(n, n_views), b = bin_ws_bytes(rec_cap, pair_cap, tile_cap);
  const size_t o = 4 * align_up(sizeof(uint32_t) * (size_t)tile_cap, 256) + sort_temp_bytes(tile_cap);
  c.take<char>(a > b ? (a > o ? a : o) : (b > o ? b : o));
  return align_up(c.off, 256);
}

cudaError_t launch_info_gain(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                             float* ig_out, uint32_t* status, int64_t pair_cap, int64_t tile_cap, void* ws,
                             cudaStream_t st) {
  const int64_t rec_cap = map.n * (int64_t)n_views;
  Carver c(ws);
  gs_proj proj;
  proj.capacity = rec_cap;
  proj.count = c.take<uint32_t>(1);
  proj.status = status;
  proj.view_info = c.take<uint32_t>(2 * (size_t)(n_views + 1));
  proj.gid = c.take<uint32_t>(rec_cap);
  proj.view = c.take<uint32_t>(rec_cap);
  proj.xyod = (float*)c.take<float4>(rec_cap);
  proj.conic_u = (float*)c.take<float4>(rec_cap);
  proj.rect = (uint16_t*)c.take<ushort4>(rec_cap);
  proj.depth_key = c.take<uint32_t>(rec_cap);
  proj.ext = (float*)c.take<float2>(rec_cap);
  const int64_t slots = ((map.n + 31) / 32) * (int64_t)n_views;
  proj.grp_mask = c.take<uint32_t>(slots);
  proj.grp_base = c.take<uint32_t>(slots + 1);
  gs_bins bins;
  bins.pair_capacity = pair_cap;
  bins.tile_capacity = tile_cap;
  bins.count = c.take<uint32_t>(1);
  bins.tile = c.take<uint32_t>(pair_cap);
  bins.rec = c.take<uint32_t>(pair_cap);
  bins.ranges = c.take<uint32_t>(2 * tile_cap);
  float* item_sum = c.take<float>(32 * tile_cap);
  uint32_t* work = c.take<uint32_t>(4);
  size_t a = project_ws_bytes(map.n, n_views), b = bin_ws_bytes(rec_cap, pair_cap, tile_cap);
  const size_t o = 4 * align_up(sizeof(uint32_t) * (size_t)tile_cap, 256) + sort_temp_bytes(tile_cap);
  void* inner = c.take<char>(a > b ? (a > o ? a : o) : (b > o ? b : o));

  cudaError_t e = launch_project(map, cams, n_views, p, proj, inner, st);
  if (e != cudaSuccess) return e;
  e = launch_bin_sort(proj, cams, n_views, p, bins, inner, st);
  if (e != cudaSuccess) return e;
  k_zero_words<<<1, 32, 0, st>>>(work, 4);
  note_launch();
  // longest tile lists first (the inner workspace is free again once binning is done)
  Carver oc(inner);
  uint32_t* ok_a = oc.take<uint32_t>(tile_cap);
  uint32_t* ov_a = oc.take<uint32_t>(tile_cap);
  uint32_t* ok_b = oc.take<uint32_t>(tile_cap);
  uint32_t* ov_b = oc.take<uint32_t>(tile_cap);
  void* otmp = oc.take<char>(sort_temp_bytes(tile_cap));
  {
    int64_t gb = (tile_cap + 255) / 256;
    if (gb > 4096) gb = 4096;
    k_tile_cost<<<(unsigned)gb, 256, 0, st>>>(bins.ranges, proj.view_info, n_views, tile_cap, ok_a);
    note_launch();
  }
  bool in_a = false;
  e = radix_sort(ok_a, nullptr, nullptr, SortBufs{ok_a, ov_a, ok_b, ov_b}, proj.view_info + 2 * n_views, tile_cap, 0,
                 16, otmp, st, &in_a);
  if (e != cudaSuccess) return e;
  const uint32_t* order = in_a ? ov_a : ov_b;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ig_items, kIgWarps * 32, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t items = tile_cap * (int64_t)((p.tile_w * p.tile_h) / (32 * kPix));
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  if (grid * kIgWarps > items) grid = (items + kIgWarps - 1) / kIgWarps;
  if (grid < 1) grid = 1;
  k_ig_items<<<(unsigned)grid, kIgWarps * 32, 0, st>>>(proj, bins, cams, n_views, p, order, item_sum, work);
  note_launch();
  k_ig_views<<<n_views, 256, 0, st>>>(proj.view_info, cams, n_views, p, item_sum, tile_cap, ig_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
