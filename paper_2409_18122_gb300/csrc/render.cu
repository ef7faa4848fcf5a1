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

__global__ void __launch_bounds__(kFwdWarps * 32) k_render_fwd(gs_map map, gs_proj proj, gs_bins bins,
                                                                const gs_camera* __restrict__ cams, int n_views,
                                                                gs_params p, gs_image img, uint32_t n_items) {
  __shared__ float4 s_stage[kFwdWarps][3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t item = blockIdx.x * kFwdWarps + warp;
  if (item >= n_items) return;
  const int wpt = warps_per_tile(p);
  TileInfo ti;
  if (!warp_tile_setup(proj, bins, cams, n_views, p, item / wpt, ti)) return;
  WarpBlock wb;
  warp_block(ti, p, (int)(item % wpt), wb);
  float4* sx = s_stage[warp][0];
  float4* sc = s_stage[warp][1];
  float4* sr = s_stage[warp][2];
  const bool inside = wb.px < ti.W && wb.py < ti.H;
  const float pxc = (float)wb.px + 0.5f, pyc = (float)wb.py + 0.5f;
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, cd = 0.f, cu = 0.f;
  int32_t last = 0, n_contrib = 0;
  bool done = !inside;
  const uint32_t beg = ti.beg, n = ti.end - ti.beg;
  const float4* rgb = reinterpret_cast<const float4*>(map.rgb);
  // software pipeline: the next group of 32 entries is loaded while this one is composited
  Entry nx;
  float4 nrgb = make_float4(0.f, 0.f, 0.f, 0.f);
  bool nv = (uint32_t)lane < n;
  if (nv) {
    load_entry(proj, bins, beg + lane, nx);
    nrgb = __ldg(rgb + __ldg(proj.gid + nx.rec));
  }
  for (uint32_t g = 0; g < n; g += 32) {
    if (!__any_sync(0xffffffffu, !done)) break;
    const Entry e = nx;
    const float4 ergb = nrgb;
    const bool ev = nv;
    nv = g + 32 + lane < n;
    if (nv) {
      load_entry(proj, bins, beg + g + 32 + lane, nx);
      nrgb = __ldg(rgb + __ldg(proj.gid + nx.rec));
    }
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
      if (done) continue;
      const float4 a = sx[b];
      const float4 k = sc[b];
      const float alpha = splat_alpha(a, k, pxc, pyc, p.alpha_max);
      if (alpha < p.alpha_min) continue;
      const float Tn = T * (1.f - alpha);
      if (Tn < p.T_min) { done = true; continue; }
      const float w = alpha * T;
      const float4 c = sr[b];
      cr += w * c.x;
      cg += w * c.y;
      cb += w * c.z;
      cd += w * a.w;
      cu += w * k.w;
      T = Tn;
      last = (int32_t)(g + b + 1);
      ++n_contrib;
    }
    __syncwarp();
  }
  if (!inside) return;
  const size_t P = (size_t)ti.W * ti.H;
  const size_t pix = (size_t)wb.py * ti.W + wb.px;
  const size_t o = (size_t)ti.pix_base + pix;
  if (img.rgb) {
    float* base = img.rgb + 3 * (size_t)ti.pix_base;
    base[pix] = cr;
    base[P + pix] = cg;
    base[2 * P + pix] = cb;
  }
  if (img.depth) img.depth[o] = cd;
  if (img.unc) img.unc[o] = cu;
  if (img.T) img.T[o] = T;
  if (img.last) img.last[o] = last;
  if (img.n_contrib) img.n_contrib[o] = n_contrib;
}

// Persistent U-only compositing: every warp takes (tile, 8x4 block) work items
// from a device counter until the batch is exhausted and writes the sum of U
// over its 32 pixels to the item's own slot (fixed shuffle tree), never
// accumulating, so the result does not depend on scheduling.
__global__ void __launch_bounds__(kIgWarps * 32) k_ig_items(gs_proj proj, gs_bins bins,
                                                             const gs_camera* __restrict__ cams, int n_views,
                                                             gs_params p, float* __restrict__ item_sum,
                                                             uint32_t* __restrict__ work) {
  __shared__ float4 s_stage[kIgWarps][2][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* sx = s_stage[warp][0];
  float4* sc = s_stage[warp][1];
  const int wpt = warps_per_tile(p);
  const uint32_t total = proj.view_info[2 * n_views];
  const uint32_t n_tiles = (int64_t)total < bins.tile_capacity ? total : (uint32_t)bins.tile_capacity;
  const uint32_t n_items = n_tiles * (uint32_t)wpt;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(work, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    TileInfo ti;
    if (!warp_tile_setup(proj, bins, cams, n_views, p, item / wpt, ti)) {
      if (lane == 0) item_sum[item] = 0.f;
      continue;
    }
    WarpBlock wb;
    warp_block(ti, p, (int)(item % wpt), wb);
    const bool inside = wb.px < ti.W && wb.py < ti.H;
    const float pxc = (float)wb.px + 0.5f, pyc = (float)wb.py + 0.5f;
    float T = 1.f, cu = 0.f;
    bool done = !inside;
    const uint32_t beg = ti.beg, n = ti.end - ti.beg;
    Entry nx;
    bool nv = (uint32_t)lane < n;
    if (nv) load_entry(proj, bins, beg + lane, nx);
    for (uint32_t g = 0; g < n; g += 32) {
      if (!__any_sync(0xffffffffu, !done)) break;
      const Entry e = nx;
      const bool ev = nv;
      nv = g + 32 + lane < n;
      if (nv) load_entry(proj, bins, beg + g + 32 + lane, nx);
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
        if (done) continue;
        const float4 a = sx[b];
        const float4 k = sc[b];
        const float alpha = splat_alpha(a, k, pxc, pyc, p.alpha_max);
        if (alpha < p.alpha_min) continue;
        const float Tn = T * (1.f - alpha);
        if (Tn < p.T_min) { done = true; continue; }
        cu += alpha * T * k.w;
        T = Tn;
      }
      __syncwarp();
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cu += __shfl_down_sync(0xffffffffu, cu, d);
    if (lane == 0) item_sum[item] = cu;
  }
}

// IG_v = (1 / P_v) * sum over the items of the view's tiles, in a fixed order.
__global__ void __launch_bounds__(256) k_ig_views(const uint32_t* __restrict__ view_info,
                                                   const gs_camera* __restrict__ cams, int n_views, gs_params p,
                                                   const float* __restrict__ item_sum, int64_t tile_cap,
                                                   float* __restrict__ ig) {
  __shared__ float s_red[32];
  const int v = blockIdx.x;
  const uint32_t wpt = (uint32_t)warps_per_tile(p);
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

}  // namespace

cudaError_t launch_render_fwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                              int n_views, const gs_params& p, const gs_image& img, cudaStream_t st) {
  const int64_t items = bins.tile_capacity * (int64_t)((p.tile_w * p.tile_h) >> 5);
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
  c.take<char>(a > b ? a : b);
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
  void* inner = c.take<char>(a > b ? a : b);

  cudaError_t e = launch_project(map, cams, n_views, p, proj, inner, st);
  if (e != cudaSuccess) return e;
  e = launch_bin_sort(proj, cams, n_views, p, bins, inner, st);
  if (e != cudaSuccess) return e;
  k_zero_words<<<1, 32, 0, st>>>(work, 4);
  note_launch();
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ig_items, kIgWarps * 32, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t items = tile_cap * (int64_t)((p.tile_w * p.tile_h) >> 5);
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  if (grid * kIgWarps > items) grid = (items + kIgWarps - 1) / kIgWarps;
  if (grid < 1) grid = 1;
  k_ig_items<<<(unsigned)grid, kIgWarps * 32, 0, st>>>(proj, bins, cams, n_views, p, item_sum, work);
  note_launch();
  k_ig_views<<<n_views, 256, 0, st>>>(proj.view_info, cams, n_views, p, item_sum, tile_cap, ig_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
