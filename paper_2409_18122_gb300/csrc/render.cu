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

__global__ void __launch_bounds__(1024) k_render_fwd(gs_map map, gs_proj proj, gs_bins bins,
                                                      const gs_camera* __restrict__ cams, int n_views, gs_params p,
                                                      gs_image img) {
  extern __shared__ float4 s_buf[];
  const int B = blockDim.x;
  float4* s_xyod = s_buf;
  float4* s_con = s_buf + B;
  float4* s_rgb = s_buf + 2 * B;
  __shared__ TileInfo ti;
  const uint32_t tile = blockIdx.x;
  if (!tile_setup(proj, bins, cams, n_views, p, tile, ti)) return;
  const int tid = threadIdx.x;
  const int px = ti.x0 + tid % p.tile_w, py = ti.y0 + tid / p.tile_w;
  const bool inside = px < ti.W && py < ti.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, cd = 0.f, cu = 0.f;
  int32_t last = 0, n_contrib = 0;
  bool done = !inside;
  const uint32_t beg = ti.beg, end = ti.end;
  for (uint32_t c0 = beg; c0 < end; c0 += B) {
    if (__syncthreads_count(done) == B) break;
    const uint32_t idx = c0 + tid;
    if (idx < end) {
      const uint32_t r = bins.rec[idx];
      s_xyod[tid] = __ldg(reinterpret_cast<const float4*>(proj.xyod) + r);
      s_con[tid] = __ldg(reinterpret_cast<const float4*>(proj.conic_u) + r);
      s_rgb[tid] = __ldg(reinterpret_cast<const float4*>(map.rgb) + proj.gid[r]);
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)B, end - c0);
    for (int j = 0; !done && j < cnt; ++j) {
      const float4 a = s_xyod[j];
      const float4 k = s_con[j];
      const float alpha = splat_alpha(a, k, pxc, pyc, p.alpha_max);
      if (alpha < p.alpha_min) continue;
      const float Tn = T * (1.f - alpha);
      if (Tn < p.T_min) { done = true; break; }
      const float w = alpha * T;
      const float4 c = s_rgb[j];
      cr += w * c.x;
      cg += w * c.y;
      cb += w * c.z;
      cd += w * a.w;
      cu += w * k.w;
      T = Tn;
      last = (int32_t)(c0 - beg) + j + 1;
      ++n_contrib;
    }
  }
  if (!inside) return;
  const size_t P = (size_t)ti.W * ti.H;
  const size_t pix = (size_t)py * ti.W + px;
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

// Persistent U-only compositing: blocks take (view, tile) work items from a
// device counter until the batch is exhausted; each tile's sum of U is written
// to its own slot (fixed-order block reduction), never accumulated.
__global__ void __launch_bounds__(1024) k_ig_tiles(gs_proj proj, gs_bins bins, const gs_camera* __restrict__ cams,
                                                    int n_views, gs_params p, float* __restrict__ tile_sum,
                                                    uint32_t* __restrict__ work) {
  extern __shared__ float4 s_buf[];
  const int B = blockDim.x;
  float4* s_xyod = s_buf;
  float4* s_con = s_buf + B;
  __shared__ TileInfo ti;
  __shared__ uint32_t s_tile;
  __shared__ float s_red[32];
  const int tid = threadIdx.x;
  const uint32_t total = proj.view_info[2 * n_views];
  const uint32_t n_tiles = (int64_t)total < bins.tile_capacity ? total : (uint32_t)bins.tile_capacity;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_tile = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    if (!tile_setup(proj, bins, cams, n_views, p, tile, ti)) continue;
    const int px = ti.x0 + tid % p.tile_w, py = ti.y0 + tid / p.tile_w;
    const bool inside = px < ti.W && py < ti.H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    float T = 1.f, cu = 0.f;
    bool done = !inside;
    const uint32_t beg = ti.beg, end = ti.end;
    for (uint32_t c0 = beg; c0 < end; c0 += B) {
      if (__syncthreads_count(done) == B) break;
      const uint32_t idx = c0 + tid;
      if (idx < end) {
        const uint32_t r = bins.rec[idx];
        s_xyod[tid] = __ldg(reinterpret_cast<const float4*>(proj.xyod) + r);
        s_con[tid] = __ldg(reinterpret_cast<const float4*>(proj.conic_u) + r);
      }
      __syncthreads();
      const int cnt = (int)min((uint32_t)B, end - c0);
      for (int j = 0; !done && j < cnt; ++j) {
        const float4 a = s_xyod[j];
        const float4 k = s_con[j];
        const float alpha = splat_alpha(a, k, pxc, pyc, p.alpha_max);
        if (alpha < p.alpha_min) continue;
        const float Tn = T * (1.f - alpha);
        if (Tn < p.T_min) { done = true; break; }
        cu += alpha * T * k.w;
        T = Tn;
      }
    }
    const float s = block_sum_fixed(cu, s_red);
    if (tid == 0) tile_sum[tile] = s;
  }
}

// IG_v = (1 / P_v) * sum over the view's tiles of tile_sum, in tile order.
__global__ void __launch_bounds__(256) k_ig_views(const uint32_t* __restrict__ view_info,
                                                   const gs_camera* __restrict__ cams, int n_views,
                                                   const float* __restrict__ tile_sum, int64_t tile_cap,
                                                   float* __restrict__ ig) {
  __shared__ float s_red[32];
  const int v = blockIdx.x;
  const uint32_t t0 = view_info[2 * v], t1 = view_info[2 * v + 2];
  const int W = cams[v].width, H = cams[v].height;
  float s = 0.f;
  // fixed assignment of tiles to threads and a fixed reduction tree: deterministic
  for (uint32_t t = t0 + threadIdx.x; t < t1 && (int64_t)t < tile_cap; t += blockDim.x) s += tile_sum[t];
  s = block_sum_fixed(s, s_red);
  if (threadIdx.x == 0) ig[v] = (W > 0 && H > 0) ? s / ((float)W * (float)H) : 0.f;
}

__global__ void k_zero_words(uint32_t* p, int n) {
  if (threadIdx.x < n) p[threadIdx.x] = 0u;
}

}  // namespace

cudaError_t launch_render_fwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                              int n_views, const gs_params& p, const gs_image& img, cudaStream_t st) {
  const int B = p.tile_w * p.tile_h;
  const size_t smem = 3 * sizeof(float4) * B;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_render_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  if (bins.tile_capacity > 0)
    k_render_fwd<<<(unsigned)bins.tile_capacity, B, smem, st>>>(map, proj, bins, cams, n_views, p, img);
    note_launch();
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
  c.take<uint32_t>(n + 1);                               // g_first
  c.take<uint32_t>(1);                                   // pair count
  c.take<uint32_t>(pair_cap);                            // tile
  c.take<uint32_t>(pair_cap);                            // rec
  c.take<uint32_t>(2 * tile_cap);                        // ranges
  c.take<float>(tile_cap);                               // tile sums
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
  proj.g_first = c.take<uint32_t>(map.n + 1);
  gs_bins bins;
  bins.pair_capacity = pair_cap;
  bins.tile_capacity = tile_cap;
  bins.count = c.take<uint32_t>(1);
  bins.tile = c.take<uint32_t>(pair_cap);
  bins.rec = c.take<uint32_t>(pair_cap);
  bins.ranges = c.take<uint32_t>(2 * tile_cap);
  float* tile_sum = c.take<float>(tile_cap);
  uint32_t* work = c.take<uint32_t>(4);
  size_t a = project_ws_bytes(map.n, n_views), b = bin_ws_bytes(rec_cap, pair_cap, tile_cap);
  void* inner = c.take<char>(a > b ? a : b);

  cudaError_t e = launch_project(map, cams, n_views, p, proj, inner, st);
  if (e != cudaSuccess) return e;
  e = launch_bin_sort(proj, cams, n_views, p, bins, inner, st);
  if (e != cudaSuccess) return e;
  k_zero_words<<<1, 32, 0, st>>>(work, 4);
  note_launch();
  const int B = p.tile_w * p.tile_h;
  const size_t smem = 2 * sizeof(float4) * B;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ig_tiles, B, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  if (grid > tile_cap) grid = tile_cap;
  if (grid < 1) grid = 1;
  k_ig_tiles<<<(unsigned)grid, B, smem, st>>>(proj, bins, cams, n_views, p, tile_sum, work);
  note_launch();
  k_ig_views<<<n_views, 256, 0, st>>>(proj.view_info, cams, n_views, tile_sum, tile_cap, ig_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
