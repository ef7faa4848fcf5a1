// render_common.cuh -- per-tile setup and the per-(pixel, Gaussian) opacity
// shared by the forward, backward and information-gain compositing kernels, so
// that all of them take identical skip / stop decisions.
#pragma once

#include "gs_common.cuh"

namespace gs {

struct TileInfo {
  bool valid;
  int view;
  int W, H;
  int x0, y0;          // pixel origin of the tile
  uint32_t pix_base;   // first pixel of the view in the concatenated images
  uint32_t beg, end;   // range in the sorted pair list
};

// Called by every thread of the block; returns whether the tile exists.
__device__ __forceinline__ bool tile_setup(const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                                           int n_views, const gs_params& p, uint32_t tile, TileInfo& ti) {
  if (threadIdx.x == 0) {
    const uint32_t total = proj.view_info[2 * n_views];
    ti.valid = tile < total && (int64_t)tile < bins.tile_capacity;
    if (ti.valid) {
      const int v = find_view(proj.view_info, n_views, tile);
      const uint32_t local = tile - proj.view_info[2 * v];
      const int W = cams[v].width, H = cams[v].height;
      const uint32_t tx = (uint32_t)((W + p.tile_w - 1) / p.tile_w);
      ti.view = v;
      ti.W = W;
      ti.H = H;
      ti.x0 = (int)(local % tx) * p.tile_w;
      ti.y0 = (int)(local / tx) * p.tile_h;
      ti.pix_base = proj.view_info[2 * v + 1];
      uint32_t n_pairs = *bins.count;
      if ((int64_t)n_pairs > bins.pair_capacity) n_pairs = (uint32_t)bins.pair_capacity;
      uint32_t b = bins.ranges[2 * (size_t)tile], e = bins.ranges[2 * (size_t)tile + 1];
      if (e > n_pairs) e = n_pairs;
      if (b > e) b = e;
      ti.beg = b;
      ti.end = e;
    }
  }
  __syncthreads();
  return ti.valid;
}

// alpha = min(alpha_max, o exp(-q/2)), q = a dx^2 + 2 b dx dy + c dy^2 with
// (dx, dy) = mu_2D - pixel centre.  xyod = (mu_x, mu_y, o, depth), con = (a, b, c, u).
// Written with explicit round-to-nearest intrinsics so that the forward,
// backward and information-gain kernels compute bit-identical alphas (and so
// take identical skip and stop decisions) whatever the compiler contracts.
// Also returns (dx, dy) and G = exp(-q/2).
__device__ __forceinline__ float splat_alpha_dxy(const float4& xyod, const float4& con, float pxc, float pyc,
                                                 float alpha_max, float& dx, float& dy, float& G) {
  dx = __fsub_rn(xyod.x, pxc);
  dy = __fsub_rn(xyod.y, pyc);
  float q = __fmul_rn(__fmul_rn(con.z, dy), dy);
  q = __fmaf_rn(__fmul_rn(con.x, dx), dx, q);
  q = __fmaf_rn(__fmul_rn(__fadd_rn(con.y, con.y), dx), dy, q);
  G = __expf(__fmul_rn(-0.5f, q));
  return fminf(alpha_max, __fmul_rn(xyod.z, G));
}

__device__ __forceinline__ float splat_alpha(const float4& xyod, const float4& con, float pxc, float pyc,
                                             float alpha_max) {
  float dx, dy, G;
  return splat_alpha_dxy(xyod, con, pxc, pyc, alpha_max, dx, dy, G);
}

// Work item of the compositing kernels: one warp renders one 8 x (4 KP) pixel
// block of one screen tile, KP pixels per lane (KP = 1 for the forward and
// information-gain kernels, 2 for the backward kernel, whose per-entry warp
// reduction is then shared by 64 pixels).  Block b of a tile covers columns
// 8 (b mod (tile_w/8)) .. +7 and rows 4 KP (b div (tile_w/8)) .. +4 KP - 1;
// lane l owns pixels (l mod 8, l div 8 + 4 q), q < KP.  Warps never wait for
// each other: each walks its tile's list on its own and stops as soon as all of
// its pixels are saturated.
struct WarpBlock {
  int px, py;                   // this lane's first pixel; the others are (px, py + 4 q)
  float bx0, bx1, by0, by1;     // pixel-centre bounds of the warp's block
};

template <int KP>
__device__ __forceinline__ int warps_per_tile(const gs_params& p) { return (p.tile_w * p.tile_h) / (32 * KP); }

// Tile of `tile`, computed by lane 0 and broadcast; returns false (warp-uniform) if the tile does not exist.
__device__ __forceinline__ bool warp_tile_setup(const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                                                int n_views, const gs_params& p, uint32_t tile, TileInfo& ti) {
  const int lane = threadIdx.x & 31;
  int f[7] = {0, 0, 0, 0, 0, 0, 0};
  if (lane == 0) {
    const uint32_t total = proj.view_info[2 * n_views];
    const bool valid = tile < total && (int64_t)tile < bins.tile_capacity;
    if (valid) {
      const int v = find_view(proj.view_info, n_views, tile);
      const uint32_t local = tile - proj.view_info[2 * v];
      const int W = cams[v].width, H = cams[v].height;
      const uint32_t tx = (uint32_t)((W + p.tile_w - 1) / p.tile_w);
      uint32_t n_pairs = *bins.count;
      if ((int64_t)n_pairs > bins.pair_capacity) n_pairs = (uint32_t)bins.pair_capacity;
      uint32_t b = bins.ranges[2 * (size_t)tile], e = bins.ranges[2 * (size_t)tile + 1];
      if (e > n_pairs) e = n_pairs;
      if (b > e) b = e;
      f[0] = 1;
      f[1] = W;
      f[2] = H;
      f[3] = (int)(local % tx) * p.tile_w;
      f[4] = (int)(local / tx) * p.tile_h;
      f[5] = (int)b;
      f[6] = (int)e;
      ti.pix_base = proj.view_info[2 * v + 1];
    }
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) f[i] = __shfl_sync(0xffffffffu, f[i], 0);
  ti.pix_base = __shfl_sync(0xffffffffu, ti.pix_base, 0);
  ti.valid = f[0] != 0;
  ti.W = f[1];
  ti.H = f[2];
  ti.x0 = f[3];
  ti.y0 = f[4];
  ti.beg = (uint32_t)f[5];
  ti.end = (uint32_t)f[6];
  return ti.valid;
}

template <int KP>
__device__ __forceinline__ void warp_block(const TileInfo& ti, const gs_params& p, int blk, WarpBlock& wb) {
  const int lane = threadIdx.x & 31;
  const int wpr = p.tile_w >> 3;
  const int wx = (blk % wpr) * 8, wy = (blk / wpr) * 4 * KP;
  wb.px = ti.x0 + wx + (lane & 7);
  wb.py = ti.y0 + wy + (lane >> 3);
  wb.bx0 = (float)(ti.x0 + wx) + 0.5f;
  wb.bx1 = wb.bx0 + 7.f;
  wb.by0 = (float)(ti.y0 + wy) + 0.5f;
  wb.by1 = wb.by0 + (float)(4 * KP - 1);
}

template <int KP>
__device__ __forceinline__ bool all_done(const bool* done) {
  bool r = true;
#pragma unroll
  for (int q = 0; q < KP; ++q) r = r && done[q];
  return r;
}

// Can the support box of an entry (mean +/- half-widths) contain a pixel centre of the block?
__device__ __forceinline__ bool box_overlaps(const float4& xyod, const float2& ext, const WarpBlock& wb) {
  return (xyod.x - ext.x <= wb.bx1) && (xyod.x + ext.x >= wb.bx0) && (xyod.y - ext.y <= wb.by1) &&
         (xyod.y + ext.y >= wb.by0);
}

// One list entry as a lane holds it.
struct Entry {
  float4 xyod, con;
  float2 ext;
  uint32_t rec;
};

__device__ __forceinline__ void load_entry(const gs_proj& proj, const gs_bins& bins, uint32_t idx, Entry& e) {
  e.rec = __ldg(bins.rec + idx);
  e.xyod = __ldg(reinterpret_cast<const float4*>(proj.xyod) + e.rec);
  e.con = __ldg(reinterpret_cast<const float4*>(proj.conic_u) + e.rec);
  e.ext = __ldg(reinterpret_cast<const float2*>(proj.ext) + e.rec);
}

// Record part of an entry whose record index is already known.
__device__ __forceinline__ void load_record(const gs_proj& proj, uint32_t rec, Entry& e) {
  e.rec = rec;
  e.xyod = __ldg(reinterpret_cast<const float4*>(proj.xyod) + rec);
  e.con = __ldg(reinterpret_cast<const float4*>(proj.conic_u) + rec);
  e.ext = __ldg(reinterpret_cast<const float2*>(proj.ext) + rec);
}

// Fixed-tree block sum (deterministic for a fixed block size); result valid in thread 0.
__device__ __forceinline__ float block_sum_fixed(float v, float* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (warp == 0) {
    s = lane < nw ? s_red[lane] : 0.f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  }
  __syncthreads();
  return s;
}

}  // namespace gs
