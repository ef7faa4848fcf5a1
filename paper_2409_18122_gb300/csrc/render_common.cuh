// render_common.cuh -- per-tile setup and the per-(pixel, Gaussian) opacity
// shared by the forward, backward and information-gain compositing kernels, so
// that all of them take identical skip / stop decisions.
#pragma once

#include "gs_common.cuh"

namespace gs {

struct TileInfo {
  bool valid;
  int W, H;
  int x0, y0;          // pixel origin of the tile
  int tw;              // tile width of the view
  int blk;             // pixel block of the tile handled by the warp
  uint32_t tile;       // global tile id
  uint32_t pix_base;   // first pixel of the view in the concatenated images
  uint32_t beg, end;   // range in the sorted pair list
};

// alpha = min(alpha_max, o exp(-q/2)), q = a dx^2 + 2 b dx dy + c dy^2 with
// (dx, dy) = mu_2D - pixel centre and conic (a, b, c).  exp(-q/2) is evaluated
// as 2^p with p = -q/2 log2(e): the conic is scaled once per Gaussian (per warp
// staging, not per pixel) to k = (-a/2, -b, -c/2) log2(e), and the exponent is staged as
// a quadratic in the lane's pixel offset (stage_exponent, alpha_raw below).
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float3 scaled_conic(const float4& co) {
  return make_float3(__fmul_rn(co.x, -0.5f * kLog2e), __fmul_rn(co.y, -kLog2e), __fmul_rn(co.z, -0.5f * kLog2e));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// alpha before the alpha_max clamp, o exp(-q/2), as 2^pw with pw a quadratic in the
// lane's offset (u, v) from the centre of its 8x4 pixel block (lane l: u = l mod 8 - 3.5,
// v = l div 8 - 1.5).  With (ex, ey) = mean - block centre and k = scaled_conic(conic),
//   pw = k.x (ex - u)^2 + k.y (ex - u)(ey - v) + k.z (ey - v)^2 + log2 o
//      = c0 + cu u + cv v + k.x u^2 + k.y u v + k.z v^2,
// so an entry's coefficients are staged once per warp and every pixel takes five fused
// multiply-adds.  Every kernel stages and evaluates it with these functions (explicit
// round-to-nearest operations), so the forward, backward and one-launch renders take
// bit-identical skip and stop decisions.
struct LaneOffsets {
  float u, v, uu, uv, vv;   // quarter-integers and their products: exact in FP32
};

__device__ __forceinline__ LaneOffsets lane_offsets(int lane) {
  LaneOffsets o;
  o.u = (float)(lane & 7) - 3.5f;
  o.v = (float)(lane >> 3) - 1.5f;
  o.uu = o.u * o.u;
  o.uv = o.u * o.v;
  o.vv = o.v * o.v;
  return o;
}

struct Exponent {
  float c0, cu, cv, kx, ky, kz;
};

// Coefficients of an entry with mean (mx, my) and conic co = (a, b, c, o) for the block
// whose centre is (ccx, ccy).
__device__ __forceinline__ Exponent stage_exponent(float mx, float my, const float4& co, float ccx, float ccy) {
  const float3 k = scaled_conic(co);
  const float ex = __fsub_rn(mx, ccx), ey = __fsub_rn(my, ccy);
  Exponent e;
  e.c0 = __fmaf_rn(__fmul_rn(k.z, ey), ey, __fmaf_rn(__fmul_rn(k.y, ex), ey, __fmaf_rn(__fmul_rn(k.x, ex), ex, __log2f(co.w))));
  e.cu = -__fmaf_rn(__fmul_rn(2.f, k.x), ex, __fmul_rn(k.y, ey));
  e.cv = -__fmaf_rn(k.y, ex, __fmul_rn(__fmul_rn(2.f, k.z), ey));
  e.kx = k.x;
  e.ky = k.y;
  e.kz = k.z;
  return e;
}

// o exp(-q/2) at the lane's pixel (before the alpha_max clamp).
__device__ __forceinline__ float alpha_raw(float c0, float cu, float cv, float kx, float ky, float kz,
                                           const LaneOffsets& lo) {
  return ex2_approx(__fmaf_rn(kz, lo.vv, __fmaf_rn(ky, lo.uv, __fmaf_rn(kx, lo.uu, __fmaf_rn(cv, lo.v, __fmaf_rn(cu, lo.u, c0))))));
}

// Work item of the compositing kernels: one warp renders one 8 x (4 KP) pixel
// block of one screen tile, KP pixels per lane (KP = 1 in every kernel: a larger
// block per warp culls less finely, which costs more than it saves).  Block b of a tile covers columns
// 8 (b mod (tile_w/8)) .. +7 and rows 4 KP (b div (tile_w/8)) .. +4 KP - 1;
// lane l owns pixels (l mod 8, l div 8 + 4 q), q < KP.  Warps never wait for
// each other: each walks its tile's list on its own and stops as soon as all of
// its pixels are saturated.
struct WarpBlock {
  int px, py;                   // this lane's first pixel; the others are (px, py + 4 q)
  float bx0, bx1, by0, by1;     // pixel-centre bounds of the warp's block
};

// Decodes warp item `item` (numbered view by view, tile by tile, block by block,
// with tile_w * tile_h / (32 KP) items per tile) into its tile and block; lane 0
// computes and broadcasts.  Returns false (warp-uniform) if the item does not exist.
template <int KP>
__device__ __forceinline__ bool warp_item_setup(const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                                                int n_views, uint32_t item, TileInfo& ti) {
  const int lane = threadIdx.x & 31;
  int f[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t pix_base = 0;
  if (lane == 0) {
    const uint32_t total = proj.view_info[kVI * n_views + 2] / KP;
    if (item < total) {
      // largest v with first_item(v) / KP <= item
      int lo = 0, hi = n_views - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (proj.view_info[kVI * mid + 2] / KP <= item) lo = mid; else hi = mid - 1;
      }
      const int v = lo;
      const uint32_t code = proj.view_info[kVI * v + 3];
      const int tw = (int)(code & 0xffu), th = (int)((code >> 8) & 0xffu);
      const uint32_t tx = code >> 16;
      const uint32_t wpt = (uint32_t)(tw * th / (32 * KP));
      const uint32_t local = item - proj.view_info[kVI * v + 2] / KP;
      const uint32_t lt = wpt ? local / wpt : 0u;
      const uint32_t tile = proj.view_info[kVI * v] + lt;
      if (code != 0u && wpt != 0u && (int64_t)tile < bins.tile_capacity) {
        uint32_t n_pairs = *bins.count;
        if ((int64_t)n_pairs > bins.pair_capacity) n_pairs = (uint32_t)bins.pair_capacity;
        uint32_t b = bins.ranges[2 * (size_t)tile], e = bins.ranges[2 * (size_t)tile + 1];
        if (e > n_pairs) e = n_pairs;
        if (b > e) b = e;
        f[0] = 1;
        f[1] = cams[v].width;
        f[2] = cams[v].height;
        f[3] = (int)(lt % tx) * tw;
        f[4] = (int)(lt / tx) * th;
        f[5] = (int)b;
        f[6] = (int)e;
        f[7] = tw;
        f[8] = (int)(local % wpt);
        f[9] = (int)tile;
        pix_base = proj.view_info[kVI * v + 1];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 10; ++i) f[i] = __shfl_sync(0xffffffffu, f[i], 0);
  ti.pix_base = __shfl_sync(0xffffffffu, pix_base, 0);
  ti.valid = f[0] != 0;
  ti.W = f[1];
  ti.H = f[2];
  ti.x0 = f[3];
  ti.y0 = f[4];
  ti.beg = (uint32_t)f[5];
  ti.end = (uint32_t)f[6];
  ti.tw = f[7];
  ti.blk = f[8];
  ti.tile = (uint32_t)f[9];
  return ti.valid;
}

// The warp item that work slot i renders: the binning's longest-list-first order when it
// was written (gs_bin_sort writes bins.item_order when the batch has at most item_capacity
// items of 32 pixels), else slot i itself.  Any order gives the same pixels.
__device__ __forceinline__ uint32_t ordered_item(const gs_bins& bins, const uint32_t* view_info, int n_views,
                                                 uint32_t i) {
  if (!bins.item_order) return i;
  const uint32_t n = view_info[kVI * n_views + 2];
  return ((int64_t)n <= bins.item_capacity && i < n) ? bins.item_order[i] : i;
}

template <int KP>
__device__ __forceinline__ void warp_block(const TileInfo& ti, WarpBlock& wb) {
  const int lane = threadIdx.x & 31;
  const int wpr = ti.tw >> 3;
  const int blk = ti.blk;
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

// Some pixel of the lane is not saturated (the information-gain kernel keeps T = 0 for
// saturated pixels and for pixels outside the image).
template <int KP>
__device__ __forceinline__ bool live(const float* T) {
  bool r = false;
#pragma unroll
  for (int q = 0; q < KP; ++q) r = r || T[q] != 0.f;
  return r;
}

// Can the support box of an entry contain a pixel centre of the warp's block?
// s0 = first half of its splat record (mu_x, mu_y, packed half-widths, u).
__device__ __forceinline__ bool box_overlaps(const float4& s0, const WarpBlock& wb) {
  float rx, ry;
  unpack_ext(s0.z, rx, ry);
  return (s0.x - rx <= wb.bx1) && (s0.x + rx >= wb.bx0) && (s0.y - ry <= wb.by1) && (s0.y + ry >= wb.by0);
}

// Second, tighter cull for entries that passed box_overlaps (co = second half of the
// splat record: a, b, c, o).  The support ellipse is q <= Q = 2 ln(o / alpha_min);
// for any pixel centre p of the block, sqrt(q(p - mu)) >= sqrt(q(c - mu)) - r with c
// the block centre and r = max over the block's corner offsets e of sqrt(q(e)) =
// sqrt(a hx^2 + 2 |b| hx hy + c hy^2) (triangle inequality in the norm sqrt(q)).  So a
// Gaussian with sqrt(q(c - mu)) > sqrt(Q) + r reaches no pixel of the block.  The
// margin keeps the test conservative under FP32 rounding.  ln_amin = ln(alpha_min).
__device__ __forceinline__ bool ellipse_reaches(const float4& s0, const float4& co, const WarpBlock& wb,
                                                float ln_amin) {
  const float hx = 0.5f * (wb.bx1 - wb.bx0), hy = 0.5f * (wb.by1 - wb.by0);
  const float dx = s0.x - (wb.bx0 + hx), dy = s0.y - (wb.by0 + hy);
  const float q = co.x * dx * dx + 2.f * co.y * dx * dy + co.z * dy * dy;
  const float r2 = co.x * hx * hx + 2.f * fabsf(co.y) * hx * hy + co.z * hy * hy;
  const float Q = 2.f * (__logf(co.w) - ln_amin);
  const float reach = sqrtf(fmaxf(Q, 0.f)) + sqrtf(fmaxf(r2, 0.f));
  return sqrtf(fmaxf(q, 0.f)) <= reach * 1.0001f + 1e-3f;
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
