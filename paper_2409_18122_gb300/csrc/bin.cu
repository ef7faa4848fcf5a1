// bin.cu -- gs_bin_sort: (tile, depth)-ordered pair list and per-tile ranges.
//
// Sec. III of RT-GuIDE sorts the Gaussians by increasing depth for each camera
// before splatting.  Here every record is duplicated once per covered screen
// tile, and the pairs are ordered by (view, tile, float32 depth, record index):
//   1. stable radix sort of the records by the IEEE bits of their depth
//      (records arrive in (Gaussian, view) order, so ties keep Gaussian order);
//   2. pair counts in that order, exclusive scan -> pair offsets;
//   3. emission: each record writes (global tile id, record index) for the tiles
//      of its rectangle in row-major order;
//   4. stable radix sort of the pairs by global tile id (which encodes the view),
//      so within a tile the depth order of step 1 is kept;
//   5. [start, end) of every tile by comparing neighbours.
#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxGrid = 4096;

inline unsigned grid_for(int64_t n_cap) {
  int64_t b = (n_cap + kBlock - 1) / kBlock;
  if (b < 1) b = 1;
  if (b > kMaxGrid) b = kMaxGrid;
  return (unsigned)b;
}

__device__ inline int64_t clamp_count(const uint32_t* n_dev, int64_t cap) {
  int64_t n = (int64_t)*n_dev;
  return n < cap ? n : cap;
}

__global__ void k_pair_counts(const gs_proj proj, const uint32_t* __restrict__ srec, uint32_t* __restrict__ cnt) {
  const int64_t n = clamp_count(proj.count, proj.capacity);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ushort4 r = reinterpret_cast<const ushort4*>(proj.rect)[srec[i]];
    cnt[i] = (uint32_t)(r.z - r.x) * (uint32_t)(r.w - r.y);
  }
}

__global__ void k_pair_total(const uint32_t* __restrict__ total, int64_t pair_cap, uint32_t* __restrict__ bins_count,
                             uint32_t* __restrict__ n_clamped, uint32_t* status) {
  const uint32_t t = *total;
  *bins_count = t;
  if ((int64_t)t > pair_cap || t == 0xFFFFFFFFu) set_flag(status, GS_FLAG_PAIR_OVERFLOW);
  *n_clamped = (int64_t)t > pair_cap ? (uint32_t)pair_cap : t;
}

// One warp per 32 consecutive records (in depth order).  The warp scans their
// tile counts, then writes the whole run of pairs with consecutive lanes on
// consecutive slots; each lane finds the record that owns its pair with a
// 5-step shuffle search over the running counts.  Writes are coalesced and
// records with many tiles are spread over the warp.
__global__ void __launch_bounds__(256) k_emit(const gs_proj proj, const gs_camera* __restrict__ cams, int tile_w,
                                               const uint32_t* __restrict__ srec, const uint32_t* __restrict__ off,
                                               int64_t pair_cap, uint32_t* __restrict__ tile_key,
                                               uint32_t* __restrict__ tile_rec) {
  const int64_t n = clamp_count(proj.count, proj.capacity);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = warp0 * 32; i0 < n; i0 += n_warps * 32) {
    const int64_t i = i0 + lane;
    uint32_t r = 0, tile0 = 0, tx = 1, w = 1, cnt = 0;
    if (i < n) {
      r = srec[i];
      const ushort4 rc = reinterpret_cast<const ushort4*>(proj.rect)[r];
      const uint32_t v = proj.view[r];
      tx = proj.view_info[kVI * v + 3] >> 16;
      tile0 = proj.view_info[kVI * v] + (uint32_t)rc.y * tx + rc.x;
      w = (uint32_t)(rc.z - rc.x);
      cnt = w * (uint32_t)(rc.w - rc.y);
      if (w == 0) w = 1;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - cnt;
    const uint64_t base = __shfl_sync(0xffffffffu, lane == 0 ? off[i0] : 0u, 0);
    for (uint32_t k0 = 0; k0 < total; k0 += 32) {
      const uint32_t k = k0 + lane;
      int pos = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, pos + step - 1);
        if (v <= k) pos += step;
      }
      const uint32_t o_tile0 = __shfl_sync(0xffffffffu, tile0, pos);
      const uint32_t o_tx = __shfl_sync(0xffffffffu, tx, pos);
      const uint32_t o_w = __shfl_sync(0xffffffffu, w, pos);
      const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, pos);
      const uint32_t o_r = __shfl_sync(0xffffffffu, r, pos);
      const uint64_t slot = base + k;
      if (k < total && slot < (uint64_t)pair_cap) {
        const uint32_t j = k - o_excl;
        const uint32_t y = j / o_w, x = j - y * o_w;
        tile_key[slot] = o_tile0 + y * o_tx + x;
        tile_rec[slot] = o_r;
      }
    }
  }
}

__global__ void k_zero_u32(uint32_t* __restrict__ p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0u;
}

__global__ void k_ranges(const uint32_t* __restrict__ tile, const uint32_t* n_dev, int64_t pair_cap,
                         int64_t tile_cap, const uint32_t* __restrict__ view_info, int n_views,
                         uint32_t* __restrict__ ranges, uint32_t* status) {
  const int64_t n = clamp_count(n_dev, pair_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && (int64_t)view_info[kVI * n_views] > tile_cap)
    set_flag(status, GS_FLAG_RANGE_OVERFLOW);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = tile[i];
    if ((int64_t)t >= tile_cap) continue;
    if (i == 0 || tile[i - 1] != t) ranges[2 * (int64_t)t] = (uint32_t)i;
    if (i == n - 1 || tile[i + 1] != t) ranges[2 * (int64_t)t + 1] = (uint32_t)(i + 1);
  }
}

int bits_for(int64_t tile_cap) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < tile_cap) ++b;
  return b;
}

}  // namespace

size_t bin_ws_bytes(int64_t rec_cap, int64_t pair_cap, int64_t tile_cap) {
  (void)tile_cap;
  Carver c(nullptr);
  c.take<uint32_t>(rec_cap);               // record keys a
  c.take<uint32_t>(rec_cap);               // record vals a
  c.take<uint32_t>(rec_cap);               // record keys b
  c.take<uint32_t>(rec_cap);               // record vals b
  c.take<uint32_t>(rec_cap + 1);           // pair counts
  c.take<uint32_t>(rec_cap + 1);           // pair offsets
  c.take<uint32_t>(pair_cap);              // pair keys (ping-pong partner)
  c.take<uint32_t>(pair_cap);              // pair vals (ping-pong partner)
  c.take<uint32_t>(4);                     // counters
  size_t t = sort_temp_bytes(rec_cap > pair_cap ? rec_cap : pair_cap);
  size_t s = scan_temp_bytes(rec_cap);
  c.take<char>(t > s ? t : s);
  return align_up(c.off, 256);
}

cudaError_t launch_bin_sort(const gs_proj& proj, const gs_camera* cams, int n_views, const gs_params& p,
                            const gs_bins& out, void* ws, cudaStream_t st) {
  const int64_t rec_cap = proj.capacity, pair_cap = out.pair_capacity, tile_cap = out.tile_capacity;
  Carver c(ws);
  uint32_t* rk_a = c.take<uint32_t>(rec_cap);
  uint32_t* rv_a = c.take<uint32_t>(rec_cap);
  uint32_t* rk_b = c.take<uint32_t>(rec_cap);
  uint32_t* rv_b = c.take<uint32_t>(rec_cap);
  uint32_t* cnt = c.take<uint32_t>(rec_cap + 1);
  uint32_t* off = c.take<uint32_t>(rec_cap + 1);
  uint32_t* pk_w = c.take<uint32_t>(pair_cap);
  uint32_t* pv_w = c.take<uint32_t>(pair_cap);
  uint32_t* ctr = c.take<uint32_t>(4);      // [0] pair total (saturated), [1] pair count clamped to capacity
  size_t t = sort_temp_bytes(rec_cap > pair_cap ? rec_cap : pair_cap);
  size_t s = scan_temp_bytes(rec_cap);
  void* tmp = c.take<char>(t > s ? t : s);

  // 1. records by depth bits (32 bits, 4 passes: result back in the a buffers)
  bool in_a = false;
  cudaError_t e = radix_sort(proj.depth_key, nullptr, nullptr, SortBufs{rk_a, rv_a, rk_b, rv_b}, proj.count,
                             rec_cap, 0, 32, tmp, st, &in_a);
  if (e != cudaSuccess) return e;
  const uint32_t* srec = in_a ? rv_a : rv_b;
  // 2. pair counts and offsets in depth order
  k_pair_counts<<<grid_for(rec_cap), kBlock, 0, st>>>(proj, srec, cnt);
  note_launch();
  e = scan_exclusive(cnt, off, proj.count, rec_cap, &ctr[0], tmp, st);
  if (e != cudaSuccess) return e;
  k_pair_total<<<1, 1, 0, st>>>(&ctr[0], pair_cap, out.count, &ctr[1], proj.status);
  note_launch();
  // 3. emission into whichever buffer makes the final pass land in `out`
  const int bits = bits_for(tile_cap);
  const int passes = sort_passes(0, bits);
  SortBufs pb;
  if (passes % 2 == 0) pb = SortBufs{out.tile, out.rec, pk_w, pv_w};
  else pb = SortBufs{pk_w, pv_w, out.tile, out.rec};
  k_emit<<<grid_for(rec_cap), kBlock, 0, st>>>(proj, cams, p.tile_w, srec, off, pair_cap, pb.keys_a, pb.vals_a);
  note_launch();
  // 4. pairs by global tile id
  e = radix_sort(pb.keys_a, nullptr, pb.vals_a, pb, &ctr[1], pair_cap, 0, bits, tmp, st, &in_a);
  if (e != cudaSuccess) return e;
  // 5. ranges
  k_zero_u32<<<grid_for(2 * tile_cap), kBlock, 0, st>>>(out.ranges, 2 * tile_cap);
  note_launch();
  k_ranges<<<grid_for(pair_cap), kBlock, 0, st>>>(out.tile, &ctr[1], pair_cap, tile_cap, proj.view_info, n_views,
                                                  out.ranges, proj.status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
