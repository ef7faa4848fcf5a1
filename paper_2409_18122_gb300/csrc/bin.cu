// bin.cu -- gs_bin_sort: (tile, depth)-ordered pair list and per-tile ranges.
//
// Sec. III of RT-GuIDE sorts the Gaussians by increasing depth for each camera
// before splatting.  Every record is duplicated once per covered screen tile and
// the pairs are ordered by (view, tile, float32 depth, record index).  The
// records of each view are contiguous (gs_project writes them view by view), so:
//   1. view segments: the first record of every view;
//   2. stable LSD radix sort of the record indices by the IEEE bits of their
//      depth, segmented by view (every view's records are sorted in place):
//      (view, depth, record) order;
//   3. the rectangles in that order and each record's pair count (written by the
//      last sort pass), and an exclusive scan of the counts: the pairs of the
//      sorted records, in order, are numbered 0 .. P-1 (records in order, the
//      tiles of a rectangle row-major);
//   4. the pairs of each view are cut into K equal chunks; one warp per chunk
//      counts its pairs per tile of the view (shared-memory histogram);
//   5. one exclusive scan over the counts laid out [global tile][chunk] gives,
//      for every (tile, chunk), the first slot of that chunk's pairs in the
//      tile's run -- and with it every tile's [start, end);
//   6. each warp walks its chunk again in the same order and writes every pair
//      straight to its slot, ranking pairs of the same tile among the lanes with
//      a warp match, so the order inside a tile is the depth order of step 2.
// No pair is ever sorted or moved twice, no block waits on another, and the
// result is deterministic.  Chunks hold equal numbers of pairs: near Gaussians,
// which come first in depth order, cover many tiles each.
#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxGrid = 4096;
// warp chunks over all views (256-candidate batch, binning: 49,152 / 65,536 / 98,304 / 131,072
// chunks 3.45 / 3.40 / 3.35 / 3.35 ms; at 131,072 the 2^24-entry count table bounds K there)
constexpr int kChunkTarget = 131072;
constexpr int kPairsPerEntry = 4;     // pairs per (tile, chunk) count entry, at least
constexpr int kWin = 1024;            // tile cells of a histogram window (shared memory per warp)
constexpr int kPlaceWin = 512;        // tile cells of a placement window (running slots per warp)
constexpr int kWinCols = 256;         // widest window, in tiles
constexpr int kBinWarps = 8;          // warps (= chunks) per block of the histogram / placement kernels

inline unsigned grid_for(int64_t n_cap) {
  int64_t b = (n_cap + kBlock - 1) / kBlock;
  if (b < 1) b = 1;
  if (b > kMaxGrid) b = kMaxGrid;
  return (unsigned)b;
}

// Chunks per view: about kChunkTarget warps in total, with at most pair_cap /
// kPairsPerEntry and 2^24 count entries (the per-(tile, chunk) table is written,
// scanned and read once per call, and each chunk walks every tile of its view, so the
// table is kept small against the pairs: the pair capacity bounds their number).
int chunks_per_view(int n_views, int64_t tile_cap, int64_t pair_cap) {
  int64_t k = (kChunkTarget + n_views - 1) / n_views;
  if (tile_cap > 0) {
    const int64_t by_table = ((int64_t)1 << 24) / tile_cap;
    const int64_t by_pairs = pair_cap / kPairsPerEntry / tile_cap;
    if (k > by_table) k = by_table;
    if (k > by_pairs) k = by_pairs;
  }
  if (k < 1) k = 1;
  return (int)k;
}

__device__ inline int64_t clamp_count(const uint32_t* n_dev, int64_t cap) {
  int64_t n = (int64_t)*n_dev;
  return n < cap ? n : cap;
}

__global__ void k_zero_u32(uint32_t* __restrict__ p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0u;
}

// seg[v] = first record of view v (seg[V] = n) for records grouped by view in
// increasing view order; a record out of that order, or with a view id >= V,
// sets GS_FLAG_BAD_RECORDS.  seg must be zeroed first, so that every entry lies in
// [0, n] even for bad input.  Thread 0 also stores the number of count entries
// that step 4 scans: K * min(total tiles, tile_cap).
__global__ void k_segments(const gs_proj proj, int n_views, int64_t tile_cap, int K, uint32_t* __restrict__ seg,
                           uint32_t* __restrict__ scan_n) {
  const int64_t n = clamp_count(proj.count, proj.capacity);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t tiles = proj.view_info[kVI * n_views];
    if (tiles > tile_cap) tiles = tile_cap;
    *scan_n = (uint32_t)(tiles * K);
    if (n == 0)
      for (int v = 0; v <= n_views; ++v) seg[v] = 0u;
  }
  // four records per thread and 16-byte load when the view array is 16-byte aligned
  const bool vec = ((uintptr_t)proj.view & 15u) == 0;
  const int64_t per = vec ? 4 : 1;
  const int64_t groups = (n + per - 1) / per;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < groups; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = j * per;
    uint32_t vv[4];
    if (vec && i0 + 4 <= n) {
      const uint4 q = reinterpret_cast<const uint4*>(proj.view)[j];
      vv[0] = q.x; vv[1] = q.y; vv[2] = q.z; vv[3] = q.w;
    } else {
      for (int k = 0; k < 4; ++k) vv[k] = (k < per && i0 + k < n) ? proj.view[i0 + k] : 0u;
    }
    int64_t prev = -1;
    if (i0 > 0) {
      prev = proj.view[i0 - 1];
      if (prev >= n_views) prev = n_views - 1;
    }
    for (int k = 0; k < per && i0 + k < n; ++k) {
      const int64_t i = i0 + k;
      int64_t v = vv[k];
      if (v >= n_views) {
        set_flag(proj.status, GS_FLAG_BAD_RECORDS);
        v = n_views - 1;
      }
      if (v < prev) set_flag(proj.status, GS_FLAG_BAD_RECORDS);
      for (int64_t u = prev + 1; u <= v; ++u) seg[u] = (uint32_t)i;
      if (i == n - 1)
        for (int64_t u = v + 1; u <= n_views; ++u) seg[u] = (uint32_t)n;
      prev = v;
    }
  }
}

// seg[v] from the projection's group offsets, for records written by gs_project without
// per-record view ids: view v's records start at grp_base[v * G] (clipped to the record
// count), G = the number of 32-Gaussian groups, which gs_project leaves in
// view_info[V][3]; seg[V] = the record count.
__global__ void k_segments_from_groups(const gs_proj proj, int n_views, int64_t tile_cap, int K,
                                       uint32_t* __restrict__ seg, uint32_t* __restrict__ scan_n) {
  const int64_t n = clamp_count(proj.count, proj.capacity);
  const int64_t n_grp = proj.view_info[kVI * n_views + 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t tiles = proj.view_info[kVI * n_views];
    if (tiles > tile_cap) tiles = tile_cap;
    *scan_n = (uint32_t)(tiles * K);
  }
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n_views;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = v < n_views ? (int64_t)proj.grp_base[v * n_grp] : n;
    seg[v] = (uint32_t)(b < n ? b : n);
  }
}

// Chunk (v, k): the sorted records [r0, r1) of view v whose first pair (as
// numbered in step 3) lies in [P_v k / K, P_v (k+1) / K) of the view's P_v pairs,
// so every chunk holds about P_v / K pairs; and the view's tile grid.
struct Chunk {
  int64_t r0, r1;
  uint32_t tile_base, n_tiles, tiles_x, tiles_y, k;
};

// First r in [lo, hi] with poff[r] >= x (hi if none).
__device__ inline int64_t lower_bound_u32(const uint32_t* __restrict__ poff, int64_t lo, int64_t hi, int64_t x) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)poff[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// First record of every chunk: bounds[v (K + 1) + k] = the first sorted record of view v whose
// first pair lies at or past P_v k / K (bounds[v (K + 1) + K] = the view's end).  One thread
// per bound, so the binary searches run side by side instead of at the start of every warp
// of the histogram and placement kernels.
__global__ void k_chunk_bounds(const uint32_t* __restrict__ seg, const uint32_t* __restrict__ poff, int n_views,
                               int K, uint32_t* __restrict__ bounds) {
  const int64_t nb = (int64_t)n_views * (K + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(i / (K + 1));
    const int k = (int)(i - (int64_t)v * (K + 1));
    int64_t s0 = seg[v], s1 = seg[v + 1];
    if (s1 < s0) s1 = s0;
    int64_t r = s1;
    if (k < K) {
      const int64_t a = poff[s0], b = poff[s1];
      const int64_t P = b > a ? b - a : 0;
      r = lower_bound_u32(poff, s0, s1, a + P * k / K);
    }
    bounds[i] = (uint32_t)r;
  }
}

__device__ inline bool chunk_of(int64_t cid, int K, const uint32_t* __restrict__ bounds,
                                const uint32_t* __restrict__ view_info, int64_t tile_cap, Chunk& c) {
  const int v = (int)(cid / K);
  c.k = (uint32_t)(cid - (int64_t)v * K);
  const uint32_t* b = bounds + (size_t)v * (K + 1) + c.k;
  c.r0 = b[0];
  c.r1 = b[1];
  if (c.r1 < c.r0) c.r1 = c.r0;
  c.tile_base = view_info[kVI * v];
  c.n_tiles = view_info[kVI * (v + 1)] - c.tile_base;
  c.tiles_x = view_info[kVI * v + 3] >> 16;
  c.tiles_y = c.tiles_x ? c.n_tiles / c.tiles_x : 0u;
  // a view whose tiles do not all fit under tile_cap is skipped (GS_FLAG_RANGE_OVERFLOW is set elsewhere)
  return c.n_tiles > 0 && (int64_t)c.tile_base + c.n_tiles <= tile_cap;
}

// The tile grid of a view is handled in windows [xa, xb) x [ya, yb) of at most
// `cells` cells (difference arrays need one extra row and column).
__device__ inline void window_size(uint32_t tx, uint32_t ty, uint32_t cells, bool extra, uint32_t& ww,
                                   uint32_t& wh) {
  const uint32_t e = extra ? 1u : 0u;
  ww = tx < (uint32_t)kWinCols ? tx : (uint32_t)kWinCols;
  wh = cells / (ww + e) - e;
  if (wh > ty) wh = ty;
  if (wh < 1) wh = 1;
}

// Step 4: per chunk, the number of its pairs in every tile of its view:
// cnt[K * global tile + k].  Each record adds the corners of its rectangle to a
// 2D difference array; a 2D prefix sum turns it into per-tile counts.
__global__ void __launch_bounds__(kBinWarps * 32) k_bin_hist(const gs_proj proj, const uint32_t* __restrict__ bounds,
                                                             const ushort4* __restrict__ srect, int n_views, int K,
                                                             int64_t tile_cap, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t s_d[kBinWarps][kWin];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cid = (int64_t)blockIdx.x * kBinWarps + warp;
  if (cid >= (int64_t)n_views * K) return;
  Chunk c;
  if (!chunk_of(cid, K, bounds, proj.view_info, tile_cap, c)) {
    // the tiles of a skipped view that lie under tile_cap are still scanned: zero counts
    for (int64_t t = lane; t < (int64_t)c.n_tiles && (int64_t)c.tile_base + t < tile_cap; t += 32)
      cnt[(size_t)K * (c.tile_base + t) + c.k] = 0u;
    return;
  }
  uint32_t* D = s_d[warp];
  uint32_t ww, wh;
  window_size(c.tiles_x, c.tiles_y, kWin, true, ww, wh);
  const uint32_t pitch = ww + 1;
  for (uint32_t ya = 0; ya < c.tiles_y; ya += wh) {
    const uint32_t yb = ya + wh < c.tiles_y ? ya + wh : c.tiles_y;
    for (uint32_t xa = 0; xa < c.tiles_x; xa += ww) {
      const uint32_t xb = xa + ww < c.tiles_x ? xa + ww : c.tiles_x;
      for (int i = lane; i < kWin; i += 32) D[i] = 0u;
      __syncwarp();
#pragma unroll 4
      for (int64_t r = c.r0 + lane; r < c.r1; r += 32) {
        const ushort4 rc = srect[r];
        const uint32_t x0 = rc.x > xa ? rc.x : xa, x1 = rc.z < xb ? rc.z : xb;
        const uint32_t y0 = rc.y > ya ? rc.y : ya, y1 = rc.w < yb ? rc.w : yb;
        if (x0 < x1 && y0 < y1) {
          atomicAdd(&D[(y0 - ya) * pitch + (x0 - xa)], 1u);
          atomicAdd(&D[(y0 - ya) * pitch + (x1 - xa)], 0xFFFFFFFFu);
          atomicAdd(&D[(y1 - ya) * pitch + (x0 - xa)], 0xFFFFFFFFu);
          atomicAdd(&D[(y1 - ya) * pitch + (x1 - xa)], 1u);
        }
      }
      __syncwarp();
      const uint32_t rows = yb - ya, cols = xb - xa;
      for (uint32_t y = lane; y < rows; y += 32) {   // prefix along x
        uint32_t run = 0;
        for (uint32_t x = 0; x < cols; ++x) {
          run += D[y * pitch + x];
          D[y * pitch + x] = run;
        }
      }
      __syncwarp();
      for (uint32_t x = lane; x < cols; x += 32) {   // prefix along y, and out
        uint32_t run = 0;
        for (uint32_t y = 0; y < rows; ++y) {
          run += D[y * pitch + x];
          cnt[(size_t)K * (c.tile_base + (ya + y) * c.tiles_x + xa + x) + c.k] = run;
        }
      }
      __syncwarp();
    }
  }
}

// Step 5b: ranges of every global tile from the scanned counts, the pair total
// and the overflow flags.  Empty tiles, and tiles past the scanned range, get [0, 0).
__global__ void k_bin_ranges(const uint32_t* __restrict__ off, const uint32_t* __restrict__ scan_n,
                             const uint32_t* __restrict__ total, int K, int64_t pair_cap, int64_t tile_cap,
                             const uint32_t* __restrict__ view_info, int n_views, uint32_t* __restrict__ ranges,
                             uint32_t* __restrict__ bins_count, uint32_t* status) {
  const int64_t lim = (int64_t)*scan_n / K;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint32_t t = *total;
    *bins_count = t;
    if ((int64_t)t > pair_cap || t == 0xFFFFFFFFu) set_flag(status, GS_FLAG_PAIR_OVERFLOW);
    if ((int64_t)view_info[kVI * n_views] > tile_cap) set_flag(status, GS_FLAG_RANGE_OVERFLOW);
  }
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < tile_cap; g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t a = 0, b = 0;
    if (g < lim) {
      a = off[(size_t)K * g];
      b = off[(size_t)K * (g + 1)];
      if ((int64_t)a > pair_cap) a = (uint32_t)pair_cap;
      if ((int64_t)b > pair_cap) b = (uint32_t)pair_cap;
      if (a == b) a = b = 0u;   // an empty tile is [0, 0)
    }
    ranges[2 * g] = a;
    ranges[2 * g + 1] = b;
  }
}

// Step 6: every pair written to its slot.  A warp takes its chunk's records 32
// at a time (a group; the next group's rectangles and record ids are loaded while
// the current one is placed).  The group's records that have pairs in the current
// window are compacted, in order, into shared memory (corner, width, first pair,
// record id and a reciprocal of the width), and their pairs are enumerated 32 at a
// time (a round; record order, each rectangle row-major), one pair per lane.  The
// record owning pair k is found from the records that start inside the round (one
// warp OR of start bits and a population count), not by a search.  The lanes of a
// round holding pairs of the same window cell belong to different records, in lane
// order: a warp match on the cell gives each its rank among them, its slot is the
// cell's running slot plus that rank, and the lowest of them advances the running
// slot for the next round.
template <bool kTileIds>
__global__ void __launch_bounds__(kBinWarps * 32, 5) k_bin_place(const gs_proj proj,
                                                                 const uint32_t* __restrict__ bounds,
                                                                 const uint32_t* __restrict__ srec,
                                                                 const ushort4* __restrict__ srect, int n_views, int K,
                                                                 int64_t tile_cap, const uint32_t* __restrict__ off,
                                                                 gs_bins out) {
  __shared__ uint32_t s_run[kBinWarps][kPlaceWin];
  __shared__ uint4 s_grp[kBinWarps][32];
  // ceil(2^32 / w) for every clipped width w <= kWinCols (a table: an integer division by a
  // variable is a long instruction sequence)
  __shared__ uint32_t s_magic[kWinCols + 1];
  for (int i = threadIdx.x; i <= kWinCols; i += blockDim.x) s_magic[i] = i > 1 ? 0xFFFFFFFFu / (uint32_t)i + 1u : 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t le = (2u << lane) - 1u;   // lanes 0 .. lane (all 32 for lane 31)
  const int64_t cid = (int64_t)blockIdx.x * kBinWarps + warp;
  if (cid >= (int64_t)n_views * K) return;
  Chunk c;
  if (!chunk_of(cid, K, bounds, proj.view_info, tile_cap, c)) return;
  uint32_t* run = s_run[warp];
  uint4* grp = s_grp[warp];
  const uint32_t cap = out.pair_capacity < 0xFFFFFFFFll ? (uint32_t)out.pair_capacity : 0xFFFFFFFFu;
  uint32_t ww, wh;
  window_size(c.tiles_x, c.tiles_y, kPlaceWin, false, ww, wh);
  for (uint32_t ya = 0; ya < c.tiles_y; ya += wh) {
    const uint32_t yb = ya + wh < c.tiles_y ? ya + wh : c.tiles_y;
    for (uint32_t xa = 0; xa < c.tiles_x; xa += ww) {
      const uint32_t xb = xa + ww < c.tiles_x ? xa + ww : c.tiles_x;
      const uint32_t cols = xb - xa, cells = (yb - ya) * cols;
#pragma unroll 4
      for (uint32_t i = lane; i < cells; i += 32) {
        const uint32_t y = ya + i / cols, x = xa + i % cols;
        run[i] = off[(size_t)K * (c.tile_base + y * c.tiles_x + x) + c.k];
      }
      ushort4 rc_next = make_ushort4(0, 0, 0, 0);
      uint32_t rec_next = 0;
      if (c.r0 + lane < c.r1) {
        rc_next = srect[c.r0 + lane];
        rec_next = srec[c.r0 + lane];
      }
      __syncwarp();
      for (int64_t g = c.r0; g < c.r1; g += 32) {
        const ushort4 rc = rc_next;
        const uint32_t rec_g = rec_next;
        const bool have = g + lane < c.r1;
        if (g + 32 + lane < c.r1) {
          rc_next = srect[g + 32 + lane];
          rec_next = srec[g + 32 + lane];
        }
        // this lane's record, clipped to the window (window-relative corner)
        uint32_t x0 = 0, y0 = 0, w = 1, cnt = 0;
        if (have) {
          const uint32_t cx0 = rc.x > xa ? rc.x : xa, cx1 = rc.z < xb ? rc.z : xb;
          const uint32_t cy0 = rc.y > ya ? rc.y : ya, cy1 = rc.w < yb ? rc.w : yb;
          if (cx0 < cx1 && cy0 < cy1) {
            x0 = cx0 - xa;
            y0 = cy0 - ya;
            w = cx1 - cx0;
            cnt = w * (cy1 - cy0);
          }
        }
        const uint32_t nz = __ballot_sync(0xffffffffu, cnt > 0u);
        if (nz == 0u) continue;
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - cnt;
        __syncwarp();   // the previous group's rounds are done with grp
        if (cnt > 0u) {
          // floor(j / w) = umulhi(j, ceil(2^32 / w)) exactly for j w < 2^32 (here j < 2^9, w <= 2^8)
          const uint32_t magic = s_magic[w];
          grp[__popc(nz & lt)] = make_uint4(x0 | (y0 << 8) | (w << 17), excl, rec_g, magic);
        }
        __syncwarp();
        // The rounds are software-pipelined: the cell, record and same-cell lanes of round
        // k0 + 32 (which read only the group table) are found while round k0 reads and
        // advances the running slots, so the two dependency chains overlap.
        uint32_t before = 0;   // records of the group whose first pair precedes the next round
        auto cell_of = [&](uint32_t k0, bool& valid, uint32_t& i, uint32_t& peers, uint32_t& o_rec, uint32_t& cx,
                           uint32_t& cy) {
          const uint32_t d = excl - k0;   // < 32 iff this lane's record starts in the round
          const uint32_t starts = __reduce_or_sync(0xffffffffu, (cnt > 0u && d < 32u) ? (1u << d) : 0u);
          const uint32_t k = k0 + lane;
          valid = k < total;
          i = 0xFFFFFFFFu;   // invalid lanes share this key and do nothing
          cy = cx = o_rec = 0;
          if (valid) {
            const uint4 e = grp[before + __popc(starts & le) - 1u];   // the owner of pair k
            const uint32_t j = k - e.y;
            const uint32_t ow = e.x >> 17;
            const uint32_t y = ow > 1u ? __umulhi(j, e.w) : j;
            cy = ((e.x >> 8) & 0x1FFu) + y;
            cx = (e.x & 0xFFu) + (j - y * ow);
            i = cy * cols + cx;
            o_rec = e.z;
          }
          before += __popc(starts);
          peers = __match_any_sync(0xffffffffu, i);   // lanes of the same window cell
        };
        bool vA;
        uint32_t iA, pA, rA, xA, yA;
        cell_of(0u, vA, iA, pA, rA, xA, yA);
        for (uint32_t k0 = 0; k0 < total; k0 += 32) {
          bool vB = false;
          uint32_t iB = 0xFFFFFFFFu, pB = 0u, rB = 0u, xB = 0u, yB = 0u;
          if (k0 + 32u < total) cell_of(k0 + 32u, vB, iB, pB, rB, xB, yB);
          const uint32_t below = pA & lt;
          uint32_t base = 0;
          if (vA) {
            base = run[iA];
            const uint32_t slot = base + __popc(below);
            if (slot < cap) {
              out.rec[slot] = rA;
              if (kTileIds) out.tile[slot] = c.tile_base + (ya + yA) * c.tiles_x + xa + xA;
            }
          }
          __syncwarp();
          if (vA && below == 0u) run[iA] = base + __popc(pA);   // lowest lane of the cell in this round
          __syncwarp();
          vA = vB;
          iA = iB;
          pA = pB;
          rA = rB;
          xA = xB;
          yA = yB;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- item order
// The warp items of the batch (32-pixel blocks of tiles; view_info[v][2] is the first item
// of view v) ordered longest tile list first, by a counting sort over kOrderBuckets buckets
// of list length, four per doubling.  The compositing kernels take their items in this
// order, so that the longest lists start first instead of wherever their tile falls.
constexpr int kOrderBuckets = 64;

// Bucket of a list of `len` pairs: 0 for the longest lists.
__device__ inline uint32_t order_bucket(uint32_t len) {
  uint32_t key = 0;   // non-decreasing in len
  if (len) {
    const uint32_t lg = 31u - __clz(len);
    const uint32_t two = lg >= 2u ? (len >> (lg - 2u)) & 3u : (len << (2u - lg)) & 3u;
    key = 4u * lg + two;
    if (key > (uint32_t)kOrderBuckets - 1u) key = kOrderBuckets - 1u;
  }
  return (uint32_t)kOrderBuckets - 1u - key;
}

// Pairs in the tile list of warp item i (0 for a view without tiles or a tile past tile_cap).
__device__ inline uint32_t item_list_len(uint32_t i, const uint32_t* __restrict__ view_info, int n_views,
                                         const uint32_t* __restrict__ ranges, int64_t tile_cap) {
  const int v = find_view(view_info, n_views, i, 2);
  const uint32_t code = view_info[kVI * v + 3];
  const uint32_t wpt = ((code & 0xffu) * ((code >> 8) & 0xffu)) / 32u;   // items per tile
  if (!wpt) return 0u;
  const uint32_t tile = view_info[kVI * v] + (i - view_info[kVI * v + 2]) / wpt;
  if ((int64_t)tile >= tile_cap) return 0u;
  return ranges[2 * (size_t)tile + 1] - ranges[2 * (size_t)tile];
}

__global__ void k_order_zero(uint32_t* __restrict__ cnt) {   // counts and cursors
  for (int i = threadIdx.x; i < 2 * kOrderBuckets; i += blockDim.x) cnt[i] = 0u;
}

// Items per bucket (nothing when the batch has more than item_cap items).
__global__ void __launch_bounds__(kBlock) k_order_count(const uint32_t* __restrict__ view_info, int n_views,
                                                        const uint32_t* __restrict__ ranges, int64_t tile_cap,
                                                        int64_t item_cap, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t s_cnt[kOrderBuckets];
  for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_cnt[i] = 0u;
  __syncthreads();
  const int64_t n = view_info[kVI * n_views + 2];
  if (n <= item_cap) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      atomicAdd(&s_cnt[order_bucket(item_list_len((uint32_t)i, view_info, n_views, ranges, tile_cap))], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
}

// Every item to its bucket's next free position; one atomic per (warp, bucket).
__global__ void __launch_bounds__(kBlock) k_order_place(const uint32_t* __restrict__ view_info, int n_views,
                                                        const uint32_t* __restrict__ ranges, int64_t tile_cap,
                                                        int64_t item_cap, const uint32_t* __restrict__ cnt,
                                                        uint32_t* __restrict__ cur, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_base[kOrderBuckets];
  const int64_t n = view_info[kVI * n_views + 2];
  if (n > item_cap) return;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {   // exclusive scan of the bucket counts, two per lane
    const uint32_t a = cnt[2 * lane], b = cnt[2 * lane + 1];
    uint32_t x = a + b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    s_base[2 * lane] = x - a - b;
    s_base[2 * lane + 1] = x - b;
  }
  __syncthreads();
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = wid * 32; w0 < n; w0 += n_warps * 32) {   // warp-uniform loop
    const int64_t i = w0 + lane;
    const bool ok = i < n;
    const uint32_t b = ok ? order_bucket(item_list_len((uint32_t)i, view_info, n_views, ranges, tile_cap))
                          : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    uint32_t pos = 0;
    if (ok && lane == leader) pos = atomicAdd(&cur[b], (uint32_t)__popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (ok) order[s_base[b] + pos + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

}  // namespace

size_t bin_ws_bytes(int64_t rec_cap, int64_t pair_cap, int64_t tile_cap, int n_views) {
  const int K = chunks_per_view(n_views, tile_cap, pair_cap);
  const int64_t cnt_cap = (int64_t)K * tile_cap + 1;
  Carver c(nullptr);
  c.take<uint32_t>(n_views + 1);           // view segments
  c.take<uint32_t>(4);                     // counters
  c.take<uint32_t>(rec_cap);               // record keys a
  c.take<uint32_t>(rec_cap);               // record vals a
  c.take<uint32_t>(rec_cap);               // record keys b
  c.take<uint32_t>(rec_cap);               // record vals b
  c.take<ushort4>(rec_cap);                // rectangles in sorted order
  c.take<uint32_t>(rec_cap + 1);           // pair counts of the sorted records
  c.take<uint32_t>(rec_cap + 1);           // ... scanned: first pair of each sorted record
  c.take<uint32_t>(cnt_cap);               // per (tile, chunk) pair counts
  c.take<uint32_t>(cnt_cap);               // ... scanned
  c.take<uint32_t>((int64_t)n_views * (K + 1));   // first sorted record of every chunk
  c.take<uint32_t>(2 * kOrderBuckets);            // item order: bucket counts and cursors
  size_t t = sort_temp_bytes(rec_cap, n_views);
  size_t s = scan_temp_bytes(cnt_cap > rec_cap ? cnt_cap : rec_cap);
  c.take<char>(t > s ? t : s);
  return align_up(c.off, 256);
}

cudaError_t launch_bin_sort(const gs_proj& proj, const gs_camera* cams, int n_views, const gs_params& p,
                            const gs_bins& out, void* ws, cudaStream_t st) {
  (void)cams;
  (void)p;
  const int64_t rec_cap = proj.capacity, tile_cap = out.tile_capacity;
  const int K = chunks_per_view(n_views, tile_cap, out.pair_capacity);
  const int64_t cnt_cap = (int64_t)K * tile_cap + 1;
  Carver c(ws);
  uint32_t* seg = c.take<uint32_t>(n_views + 1);
  uint32_t* ctr = c.take<uint32_t>(4);      // [0] count entries to scan, [1] pair total
  uint32_t* rk_a = c.take<uint32_t>(rec_cap);
  uint32_t* rv_a = c.take<uint32_t>(rec_cap);
  uint32_t* rk_b = c.take<uint32_t>(rec_cap);
  uint32_t* rv_b = c.take<uint32_t>(rec_cap);
  ushort4* srect = c.take<ushort4>(rec_cap);
  uint32_t* rcnt = c.take<uint32_t>(rec_cap + 1);
  uint32_t* poff = c.take<uint32_t>(rec_cap + 1);
  uint32_t* cnt = c.take<uint32_t>(cnt_cap);
  uint32_t* off = c.take<uint32_t>(cnt_cap);
  uint32_t* bounds = c.take<uint32_t>((int64_t)n_views * (K + 1));
  uint32_t* ocnt = c.take<uint32_t>(2 * kOrderBuckets);
  size_t t = sort_temp_bytes(rec_cap, n_views);
  size_t s = scan_temp_bytes(cnt_cap > rec_cap ? cnt_cap : rec_cap);
  void* tmp = c.take<char>(t > s ? t : s);

  // 1. view segments (from the records' view ids, or from the projection's group offsets)
  if (!proj.view) {
    k_segments_from_groups<<<grid_for(n_views + 1), kBlock, 0, st>>>(proj, n_views, tile_cap, K, seg, &ctr[0]);
    note_launch();
  } else {
    k_zero_u32<<<grid_for(n_views + 1), kBlock, 0, st>>>(seg, n_views + 1);
    note_launch();
    k_segments<<<grid_for(rec_cap), kBlock, 0, st>>>(proj, n_views, tile_cap, K, seg, &ctr[0]);
    note_launch();
  }
  // 2. record indices by depth bits within each view (4 passes: result back in the a buffers)
  // (the last pass also writes the rectangles in sorted order and their pair counts)
  bool in_a = false;
  const SortRectEpilogue epi{reinterpret_cast<const ushort4*>(proj.rect), proj.view_info, srect, rcnt, proj.status};
  cudaError_t e = radix_sort(proj.depth_key, nullptr, SortBufs{rk_a, rv_a, rk_b, rv_b}, proj.count, rec_cap, 0, 32,
                             tmp, st, &in_a, seg, n_views, &epi);
  if (e != cudaSuccess) return e;
  const uint32_t* srec = in_a ? rv_a : rv_b;
  // 3. pair numbering
  e = scan_exclusive(rcnt, poff, proj.count, rec_cap, nullptr, tmp, st);
  if (e != cudaSuccess) return e;
  // 4. chunk boundaries, per-chunk tile counts
  k_chunk_bounds<<<grid_for((int64_t)n_views * (K + 1)), kBlock, 0, st>>>(seg, poff, n_views, K, bounds);
  note_launch();
  const int64_t chunks = (int64_t)n_views * K;
  const unsigned bin_grid = (unsigned)((chunks + kBinWarps - 1) / kBinWarps);
  k_bin_hist<<<bin_grid, kBinWarps * 32, 0, st>>>(proj, bounds, srect, n_views, K, tile_cap, cnt);
  note_launch();
  // 5. slots of every (tile, chunk); ranges and totals
  e = scan_exclusive(cnt, off, &ctr[0], cnt_cap - 1, &ctr[1], tmp, st);
  if (e != cudaSuccess) return e;
  k_bin_ranges<<<grid_for(tile_cap), kBlock, 0, st>>>(off, &ctr[0], &ctr[1], K, out.pair_capacity, tile_cap,
                                                      proj.view_info, n_views, out.ranges, out.count, proj.status);
  note_launch();
  // 6. placement
  if (out.tile)
    k_bin_place<true><<<bin_grid, kBinWarps * 32, 0, st>>>(proj, bounds, srec, srect, n_views, K, tile_cap, off, out);
  else
    k_bin_place<false><<<bin_grid, kBinWarps * 32, 0, st>>>(proj, bounds, srec, srect, n_views, K, tile_cap, off, out);
  note_launch();
  // 7. warp items longest tile list first, for the compositing kernels (optional)
  if (out.item_order && out.item_capacity > 0) {
    k_order_zero<<<1, 2 * kOrderBuckets, 0, st>>>(ocnt);
    note_launch();
    const unsigned og = grid_for(out.item_capacity);
    k_order_count<<<og, kBlock, 0, st>>>(proj.view_info, n_views, out.ranges, tile_cap, out.item_capacity, ocnt);
    note_launch();
    k_order_place<<<og, kBlock, 0, st>>>(proj.view_info, n_views, out.ranges, tile_cap, out.item_capacity, ocnt,
                                         ocnt + kOrderBuckets, out.item_order);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace gs
