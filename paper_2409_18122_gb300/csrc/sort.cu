// sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs whose
// count lives in device memory.
//
// Each 8-bit pass is reduce-then-scan: (1) every partition block counts its
// digits, (2) one block turns the per-partition counts into global digit
// offsets, (3) every partition block walks its tiles in order, ranks each key
// stably inside the tile with warp ballots, stages the tile in shared
// memory in digit order and writes it out at the running digit offsets.  No
// block ever waits on another, the result is deterministic, and the launch
// shape depends only on the host-side capacity.
//
// Segmented mode: the input is cut into contiguous segments (the records of
// one view each); partitions never cross a segment and digit offsets are
// scanned per segment, so every pass keeps each segment in place and the
// result is sorted within each segment.
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kItems = 8;
constexpr int kTile = kBlock * kItems;   // 2048 keys per tile
constexpr int kRadix = 256;
// Partitions of a large sort.  More, smaller partitions keep the blocks that run at the same
// time on fewer segments, so the last pass of a binning sort, which gathers each record's
// rectangle by record index within its view, finds them in L2: at 2,048 / 4,096 / 8,192 /
// 16,384 / 32,768 partitions the binning of a 256-view batch took 3.80 / 3.56 / 3.52 / 3.61 /
// 3.89 ms (per-partition histograms and scans grow with the count).
constexpr int kMaxParts = 8192;

inline int64_t parts_for(int64_t n_cap) {
  int64_t g = (n_cap + kTile - 1) / kTile;
  if (g < 1) g = 1;
  if (g > kMaxParts) g = kMaxParts;
  return g;
}

__device__ inline int64_t count_of(const uint32_t* n_dev, int64_t n_cap) {
  int64_t n = (int64_t)*n_dev;
  return n < n_cap ? n : n_cap;
}

__device__ inline void part_range(int64_t n, int64_t& beg, int64_t& end) {
  const int64_t g = gridDim.x;
  int64_t chunk = (n + g - 1) / g;
  chunk = (chunk + kTile - 1) / kTile * kTile;
  beg = (int64_t)blockIdx.x * chunk;
  end = beg + chunk;
  if (end > n) end = n;
  if (beg > n) beg = n;
}

// Segmented partition map: pmap[0] = partition size, pmap[1 + s] = first
// partition of segment s (s = 0 .. n_seg).  Segment s of n_s elements gets
// ceil(n_s / size) partitions; size is chosen so that all fit in the grid.
__global__ void __launch_bounds__(1024) k_part_map(const uint32_t* __restrict__ seg, int n_seg, const uint32_t* n_dev,
                                                   int64_t n_cap, int grid, uint32_t* __restrict__ pmap) {
  __shared__ unsigned long long s_sum[32];
  const int64_t n = count_of(n_dev, n_cap);
  const int64_t avail = grid - n_seg > 1 ? grid - n_seg : 1;
  int64_t size = (n + avail - 1) / avail;
  size = (size + kTile - 1) / kTile * kTile;
  if (size < kTile) size = kTile;
  const int per = (n_seg + blockDim.x - 1) / blockDim.x;
  const int s0 = threadIdx.x * per;
  int s1 = s0 + per;
  if (s1 > n_seg) s1 = n_seg;
  unsigned long long acc = 0;
  for (int t = s0; t < s1; ++t) {
    const int64_t a = seg[t], b = seg[t + 1];
    if (b > a) acc += (unsigned long long)((b - a + size - 1) / size);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = acc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_sum[warp] = x;
  __syncthreads();
  unsigned long long e = x - acc;
  for (int w = 0; w < warp; ++w) e += s_sum[w];
  for (int t = s0; t < s1; ++t) {
    pmap[1 + t] = (uint32_t)e;
    const int64_t a = seg[t], b = seg[t + 1];
    if (b > a) e += (unsigned long long)((b - a + size - 1) / size);
  }
  if (threadIdx.x == blockDim.x - 1) pmap[1 + n_seg] = (uint32_t)e;
  if (threadIdx.x == 0) pmap[0] = (uint32_t)size;
}

// Element range of this block's partition (segmented mode): empty past the last.
// Returns the partition's segment.
__device__ inline int seg_part_range(const uint32_t* __restrict__ seg, int n_seg, const uint32_t* __restrict__ pmap,
                                     int64_t& beg, int64_t& end) {
  const int64_t p = blockIdx.x;
  beg = end = 0;
  if (p >= (int64_t)pmap[1 + n_seg]) return 0;
  int lo = 0, hi = n_seg - 1;   // segment: the largest s with first partition <= p
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)pmap[1 + mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  const int64_t size = pmap[0];
  const int64_t a = seg[lo], b = seg[lo + 1];
  beg = a + (p - (int64_t)pmap[1 + lo]) * size;
  end = beg + size;
  if (end > b) end = b;
  if (beg > end) beg = end;
  return lo;
}

// (1) digit counts of each partition: hist[part][digit]
__global__ void __launch_bounds__(kBlock) k_upsweep(const uint32_t* __restrict__ keys,
                                                     const uint32_t* __restrict__ seg, int n_seg,
                                                     const uint32_t* __restrict__ pmap, const uint32_t* n_dev,
                                                     int64_t n_cap, int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kWarps][kRadix];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kBlock) (&cnt[0][0])[i] = 0;
  __syncthreads();
  int64_t beg, end;
  if (pmap) seg_part_range(seg, n_seg, pmap, beg, end);
  else part_range(count_of(n_dev, n_cap), beg, end);
  for (int64_t i = beg + threadIdx.x; i < end; i += kBlock) {
    uint32_t d = (keys[i] >> shift) & 0xffu;
    atomicAdd(&cnt[warp][d], 1u);
  }
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += cnt[w][threadIdx.x];
  hist[(size_t)blockIdx.x * kRadix + threadIdx.x] = s;
}

// (2) hist[part][digit] -> exclusive prefix over parts per digit (in place);
// digit_base[digit] = exclusive prefix of the digit totals.  32 warps; warp w
// owns a contiguous range of parts, lane l owns digits l, l+32, ..., l+224, so
// every load is coalesced and independent of the previous one.
__global__ void __launch_bounds__(1024) k_scan_hist(uint32_t* __restrict__ hist, int g, uint32_t* digit_base) {
  __shared__ uint32_t wtot[32][kRadix];   // per-warp digit totals, then per-warp offsets
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (g + 31) / 32;
  const int p0 = warp * per;
  int p1 = p0 + per;
  if (p1 > g) p1 = g;
  uint32_t run[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) run[k] = 0;
  for (int p = p0; p < p1; ++p) {
#pragma unroll
    for (int k = 0; k < 8; ++k) run[k] += hist[(size_t)p * kRadix + lane + 32 * k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) wtot[warp][lane + 32 * k] = run[k];
  __syncthreads();
  // per digit: exclusive scan over the 32 warps (thread d < 256), digit totals, then digit bases
  __shared__ uint32_t dtot[kRadix];
  if (threadIdx.x < kRadix) {
    const int d = threadIdx.x;
    uint32_t acc = 0;
    for (int w = 0; w < 32; ++w) {
      const uint32_t c = wtot[w][d];
      wtot[w][d] = acc;
      acc += c;
    }
    dtot[d] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive scan of the 256 digit totals by one warp (8 per lane)
    uint32_t v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) { v[k] = dtot[lane * 8 + k]; s += v[k]; }
    uint32_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    uint32_t ex = x - s;
#pragma unroll
    for (int k = 0; k < 8; ++k) { digit_base[lane * 8 + k] = ex; ex += v[k]; }
  }
  // second sweep: each part's per-digit exclusive prefix
#pragma unroll
  for (int k = 0; k < 8; ++k) run[k] = wtot[warp][lane + 32 * k];
  for (int p = p0; p < p1; ++p) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const size_t i = (size_t)p * kRadix + lane + 32 * k;
      const uint32_t c = hist[i];
      hist[i] = run[k];
      run[k] += c;
    }
  }
}

// (2, segmented) one block per segment s: hist[part][digit] of the segment's
// partitions -> seg[s] + (elements of smaller digits in the segment) + (elements
// of this digit in earlier partitions of the segment), i.e. absolute offsets.
// Partitions are read 8 at a time so that the loads overlap.
__global__ void __launch_bounds__(kRadix) k_scan_hist_seg(uint32_t* __restrict__ hist, int g,
                                                          const uint32_t* __restrict__ seg,
                                                          const uint32_t* __restrict__ pmap) {
  __shared__ uint32_t s_tot[kRadix];
  const int s = blockIdx.x, d = threadIdx.x;
  // (malformed segments can ask for more partitions than the grid has: those are never run)
  const int64_t p0 = pmap[1 + s] < (uint32_t)g ? pmap[1 + s] : g;
  const int64_t p1 = pmap[2 + s] < (uint32_t)g ? pmap[2 + s] : g;
  uint32_t tot = 0;
  for (int64_t p = p0; p < p1; p += 8) {
    uint32_t c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = p + k < p1 ? hist[(size_t)(p + k) * kRadix + d] : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += c[k];
  }
  s_tot[d] = tot;
  __syncthreads();
  // exclusive scan of the digit totals (256 threads, 8 warps)
  const int lane = d & 31, warp = d >> 5;
  uint32_t x = tot;
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, k);
    if (lane >= k) x += y;
  }
  __syncthreads();
  if (lane == 31) s_tot[warp] = x;
  __syncthreads();
  uint32_t run = seg[s] + x - tot;
  for (int w = 0; w < warp; ++w) run += s_tot[w];
  for (int64_t p = p0; p < p1; p += 8) {
    uint32_t c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = p + k < p1 ? hist[(size_t)(p + k) * kRadix + d] : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (p + k < p1) hist[(size_t)(p + k) * kRadix + d] = run;
      run += c[k];
    }
  }
}

// (3) stable scatter of each partition's tiles (kEpi: the last pass of a binning
// sort, see SortRectEpilogue).  Four blocks per SM fit in 64 registers without spilling;
// at the unbounded 76-80 registers only three did, and the binning of a 256-view batch took
// 3.46 instead of 3.35 ms.
template <bool kEpi>
__global__ void __launch_bounds__(kBlock, 4) k_downsweep(const uint32_t* __restrict__ keys_in,
                                                       const uint32_t* __restrict__ vals_in,
                                                       const uint32_t* __restrict__ seg, int n_seg,
                                                       const uint32_t* __restrict__ pmap,
                                                       uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                       const uint32_t* n_dev, int64_t n_cap, int shift,
                                                       const uint32_t* __restrict__ hist,
                                                       const uint32_t* __restrict__ digit_base,
                                                       const SortRectEpilogue epi) {
  extern __shared__ uint32_t smem[];
  uint32_t* s_keys = smem;                              // kTile
  uint32_t* s_vals = s_keys + kTile;                    // kTile
  uint32_t* whist = s_vals + kTile;                     // kWarps * (kRadix + 1)
  uint32_t* t_cnt = whist + kWarps * (kRadix + 1);      // kRadix
  uint32_t* t_start = t_cnt + kRadix;                   // kRadix
  uint32_t* base = t_start + kRadix;                    // kRadix
  uint32_t* wsum = base + kRadix;                       // kWarps

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  int64_t beg, end;
  int segment = 0;
  if (pmap) {
    base[tid] = hist[(size_t)blockIdx.x * kRadix + tid];   // already absolute
    segment = seg_part_range(seg, n_seg, pmap, beg, end);
  } else {
    base[tid] = digit_base[tid] + hist[(size_t)blockIdx.x * kRadix + tid];
    part_range(count_of(n_dev, n_cap), beg, end);
  }

  uint32_t tiles_x = 0, tiles_y = 0;   // epilogue: the tile grid of this partition's view
  if (kEpi) {
    tiles_x = epi.view_info[4 * segment + 3] >> 16;
    const uint32_t nt = epi.view_info[4 * (segment + 1)] - epi.view_info[4 * segment];
    tiles_y = tiles_x ? nt / tiles_x : 0u;
  }
  // the keys/values of the next tile are loaded while the current one is ranked and scattered
  uint32_t nkey[kItems], nval[kItems];
  auto load_tile = [&](int64_t t0) {
    const int tn = (int)((end - t0) < kTile ? (end - t0) : kTile);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int li = warp * (kTile / kWarps) + i * 32 + lane;
      const bool ok = li < tn;
      nkey[i] = ok ? keys_in[t0 + li] : 0u;
      nval[i] = ok ? (vals_in ? vals_in[t0 + li] : (uint32_t)(t0 + li)) : 0u;
    }
  };
  if (beg < end) load_tile(beg);
  for (int64_t t0 = beg; t0 < end; t0 += kTile) {
    const int tile_n = (int)((end - t0) < kTile ? (end - t0) : kTile);
    uint32_t key[kItems], val[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      key[i] = nkey[i];
      val[i] = nval[i];
    }
    if (t0 + kTile < end) load_tile(t0 + kTile);
    for (int i = tid; i < kWarps * (kRadix + 1); i += kBlock) whist[i] = 0;
    __syncthreads();
    uint16_t rank[kItems];
    uint32_t* wh = whist + warp * (kRadix + 1);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int li = warp * (kTile / kWarps) + i * 32 + lane;
      const bool ok = li < tile_n;
      const uint32_t d = ok ? ((key[i] >> shift) & 0xffu) : (uint32_t)kRadix;
      // lanes holding the same digit: intersect the 8 digit-bit ballots (and validity)
      uint32_t peers = __ballot_sync(0xffffffffu, ok);
      if (!ok) peers = ~peers;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bb = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bb : ~bb;
      }
      const uint32_t before = wh[d];
      rank[i] = (uint16_t)(before + __popc(peers & lt_mask));
      __syncwarp();
      if ((peers & lt_mask) == 0 && ok) wh[d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: warp-exclusive offsets in place, tile totals
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        uint32_t c = whist[w * (kRadix + 1) + tid];
        whist[w * (kRadix + 1) + tid] = run;
        run += c;
      }
      t_cnt[tid] = run;
      // exclusive scan of tile totals over digits
      uint32_t x = run;
#pragma unroll
      for (int s2 = 1; s2 < 32; s2 <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, s2);
        if (lane >= s2) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncthreads();
      uint32_t before = 0;
      for (int w = 0; w < warp; ++w) before += wsum[w];
      t_start[tid] = before + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int li = warp * (kTile / kWarps) + i * 32 + lane;
      if (li < tile_n) {
        const uint32_t d = (key[i] >> shift) & 0xffu;
        const uint32_t pos = t_start[d] + whist[warp * (kRadix + 1) + d] + rank[i];
        s_keys[pos] = key[i];
        s_vals[pos] = val[i];
      }
    }
    __syncthreads();
    if (!kEpi) {
#pragma unroll
      for (int it = 0; it < kItems; ++it) {
        const int j = tid + it * kBlock;
        if (j >= tile_n) break;
        const uint32_t k = s_keys[j];
        const uint32_t d = (k >> shift) & 0xffu;
        const uint32_t g = base[d] + (uint32_t)j - t_start[d];
        vals_out[g] = s_vals[j];
        keys_out[g] = k;
      }
    } else {
      // all of this thread's rectangle gathers first, so that they are in flight together
      // (the stores below go to other arrays, but the compiler cannot know that)
      ushort4 rcs[kItems];
#pragma unroll
      for (int it = 0; it < kItems; ++it) {
        const int j = tid + it * kBlock;
        rcs[it] = j < tile_n ? epi.rect[s_vals[j]] : make_ushort4(0, 0, 0, 0);
      }
#pragma unroll
      for (int it = 0; it < kItems; ++it) {
        const int j = tid + it * kBlock;
        if (j >= tile_n) break;
        const uint32_t k = s_keys[j];
        const uint32_t d = (k >> shift) & 0xffu;
        const uint32_t g = base[d] + (uint32_t)j - t_start[d];
        vals_out[g] = s_vals[j];
        ushort4 rc = rcs[it];
        uint32_t c = 0;
        if (rc.x < rc.z && rc.y < rc.w) {
          if (rc.z <= tiles_x && rc.w <= tiles_y) c = (uint32_t)(rc.z - rc.x) * (uint32_t)(rc.w - rc.y);
          else atomicOr(epi.status, (uint32_t)GS_FLAG_BAD_RECORDS);
        }
        if (c == 0) rc = make_ushort4(0, 0, 0, 0);
        epi.out_rect[g] = rc;
        epi.out_cnt[g] = c;
      }
    }
    __syncthreads();
    base[tid] += t_cnt[tid];
    __syncthreads();
  }
}

constexpr size_t kDownSmem = sizeof(uint32_t) * (2 * kTile + kWarps * (kRadix + 1) + 3 * kRadix + kWarps);

}  // namespace

int sort_passes(int bit_begin, int bit_end) { return bit_end > bit_begin ? (bit_end - bit_begin + 7) / 8 : 0; }

size_t sort_temp_bytes(int64_t n_cap, int n_seg) {
  const int64_t g = parts_for(n_cap) + (n_seg > 1 ? n_seg : 0);
  return align_up(sizeof(uint32_t) * kRadix * g, 256) + align_up(sizeof(uint32_t) * kRadix, 256) +
         align_up(sizeof(uint32_t) * (n_seg + 2), 256);
}

cudaError_t radix_sort(const uint32_t* keys_in, const uint32_t* vals_in, SortBufs b, const uint32_t* n_dev,
                       int64_t n_cap, int bit_begin, int bit_end, void* temp, cudaStream_t st, bool* result_in_a,
                       const uint32_t* seg, int n_seg, const SortRectEpilogue* epi) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_downsweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDownSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_downsweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDownSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const SortRectEpilogue no_epi{nullptr, nullptr, nullptr, nullptr, nullptr};
  const bool segmented = seg && n_seg > 1;   // one segment sorts like the plain mode
  const int g = (int)(parts_for(n_cap) + (segmented ? n_seg : 0));
  Carver c(temp);
  uint32_t* hist = c.take<uint32_t>((size_t)kRadix * g);
  uint32_t* digit_base = c.take<uint32_t>(kRadix);
  uint32_t* pmap = c.take<uint32_t>(n_seg + 2);
  if (segmented) {
    k_part_map<<<1, 1024, 0, st>>>(seg, n_seg, n_dev, n_cap, g, pmap);
    note_launch();
  } else {
    pmap = nullptr;
  }
  const int passes = sort_passes(bit_begin, bit_end);
  const uint32_t* kin = keys_in;
  const uint32_t* vin = vals_in;
  for (int p = 0; p < passes; ++p) {
    const int shift = bit_begin + 8 * p;
    uint32_t* kout = (p % 2 == 0) ? b.keys_b : b.keys_a;
    uint32_t* vout = (p % 2 == 0) ? b.vals_b : b.vals_a;
    k_upsweep<<<g, kBlock, 0, st>>>(kin, seg, n_seg, pmap, n_dev, n_cap, shift, hist);
    note_launch();
    if (segmented) k_scan_hist_seg<<<n_seg, kRadix, 0, st>>>(hist, g, seg, pmap);
    else k_scan_hist<<<1, 1024, 0, st>>>(hist, g, digit_base);
    note_launch();
    if (epi && p == passes - 1)
      k_downsweep<true><<<g, kBlock, kDownSmem, st>>>(kin, vin, seg, n_seg, pmap, kout, vout, n_dev, n_cap, shift,
                                                      hist, digit_base, *epi);
    else
      k_downsweep<false><<<g, kBlock, kDownSmem, st>>>(kin, vin, seg, n_seg, pmap, kout, vout, n_dev, n_cap, shift,
                                                       hist, digit_base, no_epi);
    note_launch();
    kin = kout;
    vin = vout;
  }
  *result_in_a = (passes % 2 == 0);
  return cudaGetLastError();
}

}  // namespace gs
