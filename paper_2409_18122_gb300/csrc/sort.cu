// sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs whose
// count lives in device memory.
//
// Each 8-bit pass is reduce-then-scan: (1) every partition block counts its
// digits, (2) one block turns the per-partition counts into global digit
// offsets, (3) every partition block walks its tiles in order, ranks each key
// stably inside the tile with warp-level match, stages the tile in shared
// memory in digit order and writes it out at the running digit offsets.  No
// block ever waits on another, the result is deterministic, and the launch
// shape depends only on the host-side capacity.
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kItems = 8;
constexpr int kTile = kBlock * kItems;   // 2048 keys per tile
constexpr int kRadix = 256;
constexpr int kMaxParts = 2048;

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

// (1) digit counts of each partition: hist[part][digit]
__global__ void __launch_bounds__(kBlock) k_upsweep(const uint32_t* __restrict__ keys, const uint32_t* n_dev,
                                                     int64_t n_cap, int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[kWarps][kRadix];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kBlock) (&cnt[0][0])[i] = 0;
  __syncthreads();
  int64_t beg, end;
  part_range(count_of(n_dev, n_cap), beg, end);
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

// (3) stable scatter of each partition's tiles
__global__ void __launch_bounds__(kBlock) k_downsweep(const uint32_t* __restrict__ keys_in,
                                                       const uint32_t* __restrict__ vals_in,
                                                       uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                       const uint32_t* n_dev, int64_t n_cap, int shift,
                                                       const uint32_t* __restrict__ hist,
                                                       const uint32_t* __restrict__ digit_base) {
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
  base[tid] = digit_base[tid] + hist[(size_t)blockIdx.x * kRadix + tid];
  int64_t beg, end;
  part_range(count_of(n_dev, n_cap), beg, end);

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
    for (int j = tid; j < tile_n; j += kBlock) {
      const uint32_t k = s_keys[j];
      const uint32_t d = (k >> shift) & 0xffu;
      const uint32_t g = base[d] + (uint32_t)j - t_start[d];
      keys_out[g] = k;
      vals_out[g] = s_vals[j];
    }
    __syncthreads();
    base[tid] += t_cnt[tid];
    __syncthreads();
  }
}

constexpr size_t kDownSmem = sizeof(uint32_t) * (2 * kTile + kWarps * (kRadix + 1) + 3 * kRadix + kWarps);

}  // namespace

int sort_passes(int bit_begin, int bit_end) { return bit_end > bit_begin ? (bit_end - bit_begin + 7) / 8 : 0; }

size_t sort_temp_bytes(int64_t n_cap) {
  return align_up(sizeof(uint32_t) * kRadix * parts_for(n_cap), 256) + align_up(sizeof(uint32_t) * kRadix, 256);
}

cudaError_t radix_sort(const uint32_t* keys_in, const uint32_t* /*key_src*/, const uint32_t* vals_in, SortBufs b,
                       const uint32_t* n_dev, int64_t n_cap, int bit_begin, int bit_end, void* temp,
                       cudaStream_t st, bool* result_in_a) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDownSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int g = (int)parts_for(n_cap);
  Carver c(temp);
  uint32_t* hist = c.take<uint32_t>((size_t)kRadix * g);
  uint32_t* digit_base = c.take<uint32_t>(kRadix);
  const int passes = sort_passes(bit_begin, bit_end);
  const uint32_t* kin = keys_in;
  const uint32_t* vin = vals_in;
  for (int p = 0; p < passes; ++p) {
    const int shift = bit_begin + 8 * p;
    uint32_t* kout = (p % 2 == 0) ? b.keys_b : b.keys_a;
    uint32_t* vout = (p % 2 == 0) ? b.vals_b : b.vals_a;
    k_upsweep<<<g, kBlock, 0, st>>>(kin, n_dev, n_cap, shift, hist);
    note_launch();
    k_scan_hist<<<1, 1024, 0, st>>>(hist, g, digit_base);
    note_launch();
    k_downsweep<<<g, kBlock, kDownSmem, st>>>(kin, vin, kout, vout, n_dev, n_cap, shift, hist, digit_base);
    note_launch();
    kin = kout;
    vin = vout;
  }
  *result_in_a = (passes % 2 == 0);
  return cudaGetLastError();
}

}  // namespace gs
