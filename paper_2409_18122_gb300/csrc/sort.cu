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
constexpr int kItems = 16;
constexpr int kTile = kBlock * kItems;   // 4096 keys per tile
constexpr int kRadix = 256;
constexpr int kMaxParts = 1024;

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
// digit_base[digit] = exclusive prefix of the digit totals.
__global__ void __launch_bounds__(1024) k_scan_hist(uint32_t* __restrict__ hist, int g, uint32_t* digit_base) {
  // 4 groups of 256 threads; group k handles parts [k*gs, (k+1)*gs)
  __shared__ uint32_t group_tot[4][kRadix];
  __shared__ uint32_t warp_tot[kWarps];
  const int d = threadIdx.x & (kRadix - 1);
  const int grp = threadIdx.x >> 8;
  const int gsz = (g + 3) / 4;
  const int p0 = grp * gsz;
  int p1 = p0 + gsz;
  if (p1 > g) p1 = g;
  uint32_t run = 0;
  for (int p = p0; p < p1; ++p) {
    uint32_t c = hist[(size_t)p * kRadix + d];
    hist[(size_t)p * kRadix + d] = run;
    run += c;
  }
  group_tot[grp][d] = run;
  __syncthreads();
  uint32_t add = 0;
  for (int k = 0; k < grp; ++k) add += group_tot[k][d];
  if (add)
    for (int p = p0; p < p1; ++p) hist[(size_t)p * kRadix + d] += add;
  if (grp == 0) {
    uint32_t tot = group_tot[0][d] + group_tot[1][d] + group_tot[2][d] + group_tot[3][d];
    // exclusive scan of tot over the 256 digits (threads 0..255)
    const int lane = d & 31, w = d >> 5;
    uint32_t x = tot;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
      if (lane >= s) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    asm volatile("bar.sync 1, 256;");
    uint32_t before = 0;
    for (int k = 0; k < w; ++k) before += warp_tot[k];
    digit_base[d] = before + x - tot;
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

  for (int64_t t0 = beg; t0 < end; t0 += kTile) {
    const int tile_n = (int)((end - t0) < kTile ? (end - t0) : kTile);
    for (int i = tid; i < kWarps * (kRadix + 1); i += kBlock) whist[i] = 0;
    __syncthreads();
    uint32_t key[kItems], val[kItems];
    uint16_t rank[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int li = warp * (kTile / kWarps) + i * 32 + lane;
      const bool ok = li < tile_n;
      key[i] = ok ? keys_in[t0 + li] : 0u;
      val[i] = ok ? (vals_in ? vals_in[t0 + li] : (uint32_t)(t0 + li)) : 0u;
    }
    uint32_t* wh = whist + warp * (kRadix + 1);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const int li = warp * (kTile / kWarps) + i * 32 + lane;
      const uint32_t d = li < tile_n ? ((key[i] >> shift) & 0xffu) : (uint32_t)kRadix;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = wh[d];
      rank[i] = (uint16_t)(before + __popc(peers & lt_mask));
      __syncwarp();
      if ((peers & lt_mask) == 0 && d < (uint32_t)kRadix) wh[d] = before + __popc(peers);
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
      for (int s = 1; s < 32; s <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
        if (lane >= s) x += y;
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
