// scan.cu -- device-wide exclusive prefix sum with a device-side element count.
//
// Reduce-then-scan in three launches (per-partition sums, scan of the sums,
// per-partition scan with carry).  Deterministic, no inter-block waiting, and
// the element count may live in device memory (known only after an earlier
// kernel), so the launch configuration depends only on the host-side capacity.
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 512;
constexpr int kItems = 8;
static_assert(kItems == 8, "the down-sweep moves each thread's items as two 16-byte vectors");
constexpr int kTile = kBlock * kItems;
constexpr int kMaxParts = 1024;

__host__ __device__ inline int64_t parts_for(int64_t n_cap) {
  int64_t g = (n_cap + kTile - 1) / kTile;
  if (g < 1) g = 1;
  if (g > kMaxParts) g = kMaxParts;
  return g;
}

__device__ inline int64_t chunk_for(int64_t n, int64_t g) {
  int64_t c = (n + g - 1) / g;
  return (c + kTile - 1) / kTile * kTile;
}

__device__ inline int64_t count_of(const uint32_t* n_dev, int64_t n_cap) {
  if (!n_dev) return n_cap;
  int64_t n = (int64_t)*n_dev;
  return n < n_cap ? n : n_cap;
}

__device__ inline uint32_t sat32(unsigned long long v) { return v > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)v; }

// Block-wide exclusive scan of one 64-bit value per thread (blockDim = kBlock).
__device__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long warp_sums[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kBlock / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < kBlock / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  unsigned long long before = warp > 0 ? warp_sums[warp - 1] : 0;
  *total = warp_sums[kBlock / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kBlock) k_scan_reduce(const uint32_t* __restrict__ in, const uint32_t* n_dev,
                                                         int64_t n_cap, unsigned long long* partial) {
  const int64_t n = count_of(n_dev, n_cap);
  const int64_t g = gridDim.x;
  const int64_t chunk = chunk_for(n, g);
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  int64_t end = beg + chunk;
  if (end > n) end = n;
  unsigned long long s = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += kBlock) s += in[i];
  unsigned long long tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long* partial, int g, const uint32_t* n_dev,
                                                        int64_t n_cap, uint32_t* out, uint32_t* total_out) {
  __shared__ unsigned long long sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long v = threadIdx.x < g ? partial[threadIdx.x] : 0, x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = sums[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    sums[lane] = w;
  }
  __syncthreads();
  unsigned long long incl = (warp > 0 ? sums[warp - 1] : 0) + x;
  if (threadIdx.x < g) partial[threadIdx.x] = incl - v;
  if (threadIdx.x == 0) {
    unsigned long long total = sums[31];
    int64_t n = count_of(n_dev, n_cap);
    out[n] = sat32(total);
    if (total_out) *total_out = sat32(total);
  }
}

__global__ void __launch_bounds__(kBlock) k_scan_down(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                       const uint32_t* n_dev, int64_t n_cap,
                                                       const unsigned long long* partial) {
  const int64_t n = count_of(n_dev, n_cap);
  const int64_t g = gridDim.x;
  const int64_t chunk = chunk_for(n, g);
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  int64_t end = beg + chunk;
  if (end > n) end = n;
  unsigned long long carry = partial[blockIdx.x];
  // 16-byte loads and stores when both arrays allow them (i0 is a multiple of 8 elements)
  const bool vec = (((uintptr_t)in | (uintptr_t)out) & 15u) == 0;
  for (int64_t t0 = beg; t0 < end; t0 += kTile) {
    uint32_t v[kItems];
    unsigned long long s = 0;
    const int64_t i0 = t0 + (int64_t)threadIdx.x * kItems;
    const bool full = vec && i0 + kItems <= end;
    if (full) {
      const uint4 a = reinterpret_cast<const uint4*>(in + i0)[0], b = reinterpret_cast<const uint4*>(in + i0)[1];
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < kItems; ++k) v[k] = (i0 + k < end) ? in[i0 + k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) s += v[k];
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan(s, &tot) + carry;
    uint32_t o[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      o[k] = sat32(ex);
      ex += v[k];
    }
    if (full) {
      reinterpret_cast<uint4*>(out + i0)[0] = make_uint4(o[0], o[1], o[2], o[3]);
      reinterpret_cast<uint4*>(out + i0)[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
      for (int k = 0; k < kItems; ++k)
        if (i0 + k < end) out[i0 + k] = o[k];
    }
    carry += tot;
  }
}

}  // namespace

size_t scan_temp_bytes(int64_t n_cap) { return align_up(sizeof(unsigned long long) * parts_for(n_cap), 256); }

cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, int64_t n_cap,
                           uint32_t* total_out, void* temp, cudaStream_t st) {
  const int g = (int)parts_for(n_cap);
  auto* partial = (unsigned long long*)temp;
  k_scan_reduce<<<g, kBlock, 0, st>>>(in, n_dev, n_cap, partial);
  note_launch();
  k_scan_partials<<<1, 1024, 0, st>>>(partial, g, n_dev, n_cap, out, total_out);
  note_launch();
  k_scan_down<<<g, kBlock, 0, st>>>(in, out, n_dev, n_cap, partial);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
