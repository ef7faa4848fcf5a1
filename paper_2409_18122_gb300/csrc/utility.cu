// utility.cu -- the render-free view utility of RT-GuIDE (Sec. IV-A / IV-B):
// per-Gaussian uncertainty from mean displacements, the high / low uncertainty
// classes, the batched view utility xi (Eq. view_util) and the mean uncertainty
// of cuboid regions.
//
// Visibility v(x, g) of a Gaussian's mean in a view is decided in FP32 with a
// fixed sequence of separately rounded IEEE operations (no fused multiply-add),
// so a plain float32 program can take the same decisions.  Per-view results are
// reduced per block into fixed slots and then in a fixed order: deterministic.
#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kViewChunk = 256;   // views whose partial results a block keeps in shared memory at once

// Camera constants of the visibility test: rotation, centre, intrinsics, image size.
struct VisCam {
  float R[9];
  float T[3];
  float fx, fy, cx, cy;
  float W, H;
};

__device__ inline void load_vis_cam(const gs_camera& g, VisCam& c) {
#pragma unroll
  for (int i = 0; i < 9; ++i) c.R[i] = g.R[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) c.T[i] = g.T[i];
  c.fx = g.fx;
  c.fy = g.fy;
  c.cx = g.cx;
  c.cy = g.cy;
  c.W = (float)g.width;
  c.H = (float)g.height;
}

// v(x, g): t = R^T (mu - T) with each product and sum rounded separately, in the
// order ((R0 dx + R3 dy) + R6 dz); visible iff near < t_z <= range and the
// projection (fx t_x / t_z + cx, fy t_y / t_z + cy) lies in [0, W) x [0, H).
__device__ __forceinline__ bool visible(float mx, float my, float mz, const VisCam& c, float near_plane,
                                        float range) {
  const float dx = __fsub_rn(mx, c.T[0]), dy = __fsub_rn(my, c.T[1]), dz = __fsub_rn(mz, c.T[2]);
  const float tz = __fadd_rn(__fadd_rn(__fmul_rn(c.R[2], dx), __fmul_rn(c.R[5], dy)), __fmul_rn(c.R[8], dz));
  if (!(tz > near_plane) || !(tz <= range)) return false;
  const float tx = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], dx), __fmul_rn(c.R[3], dy)), __fmul_rn(c.R[6], dz));
  const float ty = __fadd_rn(__fadd_rn(__fmul_rn(c.R[1], dx), __fmul_rn(c.R[4], dy)), __fmul_rn(c.R[7], dz));
  const float u = __fadd_rn(__fdiv_rn(__fmul_rn(c.fx, tx), tz), c.cx);
  const float v = __fadd_rn(__fdiv_rn(__fmul_rn(c.fy, ty), tz), c.cy);
  return u >= 0.f && u < c.W && v >= 0.f && v < c.H;
}

// u_i = |mu_cur - mu_prev| (or its square); unchanged means keep their u.
__global__ void k_uncertainty_update(const float4* __restrict__ mo_prev, const float4* __restrict__ mo_cur,
                                     float4* __restrict__ su, int64_t n, int squared) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = mo_prev[i], b = mo_cur[i];
    const float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y), dz = __fsub_rn(b.z, a.z);
    if (dx == 0.f && dy == 0.f && dz == 0.f) continue;
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    su[i].w = squared ? d2 : __fsqrt_rn(d2);
  }
}

// Fixed-order block sum of doubles; valid in thread 0.
__device__ double block_sum_d(double v, double* s) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
  __syncthreads();
  return t;
}

// Per block: sum of u over the block's Gaussians (pass 0), or of (u - mean)^2
// (pass 1), in a fixed order, into part[block].  Gaussians with mu_z < ground_z
// are left out.
__global__ void __launch_bounds__(kBlock) k_u_moments(const float4* __restrict__ mo, const float4* __restrict__ su,
                                                      int64_t n, float ground_z, const double* __restrict__ stats,
                                                      int pass, double* __restrict__ part) {
  __shared__ double s[kWarps];
  const double mean = pass ? stats[0] : 0.0;
  double acc = 0.0;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * per;
  int64_t i1 = i0 + per;
  if (i1 > n) i1 = n;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    if (!(mo[i].z >= ground_z)) continue;
    const double u = (double)su[i].w;
    acc += pass ? (u - mean) * (u - mean) : u;
  }
  const double t = block_sum_d(acc, s);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_u_count(const float4* __restrict__ mo, int64_t n, float ground_z, unsigned long long* cnt) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += (mo[i].z >= ground_z) ? 1ull : 0ull;
  for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// stats = (mean, sigma, t_high = mean + sigma/2, t_low = mean - sigma/2, count)
__global__ void k_u_finish(const double* __restrict__ part, int g, const unsigned long long* cnt, int pass,
                           double* __restrict__ stats) {
  double t = 0.0;
  for (int b = 0; b < g; ++b) t += part[b];
  const double m = (double)*cnt;
  if (pass == 0) {
    stats[0] = m > 0 ? t / m : 0.0;
    stats[4] = m;
  } else {
    const double sigma = m > 0 ? sqrt(t / m) : 0.0;
    stats[1] = sigma;
    stats[2] = stats[0] + 0.5 * sigma;
    stats[3] = stats[0] - 0.5 * sigma;
  }
}

// Per block and view: xi mode: count of visible high-uncertainty Gaussians minus
// lambda * count of visible low ones (both counted exactly as integers, combined in
// the final pass); sum mode: sum of u over the visible Gaussians.
template <bool kSum>
__global__ void __launch_bounds__(kBlock) k_view_utility(const float4* __restrict__ mo, const float4* __restrict__ su,
                                                         int64_t n, const gs_camera* __restrict__ cams, int v0, int nv,
                                                         gs_utility_params prm, const double* __restrict__ stats,
                                                         uint32_t* __restrict__ cnt_part, float* __restrict__ sum_part,
                                                         int n_views) {
  __shared__ VisCam s_cam[kViewChunk];
  __shared__ uint32_t s_hi[kWarps][kViewChunk];
  __shared__ uint32_t s_lo[kWarps][kViewChunk];
  __shared__ float s_sum[kWarps][kViewChunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) load_vis_cam(cams[v0 + i], s_cam[i]);
  for (int i = threadIdx.x; i < kWarps * kViewChunk; i += blockDim.x) {
    (&s_hi[0][0])[i] = 0u;
    (&s_lo[0][0])[i] = 0u;
    (&s_sum[0][0])[i] = 0.f;
  }
  __syncthreads();
  const double t_hi = kSum ? 0.0 : stats[2], t_lo = kSum ? 0.0 : stats[3];
  // this block's Gaussians, 32 per warp at a time
  const int64_t per = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const int64_t i0 = (int64_t)blockIdx.x * per;
  int64_t i1 = i0 + per;
  if (i1 > n) i1 = n;
  for (int64_t base = i0 + warp * 32; base < i1; base += kBlock) {
    const int64_t i = base + lane;
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    float u = 0.f;
    bool use = false;
    if (i < i1) {
      m = mo[i];
      u = su[i].w;
      use = m.z >= prm.ground_z;
    }
    const bool hi = use && !kSum && (double)u > t_hi;
    const bool lo = use && !kSum && (double)u < t_lo;
    const bool any = __any_sync(0xffffffffu, kSum ? use : (hi || lo));
    if (!any) continue;
    for (int v = 0; v < nv; ++v) {
      const bool vis = (kSum ? use : (hi || lo)) && visible(m.x, m.y, m.z, s_cam[v], prm.near_plane, prm.range);
      if (kSum) {
        float s = vis ? u : 0.f;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
        if (lane == 0) s_sum[warp][v] += s;
      } else {
        const uint32_t bh = __ballot_sync(0xffffffffu, vis && hi), bl = __ballot_sync(0xffffffffu, vis && lo);
        if (lane == 0) {
          s_hi[warp][v] += __popc(bh);
          s_lo[warp][v] += __popc(bl);
        }
      }
    }
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const size_t o = (size_t)blockIdx.x * n_views + v0 + v;
    if (kSum) {
      float s = 0.f;
      for (int w = 0; w < kWarps; ++w) s += s_sum[w][v];
      sum_part[o] = s;
    } else {
      uint32_t h = 0, l = 0;
      for (int w = 0; w < kWarps; ++w) {
        h += s_hi[w][v];
        l += s_lo[w][v];
      }
      cnt_part[2 * o] = h;
      cnt_part[2 * o + 1] = l;
    }
  }
}

template <bool kSum>
__global__ void k_view_utility_finish(const uint32_t* __restrict__ cnt_part, const float* __restrict__ sum_part,
                                      int g, int n_views, float lambda, float* __restrict__ xi,
                                      uint32_t* __restrict__ counts) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  if (kSum) {
    float s = 0.f;
    for (int b = 0; b < g; ++b) s += sum_part[(size_t)b * n_views + v];
    xi[v] = s;
  } else {
    unsigned long long h = 0, l = 0;
    for (int b = 0; b < g; ++b) {
      h += cnt_part[2 * ((size_t)b * n_views + v)];
      l += cnt_part[2 * ((size_t)b * n_views + v) + 1];
    }
    xi[v] = (float)((double)h - (double)lambda * (double)l);
    if (counts) {
      counts[2 * v] = (uint32_t)h;
      counts[2 * v + 1] = (uint32_t)l;
    }
  }
}

// Mean uncertainty of cuboid regions: region (ix, iy, iz) with i = floor((mu - origin) / size)
// holds the Gaussians inside the grid; sums in FP64, counts exact.
__global__ void k_regions(const float4* __restrict__ mo, const float4* __restrict__ su, int64_t n,
                          gs_region_grid grid, double* __restrict__ sum, uint32_t* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 m = mo[i];
    const float fx = floorf(__fdiv_rn(__fsub_rn(m.x, grid.origin[0]), grid.size));
    const float fy = floorf(__fdiv_rn(__fsub_rn(m.y, grid.origin[1]), grid.size));
    const float fz = floorf(__fdiv_rn(__fsub_rn(m.z, grid.origin[2]), grid.size));
    if (!(fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)grid.dims[0] && fy < (float)grid.dims[1] &&
          fz < (float)grid.dims[2]))
      continue;
    const int64_t r = ((int64_t)fz * grid.dims[1] + (int64_t)fy) * grid.dims[0] + (int64_t)fx;
    atomicAdd(&sum[r], (double)su[i].w);
    atomicAdd(&count[r], 1u);
  }
}

__global__ void k_region_mean(const double* __restrict__ sum, const uint32_t* __restrict__ count, int64_t n_reg,
                              float* __restrict__ omega) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reg; r += (int64_t)gridDim.x * blockDim.x)
    omega[r] = count[r] ? (float)(sum[r] / (double)count[r]) : 0.f;
}

// Trajectory information (Eq. traj_utility): per trajectory the sum over its states
// of xi (states l = 0..L in order, FP64), and the first trajectory with the largest sum.
__global__ void k_traj_sum(const float* __restrict__ xi, int n_traj, int n_states, float* __restrict__ out,
                           int32_t* __restrict__ best) {
  __shared__ double s_best[256];
  __shared__ int s_idx[256];
  double bv = -INFINITY;
  int bi = 0x7fffffff;
  for (int t = threadIdx.x; t < n_traj; t += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < n_states; ++l) acc += (double)xi[(size_t)t * n_states + l];
    out[t] = (float)acc;
    if (acc > bv) { bv = acc; bi = t; }
  }
  s_best[threadIdx.x] = bv;
  s_idx[threadIdx.x] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -INFINITY;
    int i = 0x7fffffff;
    for (int k = 0; k < (int)blockDim.x; ++k)
      if (s_best[k] > v || (s_best[k] == v && s_idx[k] < i)) { v = s_best[k]; i = s_idx[k]; }
    *best = n_traj > 0 ? i : -1;
  }
}

// Collision check (Sec. IV-B): ordered integer key of a float, so that unsigned
// minimum = float minimum.
__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

constexpr int kColChunk = 4096;   // Gaussians per block of the collision kernel
constexpr int kColTile = 256;     // Gaussians staged in shared memory at a time

// Per block: a chunk of Gaussians against every test point (one point per thread,
// the Gaussians broadcast from shared memory).  Each thread keeps its point's
// smallest margin |p - mu| - gamma (a square root only when the pair can beat it)
// and whether some Gaussian has |p - mu|^2 < gamma^2 (separately rounded FP32).
__global__ void __launch_bounds__(kBlock) k_collision(const float4* __restrict__ mo, const float4* __restrict__ su,
                                                      int64_t n, const float4* __restrict__ pts, int n_pts,
                                                      float r_robot, float lambda_g, float ground_z,
                                                      uint32_t* __restrict__ margin_key, uint32_t* __restrict__ hit) {
  __shared__ float4 s_g[kColTile];   // (mu, gamma)
  const int64_t g0 = (int64_t)blockIdx.x * kColChunk;
  int64_t g1 = g0 + kColChunk;
  if (g1 > n) g1 = n;
  for (int p0 = 0; p0 < n_pts; p0 += kBlock) {
    const int pi = p0 + threadIdx.x;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pi < n_pts) p = pts[pi];
    float best = INFINITY;
    bool col = false;
    for (int64_t t0 = g0; t0 < g1; t0 += kColTile) {
      __syncthreads();
      const int64_t gi = t0 + threadIdx.x;
      float4 e = make_float4(0.f, 0.f, 0.f, -1.f);   // gamma < 0: no Gaussian
      if (gi < g1) {
        const float4 m = mo[gi];
        if (m.z >= ground_z) {
          const float4 s = su[gi];
          const float r = ex32(fmaxf(fmaxf(s.x, s.y), s.z));   // principal axis
          e = make_float4(m.x, m.y, m.z, __fadd_rn(r_robot, __fmul_rn(lambda_g, r)));
        }
      }
      s_g[threadIdx.x] = e;
      __syncthreads();
      const int cnt = (int)(g1 - t0 < kColTile ? g1 - t0 : kColTile);
      if (pi < n_pts) {
        for (int k = 0; k < cnt; ++k) {
          const float4 g = s_g[k];
          if (!(g.w >= 0.f)) continue;
          const float dx = __fsub_rn(p.x, g.x), dy = __fsub_rn(p.y, g.y), dz = __fsub_rn(p.z, g.z);
          const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
          col |= d2 < __fmul_rn(g.w, g.w);
          const float lim = g.w + best;   // a smaller margin needs |p - mu| < gamma + best
          if (lim > 0.f && d2 < lim * lim) best = fminf(best, sqrtf(d2) - g.w);
        }
      }
    }
    if (pi < n_pts) {
      if (best < INFINITY) atomicMin(&margin_key[pi], fkey(best));
      if (col) atomicOr(&hit[pi], 1u);
    }
  }
}

__global__ void k_collision_init(uint32_t* __restrict__ margin_key, uint32_t* __restrict__ hit, int n_pts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pts; i += (int64_t)gridDim.x * blockDim.x) {
    margin_key[i] = fkey(INFINITY);
    hit[i] = 0u;
  }
}

__global__ void k_collision_finish(uint32_t* __restrict__ margin, int n_pts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pts; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = margin[i];
    reinterpret_cast<float*>(margin)[i] = fkey_inv(k);
  }
}

__global__ void k_zero_bytes(uint8_t* p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0;
}

int utility_grid() { return 2 * device_sm_count(); }

}  // namespace

cudaError_t launch_uncertainty_update(const float* mo_prev, const float* mo_cur, float* su, int64_t n, int squared,
                                      cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > 4096) g = 4096;
  k_uncertainty_update<<<(unsigned)g, kBlock, 0, st>>>(reinterpret_cast<const float4*>(mo_prev),
                                                       reinterpret_cast<const float4*>(mo_cur),
                                                       reinterpret_cast<float4*>(su), n, squared);
  note_launch();
  return cudaGetLastError();
}

size_t thresholds_ws_bytes() {
  return align_up(sizeof(double) * 1024, 256) + align_up(sizeof(unsigned long long) * 2, 256);
}

cudaError_t launch_uncertainty_thresholds(const float* mo, const float* su, int64_t n, float ground_z, double* stats,
                                          void* ws, cudaStream_t st) {
  Carver c(ws);
  double* part = c.take<double>(1024);
  unsigned long long* cnt = c.take<unsigned long long>(2);
  int g = utility_grid();
  if (g > 1024) g = 1024;
  k_zero_bytes<<<1, 32, 0, st>>>(reinterpret_cast<uint8_t*>(cnt), sizeof(unsigned long long) * 2);
  note_launch();
  k_u_count<<<g, kBlock, 0, st>>>(reinterpret_cast<const float4*>(mo), n, ground_z, cnt);
  note_launch();
  for (int pass = 0; pass < 2; ++pass) {
    k_u_moments<<<g, kBlock, 0, st>>>(reinterpret_cast<const float4*>(mo), reinterpret_cast<const float4*>(su), n,
                                      ground_z, stats, pass, part);
    note_launch();
    k_u_finish<<<1, 1, 0, st>>>(part, g, cnt, pass, stats);
    note_launch();
  }
  return cudaGetLastError();
}

size_t utility_ws_bytes(int n_views) {
  const int g = 1024;
  return align_up(sizeof(uint32_t) * 2 * (size_t)g * n_views, 256) + align_up(sizeof(float) * (size_t)g * n_views, 256);
}

cudaError_t launch_view_utility(const float* mo, const float* su, int64_t n, const gs_camera* cams, int n_views,
                                const gs_utility_params& prm, int mode, const double* stats, float* xi,
                                uint32_t* counts, void* ws, cudaStream_t st) {
  Carver c(ws);
  uint32_t* cnt_part = c.take<uint32_t>(2 * (size_t)1024 * n_views);
  float* sum_part = c.take<float>((size_t)1024 * n_views);
  int g = utility_grid();
  if (g > 1024) g = 1024;
  const bool sum = mode == GS_XI_SUM;
  for (int v0 = 0; v0 < n_views; v0 += kViewChunk) {
    const int nv = n_views - v0 < kViewChunk ? n_views - v0 : kViewChunk;
    if (sum)
      k_view_utility<true><<<g, kBlock, 0, st>>>(reinterpret_cast<const float4*>(mo),
                                                 reinterpret_cast<const float4*>(su), n, cams, v0, nv, prm, stats,
                                                 cnt_part, sum_part, n_views);
    else
      k_view_utility<false><<<g, kBlock, 0, st>>>(reinterpret_cast<const float4*>(mo),
                                                  reinterpret_cast<const float4*>(su), n, cams, v0, nv, prm, stats,
                                                  cnt_part, sum_part, n_views);
    note_launch();
  }
  const int fb = (n_views + 255) / 256;
  if (sum) k_view_utility_finish<true><<<fb, 256, 0, st>>>(cnt_part, sum_part, g, n_views, prm.lambda, xi, counts);
  else k_view_utility_finish<false><<<fb, 256, 0, st>>>(cnt_part, sum_part, g, n_views, prm.lambda, xi, counts);
  note_launch();
  return cudaGetLastError();
}

size_t regions_ws_bytes(int64_t n_regions) {
  return align_up(sizeof(double) * (size_t)n_regions, 256) + align_up(sizeof(uint32_t) * (size_t)n_regions, 256);
}

cudaError_t launch_regions(const float* mo, const float* su, int64_t n, const gs_region_grid& grid, float* omega,
                           uint32_t* count_out, void* ws, cudaStream_t st) {
  const int64_t nr = (int64_t)grid.dims[0] * grid.dims[1] * grid.dims[2];
  Carver c(ws);
  double* sum = c.take<double>((size_t)nr);
  uint32_t* cnt = c.take<uint32_t>((size_t)nr);
  if (count_out) cnt = count_out;
  int64_t zb = ((int64_t)sizeof(double) * nr + 255) / 256;
  if (zb > 4096) zb = 4096;
  k_zero_bytes<<<(unsigned)(zb < 1 ? 1 : zb), 256, 0, st>>>(reinterpret_cast<uint8_t*>(sum), sizeof(double) * nr);
  note_launch();
  k_zero_bytes<<<(unsigned)(zb < 1 ? 1 : zb), 256, 0, st>>>(reinterpret_cast<uint8_t*>(cnt), sizeof(uint32_t) * nr);
  note_launch();
  if (n > 0) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_regions<<<(unsigned)g, 256, 0, st>>>(reinterpret_cast<const float4*>(mo), reinterpret_cast<const float4*>(su),
                                            n, grid, sum, cnt);
    note_launch();
  }
  int64_t g2 = (nr + 255) / 256;
  if (g2 > 4096) g2 = 4096;
  k_region_mean<<<(unsigned)(g2 < 1 ? 1 : g2), 256, 0, st>>>(sum, cnt, nr, omega);
  note_launch();
  return cudaGetLastError();
}

size_t trajectory_ws_bytes(int n_states_total) {
  return utility_ws_bytes(n_states_total) + align_up(sizeof(float) * (size_t)n_states_total, 256);
}

cudaError_t launch_trajectory_utility(const float* mo, const float* su, int64_t n, const gs_camera* cams, int n_traj,
                                      int n_states, const gs_utility_params& prm, int mode, const double* stats,
                                      float* traj_out, int32_t* best_out, void* ws, cudaStream_t st) {
  const int total = n_traj * n_states;
  Carver c(ws);
  void* uws = c.take<char>(utility_ws_bytes(total));
  float* xi = c.take<float>((size_t)total);
  cudaError_t e = launch_view_utility(mo, su, n, cams, total, prm, mode, stats, xi, nullptr, uws, st);
  if (e != cudaSuccess) return e;
  k_traj_sum<<<1, 256, 0, st>>>(xi, n_traj, n_states, traj_out, best_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_collision_check(const float* mo, const float* su, int64_t n, const float* pts, int n_pts,
                                   float r_robot, float lambda_g, float ground_z, float* margin_out,
                                   uint32_t* collides_out, cudaStream_t st) {
  uint32_t* key = reinterpret_cast<uint32_t*>(margin_out);
  const int ib = (n_pts + 255) / 256;
  k_collision_init<<<ib < 1 ? 1 : ib, 256, 0, st>>>(key, collides_out, n_pts);
  note_launch();
  if (n > 0 && n_pts > 0) {
    const int64_t blocks = (n + kColChunk - 1) / kColChunk;
    k_collision<<<(unsigned)blocks, kBlock, 0, st>>>(reinterpret_cast<const float4*>(mo),
                                                     reinterpret_cast<const float4*>(su), n,
                                                     reinterpret_cast<const float4*>(pts), n_pts, r_robot, lambda_g,
                                                     ground_z, key, collides_out);
    note_launch();
  }
  k_collision_finish<<<ib < 1 ? 1 : ib, 256, 0, st>>>(key, n_pts);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
