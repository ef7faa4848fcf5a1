// project.cu -- gs_project: EWA projection of every Gaussian into every view.
//
// Sec. III of RT-GuIDE: mu_2D = K R^T (mu - T) / d, d = e3^T R^T (mu - T), with the
// anisotropic EWA covariance in place of the isotropic r_2D = f r / d.
//
// Gaussian-major: one thread per Gaussian reads its 64 bytes of parameters once
// (coalesced float4 SoA loads), computes the view-independent part (rotation,
// 3D covariance, opacity, support bound) once, and loops over the cameras held
// in shared memory.  Records are compacted in (view, Gaussian) order with two
// passes (count per (view, group of 32 Gaussians), exclusive scan, write), so the
// order is deterministic, the records of every view are contiguous, no block
// waits on another and every record store of a warp is coalesced.
#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool camera_ok(const gs_camera& c, int tw, int th) {
  return c.width > 0 && c.height > 0 && c.fx > 0.f && c.fy > 0.f && isfinite(c.fx) && isfinite(c.fy) &&
         valid_tile(tw, th);
}

// Per-view table: tile, pixel and warp-item offsets (prefix sums over views), tile
// sizes, camera checks.
__global__ void __launch_bounds__(1024) k_view_info(const gs_camera* __restrict__ cams, int n_views, int def_tw,
                                                    int def_th, uint32_t* __restrict__ view_info,
                                                    uint32_t* status) {
  __shared__ unsigned long long s_sum[3][32];
  const int per = (n_views + blockDim.x - 1) / blockDim.x;
  const int v0 = threadIdx.x * per;
  int v1 = v0 + per;
  if (v1 > n_views) v1 = n_views;
  unsigned long long acc[3] = {0, 0, 0};   // tiles, pixels, warp items
  bool bad = false;
  for (int v = v0; v < v1; ++v) {
    const gs_camera& c = cams[v];
    int tw, th;
    view_tile(c, def_tw, def_th, tw, th);
    if (!camera_ok(c, tw, th)) { bad = true; continue; }
    const unsigned long long t = (unsigned long long)((c.width + tw - 1) / tw) * ((c.height + th - 1) / th);
    acc[0] += t;
    acc[1] += (unsigned long long)c.width * (unsigned long long)c.height;
    acc[2] += t * (unsigned long long)(tw * th / 32);
  }
  if (bad) set_flag(status, GS_FLAG_BAD_CAMERA);
  // block exclusive scan of the three sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x[3] = {acc[0], acc[1], acc[2]};
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x[k], d);
      if (lane >= d) x[k] += y;
    }
  }
  if (lane == 31)
    for (int k = 0; k < 3; ++k) s_sum[k][warp] = x[k];
  __syncthreads();
  unsigned long long e[3];
  for (int k = 0; k < 3; ++k) {
    unsigned long long b = 0;
    for (int w = 0; w < warp; ++w) b += s_sum[k][w];
    e[k] = b + x[k] - acc[k];
  }
  for (int v = v0; v < v1; ++v) {
    const gs_camera& c = cams[v];
    int tw, th;
    view_tile(c, def_tw, def_th, tw, th);
    const bool ok = camera_ok(c, tw, th);
    const uint32_t tx = ok ? (uint32_t)((c.width + tw - 1) / tw) : 0u;
    view_info[kVI * v + 0] = (uint32_t)e[0];
    view_info[kVI * v + 1] = (uint32_t)e[1];
    view_info[kVI * v + 2] = (uint32_t)e[2];
    view_info[kVI * v + 3] = ok ? ((uint32_t)tw | ((uint32_t)th << 8) | (tx << 16)) : 0u;
    if (ok) {
      const unsigned long long t = (unsigned long long)tx * ((c.height + th - 1) / th);
      e[0] += t;
      e[1] += (unsigned long long)c.width * (unsigned long long)c.height;
      e[2] += t * (unsigned long long)(tw * th / 32);
    }
  }
  if (threadIdx.x == blockDim.x - 1) {
    if (e[0] > 0xFFFFFFFFull || e[1] > 0xFFFFFFFFull || e[2] > 0xFFFFFFFFull) set_flag(status, GS_FLAG_RANGE_OVERFLOW);
    view_info[kVI * n_views + 0] = (uint32_t)e[0];
    view_info[kVI * n_views + 1] = (uint32_t)e[1];
    view_info[kVI * n_views + 2] = (uint32_t)e[2];
    view_info[kVI * n_views + 3] = 0u;
  }
}

__device__ __forceinline__ void stage_cams(const gs_camera* __restrict__ cams, const uint32_t* __restrict__ view_info,
                                           int v0, int nv, const gs_params& p, CamC* s_cam) {
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const gs_camera g = cams[v0 + i];
    CamC c;
    load_cam(g, p.guard, p.tile_w, p.tile_h, c);
    if (!camera_ok(g, c.tw, c.th)) {
      c.W = 0;  // marks the view unusable
      c.H = 0;
    }
    c.tile_base = view_info[kVI * (v0 + i)];
    c.pix_base = view_info[kVI * (v0 + i) + 1];
    s_cam[i] = c;
  }
}

// One warp = one group of 32 consecutive Gaussians.  Count pass: per view, the
// ballot of visible lanes is stored (grp_mask, entry view * G + group) and its
// popcount counted.  Write pass: the visible lanes of a (view, group) write their
// records to consecutive slots grp_base + rank, so every store instruction of the
// warp is contiguous.
template <bool kWrite>
__global__ void __launch_bounds__(kBlock) k_project(gs_map map, const gs_camera* __restrict__ cams, int n_views,
                                                     gs_params p, const uint32_t* __restrict__ view_info,
                                                     uint32_t* __restrict__ counts, gs_proj out) {
  __shared__ CamC s_cam[kMaxViewsPerChunk];
  const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t grp = g >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const bool active = g < map.n;
  const bool grp_active = __any_sync(0xffffffffu, active);
  const int64_t n_grp = (map.n + 31) >> 5;
  float4 mo = make_float4(0.f, 0.f, 0.f, 0.f), su = mo, q = mo, col = mo;
  GaussPre pre;
  pre.valid = false;
  if (active) {
    mo = __ldg(reinterpret_cast<const float4*>(map.mo) + g);
    su = __ldg(reinterpret_cast<const float4*>(map.su) + g);
    q = __ldg(reinterpret_cast<const float4*>(map.q) + g);
    if (kWrite && out.color_d) col = __ldg(reinterpret_cast<const float4*>(map.rgb) + g);
    pre = gauss_pre(mo, su, q, p.alpha_min);
    if (!kWrite && !(finite4(mo) && isfinite(su.x) && isfinite(su.y) && isfinite(su.z) && finite4(q)))
      set_flag(out.status, GS_FLAG_NONFINITE);
  }
  for (int v0 = 0; v0 < n_views; v0 += kMaxViewsPerChunk) {
    const int nv = min(kMaxViewsPerChunk, n_views - v0);
    __syncthreads();
    stage_cams(cams, view_info, v0, nv, p, s_cam);
    __syncthreads();
    if (!grp_active) continue;
    uint32_t m_ahead = 0;   // write pass: the visibility masks of the next 32 views, one per lane
    for (int i = 0; i < nv; ++i) {
      const CamC& c = s_cam[i];
      const size_t slot = (size_t)(v0 + i) * n_grp + grp;
      ViewProj vp;
      if (!kWrite) {
        const bool vis = active && pre.valid && c.W > 0 && view_proj(mo, pre, c, p.near_plane, p.eps2d, vp);
        const uint32_t m = __ballot_sync(0xffffffffu, vis);
        if (lane == 0) {
          out.grp_mask[slot] = m;
          counts[slot] = __popc(m);
        }
        continue;
      }
      // write pass: only the (Gaussian, view) pairs the count pass found visible are projected again
      if ((i & 31) == 0)
        m_ahead = i + lane < nv ? out.grp_mask[(size_t)(v0 + i + lane) * n_grp + grp] : 0u;
      const uint32_t m = __shfl_sync(0xffffffffu, m_ahead, i & 31);
      if (!(m & (1u << lane))) continue;
      if (view_proj(mo, pre, c, p.near_plane, p.eps2d, vp)) {
        const uint32_t dst = out.grp_base[slot] + __popc(m & lt);
        if ((int64_t)dst < out.capacity) {
          out.gid[dst] = (uint32_t)g;
          out.view[dst] = (uint32_t)(v0 + i);
          float4* sp = reinterpret_cast<float4*>(out.splat) + 2 * (size_t)dst;
          sp[0] = make_float4(vp.mx, vp.my, pack_ext(vp.rx, vp.ry), su.w);
          sp[1] = make_float4(vp.ca, vp.cb, vp.cc, pre.o);
          if (out.color_d) reinterpret_cast<float4*>(out.color_d)[dst] = make_float4(col.x, col.y, col.z, vp.depth);
          reinterpret_cast<ushort4*>(out.rect)[dst] =
              make_ushort4((unsigned short)vp.x0, (unsigned short)vp.y0, (unsigned short)vp.x1, (unsigned short)vp.y1);
          out.depth_key[dst] = __float_as_uint(vp.depth);
        }
      }
    }
  }
}

__global__ void k_record_count(const gs_proj out, int64_t n_slots) {
  const uint32_t total = out.grp_base[n_slots];
  *out.count = (int64_t)total > out.capacity ? (uint32_t)out.capacity : total;
  if ((int64_t)total > out.capacity) set_flag(out.status, GS_FLAG_RECORD_OVERFLOW);
}

}  // namespace

size_t project_ws_bytes(int64_t n, int n_views) {
  const int64_t slots = ((n + 31) / 32) * (int64_t)n_views;
  return align_up(sizeof(uint32_t) * (size_t)(slots + 1), 256) + scan_temp_bytes(slots);
}

cudaError_t launch_project(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                           const gs_proj& out, void* ws, cudaStream_t st) {
  const int64_t slots = ((map.n + 31) / 32) * (int64_t)n_views;
  Carver c(ws);
  uint32_t* counts = c.take<uint32_t>((size_t)slots + 1);
  void* scan_tmp = c.take<char>(scan_temp_bytes(slots));
  k_view_info<<<1, 1024, 0, st>>>(cams, n_views, p.tile_w, p.tile_h, out.view_info, out.status);
  note_launch();
  const int64_t blocks = (map.n + kBlock - 1) / kBlock;
  if (blocks > 0) {
    k_project<false><<<(unsigned)blocks, kBlock, 0, st>>>(map, cams, n_views, p, out.view_info, counts, out);
    note_launch();
  }
  cudaError_t e = scan_exclusive(counts, out.grp_base, nullptr, slots, nullptr, scan_tmp, st);
  if (e != cudaSuccess) return e;
  if (blocks > 0) {
    k_project<true><<<(unsigned)blocks, kBlock, 0, st>>>(map, cams, n_views, p, out.view_info, counts, out);
    note_launch();
  }
  k_record_count<<<1, 1, 0, st>>>(out, slots);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
