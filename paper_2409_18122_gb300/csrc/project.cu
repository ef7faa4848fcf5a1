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
constexpr int kWarps = kBlock / 32;

__device__ __forceinline__ bool camera_ok(const gs_camera& c, int tw, int th) {
  return c.width > 0 && c.height > 0 && c.fx > 0.f && c.fy > 0.f && isfinite(c.fx) && isfinite(c.fy) &&
         valid_tile(tw, th);
}

// Pixels of a view in the image layout: W x H, a negative size counting as zero.
__device__ __forceinline__ unsigned long long view_pixels(const gs_camera& c) {
  return (unsigned long long)(c.width > 0 ? c.width : 0) * (unsigned long long)(c.height > 0 ? c.height : 0);
}

// Per-view table: tile, pixel and warp-item offsets (prefix sums over views), tile
// sizes, camera checks.
__global__ void __launch_bounds__(1024) k_view_info(const gs_camera* __restrict__ cams, int n_views, int def_tw,
                                                    int def_th, uint32_t n_groups, uint32_t* __restrict__ view_info,
                                                    uint32_t* status) {
  __shared__ unsigned long long s_sum[3][32];
  const int per = (n_views + blockDim.x - 1) / blockDim.x;
  const int v0 = threadIdx.x * per;
  int v1 = v0 + per;
  if (v1 > n_views) v1 = n_views;
  // every view keeps its W x H pixels in the image layout, so that the layout is the same
  // whatever the device decides about a camera; an invalid camera gets no tiles and no warp
  // items (its pixels are never written)
  unsigned long long acc[3] = {0, 0, 0};   // tiles, pixels, warp items
  bool bad = false;
  for (int v = v0; v < v1; ++v) {
    const gs_camera& c = cams[v];
    int tw, th;
    view_tile(c, def_tw, def_th, tw, th);
    acc[1] += view_pixels(c);
    if (!camera_ok(c, tw, th)) { bad = true; continue; }
    const unsigned long long t = (unsigned long long)((c.width + tw - 1) / tw) * ((c.height + th - 1) / th);
    acc[0] += t;
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
    e[1] += view_pixels(c);
    if (ok) {
      const unsigned long long t = (unsigned long long)tx * ((c.height + th - 1) / th);
      e[0] += t;
      e[2] += t * (unsigned long long)(tw * th / 32);
    }
  }
  if (threadIdx.x == blockDim.x - 1) {
    if (e[0] > 0xFFFFFFFFull || e[1] > 0xFFFFFFFFull || e[2] > 0xFFFFFFFFull) set_flag(status, GS_FLAG_RANGE_OVERFLOW);
    view_info[kVI * n_views + 0] = (uint32_t)e[0];
    view_info[kVI * n_views + 1] = (uint32_t)e[1];
    view_info[kVI * n_views + 2] = (uint32_t)e[2];
    view_info[kVI * n_views + 3] = n_groups;   // groups of 32 Gaussians: the stride of grp_mask / grp_base
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

// One warp = one group of 32 consecutive Gaussians.  For every view the lanes
// test their Gaussian cheaply (near plane, guard band: frustum_ok; in the write
// pass, the count pass's visibility bit) and queue the (view, lane) pairs that
// pass in shared memory; whenever 32 are queued, each lane takes one and runs the
// full projection, so the expensive EWA path runs with every lane busy whatever
// the fraction of Gaussians a view sees.  Count pass: the visible lanes of each
// (view, group) become a ballot mask (grp_mask, entry view * G + group) and its
// popcount.  Write pass: every visible pair writes its record to
// grp_base[(view, group)] + (visible lanes below it), i.e. in (view, Gaussian) order.
template <bool kWrite>
__global__ void __launch_bounds__(kBlock) k_project(gs_map map, const gs_camera* __restrict__ cams, int n_views,
                                                     gs_params p, const uint32_t* __restrict__ view_info,
                                                     uint32_t* __restrict__ counts, gs_proj out) {
  __shared__ CamC s_cam[kMaxViewsPerChunk];
  __shared__ float4 s_g[kWarps][4][32];                  // per lane: mo, (S0..S3), (S4, S5, Q, o), (rgb, u)
  __shared__ uint32_t s_q[kWarps][64];                   // queued (view in chunk << 5 | lane)
  __shared__ uint32_t s_mask[kWarps][kMaxViewsPerChunk];   // per view of the chunk: visible lanes
  __shared__ uint32_t s_base[kWarps][kMaxViewsPerChunk];   // write pass: first record of (view, group)
  const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t grp = g >> 5;
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
  s_g[warp][0][lane] = mo;
  s_g[warp][1][lane] = make_float4(pre.S[0], pre.S[1], pre.S[2], pre.S[3]);
  s_g[warp][2][lane] = make_float4(pre.S[4], pre.S[5], pre.Q, pre.o);
  s_g[warp][3][lane] = make_float4(col.x, col.y, col.z, su.w);
  const bool usable = active && pre.valid;
  uint32_t* queue = s_q[warp];
  uint32_t* vmask = s_mask[warp];
  // count pass: a sphere holding the centres of the group's usable Gaussians, for the group
  // cull of every view (group_may_meet); its radius carries a margin against rounding
  float gc[3] = {0.f, 0.f, 0.f}, grad = 0.f;
  const uint32_t use_mask = __ballot_sync(0xffffffffu, usable);
  if (!kWrite && use_mask) {
    float sx = usable ? mo.x : 0.f, sy = usable ? mo.y : 0.f, sz = usable ? mo.z : 0.f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, d);
      sy += __shfl_xor_sync(0xffffffffu, sy, d);
      sz += __shfl_xor_sync(0xffffffffu, sz, d);
    }
    const float inv = 1.f / (float)__popc(use_mask);
    gc[0] = sx * inv;
    gc[1] = sy * inv;
    gc[2] = sz * inv;
    float r2 = 0.f;
    if (usable) {
      const float ex = mo.x - gc[0], ey = mo.y - gc[1], ez = mo.z - gc[2];
      r2 = ex * ex + ey * ey + ez * ez;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, d));
    grad = sqrtf(r2) * 1.001f + 1e-4f;
  }

  // full projection of up to 32 queued pairs, one per lane
  auto drain = [&](int v0, int count) {
    if (lane < count) {
      const uint32_t e = queue[lane];
      const int gl = e & 31, vi = e >> 5;
      const float4 gmo = s_g[warp][0][gl], s0 = s_g[warp][1][gl], s1 = s_g[warp][2][gl];
      GaussPre gp;
      gp.valid = true;
      gp.S[0] = s0.x; gp.S[1] = s0.y; gp.S[2] = s0.z; gp.S[3] = s0.w; gp.S[4] = s1.x; gp.S[5] = s1.y;
      gp.Q = s1.z;
      gp.o = s1.w;
      ViewProj vp;
      const bool vis = view_proj<kWrite>(gmo, gp, s_cam[vi], p.near_plane, p.eps2d, vp);
      if (!kWrite) {
        if (vis) atomicOr(&vmask[vi], 1u << gl);
      } else if (vis) {
        const uint32_t dst = s_base[warp][vi] + __popc(vmask[vi] & ((1u << gl) - 1u));
        if ((int64_t)dst < out.capacity) {
          const float4 cu = s_g[warp][3][gl];
          if (out.gid) out.gid[dst] = (uint32_t)((grp << 5) + gl);
          if (out.view) out.view[dst] = (uint32_t)(v0 + vi);
          float4* sp = reinterpret_cast<float4*>(out.splat) + 2 * (size_t)dst;
          sp[0] = make_float4(vp.mx, vp.my, pack_ext(vp.rx, vp.ry), cu.w);
          sp[1] = make_float4(vp.ca, vp.cb, vp.cc, gp.o);
          if (out.color_d) reinterpret_cast<float4*>(out.color_d)[dst] = make_float4(cu.x, cu.y, cu.z, vp.depth);
          reinterpret_cast<ushort4*>(out.rect)[dst] =
              make_ushort4((unsigned short)vp.x0, (unsigned short)vp.y0, (unsigned short)vp.x1, (unsigned short)vp.y1);
          out.depth_key[dst] = __float_as_uint(vp.depth);
        }
      }
    }
    __syncwarp();
  };

  for (int v0 = 0; v0 < n_views; v0 += kMaxViewsPerChunk) {
    const int nv = min(kMaxViewsPerChunk, n_views - v0);
    __syncthreads();
    stage_cams(cams, view_info, v0, nv, p, s_cam);
    __syncthreads();
    if (!grp_active) continue;
    for (int i = lane; i < nv; i += 32) {
      const size_t slot = (size_t)(v0 + i) * n_grp + grp;
      vmask[i] = kWrite ? out.grp_mask[slot] : 0u;
      if (kWrite) s_base[warp][i] = out.grp_base[slot];
    }
    __syncwarp();
    int qn = 0;   // queued pairs (warp-uniform)
    // 32 views at a time, one per lane, are first tested for the whole group: in the count
    // pass a view whose frustum the group's sphere cannot meet is skipped, in the write pass
    // a view in which none of the group is visible; the lanes then test their own Gaussian
    // against each remaining view in turn
    for (int vb = 0; vb < nv; vb += 32) {
      const int iv = vb + lane;
      bool cand = false;
      if (iv < nv) {
        if (kWrite) cand = vmask[iv] != 0u;
        else cand = use_mask != 0u && s_cam[iv].W > 0 && group_may_meet(gc, grad, s_cam[iv], p.near_plane);
      }
      uint32_t cm = __ballot_sync(0xffffffffu, cand);
      while (cm) {
        const int i = vb + __ffs(cm) - 1;
        cm &= cm - 1u;
        bool take;
        if (kWrite) take = (vmask[i] >> lane) & 1u;
        else take = usable && frustum_ok(mo, s_cam[i], p.near_plane);
        const uint32_t m = __ballot_sync(0xffffffffu, take);
        if (take) queue[qn + __popc(m & lt)] = ((uint32_t)i << 5) | (uint32_t)lane;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
          drain(v0, 32);
          const uint32_t rest = lane + 32 < qn ? queue[lane + 32] : 0u;
          __syncwarp();
          if (lane + 32 < qn) queue[lane] = rest;
          qn -= 32;
          __syncwarp();
        }
      }
    }
    drain(v0, qn);
    if (!kWrite) {
      for (int i = lane; i < nv; i += 32) {
        const size_t slot = (size_t)(v0 + i) * n_grp + grp;
        const uint32_t m = vmask[i];
        out.grp_mask[slot] = m;
        counts[slot] = __popc(m);
      }
    }
    __syncwarp();
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
  k_view_info<<<1, 1024, 0, st>>>(cams, n_views, p.tile_w, p.tile_h, (uint32_t)((map.n + 31) / 32), out.view_info,
                                  out.status);
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
