// small.cu -- gs_render_small: the forward render of a small map in one launch.
//
// Sec. III of RT-GuIDE: the Gaussians of each view are sorted by increasing depth and
// composited front to back.  The tiled path (gs_project, gs_bin_sort, gs_render_fwd) runs
// about 35 kernels whose launch latencies, not their work, set the time of a render of a
// few thousand Gaussians.  Here one launch does everything: each CTA takes screen tiles
// (a fixed stride over all views' tiles), projects every Gaussian of the map for the tile's
// view with the same FP32 decision arithmetic as gs_project, keeps in shared memory, in
// Gaussian-id order, those whose tile rectangle covers the tile, sorts them stably by their
// depth key (so the list is the tile's list of gs_bin_sort), and composites the tile's 8x4
// pixel blocks with the forward kernel's alpha and update sequence.  Images, T, `last` and
// the contributor counts are therefore bit for bit those of the tiled path.  No workspace.
#include "gs_common.cuh"
#include "gs_internal.h"
#include "render_common.cuh"

namespace gs {
namespace {

constexpr int kThreads = 512;   // a multiple of 256 (the sort's digits)
constexpr int kWarps = kThreads / 32;
static_assert(kThreads % 256 == 0, "one thread per digit in the sort's digit loops");
constexpr int kList = GS_SMALL_MAX_LIST;   // Gaussians of one tile that fit in shared memory

struct SmallSmem {
  float4 m[kList];                  // (mu_x, mu_y, packed half-widths, u), in Gaussian-id order
  float4 co[kList];                 // (a, b, c, o): conic and opacity
  float4 cd[kList];                 // (r, g, b, t_z)
  uint32_t key[2][kList];           // depth key bits, ping-pong of the sort
  uint16_t idx[2][kList];           // entry of each key
  uint32_t cnt[kWarps][256];        // per-warp digit counts of one sort chunk
  uint32_t base[256];               // first slot of every digit (sort pass)
  uint32_t run[256];                // slots of every digit used by earlier chunks
  uint32_t wsum[kWarps];
  CamC cam;
  int n_list;
  int tile_x, tile_y;               // the tile, in the view's tile grid
  uint32_t pix_base;                // first pixel of the view in the image layout
  int view_ok;
};

constexpr uint64_t kMaxTiles = 1ull << 20;   // tiles over all views this entry point renders

__device__ __forceinline__ bool small_camera_ok(const gs_camera& c, int tw, int th) {
  return c.width > 0 && c.height > 0 && c.fx > 0.f && c.fy > 0.f && isfinite(c.fx) && isfinite(c.fy) &&
         valid_tile(tw, th);
}

// The view and tile of global tile t (views in order, each with its own tile grid; an
// invalid camera has no tiles but keeps its pixels in the layout).  False past the last
// tile, or if the tiles or pixels before t exceed what this entry point handles (then
// *range is set).  Thread 0 only.
__device__ bool locate_tile(const gs_camera* cams, int n_views, const gs_params& p, uint64_t t, SmallSmem& s,
                            bool* range) {
  uint64_t tile0 = 0, pix0 = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs_camera& c = cams[v];
    int tw, th;
    view_tile(c, p.tile_w, p.tile_h, tw, th);
    const bool ok = small_camera_ok(c, tw, th);
    const uint64_t tx = ok ? (uint64_t)((c.width + tw - 1) / tw) : 0u;
    const uint64_t ty = ok ? (uint64_t)((c.height + th - 1) / th) : 0u;
    if (t < tile0 + tx * ty) {
      if (tile0 + tx * ty > kMaxTiles || pix0 + (uint64_t)c.width * (uint64_t)c.height > 0xFFFFFFFFull) {
        *range = true;
        return false;
      }
      load_cam(c, p.guard, p.tile_w, p.tile_h, s.cam);
      const uint64_t lt = t - tile0;
      s.tile_x = (int)(lt % tx);
      s.tile_y = (int)(lt / tx);
      s.pix_base = (uint32_t)pix0;
      return true;
    }
    tile0 += tx * ty;
    pix0 += (uint64_t)(c.width > 0 ? c.width : 0) * (uint64_t)(c.height > 0 ? c.height : 0);
  }
  return false;
}

// Stable LSD radix sort of the n (key, idx) pairs in buffer 0 by the 32 key bits (four
// 8-bit passes, the result back in buffer 0).  Items are ranked in chunks of kThreads in
// list order: within a chunk by warp (lower warps first) and lane (warp match), across
// chunks by a running count per digit, so equal keys keep their order.  Threads 0..255 own
// one digit each in the digit loops.
__device__ void sort_list(SmallSmem& s, int n) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass, src = pass & 1, dst = src ^ 1;
    // digit totals -> first slot of every digit
    if (tid < 256) s.run[tid] = 0u;
    __syncthreads();
    for (int i = tid; i < n; i += kThreads) atomicAdd(&s.run[(s.key[src][i] >> shift) & 0xffu], 1u);
    __syncthreads();
    if (warp == 0) {
      uint32_t v[8], t = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) { v[k] = s.run[lane * 8 + k]; t += v[k]; }
      uint32_t x = t;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
      }
      uint32_t e = x - t;
#pragma unroll
      for (int k = 0; k < 8; ++k) { s.base[lane * 8 + k] = e; e += v[k]; }
    }
    __syncthreads();
    if (tid < 256) s.run[tid] = 0u;
    for (int c0 = 0; c0 < n; c0 += kThreads) {
      for (int i = lane; i < 256; i += 32) s.cnt[warp][i] = 0u;
      __syncthreads();
      const int i = c0 + tid;
      const bool ok = i < n;
      const uint32_t k = ok ? s.key[src][i] : 0u;
      const uint32_t d = ok ? (k >> shift) & 0xffu : 256u + (uint32_t)lane;   // invalid lanes match nobody
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (ok && (peers & lt) == 0u) s.cnt[warp][d] = __popc(peers);
      __syncthreads();
      if (ok) {
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s.cnt[w][d];
        const uint32_t pos = s.base[d] + s.run[d] + before + __popc(peers & lt);
        s.key[dst][pos] = k;
        s.idx[dst][pos] = s.idx[src][i];
      }
      __syncthreads();
      if (tid < 256) {
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) add += s.cnt[w][tid];
        s.run[tid] += add;
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_render_small(gs_map map, const gs_camera* __restrict__ cams,
                                                           int n_views, gs_params p, gs_image img,
                                                           uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  SmallSmem& s = *reinterpret_cast<SmallSmem*>(s_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const float ln_amin = __logf(p.alpha_min);
  const float4* MO = reinterpret_cast<const float4*>(map.mo);
  const float4* SU = reinterpret_cast<const float4*>(map.su);
  const float4* Q = reinterpret_cast<const float4*>(map.q);
  const float4* RGB = reinterpret_cast<const float4*>(map.rgb);
  if (blockIdx.x == 0 && tid == 0) {
    for (int v = 0; v < n_views; ++v) {
      int tw, th;
      view_tile(cams[v], p.tile_w, p.tile_h, tw, th);
      if (!small_camera_ok(cams[v], tw, th)) set_flag(status, GS_FLAG_BAD_CAMERA);
    }
  }
  for (uint64_t t = blockIdx.x;; t += gridDim.x) {
    __syncthreads();   // the previous tile is done with shared memory
    if (tid == 0) {
      bool range = false;
      s.view_ok = locate_tile(cams, n_views, p, t, s, &range) ? 1 : 0;
      if (range) set_flag(status, GS_FLAG_RANGE_OVERFLOW);
      s.n_list = 0;
    }
    __syncthreads();
    if (!s.view_ok) break;   // past the last tile of the last view
    const CamC& cam = s.cam;
    const int tx = s.tile_x, ty = s.tile_y;
    // 1. the Gaussians whose tile rectangle covers this tile, in Gaussian-id order
    for (int64_t g0 = 0; g0 < map.n; g0 += kThreads) {
      const int64_t g = g0 + tid;
      bool take = false;
      float4 mo = make_float4(0.f, 0.f, 0.f, 0.f), su = mo;
      GaussPre pre;
      ViewProj vp;
      if (g < map.n) {
        mo = __ldg(MO + g);
        su = __ldg(SU + g);
        const float4 q = __ldg(Q + g);
        pre = gauss_pre(mo, su, q, p.alpha_min);
        if (t == blockIdx.x && blockIdx.x == 0 &&
            !(finite4(mo) && isfinite(su.x) && isfinite(su.y) && isfinite(su.z) && finite4(q)))
          set_flag(status, GS_FLAG_NONFINITE);
        take = view_proj<true>(mo, pre, cam, p.near_plane, p.eps2d, vp) && vp.x0 <= tx && tx < vp.x1 &&
               vp.y0 <= ty && ty < vp.y1;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, take);
      if (lane == 0) s.wsum[warp] = __popc(m);
      __syncthreads();
      int pos = s.n_list + __popc(m & lt);
      for (int w = 0; w < warp; ++w) pos += s.wsum[w];
      if (take && pos < kList) {
        const float4 c = __ldg(RGB + g);
        s.m[pos] = make_float4(vp.mx, vp.my, pack_ext(vp.rx, vp.ry), su.w);
        s.co[pos] = make_float4(vp.ca, vp.cb, vp.cc, pre.o);
        s.cd[pos] = make_float4(c.x, c.y, c.z, vp.depth);
        s.key[0][pos] = __float_as_uint(vp.depth);
        s.idx[0][pos] = (uint16_t)pos;
      }
      __syncthreads();
      if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < kWarps; ++w) tot += s.wsum[w];
        s.n_list += tot;
      }
      __syncthreads();
    }
    const int n_all = s.n_list;
    if (n_all > kList) {   // the tile's list does not fit: nothing is written for it
      if (tid == 0) set_flag(status, GS_FLAG_PAIR_OVERFLOW);
      continue;
    }
    // 2. depth order (ties keep the Gaussian-id order)
    sort_list(s, n_all);
    // 3. front-to-back compositing of the tile's 8x4 pixel blocks, one warp per block
    const int wpr = cam.tw >> 3, nb = (cam.tw * cam.th) >> 5;
    const float amax = p.alpha_max;
    for (int b = warp; b < nb; b += kWarps) {
      const int x0 = tx * cam.tw + (b % wpr) * 8, y0 = ty * cam.th + (b / wpr) * 4;
      WarpBlock wb;
      wb.px = x0 + (lane & 7);
      wb.py = y0 + (lane >> 3);
      wb.bx0 = (float)x0 + 0.5f;
      wb.bx1 = wb.bx0 + 7.f;
      wb.by0 = (float)y0 + 0.5f;
      wb.by1 = wb.by0 + 3.f;
      const LaneOffsets lo = lane_offsets(lane);
      const float ccx = wb.bx0 + 3.5f, ccy = wb.by0 + 1.5f;   // centre of the 8x4 block
      const bool inside = wb.px < cam.W && wb.py < cam.H;
      bool done = !inside;
      float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, cdp = 0.f, cu = 0.f;
      int32_t last = 0, n_contrib = 0;
      for (int g = 0; g < n_all; g += 32) {
        if (!__any_sync(0xffffffffu, !done)) break;
        const int j = g + lane;
        bool ov = false;
        Exponent ex{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // this lane's entry, staged as the tiled forward does
        if (j < n_all) {
          const int e = s.idx[0][j];
          ov = box_overlaps(s.m[e], wb) && ellipse_reaches(s.m[e], s.co[e], wb, ln_amin);
          if (ov) ex = stage_exponent(s.m[e].x, s.m[e].y, s.co[e], ccx, ccy);
        }
        uint32_t mk = __ballot_sync(0xffffffffu, ov);
        while (mk) {
          const int k = __ffs(mk) - 1;
          mk &= mk - 1u;
          // the entry's coefficients from the lane that staged it (every lane takes part)
          const float c0 = __shfl_sync(0xffffffffu, ex.c0, k), cu_ = __shfl_sync(0xffffffffu, ex.cu, k);
          const float cv = __shfl_sync(0xffffffffu, ex.cv, k), kx = __shfl_sync(0xffffffffu, ex.kx, k);
          const float ky = __shfl_sync(0xffffffffu, ex.ky, k), kz = __shfl_sync(0xffffffffu, ex.kz, k);
          if (done) continue;
          const int e = s.idx[0][g + k];
          const float4 mu = s.m[e];
          const float alpha = fminf(amax, alpha_raw(c0, cu_, cv, kx, ky, kz, lo));
          if (alpha < p.alpha_min) continue;
          const float w = alpha * T;
          const float Tn = T - w;   // T (1 - alpha)
          if (Tn < p.T_min) { done = true; continue; }
          const float4 c = s.cd[e];
          cr += w * c.x;
          cg += w * c.y;
          cb += w * c.z;
          cdp += w * c.w;
          cu += w * mu.w;
          T = Tn;
          last = g + k + 1;
          ++n_contrib;
        }
      }
      if (inside) {
        const size_t P = (size_t)cam.W * cam.H;
        const size_t pix = (size_t)wb.py * cam.W + wb.px;
        const size_t o = (size_t)s.pix_base + pix;
        if (img.rgb) {
          float* base = img.rgb + 3 * (size_t)s.pix_base;
          base[pix] = cr;
          base[P + pix] = cg;
          base[2 * P + pix] = cb;
        }
        if (img.depth) img.depth[o] = cdp;
        if (img.unc) img.unc[o] = cu;
        if (img.T) img.T[o] = T;
        if (img.last) img.last[o] = last;
        if (img.n_contrib) img.n_contrib[o] = n_contrib;
      }
    }
  }
}

}  // namespace

cudaError_t launch_render_small(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                                const gs_image& img, uint32_t* status, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_render_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallSmem));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  // one CTA per SM walks the tiles of all views with a fixed stride (the number of tiles
  // lives in the cameras, in device memory)
  k_render_small<<<(unsigned)device_sm_count(), kThreads, sizeof(SmallSmem), st>>>(map, cams, n_views, p, img,
                                                                                     status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
