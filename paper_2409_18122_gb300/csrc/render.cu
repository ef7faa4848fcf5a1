// render.cu -- front-to-back compositing (gs_render_fwd) and the batched
// information-gain pass (gs_info_gain_batch).
//
// Sec. III of RT-GuIDE: C(p) = sum_i c_i f_i(p) prod_{j<i} (1 - f_j(p)), depth with
// d_i in place of c_i; Sec. IV-A: the per-Gaussian uncertainty u_i composited the
// same way gives the rendered information channel, whose per-view mean scores a
// candidate view (Eq. (nbv) with the Jacobian replaced by the blend weights).
//
// One thread block per screen tile (tile_w x tile_h threads, one pixel each).
// The tile's depth-sorted list is walked in chunks of blockDim entries staged
// in shared memory; each thread leaves the inner loop as soon as its pixel is
// saturated, so a warp stops issuing once all its lanes are done, and the
// block stops loading chunks once every pixel is done (__syncthreads_count).
#include "gs_common.cuh"
#include "gs_internal.h"
#include "render_common.cuh"

namespace gs {
namespace {

constexpr int kFwdWarps = 2;   // warps (work items) per CTA: small CTAs free their slot as soon as both finish
constexpr int kIgWarps = 8;    // warps per CTA of the persistent information-gain kernel
constexpr int kIgRing = 64;    // staged entries per warp of the information-gain kernel (a ring)
constexpr int kPix = 1;        // pixels per lane of the forward and information-gain kernels
// Chunk depth: overlapping entries whose alphas are computed together, a template argument
// of both compositing kernels chosen per launch by gs_params (forward 1, 2 or 4, default 2;
// information gain 4, 8 or 16, default 8)
constexpr int kFwdBatchDefault = 2;
constexpr int kIgBatchDefault = 8;

// The list walk of all compositing kernels is a four-stage software pipeline
// over groups of 32 entries (one per lane).  While group g is composited, the
// alpha/colour data of group g+32 is fetched -- only for entries whose support
// box touches the warp's pixel block, decided from their means fetched one
// iteration earlier -- the means of group g+64 are fetched, and the list
// indices of group g+96.  Every fetch is issued one iteration before it is
// used and none depends on a value loaded in the same iteration.

template <int kFwdBatch>
__global__ void __launch_bounds__(kFwdWarps * 32, 12) k_render_fwd(gs_map map, gs_proj proj, gs_bins bins,
                                                                const gs_camera* __restrict__ cams, int n_views,
                                                                gs_params p, gs_image img, uint32_t n_items) {
  // staged entries: (c0, cu, cv, u), (k.x, k.y, k.z, lane), (r, g, b, depth) (stage_exponent)
  __shared__ float4 s_stage[kFwdWarps][3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t item = blockIdx.x * kFwdWarps + warp;
  if (item >= n_items) return;
  static_assert(kPix == 1, "the binning's item order numbers 32-pixel blocks");
  item = ordered_item(bins, proj.view_info, n_views, item);
  TileInfo ti;
  if (!warp_item_setup<kPix>(proj, bins, cams, n_views, item, ti)) return;
  WarpBlock wb;
  warp_block<kPix>(ti, wb);
  float4* sm = s_stage[warp][0];
  float4* sc = s_stage[warp][1];
  float4* sk = s_stage[warp][2];
  const float ln_amin = __logf(p.alpha_min);
  const LaneOffsets lo = lane_offsets(lane);
  const float ccx = wb.bx0 + 3.5f, ccy = wb.by0 + 1.5f;   // centre of the 8x4 block
  bool inside[kPix], done[kPix];
  float T[kPix], cr[kPix], cg[kPix], cb[kPix], cd[kPix], cu[kPix];
  int32_t last[kPix], n_contrib[kPix];
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    inside[q] = wb.px < ti.W && wb.py + 4 * q < ti.H;
    done[q] = !inside[q];
    T[q] = 1.f;
    cr[q] = cg[q] = cb[q] = cd[q] = cu[q] = 0.f;
    last[q] = n_contrib[q] = 0;
  }
  const uint32_t n = ti.end - ti.beg;
  const uint32_t* rl = bins.rec + ti.beg;
  const float4* SP = reinterpret_cast<const float4*>(proj.splat);
  const float4* CD = reinterpret_cast<const float4*>(proj.color_d);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t rA = 0, rB = 0, rC = 0;
  if ((uint32_t)lane < n) rA = __ldg(rl + lane);
  if (32u + lane < n) rB = __ldg(rl + 32 + lane);
  if (64u + lane < n) rC = __ldg(rl + 64 + lane);
  float4 mA = z4, mB = z4;
  if ((uint32_t)lane < n) mA = __ldg(SP + 2 * (size_t)rA);
  if (32u + lane < n) mB = __ldg(SP + 2 * (size_t)rB);
  bool ovA = (uint32_t)lane < n && box_overlaps(mA, wb);
  float4 cA = z4, kA = z4;
  if (ovA) {
    cA = __ldg(SP + 2 * (size_t)rA + 1);
    kA = __ldg(CD + rA);
  }
  for (uint32_t g = 0; g < n; g += 32) {
    if (!__any_sync(0xffffffffu, !all_done<kPix>(done))) break;
    const bool ovB = g + 32 + lane < n && box_overlaps(mB, wb);
    float4 cB = z4, kB = z4;
    if (ovB) {
      cB = __ldg(SP + 2 * (size_t)rB + 1);
      kB = __ldg(CD + rB);
    }
    float4 mC = z4;
    if (g + 64 + lane < n) mC = __ldg(SP + 2 * (size_t)rC);
    uint32_t rD = 0;
    if (g + 96 + lane < n) rD = __ldg(rl + g + 96 + lane);
    ovA = ovA && ellipse_reaches(mA, cA, wb, ln_amin);
    const uint32_t m = __ballot_sync(0xffffffffu, ovA);
    if (m) {
      // the overlapping entries, compacted in list order: (c0, cu, cv, u), (k, position in
      // the group), colour; padded to whole batches with entries of c0 = -inf (alpha = 0:
      // always skipped)
      const int n_ov = __popc(m);
      const int n_pad = (n_ov + kFwdBatch - 1) / kFwdBatch * kFwdBatch;
      if (ovA) {
        const int s = __popc(m & lt);
        const Exponent e = stage_exponent(mA.x, mA.y, cA, ccx, ccy);
        sm[s] = make_float4(e.c0, e.cu, e.cv, mA.w);
        sc[s] = make_float4(e.kx, e.ky, e.kz, __int_as_float(lane));
        sk[s] = kA;
      }
      if (lane >= n_ov && lane < n_pad) {   // slots [n_ov, n_pad): disjoint from the staged ones
        sm[lane] = make_float4(-INFINITY, 0.f, 0.f, 0.f);
        sc[lane] = z4;
      }
      __syncwarp();
      // kFwdBatch entries at a time: their alphas are independent and computed
      // together; the transmittance updates then run in list order
      for (int i0 = 0; i0 < n_ov && !all_done<kPix>(done); i0 += kFwdBatch) {
        float al[kFwdBatch][kPix];
#pragma unroll
        for (int k = 0; k < kFwdBatch; ++k) {
          const int i = i0 + k;
          const float4 e0 = sm[i];
          const float4 e1 = sc[i];
#pragma unroll
          for (int q = 0; q < kPix; ++q)
            al[k][q] = fminf(p.alpha_max, alpha_raw(e0.x, e0.y, e0.z, e1.x, e1.y, e1.z, lo));
        }
#pragma unroll
        for (int k = 0; k < kFwdBatch; ++k) {
          const int i = i0 + k;
#pragma unroll
          for (int q = 0; q < kPix; ++q) {
            if (done[q]) continue;
            const float alpha = al[k][q];
            if (alpha < p.alpha_min) continue;
            const float w = alpha * T[q];
            const float Tn = T[q] - w;      // T (1 - alpha)
            if (Tn < p.T_min) { done[q] = true; continue; }
            const float4 c = sk[i];
            cr[q] += w * c.x;
            cg[q] += w * c.y;
            cb[q] += w * c.z;
            cd[q] += w * c.w;
            cu[q] += w * sm[i].w;
            T[q] = Tn;
            last[q] = (int32_t)(g + __float_as_int(sc[i].w) + 1);
            ++n_contrib[q];
          }
        }
      }
      __syncwarp();
    }
    mA = mB; ovA = ovB; cA = cB; kA = kB;
    rB = rC; mB = mC;
    rC = rD;
  }
  const size_t P = (size_t)ti.W * ti.H;
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    if (!inside[q]) continue;
    const size_t pix = (size_t)(wb.py + 4 * q) * ti.W + wb.px;
    const size_t o = (size_t)ti.pix_base + pix;
    if (img.rgb) {
      float* base = img.rgb + 3 * (size_t)ti.pix_base;
      base[pix] = cr[q];
      base[P + pix] = cg[q];
      base[2 * P + pix] = cb[q];
    }
    if (img.depth) img.depth[o] = cd[q];
    if (img.unc) img.unc[o] = cu[q];
    if (img.T) img.T[o] = T[q];
    if (img.last) img.last[o] = last[q];
    if (img.n_contrib) img.n_contrib[o] = n_contrib[q];
  }
}

// Staged form of an entry for the information-gain kernel: s0 = (c0, cu, cv, u),
// s1 = (k.x, k.y, k.z, 0) (stage_exponent).
__device__ __forceinline__ void ig_stage(const float4& m, const float4& co, float ccx, float ccy, float4& s0,
                                         float4& s1) {
  const Exponent e = stage_exponent(m.x, m.y, co, ccx, ccy);
  s0 = make_float4(e.c0, e.cu, e.cv, m.w);
  s1 = make_float4(e.kx, e.ky, e.kz, 0.f);
}

// Composites `chunks` whole chunks of kIgBatch staged entries, starting at ring position
// `head` (a multiple of kIgBatch, so no chunk wraps): the alphas of a chunk are independent
// and computed together, the transmittance updates then run in list order.  A lane leaves
// as soon as its pixel is saturated.
template <int kIgBatch>
__device__ __forceinline__ void composite_chunks(const float4* sm, const float4* sc, uint32_t head, uint32_t chunks,
                                                 const LaneOffsets& lo, const gs_params& p, float& T, float& cu) {
  for (uint32_t c = 0; c < chunks && T != 0.f; ++c) {
    const uint32_t b0 = (head + c * kIgBatch) & (kIgRing - 1);
    float al[kIgBatch], uu[kIgBatch];
#pragma unroll
    for (int k = 0; k < kIgBatch; ++k) {
      const float4 e0 = sm[b0 + k];
      const float4 e1 = sc[b0 + k];
      uu[k] = e0.w;
      al[k] = fminf(p.alpha_max, alpha_raw(e0.x, e0.y, e0.z, e1.x, e1.y, e1.z, lo));
    }
#pragma unroll
    for (int k = 0; k < kIgBatch; ++k) {
      const float alpha = al[k];
      if (alpha < p.alpha_min) continue;
      const float w = T * alpha;   // T (1 - alpha) taken as T - w: one instruction less
      const float Tn = T - w;
      if (Tn < p.T_min) { T = 0.f; continue; }
      cu += w * uu[k];
      T = Tn;
    }
  }
}

// Persistent U-only compositing: every warp takes (tile, pixel block) work items
// from a device counter, longest tile list first, until the batch is exhausted,
// and writes the sum of U over its pixels to the item's own slot (fixed shuffle
// tree), never accumulating, so the result does not depend on scheduling.
template <int kIgBatch>
__global__ void __launch_bounds__(kIgWarps * 32) k_ig_items(gs_proj proj, gs_bins bins,
                                                             const gs_camera* __restrict__ cams, int n_views,
                                                             gs_params p, const uint32_t* __restrict__ order,
                                                             float* __restrict__ item_sum, int64_t item_cap,
                                                             uint32_t* __restrict__ work) {
  // staged entries of each warp, a ring of kIgRing: (C0, Cu, Cv, u), (k.x, k.y, k.z, 0) (ig_stage)
  __shared__ float4 s_stage[kIgWarps][2][kIgRing];
  static_assert(kIgRing % kIgBatch == 0 && kIgRing >= 32 + kIgBatch, "ring holds a group plus a partial chunk");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  float4* sm = s_stage[warp][0];
  float4* sc = s_stage[warp][1];
  uint32_t n_items = proj.view_info[kVI * n_views + 2] / kPix;
  if ((int64_t)n_items > item_cap) n_items = (uint32_t)item_cap;
  const float4* SP = reinterpret_cast<const float4*>(proj.splat);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(work, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    // items are handed out longest tile list first; each writes its own slot
    const uint32_t slot = __ldg(order + item);
    TileInfo ti;
    if (!warp_item_setup<kPix>(proj, bins, cams, n_views, slot, ti)) {
      if (lane == 0) item_sum[slot] = 0.f;
      continue;
    }
    WarpBlock wb;
    warp_block<kPix>(ti, wb);
    static_assert(kPix == 1, "one pixel per lane: the staged exponent and the live-pixel box assume it");
    const float ln_amin = __logf(p.alpha_min);
    const float bx_full = wb.bx0, by_full = wb.by0;   // centre of the block's first pixel
    const float ccx = bx_full + 3.5f, ccy = by_full + 1.5f;   // centre of the 8x4 block
    const LaneOffsets lo = lane_offsets(lane);
    // T = 0 marks a saturated pixel (and one outside the image): the stop rule sets it,
    // and a zero T adds nothing and stays zero, so no separate flag is kept
    float T = (wb.px < ti.W && wb.py < ti.H) ? 1.f : 0.f, cu = 0.f;
    const uint32_t n = ti.end - ti.beg;
    const uint32_t* rl = bins.rec + ti.beg;
    uint32_t rA = 0, rB = 0, rC = 0;
    if ((uint32_t)lane < n) rA = __ldg(rl + lane);
    if (32u + lane < n) rB = __ldg(rl + 32 + lane);
    if (64u + lane < n) rC = __ldg(rl + 64 + lane);
    float4 mA = z4, mB = z4;
    if ((uint32_t)lane < n) mA = __ldg(SP + 2 * (size_t)rA);
    if (32u + lane < n) mB = __ldg(SP + 2 * (size_t)rB);
    bool ovA = (uint32_t)lane < n && box_overlaps(mA, wb);
    float4 cA = z4;
    if (ovA) cA = __ldg(SP + 2 * (size_t)rA + 1);
    uint32_t head = 0, tail = 0;   // ring entries [head, tail) are staged and not yet composited
    for (uint32_t g = 0; g < n; g += 32) {
      const uint32_t lm = __ballot_sync(0xffffffffu, T != 0.f);
      if (!lm) break;
      // the culls below test the bounding box of the block's live pixels (lane l holds pixel
      // (l mod 8, l div 8)): an entry that reaches only saturated pixels adds nothing
      {
        const uint32_t cols = (lm | (lm >> 8) | (lm >> 16) | (lm >> 24)) & 0xFFu;
        const uint32_t rows = ((lm & 0xFFu) ? 1u : 0u) | ((lm & 0xFF00u) ? 2u : 0u) |
                              ((lm & 0xFF0000u) ? 4u : 0u) | ((lm & 0xFF000000u) ? 8u : 0u);
        wb.bx0 = bx_full + (float)(__ffs(cols) - 1);
        wb.bx1 = bx_full + (float)(31 - __clz(cols));
        wb.by0 = by_full + (float)(__ffs(rows) - 1);
        wb.by1 = by_full + (float)(31 - __clz(rows));
      }
      const bool ovB = g + 32 + lane < n && box_overlaps(mB, wb);
      float4 cB = z4;
      if (ovB) cB = __ldg(SP + 2 * (size_t)rB + 1);
      float4 mC = z4;
      if (g + 64 + lane < n) mC = __ldg(SP + 2 * (size_t)rC);
      uint32_t rD = 0;
      if (g + 96 + lane < n) rD = __ldg(rl + g + 96 + lane);
      ovA = ovA && ellipse_reaches(mA, cA, wb, ln_amin);
      const uint32_t m = __ballot_sync(0xffffffffu, ovA);
      if (m) {
        // the overlapping entries join the ring in list order; whole chunks of kIgBatch
        // are composited at once and a partial chunk waits for the next group's entries
        if (ovA) {
          const uint32_t s = (tail + __popc(m & lt)) & (kIgRing - 1);
          ig_stage(mA, cA, ccx, ccy, sm[s], sc[s]);
        }
        tail += __popc(m);
        __syncwarp();
        const uint32_t chunks = (tail - head) / kIgBatch;
        composite_chunks<kIgBatch>(sm, sc, head, chunks, lo, p, T, cu);
        head += chunks * kIgBatch;
        __syncwarp();
      }
      mA = mB; ovA = ovB; cA = cB;
      rB = rC; mB = mC;
      rC = rD;
    }
    // the last partial chunk, padded with entries of C0 = -inf (alpha = 0: adds nothing)
    if (tail != head && __any_sync(0xffffffffu, T != 0.f)) {
      const uint32_t b0 = head & (kIgRing - 1);
      if ((uint32_t)lane >= tail - head && (uint32_t)lane < kIgBatch) {
        sm[b0 + lane] = make_float4(-INFINITY, 0.f, 0.f, 0.f);
        sc[b0 + lane] = z4;
      }
      __syncwarp();
      composite_chunks<kIgBatch>(sm, sc, head, 1u, lo, p, T, cu);
      __syncwarp();
    }
    float su = cu;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) su += __shfl_down_sync(0xffffffffu, su, d);
    if (lane == 0) item_sum[slot] = su;
  }
}

// IG_v = (1 / P_v) * sum over the view's warp items, in a fixed order.
__global__ void __launch_bounds__(256) k_ig_views(const uint32_t* __restrict__ view_info,
                                                   const gs_camera* __restrict__ cams, int n_views,
                                                   const float* __restrict__ item_sum, int64_t item_cap,
                                                   float* __restrict__ ig) {
  __shared__ float s_red[32];
  const int v = blockIdx.x;
  const uint32_t i0 = view_info[kVI * v + 2] / kPix;
  uint32_t i1 = view_info[kVI * (v + 1) + 2] / kPix;
  if ((int64_t)i1 > item_cap) i1 = (uint32_t)item_cap;
  const int W = cams[v].width, H = cams[v].height;
  float s = 0.f;
  // fixed assignment of items to threads and a fixed reduction tree: deterministic
  for (int64_t i = (int64_t)i0 + threadIdx.x; i < (int64_t)i1; i += blockDim.x) s += item_sum[i];
  s = block_sum_fixed(s, s_red);
  if (threadIdx.x == 0) ig[v] = (W > 0 && H > 0) ? s / ((float)W * (float)H) : 0.f;
}

__global__ void k_zero_words(uint32_t* p, int n) {
  if (threadIdx.x < n) p[threadIdx.x] = 0u;
}

// Sort key of each warp item for longest-first scheduling:
// 0xFFFF - min(length of its tile's list, 0xFFFF).
__global__ void k_item_cost(const gs_proj proj, const gs_bins bins, int n_views, int64_t item_cap,
                            uint32_t* __restrict__ key) {
  uint32_t n = proj.view_info[kVI * n_views + 2] / kPix;
  if ((int64_t)n > item_cap) n = (uint32_t)item_cap;
  // 64-bit index: a 32-bit one could wrap past n when n is near 2^32 and never leave the loop
  for (int64_t i64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i64 < (int64_t)n;
       i64 += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)i64;
    const int v = find_view(proj.view_info, n_views, i * kPix, 2);
    const uint32_t code = proj.view_info[kVI * v + 3];
    const uint32_t wpt = ((code & 0xffu) * ((code >> 8) & 0xffu)) / (32 * kPix);
    uint32_t len = 0;
    if (wpt) {
      const uint32_t tile = proj.view_info[kVI * v] + (i - proj.view_info[kVI * v + 2] / kPix) / wpt;
      if ((int64_t)tile < bins.tile_capacity) len = bins.ranges[2 * (size_t)tile + 1] - bins.ranges[2 * (size_t)tile];
    }
    key[i] = 0xFFFFu - (len < 0xFFFFu ? len : 0xFFFFu);
  }
}

// The persistent compositing kernel at one chunk depth: one CTA per resident slot.
template <int kB>
cudaError_t launch_ig_items(const gs_proj& proj, const gs_bins& bins, const gs_camera* cams, int n_views,
                            const gs_params& p, const uint32_t* order, float* item_sum, int64_t item_cap,
                            uint32_t* work, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ig_items<kB>, kIgWarps * 32, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  if (grid * kIgWarps > item_cap) grid = (item_cap + kIgWarps - 1) / kIgWarps;
  if (grid < 1) grid = 1;
  k_ig_items<kB><<<(unsigned)grid, kIgWarps * 32, 0, st>>>(proj, bins, cams, n_views, p, order, item_sum, item_cap,
                                                           work);
  note_launch();
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_render_fwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_camera* cams,
                              int n_views, const gs_params& p, const gs_image& img, cudaStream_t st) {
  const int64_t items = bins.tile_capacity * (32 / kPix);   // upper bound: at most 32 items per tile
  if (items > 0) {
    const unsigned grid = (unsigned)((items + kFwdWarps - 1) / kFwdWarps);
    const int b = p.fwd_batch ? p.fwd_batch : kFwdBatchDefault;
    if (b == 1)
      k_render_fwd<1><<<grid, kFwdWarps * 32, 0, st>>>(map, proj, bins, cams, n_views, p, img, (uint32_t)items);
    else if (b == 4)
      k_render_fwd<4><<<grid, kFwdWarps * 32, 0, st>>>(map, proj, bins, cams, n_views, p, img, (uint32_t)items);
    else
      k_render_fwd<2><<<grid, kFwdWarps * 32, 0, st>>>(map, proj, bins, cams, n_views, p, img, (uint32_t)items);
    note_launch();
  }
  return cudaGetLastError();
}

size_t ig_ws_bytes(int64_t n, int n_views, int64_t rec_cap, int64_t pair_cap, int64_t tile_cap) {
  if (rec_cap <= 0) rec_cap = n * (int64_t)n_views;
  Carver c(nullptr);
  c.take<uint32_t>(1);                                   // record count
  c.take<uint32_t>(kVI * (size_t)(n_views + 1));         // view info
  c.take<float4>(2 * (size_t)rec_cap);                   // splat (no view ids: segments from grp_base)
  c.take<ushort4>(rec_cap);                              // rect
  c.take<uint32_t>(rec_cap);                             // depth key
  const int64_t slots = ((n + 31) / 32) * (int64_t)n_views;
  c.take<uint32_t>(slots);                               // grp_mask
  c.take<uint32_t>(slots + 1);                           // grp_base
  c.take<uint32_t>(1);                                   // pair count
  c.take<uint32_t>(pair_cap);                            // rec
  c.take<uint32_t>(2 * tile_cap);                        // ranges
  size_t a = project_ws_bytes(n, n_views), b = bin_ws_bytes(rec_cap, pair_cap, tile_cap, n_views);
  const size_t o = ig_composite_ws_bytes(tile_cap);
  c.take<char>(a > b ? (a > o ? a : o) : (b > o ? b : o));
  return align_up(c.off, 256);
}

size_t ig_composite_ws_bytes(int64_t tile_cap) {
  const int64_t item_cap = 32 * tile_cap;
  Carver c(nullptr);
  c.take<float>(item_cap);       // per-item sums
  c.take<uint32_t>(4);           // work counter
  c.take<uint32_t>(item_cap);    // order keys / values, ping-pong
  c.take<uint32_t>(item_cap);
  c.take<uint32_t>(item_cap);
  c.take<uint32_t>(item_cap);
  c.take<char>(sort_temp_bytes(item_cap));
  return align_up(c.off, 256);
}

cudaError_t launch_ig_composite(const gs_proj& proj, const gs_bins& bins, const gs_camera* cams, int n_views,
                                const gs_params& p, float* ig_out, void* ws, cudaStream_t st) {
  const int64_t item_cap = 32 * bins.tile_capacity;
  Carver c(ws);
  float* item_sum = c.take<float>(item_cap);
  uint32_t* work = c.take<uint32_t>(4);
  uint32_t* ok_a = c.take<uint32_t>(item_cap);
  uint32_t* ov_a = c.take<uint32_t>(item_cap);
  uint32_t* ok_b = c.take<uint32_t>(item_cap);
  uint32_t* ov_b = c.take<uint32_t>(item_cap);
  void* otmp = c.take<char>(sort_temp_bytes(item_cap));
  k_zero_words<<<1, 32, 0, st>>>(work, 4);
  note_launch();
  // longest tile lists first
  {
    int64_t gb = (item_cap + 255) / 256;
    if (gb > 4096) gb = 4096;
    k_item_cost<<<(unsigned)gb, 256, 0, st>>>(proj, bins, n_views, item_cap, ok_a);
    note_launch();
  }
  bool in_a = false;
  cudaError_t e = radix_sort(ok_a, nullptr, SortBufs{ok_a, ov_a, ok_b, ov_b},
                             proj.view_info + kVI * n_views + 2, item_cap, 0, 16, otmp, st, &in_a);
  if (e != cudaSuccess) return e;
  const uint32_t* order = in_a ? ov_a : ov_b;
  const int b = p.ig_batch ? p.ig_batch : kIgBatchDefault;
  e = b == 4 ? launch_ig_items<4>(proj, bins, cams, n_views, p, order, item_sum, item_cap, work, st)
    : b == 16 ? launch_ig_items<16>(proj, bins, cams, n_views, p, order, item_sum, item_cap, work, st)
              : launch_ig_items<8>(proj, bins, cams, n_views, p, order, item_sum, item_cap, work, st);
  if (e != cudaSuccess) return e;
  k_ig_views<<<n_views, 256, 0, st>>>(proj.view_info, cams, n_views, item_sum, item_cap, ig_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_info_gain(const gs_map& map, const gs_camera* cams, int n_views, const gs_params& p,
                             float* ig_out, uint32_t* status, int64_t rec_cap, int64_t pair_cap, int64_t tile_cap,
                             void* ws, cudaStream_t st) {
  if (rec_cap <= 0) rec_cap = map.n * (int64_t)n_views;
  Carver c(ws);
  gs_proj proj;
  proj.capacity = rec_cap;
  proj.count = c.take<uint32_t>(1);
  proj.status = status;
  proj.view_info = c.take<uint32_t>(kVI * (size_t)(n_views + 1));
  proj.gid = nullptr;    // Gaussian ids are not needed to score views
  proj.view = nullptr;   // nor view ids: binning finds each view's records through grp_base
  proj.splat = (float*)c.take<float4>(2 * (size_t)rec_cap);
  proj.color_d = nullptr;   // not needed to score views: the projection skips the colours
  proj.rect = (uint16_t*)c.take<ushort4>(rec_cap);
  proj.depth_key = c.take<uint32_t>(rec_cap);
  const int64_t slots = ((map.n + 31) / 32) * (int64_t)n_views;
  proj.grp_mask = c.take<uint32_t>(slots);
  proj.grp_base = c.take<uint32_t>(slots + 1);
  gs_bins bins;
  bins.pair_capacity = pair_cap;
  bins.tile_capacity = tile_cap;
  bins.count = c.take<uint32_t>(1);
  bins.tile = nullptr;   // compositing needs only the record of each pair and the ranges
  bins.rec = c.take<uint32_t>(pair_cap);
  bins.ranges = c.take<uint32_t>(2 * tile_cap);
  bins.item_order = nullptr;   // the compositing orders its items by exact list length itself
  bins.item_capacity = 0;
  size_t a = project_ws_bytes(map.n, n_views), b = bin_ws_bytes(rec_cap, pair_cap, tile_cap, n_views);
  const size_t o = ig_composite_ws_bytes(tile_cap);
  void* inner = c.take<char>(a > b ? (a > o ? a : o) : (b > o ? b : o));

  cudaError_t e = launch_project(map, cams, n_views, p, proj, inner, st);
  if (e != cudaSuccess) return e;
  e = launch_bin_sort(proj, cams, n_views, p, bins, inner, st);
  if (e != cudaSuccess) return e;
  // the inner workspace is free again once binning is done
  return launch_ig_composite(proj, bins, cams, n_views, p, ig_out, inner, st);
}

}  // namespace gs
