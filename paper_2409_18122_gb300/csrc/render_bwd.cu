// render_bwd.cu -- gs_render_bwd: adjoint of the compositing and the projection.
//
// Eq. (2) of RT-GuIDE refines the map by back-propagating the rendering loss.
// For a pixel with contributors i = 1..n (front to back), w_i = alpha_i T_i and
// out_ch = sum_i w_i x_i,ch, the derivative with respect to alpha_i is
//   dL/dalpha_i = sum_ch g_ch (x_i,ch T_i - S_i,ch / (1 - alpha_i)),
//   S_i,ch = sum_{j>i} w_j x_j,ch.
// The kernel replays each tile back to front starting from the saved final
// transmittance and last index, recovering T_i = T_{i+1} / (1 - alpha_i), so no
// per-pixel contributor list is stored.  Per-Gaussian screen-space gradients are
// summed over the 32 pixels of a warp through shared memory (rows of lane values, each
// summed by one lane) and added with one scalar atomic per nonzero term; a second
// kernel maps them through the projection per Gaussian (records of one Gaussian
// are contiguous), without atomics.
#include "gs_common.cuh"
#include "gs_internal.h"
#include "render_common.cuh"

namespace gs {
namespace {

constexpr int kBwdWarps = 2;   // warps (work items) per CTA
// The ten gradient terms of each entry are summed over the warp's 32 pixels through shared
// memory: every lane writes its terms of up to kRedBatch entries as rows of 32 values, then
// each lane sums whole rows (eight 16-byte loads) and adds the sum to the record's slot.
// Three entries make 30 rows, one per lane.  Measured on the 500k-Gaussian mapping step
// (backward pass): 12-shuffle reduce-scatter per entry 1.145 ms; batches of 2 / 3 / 4 / 8
// entries 1.11 / 1.06 / 1.18 / 1.36 ms (two passes over the rows, and less occupancy).
constexpr int kRedBatch = 3;
constexpr int kRedPitch = 36;   // floats per row: 16-byte aligned, conflict-free vector reads
constexpr int kPix = 1;        // pixels per lane (8x4 blocks: finer culling beats sharing reductions)

__global__ void __launch_bounds__(kBwdWarps * 32, 14) k_render_bwd(gs_map map, gs_proj proj, gs_bins bins,
                                                                const gs_camera* __restrict__ cams, int n_views,
                                                                gs_params p, gs_image fwd, gs_image_grad grad,
                                                                float4* __restrict__ g2d, uint32_t n_items) {
  __shared__ float4 s_stage[kBwdWarps][3][32];   // (mu), (colour, depth), (scaled conic, o)
  static_assert(kPix == 1, "the entry body below is written for one pixel per lane");
  __shared__ uint32_t s_rec[kBwdWarps][32];
  __shared__ __align__(16) float s_red[kBwdWarps][kRedBatch * 10 * kRedPitch];
  __shared__ uint32_t s_rrec[kBwdWarps][kRedBatch];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t item = blockIdx.x * kBwdWarps + warp;
  if (item >= n_items) return;
  item = ordered_item(bins, proj.view_info, n_views, item);   // longest tile lists first
  TileInfo ti;
  if (!warp_item_setup<kPix>(proj, bins, cams, n_views, item, ti)) return;
  WarpBlock wb;
  warp_block<kPix>(ti, wb);
  float4* sx = s_stage[warp][0];
  float4* sr = s_stage[warp][1];
  float4* sk = s_stage[warp][2];
  uint32_t* srec = s_rec[warp];
  float* red = s_red[warp];
  uint32_t* rrec = s_rrec[warp];
  int nb = 0;   // entries waiting in the batch (warp-uniform)
  // Sums each batched entry's ten terms over the warp (one row of 32 lane values per term,
  // rows spread over the lanes) and adds them to the record's gradient slots:
  // (v0, v1, v2, v3), (v4, v5, v6, -), (v7, v8, v9, -).
  auto flush = [&](int count) {
    __syncwarp();
    for (int r = lane; r < count * 10; r += 32) {
      const float4* row = reinterpret_cast<const float4*>(red + r * kRedPitch);
      float4 a = row[0];
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        const float4 c = row[k];
        a.x += c.x;
        a.y += c.y;
        a.z += c.z;
        a.w += c.w;
      }
      const float sum = (a.x + a.y) + (a.z + a.w);
      const int e = r / 10, j = r - 10 * e;
      if (sum != 0.f) atomicAdd(reinterpret_cast<float*>(g2d + 3 * (size_t)rrec[e]) + (j < 7 ? j : j + 1), sum);
    }
    __syncwarp();
  };
  const float pxc = (float)wb.px + 0.5f;
  const float ln_amin = __logf(p.alpha_min);
  const LaneOffsets lo = lane_offsets(lane);
  const float ccx = wb.bx0 + 3.5f, ccy = wb.by0 + 1.5f;   // centre of the 8x4 block
  const size_t P = (size_t)ti.W * ti.H;
  float pyc[kPix], T[kPix], gr[kPix], gg[kPix], gb[kPix], gd[kPix];
  float Sr[kPix], Sg[kPix], Sb[kPix], Sd[kPix];
  bool inside[kPix];
  int last[kPix];
#pragma unroll
  for (int q = 0; q < kPix; ++q) {
    const int py = wb.py + 4 * q;
    pyc[q] = (float)py + 0.5f;
    inside[q] = wb.px < ti.W && py < ti.H;
    T[q] = 1.f;
    gr[q] = gg[q] = gb[q] = gd[q] = 0.f;
    Sr[q] = Sg[q] = Sb[q] = Sd[q] = 0.f;
    last[q] = 0;
    if (inside[q]) {
      const size_t pix = (size_t)py * ti.W + wb.px;
      const size_t o = (size_t)ti.pix_base + pix;
      T[q] = fwd.T[o];
      last[q] = fwd.last[o];
      if (grad.rgb) {
        const float* base = grad.rgb + 3 * (size_t)ti.pix_base;
        gr[q] = base[pix];
        gg[q] = base[P + pix];
        gb[q] = base[2 * P + pix];
      }
      if (grad.depth) gd[q] = grad.depth[o];
    }
  }
  int my_last = 0;
#pragma unroll
  for (int q = 0; q < kPix; ++q) my_last = max(my_last, last[q]);
  const int wlast = (int)__reduce_max_sync(0xffffffffu, (unsigned)my_last);
  if (wlast == 0) return;
  // groups of 32 entries are walked from the last one any lane used back to the
  // first, with the same four-stage pipeline as the forward kernel (alpha and
  // colour data of the next group, means of the one after, list indices of the
  // one after that)
  const uint32_t* rl = bins.rec + ti.beg;
  const float4* SP = reinterpret_cast<const float4*>(proj.splat);
  const float4* CD = reinterpret_cast<const float4*>(proj.color_d);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  int g = ((wlast - 1) >> 5) << 5;
  uint32_t rA = 0, rB = 0, rC = 0;
  if (g + lane < wlast) rA = __ldg(rl + g + lane);
  if (g >= 32) rB = __ldg(rl + g - 32 + lane);
  if (g >= 64) rC = __ldg(rl + g - 64 + lane);
  float4 mA = z4, mB = z4;
  if (g + lane < wlast) mA = __ldg(SP + 2 * (size_t)rA);
  if (g >= 32) mB = __ldg(SP + 2 * (size_t)rB);
  bool ovA = g + lane < wlast && box_overlaps(mA, wb);
  float4 cA = z4, kA = z4;
  if (ovA) {
    cA = __ldg(SP + 2 * (size_t)rA + 1);
    kA = __ldg(CD + rA);
  }
  for (; g >= 0; g -= 32) {
    const bool ovB = g >= 32 && box_overlaps(mB, wb);
    float4 cB = z4, kB = z4;
    if (ovB) {
      cB = __ldg(SP + 2 * (size_t)rB + 1);
      kB = __ldg(CD + rB);
    }
    float4 mC = z4;
    if (g >= 64) mC = __ldg(SP + 2 * (size_t)rC);
    uint32_t rD = 0;
    if (g >= 96) rD = __ldg(rl + g - 96 + lane);
    ovA = ovA && ellipse_reaches(mA, cA, wb, ln_amin);
    uint32_t m = __ballot_sync(0xffffffffu, ovA);
    if (m) {
      if (ovA) {
        const Exponent e = stage_exponent(mA.x, mA.y, cA, ccx, ccy);
        sx[lane] = make_float4(mA.x, mA.y, e.cu, e.cv);
        sr[lane] = kA;
        sk[lane] = make_float4(e.kx, e.ky, e.kz, e.c0);
        srec[lane] = rA;
      }
      __syncwarp();
      while (m) {
        const int b = 31 - __clz(m);
        m ^= 1u << b;
        const int pos = g + b;   // position in the tile's list
        const float4 mu = sx[b];
        const float4 ks = sk[b];
        // the alpha of the forward pass (same staged coefficients, same operations); ar = o G
        float dx = 0.f, dy = 0.f, ar = 0.f, al = 0.f;
        const bool live = inside[0] && pos < last[0];
        if (live) {
          ar = alpha_raw(ks.w, mu.z, mu.w, ks.x, ks.y, ks.z, lo);
          al = fminf(p.alpha_max, ar);
          dx = __fsub_rn(mu.x, pxc);
          dy = __fsub_rn(mu.y, pyc[0]);
        }
        const bool contrib = live && !(al < p.alpha_min);
        if (!__any_sync(0xffffffffu, contrib)) continue;
        // A lane that does not contribute runs the same arithmetic with alpha = ar = dx = dy = 0:
        // its T and suffix sums stay exactly unchanged (T * 1, S + 0) and every term is zero.
        if (!contrib) al = ar = dx = dy = 0.f;
        const float4 c = sr[b];
        const float inv = __fdividef(1.f, 1.f - al);   // 1 - alpha in [1 - alpha_max, 1]: approximate reciprocal
        const float Ti = T[0] * inv;
        const float w = al * Ti;
        const float dalpha = (gr[0] * c.x + gg[0] * c.y + gb[0] * c.z + gd[0] * c.w) * Ti -
                             (gr[0] * Sr[0] + gg[0] * Sg[0] + gb[0] * Sb[0] + gd[0] * Sd[0]) * inv;
        Sr[0] += w * c.x;
        Sg[0] += w * c.y;
        Sb[0] += w * c.z;
        Sd[0] += w * c.w;
        T[0] = Ti;
        const bool free = ar < p.alpha_max;   // alpha not clamped
        const float dq = free ? -0.5f * al * dalpha : 0.f;    // dL/dq
        // dL/dmu_2D = 2 (a P + b Q, b P + c Q) with P = sum dq dx, Q = sum dq dy (dx = mu_x - p_x):
        // the conic is the record's, so P and Q are summed and k_proj_adjoint applies it
        float v[10];
        v[0] = dq * dx;              // P
        v[1] = dq * dy;              // Q
        v[2] = v[0] * dx;            // dL/da
        v[3] = 2.f * v[0] * dy;      // dL/db
        v[4] = v[1] * dy;            // dL/dc
        v[5] = free ? dalpha * ar : 0.f;          // o dL/do (k_proj_adjoint divides by o)
        v[6] = gd[0] * w;
        v[7] = gr[0] * w;
        v[8] = gg[0] * w;
        v[9] = gb[0] * w;
        // this lane's terms join the batch; a full batch is summed and added
#pragma unroll
        for (int j = 0; j < 10; ++j) red[(nb * 10 + j) * kRedPitch + lane] = v[j];
        if (lane == 0) rrec[nb] = srec[b];
        if (++nb == kRedBatch) {
          flush(nb);
          nb = 0;
        }
      }
      __syncwarp();
    }
    mA = mB; ovA = ovB; cA = cB; kA = kB; rA = rB;
    rB = rC; mB = mC;
    rC = rD;
  }
  if (nb) flush(nb);
}

__global__ void k_zero_g2d(float4* __restrict__ g2d, const uint32_t* count, int64_t cap) {
  int64_t n = (int64_t)*count;
  if (n > cap) n = cap;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
    g2d[i] = z;
}

// Projection adjoint: one thread per Gaussian, gathering its records (one per
// view it is visible in, found through the group masks) without atomics.
__global__ void __launch_bounds__(256) k_proj_adjoint(gs_map map, gs_proj proj, const gs_camera* __restrict__ cams,
                                                      int n_views, const float4* __restrict__ g2d, gs_map_grad out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= map.n) return;
  const int64_t nrec = (int64_t)*proj.count;
  const int64_t grp = g >> 5, n_grp = (map.n + 31) >> 5;   // mask entry of (view v, group) at v * n_grp + group
  const uint32_t bit = 1u << (g & 31), lt = bit - 1u;
  bool any = false;
  for (int v = 0; v < n_views; ++v) any |= (proj.grp_mask[v * n_grp + grp] & bit) != 0;
  float gmu[3] = {0.f, 0.f, 0.f}, go = 0.f, grgb[3] = {0.f, 0.f, 0.f};
  float M3[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  const float4 mo = reinterpret_cast<const float4*>(map.mo)[g];
  const float4 su = reinterpret_cast<const float4*>(map.su)[g];
  const float4 qv = reinterpret_cast<const float4*>(map.q)[g];
  float Rq[9], s2[3], S3[3][3], qn[4], qnorm = 1.f;
  if (any) {
    qnorm = sqrtf(qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w);
    const float w = qv.x / qnorm, x = qv.y / qnorm, y = qv.z / qnorm, z = qv.w / qnorm;
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    Rq[0] = 1.f - 2.f * (y * y + z * z); Rq[1] = 2.f * (x * y - w * z);       Rq[2] = 2.f * (x * z + w * y);
    Rq[3] = 2.f * (x * y + w * z);       Rq[4] = 1.f - 2.f * (x * x + z * z); Rq[5] = 2.f * (y * z - w * x);
    Rq[6] = 2.f * (x * z - w * y);       Rq[7] = 2.f * (y * z + w * x);       Rq[8] = 1.f - 2.f * (x * x + y * y);
    s2[0] = expf(2.f * su.x); s2[1] = expf(2.f * su.y); s2[2] = expf(2.f * su.z);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        S3[i][j] = Rq[3 * i] * s2[0] * Rq[3 * j] + Rq[3 * i + 1] * s2[1] * Rq[3 * j + 1] + Rq[3 * i + 2] * s2[2] * Rq[3 * j + 2];
  }
  for (int v = 0; v < n_views && any; ++v) {
    const uint32_t m = proj.grp_mask[v * n_grp + grp];
    if (!(m & bit)) continue;
    const uint32_t r = proj.grp_base[v * n_grp + grp] + __popc(m & lt);
    if ((int64_t)r >= nrec) continue;
    const float4 A = g2d[3 * (size_t)r], Bv = g2d[3 * (size_t)r + 1], Cv = g2d[3 * (size_t)r + 2];
    const float4 con = reinterpret_cast<const float4*>(proj.splat)[2 * (size_t)r + 1];
    grgb[0] += Cv.x; grgb[1] += Cv.y; grgb[2] += Cv.z;
    go += Bv.y / con.w;   // the compositing summed o dL/do (o = con.w >= alpha_min > 0)
    // slots A.x, A.y hold P = sum dq dx, Q = sum dq dy: dL/dmu_2D = 2 (a P + b Q, b P + c Q)
    const float gmx = 2.f * (con.x * A.x + con.y * A.y), gmy = 2.f * (con.y * A.x + con.z * A.y);
    const float ga = A.z, gb = A.w, gc = Bv.x, gdep = Bv.z;
    const gs_camera& cam = cams[v];
    const float* R = cam.R;
    const float dx = mo.x - cam.T[0], dy = mo.y - cam.T[1], dz = mo.z - cam.T[2];
    const float tx = R[0] * dx + R[3] * dy + R[6] * dz;
    const float ty = R[1] * dx + R[4] * dy + R[7] * dz;
    const float tz = R[2] * dx + R[5] * dy + R[8] * dz;
    // dL/dSigma2D = -C G_C C (symmetric-matrix gradients)
    const float C00 = con.x, C01 = con.y, C11 = con.z;
    const float G00 = ga, G01 = 0.5f * gb, G11 = gc;
    const float t00 = G00 * C00 + G01 * C01, t01 = G00 * C01 + G01 * C11;
    const float t10 = G01 * C00 + G11 * C01, t11 = G01 * C01 + G11 * C11;
    const float S00 = -(C00 * t00 + C01 * t10), S01 = -(C00 * t01 + C01 * t11);
    const float S11 = -(C01 * t01 + C11 * t11);
    const float iz = 1.f / tz, iz2 = iz * iz;
    const float J00 = cam.fx * iz, J02 = -cam.fx * tx * iz2, J11 = cam.fy * iz, J12 = -cam.fy * ty * iz2;
    float T3[2][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      T3[0][m] = J00 * R[3 * m + 0] + J02 * R[3 * m + 2];
      T3[1][m] = J11 * R[3 * m + 1] + J12 * R[3 * m + 2];
    }
    const float GS[2][2] = {{S00, S01}, {S01, S11}};
    // M3 += T3^T GS T3
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float u0 = GS[0][0] * T3[0][i] + GS[1][0] * T3[1][i];
      const float u1 = GS[0][1] * T3[0][i] + GS[1][1] * T3[1][i];
#pragma unroll
      for (int j = 0; j < 3; ++j) M3[i][j] += u0 * T3[0][j] + u1 * T3[1][j];
    }
    // GT3 = 2 GS T3 S3; GJ = GT3 R (GJ[r][k] = sum_m GT3[r][m] R[m][k])
    float GT3[2][3];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const float h0 = GS[rr][0] * T3[0][0] + GS[rr][1] * T3[1][0];
      const float h1 = GS[rr][0] * T3[0][1] + GS[rr][1] * T3[1][1];
      const float h2 = GS[rr][0] * T3[0][2] + GS[rr][1] * T3[1][2];
#pragma unroll
      for (int m = 0; m < 3; ++m) GT3[rr][m] = 2.f * (h0 * S3[0][m] + h1 * S3[1][m] + h2 * S3[2][m]);
    }
    float GJ[2][3];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) GJ[rr][kk] = GT3[rr][0] * R[kk] + GT3[rr][1] * R[3 + kk] + GT3[rr][2] * R[6 + kk];
    const float iz3 = iz2 * iz;
    const float gtx = GJ[0][2] * (-cam.fx * iz2) + gmx * cam.fx * iz;
    const float gty = GJ[1][2] * (-cam.fy * iz2) + gmy * cam.fy * iz;
    const float gtz = GJ[0][0] * (-cam.fx * iz2) + GJ[0][2] * (2.f * cam.fx * tx * iz3) + GJ[1][1] * (-cam.fy * iz2) +
                      GJ[1][2] * (2.f * cam.fy * ty * iz3) - gmx * cam.fx * tx * iz2 - gmy * cam.fy * ty * iz2 + gdep;
#pragma unroll
    for (int m = 0; m < 3; ++m) gmu[m] += R[3 * m + 0] * gtx + R[3 * m + 1] * gty + R[3 * m + 2] * gtz;
  }
  float4 dmo = make_float4(0.f, 0.f, 0.f, 0.f), dsu = dmo, dq = dmo, drgb = dmo;
  if (any) {
    // dL/dRq = 2 M3 Rq diag(s2); dL/ds2_k = (Rq^T M3 Rq)_kk
    float GR[9], gs2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int kk = 0; kk < 3; ++kk)
        GR[3 * i + kk] = 2.f * (M3[i][0] * Rq[kk] + M3[i][1] * Rq[3 + kk] + M3[i][2] * Rq[6 + kk]) * s2[kk];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) s += Rq[3 * i + kk] * M3[i][j] * Rq[3 * j + kk];
      gs2[kk] = s;
    }
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    const float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    const float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] -
                            2.f * x * GR[8]);
    const float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] -
                            2.f * y * GR[8]);
    const float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] +
                            y * GR[7]);
    const float dot = w * gw + x * gx + y * gy + z * gz;
    const float inv = 1.f / qnorm;
    dq = make_float4((gw - w * dot) * inv, (gx - x * dot) * inv, (gy - y * dot) * inv, (gz - z * dot) * inv);
    const float o = 1.f / (1.f + expf(-mo.w));
    dmo = make_float4(gmu[0], gmu[1], gmu[2], go * o * (1.f - o));
    dsu = make_float4(2.f * s2[0] * gs2[0], 2.f * s2[1] * gs2[1], 2.f * s2[2] * gs2[2], 0.f);
    drgb = make_float4(grgb[0], grgb[1], grgb[2], 0.f);
  }
  reinterpret_cast<float4*>(out.dmo)[g] = dmo;
  reinterpret_cast<float4*>(out.dsu)[g] = dsu;
  reinterpret_cast<float4*>(out.dq)[g] = dq;
  reinterpret_cast<float4*>(out.drgb)[g] = drgb;
}

}  // namespace

size_t bwd_ws_bytes(int64_t rec_cap) { return align_up(sizeof(float4) * 3 * (size_t)rec_cap, 256); }

cudaError_t launch_render_bwd(const gs_map& map, const gs_proj& proj, const gs_bins& bins, const gs_image& fwd,
                              const gs_image_grad& g, const gs_camera* cams, int n_views, const gs_params& p,
                              const gs_map_grad& out, void* ws, cudaStream_t st) {
  float4* g2d = (float4*)ws;
  int64_t zb = (3 * proj.capacity + 255) / 256;
  if (zb > 4096) zb = 4096;
  if (zb < 1) zb = 1;
  k_zero_g2d<<<(unsigned)zb, 256, 0, st>>>(g2d, proj.count, proj.capacity);
  note_launch();
  const int64_t items = bins.tile_capacity * (32 / kPix);   // upper bound: at most 32 / kPix items per tile
  if (items > 0) {
    k_render_bwd<<<(unsigned)((items + kBwdWarps - 1) / kBwdWarps), kBwdWarps * 32, 0, st>>>(
        map, proj, bins, cams, n_views, p, fwd, g, g2d, (uint32_t)items);
    note_launch();
  }
  if (map.n > 0) {
    k_proj_adjoint<<<(unsigned)((map.n + 255) / 256), 256, 0, st>>>(map, proj, cams, n_views, g2d, out);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace gs
