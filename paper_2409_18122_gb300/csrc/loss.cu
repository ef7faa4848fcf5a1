// loss.cu -- the mapping loss of Eq. 3 (L1 depth + L1 colour + SSIM) and its gradient
// with respect to the rendered images.
//
// Two tiled passes over 32x16-pixel output tiles of each (view, channel), one CTA each:
//   pass 1  loads the tile of x (render) and y (reference) with a 5-pixel halo into shared
//           memory, blurs the five moments x, y, x^2, y^2, xy with the separable 11-tap
//           window (rows, then columns), evaluates S(p) and the partial derivatives of S
//           with respect to the three moments that depend on x (m1 = G*x, m2 = G*x^2,
//           m12 = G*xy), stores those as three planes and reduces S and the L1 terms of the
//           tile into one FP64 partial per CTA;
//   pass 2  blurs the three derivative planes with the same window (the adjoint of the
//           zero-padded correlation with a symmetric window is itself) and forms
//           dS/dx = G*dm1 + 2 x G*dm2 + y G*dm12, then dL/dx with the L1 sign term.
// A one-CTA kernel sums the partials in FP64 in a fixed order.  Without the SSIM term
// (w_ssim = 0) the loss is elementwise: one flat kernel over the colour and one over the
// depth array (contiguous chunks per block, fixed partial slots) replaces both passes.
#include <math.h>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kLTW = 32, kLTH = 16;           // output tile
constexpr int kR = 5, kWin = 2 * kR + 1;      // 11-tap window
constexpr int kInW = kLTW + 2 * kR, kInH = kLTH + 2 * kR;
constexpr int kLossThreads = 256;             // 8 warps: warp w owns output rows 2w, 2w+1
constexpr int kLossViewsPerLaunch = 64;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;
static_assert(kLossThreads == kLTW * kLTH / 2, "two output pixels per thread");

struct LossView {
  int64_t pix_base;  // first pixel of the view in the concatenated images
  int32_t W, H, tile_base, pad;
};

struct LossArgs {
  const float* rgb;
  const float* depth;
  const float* rgb_ref;
  const float* depth_ref;
  float* d_rgb;
  float* d_depth;
  float* dm;        // [3][3P] derivative planes (dS/dm1, dS/dm2, dS/dm12), rgb layout
  double* part;     // [slots][3] per-CTA (sum S, sum |dc|, sum |dd|)
  int64_t P;        // total pixels of all views
  float w_d, w_c, w_s, inv_n, inv_3n;
  float g[kWin];
  int32_t n_views;  // views in this launch
  int32_t part_base;
  LossView v[kLossViewsPerLaunch];
};

__device__ __forceinline__ int loss_view_of(const LossArgs& a, int t) {
  int v = 0;
  for (int i = 1; i < a.n_views; ++i) v = (a.v[i].tile_base <= t) ? i : v;
  return v;
}

__device__ __forceinline__ float sgnf(float d) { return (float)(d > 0.f) - (float)(d < 0.f); }

struct TileGeo {
  int W, H, x0, y0;
  int64_t pix, base;  // first pixel of the view; first element of this (view, channel) plane
};

__device__ __forceinline__ TileGeo tile_geo(const LossArgs& a, int t, int ch) {
  const int vi = loss_view_of(a, t);
  TileGeo g;
  g.W = a.v[vi].W;
  g.H = a.v[vi].H;
  const int tiles_x = (g.W + kLTW - 1) / kLTW;
  const int lt = t - a.v[vi].tile_base;
  g.x0 = (lt % tiles_x) * kLTW;
  g.y0 = (lt / tiles_x) * kLTH;
  g.pix = a.v[vi].pix_base;
  g.base = 3 * g.pix + (int64_t)ch * g.W * g.H;
  return g;
}

// Loads NP planes (src[k] + base) of a halo tile into s[k], zero outside the image.
template <int NP>
__device__ __forceinline__ void load_halo(const float* const* src, const TileGeo& g, float (*s)[kInH][kInW]) {
  for (int i = threadIdx.x; i < kInH * kInW; i += kLossThreads) {
    const int r = i / kInW, c = i - r * kInW;
    const int gx = g.x0 - kR + c, gy = g.y0 - kR + r;
    const bool in = gx >= 0 && gx < g.W && gy >= 0 && gy < g.H;
    const int64_t o = g.base + (int64_t)gy * g.W + gx;
#pragma unroll
    for (int k = 0; k < NP; ++k) s[k][r][c] = in ? src[k][o] : 0.f;
  }
}

// Row pass then column pass of the separable window over NP planes; out[k][q] is the
// blurred value of plane k at output row 2 * warp + q, column lane.
template <int NP>
__device__ __forceinline__ void blur_tile(const LossArgs& a, float (*s_in)[kInH][kInW], float (*s_h)[kInH][kLTW],
                                          float (&out)[NP][2]) {
  for (int i = threadIdx.x; i < kInH * kLTW; i += kLossThreads) {
    const int r = i / kLTW, c = i % kLTW;
    float acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.f;
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
#pragma unroll
      for (int k = 0; k < NP; ++k) acc[k] = fmaf(a.g[j], s_in[k][r][c + j], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) s_h[k][r][c] = acc[k];
  }
  __syncthreads();
  const int c = threadIdx.x & 31, r0 = 2 * (threadIdx.x >> 5);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    float h[kWin + 1];
#pragma unroll
    for (int j = 0; j <= kWin; ++j) h[j] = s_h[k][r0 + j][c];
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
      a0 = fmaf(a.g[j], h[j], a0);
      a1 = fmaf(a.g[j], h[j + 1], a1);
    }
    out[k][0] = a0;
    out[k][1] = a1;
  }
}

// Block sum of three per-thread values into one FP64 partial (fixed order).
__device__ __forceinline__ void block_partial(float v0, float v1, float v2, double* dst) {
  __shared__ float s_red[3][kLossThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    v2 += __shfl_xor_sync(0xffffffffu, v2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = v0;
    s_red[1][threadIdx.x >> 5] = v1;
    s_red[2][threadIdx.x >> 5] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) {
      t0 += (double)s_red[0][w];
      t1 += (double)s_red[1][w];
      t2 += (double)s_red[2][w];
    }
    dst[0] = t0;
    dst[1] = t1;
    dst[2] = t2;
  }
}

__global__ void __launch_bounds__(kLossThreads) k_loss_fwd(const __grid_constant__ LossArgs a) {
  const int t = blockIdx.x, ch = blockIdx.y;
  const TileGeo g = tile_geo(a, t, ch);
  const int c = threadIdx.x & 31, r0 = 2 * (threadIdx.x >> 5);
  float s_sum = 0.f, l1c = 0.f, l1d = 0.f;

  __shared__ float s_in[5][kInH][kInW];  // x, y, x^2, y^2, xy
  __shared__ float s_h[5][kInH][kLTW];
  for (int i = threadIdx.x; i < kInH * kInW; i += kLossThreads) {
    const int r = i / kInW, cc = i - r * kInW;
    const int gx = g.x0 - kR + cc, gy = g.y0 - kR + r;
    const bool in = gx >= 0 && gx < g.W && gy >= 0 && gy < g.H;
    const int64_t o = g.base + (int64_t)gy * g.W + gx;
    const float xv = in ? a.rgb[o] : 0.f, yv = in ? a.rgb_ref[o] : 0.f;
    s_in[0][r][cc] = xv;
    s_in[1][r][cc] = yv;
    s_in[2][r][cc] = xv * xv;
    s_in[3][r][cc] = yv * yv;
    s_in[4][r][cc] = xv * yv;
  }
  __syncthreads();
  float m[5][2];
  blur_tile<5>(a, s_in, s_h, m);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int px = g.x0 + c, py = g.y0 + r0 + q;
    if (px >= g.W || py >= g.H) continue;
    const int64_t o = g.base + (int64_t)py * g.W + px;
    const float mx = m[0][q], my = m[1][q];
    const float sxx = m[2][q] - mx * mx, syy = m[3][q] - my * my, sxy = m[4][q] - mx * my;
    const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
    const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
    const float iD = __frcp_rn(B1 * B2);
    const float S = A1 * A2 * iD;
    s_sum += S;
    if (a.d_rgb) {
      // dS/dm1 = 2 my (A2 - A1) / D - 2 mx S (1/B1 - 1/B2);  dS/dm2 = -S / B2;  dS/dm12 = 2 A1 / D
      a.dm[o] = 2.f * iD * (my * (A2 - A1) - mx * S * (B2 - B1));
      a.dm[3 * a.P + o] = -S * B1 * iD;
      a.dm[6 * a.P + o] = 2.f * A1 * iD;
    }
    l1c += fabsf(s_in[0][r0 + q + kR][c + kR] - s_in[1][r0 + q + kR][c + kR]);
  }

  if (ch == 0 && (a.depth || a.d_depth)) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int px = g.x0 + c, py = g.y0 + r0 + q;
      if (px >= g.W || py >= g.H) continue;
      const int64_t o = g.pix + (int64_t)py * g.W + px;
      const float dd = a.depth ? a.depth[o] - a.depth_ref[o] : 0.f;
      l1d += fabsf(dd);
      if (a.d_depth) a.d_depth[o] = a.w_d * sgnf(dd) * a.inv_n;
    }
  }
  block_partial(s_sum, l1c, l1d, a.part + 3 * ((int64_t)a.part_base + 3 * t + ch));
}

__global__ void __launch_bounds__(kLossThreads) k_loss_ssim_bwd(const __grid_constant__ LossArgs a) {
  __shared__ float s_in[3][kInH][kInW];
  __shared__ float s_h[3][kInH][kLTW];
  const int t = blockIdx.x, ch = blockIdx.y;
  const TileGeo g = tile_geo(a, t, ch);
  const float* src[3] = {a.dm, a.dm + 3 * a.P, a.dm + 6 * a.P};
  load_halo<3>(src, g, s_in);
  __syncthreads();
  float b[3][2];
  blur_tile<3>(a, s_in, s_h, b);
  const int c = threadIdx.x & 31, r0 = 2 * (threadIdx.x >> 5);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int px = g.x0 + c, py = g.y0 + r0 + q;
    if (px >= g.W || py >= g.H) continue;
    const int64_t o = g.base + (int64_t)py * g.W + px;
    const float x = a.rgb[o], y = a.rgb_ref[o];
    const float dS = fmaf(y, b[2][q], fmaf(2.f * x, b[1][q], b[0][q]));
    a.d_rgb[o] = a.w_c * sgnf(x - y) * a.inv_n - a.w_s * a.inv_3n * dS;
  }
}

// Loss without the SSIM term: elementwise over the flat arrays.  Block b takes the
// contiguous elements [b chunk, (b + 1) chunk) and stores its sum of |x - y| in field
// `field` of partial slot slot0 + b (other fields zero); g = w sign(x - y) / N_p if g.
// x == NULL (no depth): differences are zero.
__global__ void __launch_bounds__(kLossThreads) k_loss_l1(const float* __restrict__ x, const float* __restrict__ y,
                                                          float* __restrict__ g, int64_t n, int64_t chunk, float w,
                                                          float inv_n, int field, double* __restrict__ part,
                                                          int64_t slot0) {
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  float acc = 0.f;
#pragma unroll 4
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kLossThreads) {
    const float d = x ? x[i] - y[i] : 0.f;
    acc += fabsf(d);
    if (g) g[i] = w * sgnf(d) * inv_n;
  }
  block_partial(0.f, field == 1 ? acc : 0.f, field == 2 ? acc : 0.f, part + 3 * (slot0 + blockIdx.x));
}

__global__ void __launch_bounds__(kLossThreads)
    k_loss_finish(const double* part, int64_t n_slots, float w_d, float w_c, float w_s, bool ssim, double n_pix,
                  float* out) {
  __shared__ double s[3][kLossThreads];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n_slots; i += kLossThreads)
    for (int k = 0; k < 3; ++k) acc[k] += part[3 * i + k];
  for (int k = 0; k < 3; ++k) s[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int h = kLossThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double l1d = s[2][0] / n_pix, l1c = s[1][0] / n_pix;
    const double ss = ssim ? s[0][0] / (3.0 * n_pix) : (double)NAN;
    double L = (double)w_d * l1d + (double)w_c * l1c;
    if (ssim) L += (double)w_s * (1.0 - ss);
    out[0] = (float)L;
    out[1] = (float)l1d;
    out[2] = (float)l1c;
    out[3] = (float)ss;
  }
}

struct LossLayout {
  int64_t P = 0, tiles = 0;
};

bool loss_layout(const int32_t* sizes, int n_views, LossLayout& lay) {
  if (!sizes || n_views < 1) return false;
  for (int v = 0; v < n_views; ++v) {
    const int64_t W = sizes[2 * v], H = sizes[2 * v + 1];
    if (W < 1 || H < 1 || W > 65536 || H > 65536) return false;
    lay.P += W * H;
    lay.tiles += ((W + kLTW - 1) / kLTW) * ((H + kLTH - 1) / kLTH);
  }
  return lay.P <= ((int64_t)1 << 36) && lay.tiles <= ((int64_t)1 << 30);
}

}  // namespace

size_t image_loss_ws_bytes(const int32_t* sizes, int n_views) {
  LossLayout lay;
  if (!loss_layout(sizes, n_views, lay)) return 0;
  Carver cv(nullptr);
  cv.take<float>(9 * lay.P);
  cv.take<double>(9 * lay.tiles);
  return align_up(cv.off, 256);
}

cudaError_t launch_image_loss(const int32_t* sizes, int n_views, const float* rgb, const float* depth,
                              const float* rgb_ref, const float* depth_ref, const gs_loss_weights& w,
                              float* loss_out, float* d_rgb, float* d_depth, void* ws, cudaStream_t st) {
  LossLayout lay;
  if (!loss_layout(sizes, n_views, lay)) return cudaErrorInvalidValue;
  Carver cv(ws);
  float* dm = cv.take<float>(9 * lay.P);
  double* part = cv.take<double>(9 * lay.tiles);
  const bool ssim = w.w_ssim != 0.f;

  LossArgs a{};
  a.rgb = rgb;
  a.depth = depth;
  a.rgb_ref = rgb_ref;
  a.depth_ref = depth_ref;
  a.d_rgb = d_rgb;
  a.d_depth = d_depth;
  a.dm = dm;
  a.part = part;
  a.P = lay.P;
  a.w_d = w.w_depth;
  a.w_c = w.w_rgb;
  a.w_s = w.w_ssim;
  a.inv_n = (float)(1.0 / (double)lay.P);
  a.inv_3n = (float)(1.0 / (3.0 * (double)lay.P));
  {  // normalised Gaussian window, sigma 1.5
    double gw[kWin], sum = 0.0;
    for (int j = 0; j < kWin; ++j) {
      const double k = j - kR;
      gw[j] = exp(-k * k / (2.0 * 1.5 * 1.5));
      sum += gw[j];
    }
    for (int j = 0; j < kWin; ++j) a.g[j] = (float)(gw[j] / sum);
  }

  int64_t pix = 0, slot = 0;
  if (!ssim) {
    // elementwise: contiguous chunks of at least 4096 elements (at most P / 1024 + 2 partial
    // slots, within the 3 x tiles the workspace holds), about 8 blocks per SM of 152
    int64_t chunk = (3 * lay.P + 152 * 8 - 1) / (152 * 8);
    chunk = (chunk + 4 * kLossThreads - 1) / (4 * kLossThreads) * (4 * kLossThreads);
    if (chunk < 4096) chunk = 4096;
    const int64_t nb_c = (3 * lay.P + chunk - 1) / chunk, nb_d = (lay.P + chunk - 1) / chunk;
    k_loss_l1<<<(unsigned)nb_c, kLossThreads, 0, st>>>(rgb, rgb_ref, d_rgb, 3 * lay.P, chunk, w.w_rgb, a.inv_n, 1,
                                                       part, 0);
    note_launch();
    k_loss_l1<<<(unsigned)nb_d, kLossThreads, 0, st>>>(depth, depth_ref, d_depth, lay.P, chunk, w.w_depth, a.inv_n,
                                                       2, part, nb_c);
    note_launch();
    slot = nb_c + nb_d;
  }
  for (int v0 = 0; v0 < n_views && ssim; v0 += kLossViewsPerLaunch) {
    const int nv = n_views - v0 < kLossViewsPerLaunch ? n_views - v0 : kLossViewsPerLaunch;
    a.n_views = nv;
    a.part_base = (int32_t)slot;
    int32_t tb = 0;
    for (int i = 0; i < nv; ++i) {
      const int W = sizes[2 * (v0 + i)], H = sizes[2 * (v0 + i) + 1];
      a.v[i].pix_base = pix;
      a.v[i].W = W;
      a.v[i].H = H;
      a.v[i].tile_base = tb;
      a.v[i].pad = 0;
      pix += (int64_t)W * H;
      tb += ((W + kLTW - 1) / kLTW) * ((H + kLTH - 1) / kLTH);
    }
    const dim3 grid((unsigned)tb, 3);
    k_loss_fwd<<<grid, kLossThreads, 0, st>>>(a);
    note_launch();
    if (d_rgb) {
      k_loss_ssim_bwd<<<grid, kLossThreads, 0, st>>>(a);
      note_launch();
    }
    slot += 3 * (int64_t)tb;
  }
  k_loss_finish<<<1, kLossThreads, 0, st>>>(part, slot, w.w_depth, w.w_rgb, w.w_ssim, ssim, (double)lay.P,
                                            loss_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
