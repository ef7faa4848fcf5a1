// gs_common.cuh -- device-side building blocks shared by the splatting kernels.
//
// Projection arithmetic follows RT-GuIDE (arXiv 2409.18122) Sec. III: world-to-
// camera t = R^T (mu - T), depth d = t_z, mu_2D = K t / t_z, generalised to the
// EWA 2D covariance J W Sigma W^T J^T of an anisotropic Gaussian.
//
// The integer outcomes of the projection -- whether a Gaussian is culled for a
// view, its depth sort key and its tile rectangle -- are computed with a fixed
// sequence of correctly rounded IEEE-754 float operations written as explicit
// __f*_rn intrinsics (never contracted or reordered by the compiler), plus the
// exp/log below.  The results are therefore reproducible bit for bit by any
// IEEE-754 implementation that performs the same operations.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

// ---------------------------------------------------------------- constants
constexpr int kMaxViewsPerChunk = 128;   // cameras staged in shared memory at a time

// view_info layout: [V+1][4] = (first global tile, first pixel, first warp item,
// tile_w | tile_h << 8 | tiles_x << 16); a warp item is an 8x4 pixel block of a tile.
constexpr int kVI = 4;

__host__ __device__ __forceinline__ bool valid_tile(int tw, int th) {
  const int b = tw * th;
  return (tw == 8 || tw == 16 || tw == 32 || tw == 64) && th >= 8 && th % 8 == 0 &&
         (b == 64 || b == 128 || b == 256 || b == 512 || b == 1024);
}

// Per-view constants derived from a gs_camera, staged in shared memory.  The
// first 64 bytes (rotation, centre, guard slopes, focal lengths) are what the
// cull of every (Gaussian, view) pair reads, as four 16-byte loads.
struct __align__(16) CamC {
  float R[9];
  float T[3];
  float gx, gy;          // guard-band slopes guard * (W/2) / fx, guard * (H/2) / fy
  float fx, fy;
  float cx, cy;
  int W, H;
  int tw, th;            // this view's tile size (powers of two)
  int sx, sy;            // log2 of tw, th
  int tiles_x, tiles_y;
  uint32_t tile_base;
  uint32_t pix_base;
};

// ---------------------------------------------------------------- float math
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// e^x for the projection: Cody & Waite additive range reduction x = k ln2 + r
// (ln 2 split into 355/512 and a correction so that k * hi is exact), the
// Taylor series of e^r to r^7 in Horner form, and 2^k from the exponent bits.
// Input clamped to [-87, 88] so 2^k stays normal.
__device__ __forceinline__ float ex32(float x) {
  if (x < -87.0f) x = -87.0f;
  if (x > 88.0f) x = 88.0f;
  float kf = rintf(fmul(x, 1.44269504088896341f));
  float r = ffma(-kf, 0.693359375f, x);
  r = ffma(-kf, -2.12194440054690583e-4f, r);
  float p = 0x1.a01a02p-13f;       // 1/7!
  p = ffma(p, r, 0x1.6c16c2p-10f);  // 1/6!
  p = ffma(p, r, 0x1.111112p-7f);   // 1/5!
  p = ffma(p, r, 0x1.555556p-5f);   // 1/4!
  p = ffma(p, r, 0x1.555556p-3f);   // 1/3!
  p = ffma(p, r, 0.5f);
  p = ffma(p, r, 1.0f);
  p = ffma(p, r, 1.0f);
  int k = (int)kf;
  float scale = __uint_as_float((uint32_t)(k + 127) << 23);
  return fmul(p, scale);
}

// ln y for finite normal y > 0: y = m 2^e, m in [sqrt(1/2), sqrt(2)),
// ln m = 2 atanh(s) with s = (m - 1)/(m + 1), odd series to s^13.
__device__ __forceinline__ float lg32(float y) {
  uint32_t b = __float_as_uint(y);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > 1.41421354f) { m = fmul(m, 0.5f); e += 1; }
  float s = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
  float s2 = fmul(s, s);
  float p = 0x1.3b13b2p-4f;          // 1/13
  p = ffma(p, s2, 0x1.745d18p-4f);   // 1/11
  p = ffma(p, s2, 0x1.c71c72p-4f);   // 1/9
  p = ffma(p, s2, 0x1.24924ap-3f);   // 1/7
  p = ffma(p, s2, 0x1.99999ap-3f);   // 1/5
  p = ffma(p, s2, 0x1.555556p-2f);   // 1/3
  float t = fmul(s, s2);
  float lm = ffma(t, p, s);
  lm = fadd(lm, lm);
  float ef = (float)e;
  return ffma(ef, 0.693359375f, ffma(ef, -2.12194440054690583e-4f, lm));
}

// ---------------------------------------------------------------- per Gaussian
// View-independent part of the projection.
struct GaussPre {
  bool valid;
  float S[6];     // 3D covariance upper triangle 00 01 02 11 12 22
  float Q;        // alpha >= alpha_min  <=>  q <= Q
  float o;        // opacity
};

__device__ __forceinline__ bool finite4(float4 a) {
  return isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w);
}

__device__ __forceinline__ float sym3(const float* S, int i, int j) {
  // upper-triangle index of (i, j)
  int a = i < j ? i : j, b = i < j ? j : i;
  return S[a == 0 ? b : (a == 1 ? 2 + b : 5)];
}

// Rotation matrix (row-major) of the normalised quaternion (w, x, y, z), with the
// same operation order as the decision arithmetic requires.
__device__ __forceinline__ void quat_rot_dec(float w, float x, float y, float z, float* R) {
  float xx = fmul(x, x), yy = fmul(y, y), zz = fmul(z, z);
  float xy = fmul(x, y), xz = fmul(x, z), yz = fmul(y, z);
  float wx = fmul(w, x), wy = fmul(w, y), wz = fmul(w, z), t;
  t = fadd(yy, zz); R[0] = fsub(1.0f, fadd(t, t));
  t = fsub(xy, wz); R[1] = fadd(t, t);
  t = fadd(xz, wy); R[2] = fadd(t, t);
  t = fadd(xy, wz); R[3] = fadd(t, t);
  t = fadd(xx, zz); R[4] = fsub(1.0f, fadd(t, t));
  t = fsub(yz, wx); R[5] = fadd(t, t);
  t = fsub(xz, wy); R[6] = fadd(t, t);
  t = fadd(yz, wx); R[7] = fadd(t, t);
  t = fadd(xx, yy); R[8] = fsub(1.0f, fadd(t, t));
}

__device__ __forceinline__ GaussPre gauss_pre(float4 mo, float4 su, float4 q, float alpha_min) {
  GaussPre g;
  g.valid = false;
  g.Q = 0.f;
  g.o = 0.f;
  if (!finite4(mo) || !isfinite(su.x) || !isfinite(su.y) || !isfinite(su.z) || !finite4(q)) return g;
  float n2 = ffma(q.x, q.x, ffma(q.y, q.y, ffma(q.z, q.z, fmul(q.w, q.w))));
  if (!(n2 > 0.0f) || !isfinite(n2)) return g;
  float rn = __fsqrt_rn(n2);
  float w = fdiv(q.x, rn), x = fdiv(q.y, rn), y = fdiv(q.z, rn), z = fdiv(q.w, rn);
  float R[9];
  quat_rot_dec(w, x, y, z, R);
  float s2[3] = {ex32(fadd(su.x, su.x)), ex32(fadd(su.y, su.y)), ex32(fadd(su.z, su.z))};
  float A[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) A[3 * i + k] = fmul(R[3 * i + k], s2[k]);
  const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    int i = I[e], j = J[e];
    g.S[e] = ffma(A[3 * i + 0], R[3 * j + 0], ffma(A[3 * i + 1], R[3 * j + 1], fmul(A[3 * i + 2], R[3 * j + 2])));
  }
  float o = fdiv(1.0f, fadd(1.0f, ex32(-mo.w)));
  g.o = o;
  if (alpha_min > 0.0f) {
    float inv = fdiv(1.0f, alpha_min);
    float xo = fmul(o, inv);
    if (!(xo >= 1.0f)) return g;
    float l = lg32(xo);
    g.Q = fadd(l, l);
  } else {
    if (!(o > 0.0f)) return g;
    g.Q = __int_as_float(0x7f800000);  // +inf: unbounded support
  }
  g.valid = true;
  return g;
}

// Support half-widths (rx, ry) of a record as two IEEE half floats rounded up, in
// the bits of one float (rx in the low 16 bits): a conservative bound, used only to
// skip Gaussians that cannot reach a pixel block.
__device__ __forceinline__ float pack_ext(float rx, float ry) {
  const uint32_t lo = __half_as_ushort(__float2half_ru(rx));
  const uint32_t hi = __half_as_ushort(__float2half_ru(ry));
  return __uint_as_float(lo | (hi << 16));
}

__device__ __forceinline__ void unpack_ext(float e, float& rx, float& ry) {
  const uint32_t b = __float_as_uint(e);
  rx = __half2float(__ushort_as_half((unsigned short)(b & 0xffffu)));
  ry = __half2float(__ushort_as_half((unsigned short)(b >> 16)));
}

// ---------------------------------------------------------------- per view
struct ViewProj {
  float mx, my;      // mu_2D
  float depth;       // t_z
  float ca, cb, cc;  // conic
  float rx, ry;      // support half-widths in pixels
  int x0, y0, x1, y1;  // tile rect, ends exclusive
};

// Returns true if the Gaussian is visible in the view and fills `vp`.
// The first culls of view_proj (near plane, guard band), with the same operations:
// view_proj can only accept a pair this accepts.
__device__ __forceinline__ bool frustum_ok(float4 mo, const CamC& c, float near_plane) {
  const float4* c4 = reinterpret_cast<const float4*>(&c);
  const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2], q3 = c4[3];
  const float dx = fsub(mo.x, q2.y), dy = fsub(mo.y, q2.z), dz = fsub(mo.z, q2.w);
  const float tx = ffma(q1.z, dz, ffma(q0.w, dy, fmul(q0.x, dx)));
  const float ty = ffma(q1.w, dz, ffma(q1.x, dy, fmul(q0.y, dx)));
  const float tz = ffma(q2.x, dz, ffma(q1.y, dy, fmul(q0.z, dx)));
  return tz > near_plane && !(fabsf(tx) > fmul(q3.x, tz)) && !(fabsf(ty) > fmul(q3.y, tz));
}

// Group cull: false only if no centre within `rad` of (gc) can pass frustum_ok for the
// view.  For a point p with |p - gc| <= rad and t = R^T (p - T): t_z <= t_z(gc) + rad, and
// its signed distance to each side plane t_x = +-gx t_z (t_y = +-gy t_z) differs from the
// centre's by at most rad.  `m` covers the rounding of frustum_ok's FP32 evaluation (a few
// ulp of |p - T|) with a wide margin, so the cull never drops a pair frustum_ok accepts.
__device__ __forceinline__ bool group_may_meet(const float* gc, float rad, const CamC& c, float near_plane) {
  const float dx = gc[0] - c.T[0], dy = gc[1] - c.T[1], dz = gc[2] - c.T[2];
  const float tx = c.R[0] * dx + c.R[3] * dy + c.R[6] * dz;
  const float ty = c.R[1] * dx + c.R[4] * dy + c.R[7] * dz;
  const float tz = c.R[2] * dx + c.R[5] * dy + c.R[8] * dz;
  const float m = 1e-4f * (fabsf(dx) + fabsf(dy) + fabsf(dz) + rad) + 1e-4f;
  const float r = rad + m;
  if (tz + r <= near_plane) return false;
  const float kx = r * sqrtf(1.f + c.gx * c.gx) * 1.0001f;
  const float ky = r * sqrtf(1.f + c.gy * c.gy) * 1.0001f;
  if (tx - c.gx * tz > kx || -tx - c.gx * tz > kx) return false;
  if (ty - c.gy * tz > ky || -ty - c.gy * tz > ky) return false;
  return true;
}

// kFull = false: only the decision (the same operations up to the rectangle test; the
// record's conic, mean and depth are not formed), for the projection's count pass.
template <bool kFull = true>
__device__ __forceinline__ bool view_proj(float4 mo, const GaussPre& g, const CamC& c, float near_plane,
                                          float eps2d, ViewProj& vp) {
  if (!g.valid) return false;
  const float4* c4 = reinterpret_cast<const float4*>(&c);
  const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2], q3 = c4[3];
  const float R[9] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x};
  float dx = fsub(mo.x, q2.y), dy = fsub(mo.y, q2.z), dz = fsub(mo.z, q2.w);
  float tx = ffma(R[6], dz, ffma(R[3], dy, fmul(R[0], dx)));
  float ty = ffma(R[7], dz, ffma(R[4], dy, fmul(R[1], dx)));
  float tz = ffma(R[8], dz, ffma(R[5], dy, fmul(R[2], dx)));
  if (!(tz > near_plane)) return false;
  if (fabsf(tx) > fmul(q3.x, tz)) return false;
  if (fabsf(ty) > fmul(q3.y, tz)) return false;
  const float fx = q3.z, fy = q3.w;
  float iz = fdiv(1.0f, tz);
  float u = fmul(tx, iz), v = fmul(ty, iz);
  float mux = ffma(fx, u, c.cx), muy = ffma(fy, v, c.cy);
  float j00 = fmul(fx, iz), j11 = fmul(fy, iz);
  float j02 = -fmul(j00, u), j12 = -fmul(j11, v);
  float T0[3], T1[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    T0[m] = ffma(j00, R[3 * m + 0], fmul(j02, R[3 * m + 2]));
    T1[m] = ffma(j11, R[3 * m + 1], fmul(j12, R[3 * m + 2]));
  }
  float B0[3], B1[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    B0[m] = ffma(T0[0], sym3(g.S, 0, m), ffma(T0[1], sym3(g.S, 1, m), fmul(T0[2], sym3(g.S, 2, m))));
    B1[m] = ffma(T1[0], sym3(g.S, 0, m), ffma(T1[1], sym3(g.S, 1, m), fmul(T1[2], sym3(g.S, 2, m))));
  }
  float a = fadd(ffma(B0[0], T0[0], ffma(B0[1], T0[1], fmul(B0[2], T0[2]))), eps2d);
  float b = ffma(B0[0], T1[0], ffma(B0[1], T1[1], fmul(B0[2], T1[2])));
  float cc = fadd(ffma(B1[0], T1[0], ffma(B1[1], T1[1], fmul(B1[2], T1[2]))), eps2d);
  float det = ffma(a, cc, -fmul(b, b));
  if (!(det > 0.0f)) return false;
  float rx = __fsqrt_rn(fmul(g.Q, a)), ry = __fsqrt_rn(fmul(g.Q, cc));
  float px = fsub(mux, 0.5f), py = fsub(muy, 0.5f);
  float xlo = ceilf(fsub(px, rx)), xhi = floorf(fadd(px, rx));
  float ylo = ceilf(fsub(py, ry)), yhi = floorf(fadd(py, ry));
  xlo = fmaxf(xlo, 0.0f);
  ylo = fmaxf(ylo, 0.0f);
  xhi = fminf(xhi, (float)(c.W - 1));
  yhi = fminf(yhi, (float)(c.H - 1));
  if (!(xlo <= xhi) || !(ylo <= yhi)) return false;
  if (!kFull) return true;
  // pixel -> tile: the coordinates are >= 0 and tile sizes are powers of two
  vp.x0 = (int)xlo >> c.sx;
  vp.y0 = (int)ylo >> c.sy;
  vp.x1 = ((int)xhi >> c.sx) + 1;
  vp.y1 = ((int)yhi >> c.sy) + 1;
  vp.mx = mux;
  vp.my = muy;
  vp.rx = rx;
  vp.ry = ry;
  vp.depth = tz;
  float idet = fdiv(1.0f, det);
  vp.ca = fmul(cc, idet);
  vp.cb = -fmul(b, idet);
  vp.cc = fmul(a, idet);
  return true;
}

// Tile size of a view: the camera's own if set, else the default.
__device__ __forceinline__ void view_tile(const gs_camera& g, int def_w, int def_h, int& tw, int& th) {
  tw = (g.tile_w > 0 && g.tile_h > 0) ? g.tile_w : def_w;
  th = (g.tile_w > 0 && g.tile_h > 0) ? g.tile_h : def_h;
}

// Camera -> per-view constants (guard slopes computed with the same operations
// on every device so the cull decision is reproducible).
__device__ __forceinline__ void load_cam(const gs_camera& g, float guard, int def_tw, int def_th, CamC& c) {
  int tile_w, tile_h;
  view_tile(g, def_tw, def_th, tile_w, tile_h);
  c.tw = tile_w;
  c.th = tile_h;
  c.sx = __ffs(tile_w) - 1;
  c.sy = __ffs(tile_h) - 1;
  c.fx = g.fx; c.fy = g.fy; c.cx = g.cx; c.cy = g.cy;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.R[i] = g.R[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) c.T[i] = g.T[i];
  c.W = g.width;
  c.H = g.height;
  c.gx = fdiv(fmul(guard, fmul(0.5f, (float)g.width)), g.fx);
  c.gy = fdiv(fmul(guard, fmul(0.5f, (float)g.height)), g.fy);
  c.tiles_x = (g.width + tile_w - 1) / tile_w;
  c.tiles_y = (g.height + tile_h - 1) / tile_h;
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ void set_flag(uint32_t* status, uint32_t f) {
  if (status) atomicOr(status, f);
}

// Largest v with view_info[v].field <= key (field 0: first tile, 2: first warp item).
__device__ __forceinline__ int find_view(const uint32_t* view_info, int n_views, uint32_t key, int field) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (view_info[kVI * mid + field] <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace gs
