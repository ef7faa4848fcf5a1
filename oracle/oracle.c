/*
 * oracle.c -- plain, slow FP64 CPU oracle for the tile-based Gaussian-splatting
 * path (projection, depth-ordered compositing, tile binning, analytic gradient).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant generator with the CUDA path; it is built from this file alone.
 *
 * What it follows (RT-GuIDE, arXiv 2409.18122):
 *   - Sec. III "Gaussian Splatting": Gaussians are sorted by increasing depth
 *     relative to the camera and splatted; projected mean mu_2D = K R^T (mu - T)/d,
 *     d = e3^T R^T (mu - T); pixel colour C(p) = sum_i c_i f_i(p) prod_{j<i}(1 - f_j(p)),
 *     f_i(p) = alpha_i exp(-|p - mu_2D|^2 / (2 r_2D^2)); depth by replacing c_i with d_i.
 *     The paper's Gaussians are isotropic; this oracle uses the anisotropic EWA
 *     generalisation (2D covariance J W Sigma W^T J^T), which reduces to the paper's
 *     r_2D = f r / d for an isotropic Gaussian on the optical axis with no dilation.
 *   - Eq. (2) / Sec. IV-A: map parameters are refined by back-propagation; the
 *     analytic gradient below is the chain rule of the compositing formula above,
 *     computed from explicit per-pixel contributor lists and suffix sums.
 *   - Eq. (nbv), Sec. IV-A: per-Gaussian uncertainty u_i is composited like a colour
 *     channel; its per-view mean is the rendered information-gain proxy.
 *
 * Readings where the paper is silent (opacity clamp 0.99, skip alpha < 1/255,
 * stop before adding when T(1 - alpha) < 1e-4, low-pass dilation eps2d, near plane,
 * guard band, opacity-aware elliptical support box, pixel centres at (u+0.5, v+0.5),
 * ties in depth broken by Gaussian id) are inputs in `prm`.
 *
 * Precision: every value (means, covariances, conics, opacities, weights, colours,
 * depth, gradients) is computed in FP64 from the FP32 inputs.  The integer
 * decisions -- whether a Gaussian is culled for a view, its depth-ordering key and
 * its tile rectangle -- are decided in FP32 with a fixed sequence of correctly
 * rounded IEEE operations (add, sub, mul, div, sqrt, fma, floor, ceil) and the
 * exp/log below, so that both implementations take the same decision bit for bit.
 * exp and log are Cody-Waite style range reductions followed by series, written
 * from the mathematics (see ex32 / lg32).
 *
 * Compile:  gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared oracle.c -o liboracle.so -lm
 * (-ffp-contract=off is required: the FP32 decision path must not be contracted.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* parameter block layout (doubles)                                          */
/* ------------------------------------------------------------------------- */
enum { P_TILE_W = 0, P_TILE_H, P_EPS2D, P_NEAR, P_GUARD, P_ALPHA_MIN, P_ALPHA_MAX, P_T_MIN, P_COUNT };

/* camera block: 16 floats per view: fx fy cx cy R00..R22 (camera-to-world, row-major) Tx Ty Tz;
 * plus 4 ints per view: width height tile_w tile_h (tile size of that view).  */
#define CAMF 16

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* FP32 exp and log (decision path)                                          */
/* ------------------------------------------------------------------------- */
static float f_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t u_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* e^x: x = k ln2 + r with k = rint(x log2 e) and ln 2 split in two parts
 * (Cody & Waite 1980), |r| <= ln2/2, e^r by its Taylor series to r^7 in Horner
 * form, times 2^k built from the exponent bits.  Inputs are clamped to
 * [-87, 88] so that 2^k stays a normal float. */
float ex32(float x) {
  if (x < -87.0f) x = -87.0f;
  if (x > 88.0f) x = 88.0f;
  const float log2e = 1.44269504088896341f;
  const float ln2_hi = 0.693359375f;          /* 355/512: k*ln2_hi is exact */
  const float ln2_lo = -2.12194440054690583e-4f;
  float kf = rintf(x * log2e);
  float r = fmaf(-kf, ln2_hi, x);
  r = fmaf(-kf, ln2_lo, r);
  float p = 0x1.a01a02p-13f;                  /* float(1/5040) */
  p = fmaf(p, r, 0x1.6c16c2p-10f);            /* 1/720 */
  p = fmaf(p, r, 0x1.111112p-7f);             /* 1/120 */
  p = fmaf(p, r, 0x1.555556p-5f);             /* 1/24 */
  p = fmaf(p, r, 0x1.555556p-3f);             /* 1/6 */
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  int k = (int)kf;
  float scale = f_bits((uint32_t)(k + 127) << 23);
  return p * scale;
}

/* ex32 of every element (the collision check's radii). */
void or_ex32v(int64_t n, const float* x, float* y) {
  for (int64_t i = 0; i < n; ++i) y[i] = ex32(x[i]);
}

/* ln y for finite y > 0 (normal): y = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s), s = (m-1)/(m+1), by the odd series 2(s + s^3/3 + ... + s^13/13);
 * ln y = e ln2 + ln m with the same two-part ln 2. */
float lg32(float y) {
  uint32_t b = u_bits(y);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = f_bits((b & 0x7fffffu) | 0x3f800000u);
  if (m > 1.41421354f) { m = m * 0.5f; e += 1; }
  float s = (m - 1.0f) / (m + 1.0f);
  float s2 = s * s;
  float p = 0x1.3b13b2p-4f;                   /* float(1/13) */
  p = fmaf(p, s2, 0x1.745d18p-4f);            /* 1/11 */
  p = fmaf(p, s2, 0x1.c71c72p-4f);            /* 1/9 */
  p = fmaf(p, s2, 0x1.24924ap-3f);            /* 1/7 */
  p = fmaf(p, s2, 0x1.99999ap-3f);            /* 1/5 */
  p = fmaf(p, s2, 0x1.555556p-2f);            /* 1/3 */
  float t = s * s2;
  float lm = fmaf(t, p, s);
  lm = lm + lm;
  const float ln2_hi = 0.693359375f;
  const float ln2_lo = -2.12194440054690583e-4f;
  float ef = (float)e;
  return fmaf(ef, ln2_hi, fmaf(ef, ln2_lo, lm));
}

/* ------------------------------------------------------------------------- */
/* FP32 decision path: cull / depth key / tile rectangle                      */
/* ------------------------------------------------------------------------- */
typedef struct {
  int valid;          /* finite parameters, non-degenerate quaternion, opacity above floor */
  float S[6];         /* 3D covariance upper triangle: 00 01 02 11 12 22 */
  float Q;            /* support bound on the Mahalanobis distance q: alpha >= alpha_min <=> q <= Q */
} dec_gauss;

static int finite4(const float* a) { return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]) && isfinite(a[3]); }

static dec_gauss dec_gaussian(const float* mo, const float* su, const float* q, const double* prm) {
  dec_gauss d;
  memset(&d, 0, sizeof d);
  if (!finite4(mo) || !isfinite(su[0]) || !isfinite(su[1]) || !isfinite(su[2]) || !finite4(q)) return d;
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float n2 = fmaf(w, w, fmaf(x, x, fmaf(y, y, z * z)));
  if (!(n2 > 0.0f) || !isfinite(n2)) return d;
  float rn = sqrtf(n2);
  w = w / rn; x = x / rn; y = y / rn; z = z / rn;
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z, t;
  float R[9];
  t = yy + zz; R[0] = 1.0f - (t + t);
  t = xy - wz; R[1] = t + t;
  t = xz + wy; R[2] = t + t;
  t = xy + wz; R[3] = t + t;
  t = xx + zz; R[4] = 1.0f - (t + t);
  t = yz - wx; R[5] = t + t;
  t = xz - wy; R[6] = t + t;
  t = yz + wx; R[7] = t + t;
  t = xx + yy; R[8] = 1.0f - (t + t);
  float s2[3];
  for (int k = 0; k < 3; ++k) s2[k] = ex32(su[k] + su[k]);
  float A[9];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) A[3 * i + k] = R[3 * i + k] * s2[k];
  int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  for (int e = 0; e < 6; ++e) {
    int i = ij[e][0], j = ij[e][1];
    d.S[e] = fmaf(A[3 * i + 0], R[3 * j + 0], fmaf(A[3 * i + 1], R[3 * j + 1], A[3 * i + 2] * R[3 * j + 2]));
  }
  /* opacity o = 1/(1+e^-logit); cull when o * (1/alpha_min) < 1 */
  float amin = (float)prm[P_ALPHA_MIN];
  float o = 1.0f / (1.0f + ex32(-mo[3]));
  if (amin > 0.0f) {
    float inv = 1.0f / amin;
    float xo = o * inv;
    if (!(xo >= 1.0f)) return d;
    float l = lg32(xo);
    d.Q = l + l;
  } else {
    if (!(o > 0.0f)) return d;
    d.Q = INFINITY;
  }
  d.valid = 1;
  return d;
}

static float sym3(const float* S, int i, int j) {
  static const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return S[idx[i][j]];
}

/* Returns 1 if visible; fills the depth key bits and the tile rectangle [x0,x1) x [y0,y1). */
static int dec_view(const float* mo, const dec_gauss* dg, const float* cam, const int* wh, const double* prm,
                    uint32_t* dkey, int* rect) {
  if (!dg->valid) return 0;
  float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
  const float* R = cam + 4;
  const float* T = cam + 13;
  int W = wh[0], H = wh[1];
  int tw = wh[2], th = wh[3];
  float near = (float)prm[P_NEAR], guard = (float)prm[P_GUARD], eps = (float)prm[P_EPS2D];
  if (W <= 0 || H <= 0) return 0;
  float dx = mo[0] - T[0], dy = mo[1] - T[1], dz = mo[2] - T[2];
  float tx = fmaf(R[6], dz, fmaf(R[3], dy, R[0] * dx));
  float ty = fmaf(R[7], dz, fmaf(R[4], dy, R[1] * dx));
  float tz = fmaf(R[8], dz, fmaf(R[5], dy, R[2] * dx));
  if (!(tz > near)) return 0;
  float gx = (guard * (0.5f * (float)W)) / fx;
  float gy = (guard * (0.5f * (float)H)) / fy;
  if (fabsf(tx) > gx * tz) return 0;
  if (fabsf(ty) > gy * tz) return 0;
  float iz = 1.0f / tz;
  float u = tx * iz, v = ty * iz;
  float mux = fmaf(fx, u, cx), muy = fmaf(fy, v, cy);
  float j00 = fx * iz, j11 = fy * iz;
  float j02 = -(j00 * u), j12 = -(j11 * v);
  float T3[2][3];
  for (int m = 0; m < 3; ++m) {
    T3[0][m] = fmaf(j00, R[3 * m + 0], j02 * R[3 * m + 2]);
    T3[1][m] = fmaf(j11, R[3 * m + 1], j12 * R[3 * m + 2]);
  }
  float B[2][3];
  for (int r = 0; r < 2; ++r)
    for (int m = 0; m < 3; ++m)
      B[r][m] = fmaf(T3[r][0], sym3(dg->S, 0, m), fmaf(T3[r][1], sym3(dg->S, 1, m), T3[r][2] * sym3(dg->S, 2, m)));
  float a = fmaf(B[0][0], T3[0][0], fmaf(B[0][1], T3[0][1], B[0][2] * T3[0][2])) + eps;
  float b = fmaf(B[0][0], T3[1][0], fmaf(B[0][1], T3[1][1], B[0][2] * T3[1][2]));
  float c = fmaf(B[1][0], T3[1][0], fmaf(B[1][1], T3[1][1], B[1][2] * T3[1][2])) + eps;
  float det = fmaf(a, c, -(b * b));
  if (!(det > 0.0f)) return 0;
  float rx = sqrtf(dg->Q * a), ry = sqrtf(dg->Q * c);
  float px = mux - 0.5f, py = muy - 0.5f;
  float xlo = ceilf(px - rx), xhi = floorf(px + rx);
  float ylo = ceilf(py - ry), yhi = floorf(py + ry);
  xlo = fmaxf(xlo, 0.0f); ylo = fmaxf(ylo, 0.0f);
  xhi = fminf(xhi, (float)(W - 1)); yhi = fminf(yhi, (float)(H - 1));
  if (!(xlo <= xhi) || !(ylo <= yhi)) return 0;
  rect[0] = (int)xlo / tw;
  rect[1] = (int)ylo / th;
  rect[2] = (int)xhi / tw + 1;
  rect[3] = (int)yhi / th + 1;
  *dkey = u_bits(tz);
  return 1;
}

/* ------------------------------------------------------------------------- */
/* FP64 value path: projection of one Gaussian into one view                  */
/* ------------------------------------------------------------------------- */
typedef struct {
  double mean[2], conic[3], cov[3], depth, opac;
  double t[3];           /* view-space position */
  double Rq[9], s2[3], S3[9], qn[4], qnorm;
} val_proj;

static void val_project(const double* mo, const double* su, const double* q, const float* camf, const double* prm,
                        val_proj* P) {
  double fx = camf[0], fy = camf[1], cx = camf[2], cy = camf[3];
  double R[9], T[3];
  for (int i = 0; i < 9; ++i) R[i] = camf[4 + i];
  for (int i = 0; i < 3; ++i) T[i] = camf[13 + i];
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
  P->qn[0] = w; P->qn[1] = x; P->qn[2] = y; P->qn[3] = z; P->qnorm = nq;
  double* Rq = P->Rq;
  Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z);     Rq[2] = 2 * (x * z + w * y);
  Rq[3] = 2 * (x * y + w * z);     Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
  Rq[6] = 2 * (x * z - w * y);     Rq[7] = 2 * (y * z + w * x);     Rq[8] = 1 - 2 * (x * x + y * y);
  for (int k = 0; k < 3; ++k) P->s2[k] = exp(2.0 * su[k]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += Rq[3 * i + k] * P->s2[k] * Rq[3 * j + k];
      P->S3[3 * i + j] = s;
    }
  /* t = R^T (mu - T) */
  double d[3] = {mo[0] - T[0], mo[1] - T[1], mo[2] - T[2]};
  for (int k = 0; k < 3; ++k) P->t[k] = R[0 * 3 + k] * d[0] + R[1 * 3 + k] * d[1] + R[2 * 3 + k] * d[2];
  double tx = P->t[0], ty = P->t[1], tz = P->t[2];
  P->mean[0] = fx * tx / tz + cx;
  P->mean[1] = fy * ty / tz + cy;
  P->depth = tz;
  /* J (2x3) and W = R^T; T3 = J W */
  double J[2][3] = {{fx / tz, 0.0, -fx * tx / (tz * tz)}, {0.0, fy / tz, -fy * ty / (tz * tz)}};
  double T3[2][3];
  for (int r = 0; r < 2; ++r)
    for (int m = 0; m < 3; ++m) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += J[r][k] * R[3 * m + k]; /* W[k][m] = R[m][k] */
      T3[r][m] = s;
    }
  double C2[2][2];
  for (int r = 0; r < 2; ++r)
    for (int s = 0; s < 2; ++s) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += T3[r][i] * P->S3[3 * i + j] * T3[s][j];
      C2[r][s] = acc;
    }
  double eps = prm[P_EPS2D];
  double A = C2[0][0] + eps, B = C2[0][1], Cc = C2[1][1] + eps;
  P->cov[0] = A; P->cov[1] = B; P->cov[2] = Cc;
  double det = A * Cc - B * B;
  P->conic[0] = Cc / det; P->conic[1] = -B / det; P->conic[2] = A / det;
  P->opac = 1.0 / (1.0 + exp(-mo[3]));
}

/* ------------------------------------------------------------------------- */
/* projection entry point (dense [V][N] outputs)                              */
/* ------------------------------------------------------------------------- */
void or_project(int64_t N, const float* mo32, const float* su32, const float* q32,
                const double* mo64, const double* su64, const double* q64,
                int V, const float* cam, const int* camwh, const double* prm,
                int8_t* vis, uint32_t* dkey, int32_t* rect,
                double* mean2d, double* conic, double* cov2d, double* depth, double* opac) {
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < N; ++g) {
    dec_gauss dg = dec_gaussian(mo32 + 4 * g, su32 + 4 * g, q32 + 4 * g, prm);
    for (int v = 0; v < V; ++v) {
      int64_t o = (int64_t)v * N + g;
      uint32_t key = 0;
      int r4[4] = {0, 0, 0, 0};
      int ok = dec_view(mo32 + 4 * g, &dg, cam + CAMF * v, camwh + 4 * v, prm, &key, r4);
      vis[o] = (int8_t)ok;
      dkey[o] = key;
      for (int k = 0; k < 4; ++k) rect[4 * o + k] = r4[k];
      if (ok) {
        val_proj P;
        val_project(mo64 + 4 * g, su64 + 4 * g, q64 + 4 * g, cam + CAMF * v, prm, &P);
        mean2d[2 * o] = P.mean[0]; mean2d[2 * o + 1] = P.mean[1];
        for (int k = 0; k < 3; ++k) { conic[3 * o + k] = P.conic[k]; cov2d[3 * o + k] = P.cov[k]; }
        depth[o] = P.depth;
        opac[o] = P.opac;
      } else {
        mean2d[2 * o] = mean2d[2 * o + 1] = 0;
        for (int k = 0; k < 3; ++k) conic[3 * o + k] = cov2d[3 * o + k] = 0;
        depth[o] = 0; opac[o] = 0;
      }
    }
  }
}

/* ------------------------------------------------------------------------- */
/* per-view depth order of the visible Gaussians: ascending (key, id)         */
/* ------------------------------------------------------------------------- */
typedef struct { uint32_t key; int64_t id; } key_id;
static int cmp_key_id(const void* A, const void* B) {
  const key_id* a = (const key_id*)A;
  const key_id* b = (const key_id*)B;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->id != b->id) return a->id < b->id ? -1 : 1;
  return 0;
}

typedef struct {
  int64_t n;          /* number of visible Gaussians */
  int64_t* id;        /* in compositing order */
  val_proj* P;        /* their FP64 projections (same order) */
} view_list;

static void build_view_list(int64_t N, const float* mo32, const float* su32, const float* q32,
                            const double* mo64, const double* su64, const double* q64,
                            const float* camf, const int* wh, const double* prm, view_list* L) {
  key_id* tmp = (key_id*)malloc(sizeof(key_id) * (size_t)(N > 0 ? N : 1));
  int64_t n = 0;
  for (int64_t g = 0; g < N; ++g) {
    dec_gauss dg = dec_gaussian(mo32 + 4 * g, su32 + 4 * g, q32 + 4 * g, prm);
    uint32_t key;
    int r4[4];
    if (dec_view(mo32 + 4 * g, &dg, camf, wh, prm, &key, r4)) { tmp[n].key = key; tmp[n].id = g; ++n; }
  }
  qsort(tmp, (size_t)n, sizeof(key_id), cmp_key_id);
  L->n = n;
  L->id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  L->P = (val_proj*)malloc(sizeof(val_proj) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    int64_t g = tmp[i].id;
    L->id[i] = g;
    val_project(mo64 + 4 * g, su64 + 4 * g, q64 + 4 * g, camf, prm, &L->P[i]);
  }
  free(tmp);
}

static void free_view_list(view_list* L) { free(L->id); free(L->P); }

/* ------------------------------------------------------------------------- */
/* brute-force compositing of selected pixels                                 */
/* pix: K x 3 int32 (view, u, v).  out: K x 5 doubles (r, g, b, depth, unc).   */
/* last_id: id of the last contributing Gaussian (-1 if none).                */
/* n_contrib: number of contributing Gaussians; n_clamp: how many hit the      */
/* alpha clamp.  knife: 1 if a skip or stop decision at this pixel lies within */
/* relative `delta` of its threshold (a decision that FP32 may take otherwise).*/
/* ------------------------------------------------------------------------- */
void or_render(int64_t N, const float* mo32, const float* su32, const float* q32,
               const double* mo64, const double* su64, const double* q64, const double* rgb64,
               int V, const float* cam, const int* camwh, const double* prm,
               int64_t K, const int32_t* pix, double delta,
               double* out, double* tfinal, int64_t* last_id, int32_t* n_contrib, int32_t* n_clamp, int8_t* knife) {
  const double amin = prm[P_ALPHA_MIN], amax = prm[P_ALPHA_MAX], tmin = prm[P_T_MIN];
  view_list* L = (view_list*)calloc((size_t)(V > 0 ? V : 1), sizeof(view_list));
  char* need = (char*)calloc((size_t)(V > 0 ? V : 1), 1);
  for (int64_t k = 0; k < K; ++k) need[pix[3 * k]] = 1;
  for (int v = 0; v < V; ++v)
    if (need[v]) build_view_list(N, mo32, su32, q32, mo64, su64, q64, cam + CAMF * v, camwh + 4 * v, prm, &L[v]);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < K; ++k) {
    int v = pix[3 * k];
    double px = pix[3 * k + 1] + 0.5, py = pix[3 * k + 2] + 0.5;
    double T = 1.0, acc[5] = {0, 0, 0, 0, 0};
    int64_t last = -1;
    int nc = 0, ncl = 0, kn = 0;
    const view_list* Lv = &L[v];
    for (int64_t i = 0; i < Lv->n; ++i) {
      const val_proj* P = &Lv->P[i];
      int64_t g = Lv->id[i];
      double dx = px - P->mean[0], dy = py - P->mean[1];
      double q = P->conic[0] * dx * dx + 2.0 * P->conic[1] * dx * dy + P->conic[2] * dy * dy;
      double a_raw = P->opac * exp(-0.5 * q);
      if (amin > 0 && fabs(a_raw - amin) <= delta * amin) kn = 1;
      double alpha = a_raw < amax ? a_raw : amax;
      if (alpha < amin) continue;
      double Tn = T * (1.0 - alpha);
      if (tmin > 0 && fabs(Tn - tmin) <= delta * tmin) kn = 1;
      if (Tn < tmin) break;
      double w = alpha * T;
      acc[0] += w * rgb64[4 * g + 0];
      acc[1] += w * rgb64[4 * g + 1];
      acc[2] += w * rgb64[4 * g + 2];
      acc[3] += w * P->depth;
      acc[4] += w * su64[4 * g + 3];
      T = Tn;
      last = g;
      ++nc;
      if (a_raw >= amax) ++ncl;
    }
    for (int c = 0; c < 5; ++c) out[5 * k + c] = acc[c];
    tfinal[k] = T;
    last_id[k] = last;
    n_contrib[k] = nc;
    n_clamp[k] = ncl;
    knife[k] = (int8_t)kn;
  }
  for (int v = 0; v < V; ++v)
    if (need[v]) free_view_list(&L[v]);
  free(L);
  free(need);
}

/* ------------------------------------------------------------------------- */
/* analytic gradient                                                          */
/* Pixels with a non-zero image gradient are listed explicitly: pix is K x 3   */
/* int32 (view, u, v) and gpix K x 4 doubles (dL/dR, dL/dG, dL/dB, dL/dDepth). */
/* Outputs per Gaussian (N x 4 each, zero-initialised here): dmo = (dmu_x,      */
/* dmu_y, dmu_z, dlogit), dsu = (dls_0..2, 0), dq = (dw, dx, dy, dz),          */
/* drgb = (dr, dg, db, 0).                                                     */
/* g2d (optional, V x N x 8): per view screen-space gradients                  */
/*   (dmean_x, dmean_y, dconic_a, dconic_b, dconic_c, dopacity, ddepth, 0).    */
/* ------------------------------------------------------------------------- */
static void atomic_add(double* p, double v) {
#pragma omp atomic
  *p += v;
}

void or_grad(int64_t N, const float* mo32, const float* su32, const float* q32,
             const double* mo64, const double* su64, const double* q64, const double* rgb64,
             int V, const float* cam, const int* camwh, const double* prm,
             int64_t K, const int32_t* pix, const double* gpix_all,
             double* dmo, double* dsu, double* dq, double* drgb, double* g2d) {
  const double amin = prm[P_ALPHA_MIN], amax = prm[P_ALPHA_MAX], tmin = prm[P_T_MIN];
  memset(dmo, 0, sizeof(double) * 4 * (size_t)N);
  memset(dsu, 0, sizeof(double) * 4 * (size_t)N);
  memset(dq, 0, sizeof(double) * 4 * (size_t)N);
  memset(drgb, 0, sizeof(double) * 4 * (size_t)N);
  double* G = (double*)calloc((size_t)V * (size_t)N * 8 + 1, sizeof(double));
  for (int v = 0; v < V; ++v) {
    const float* camf = cam + CAMF * v;
    int64_t any = 0;
    for (int64_t k = 0; k < K; ++k) any |= (pix[3 * k] == v);
    if (!any) continue;
    view_list L;
    build_view_list(N, mo32, su32, q32, mo64, su64, q64, camf, camwh + 4 * v, prm, &L);
    double* Gv = G + (size_t)v * (size_t)N * 8;
#pragma omp parallel
    {
      int64_t cap = L.n > 0 ? L.n : 1;
      int64_t* ci = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);     /* list position */
      double* ca = (double*)malloc(sizeof(double) * (size_t)cap);        /* alpha */
      double* cT = (double*)malloc(sizeof(double) * (size_t)cap);        /* T before */
      double* cG = (double*)malloc(sizeof(double) * (size_t)cap);        /* exp(-q/2) */
      char* cc = (char*)malloc((size_t)cap);                               /* clamped */
#pragma omp for schedule(dynamic, 16)
      for (int64_t kp = 0; kp < K; ++kp) {
        if (pix[3 * kp] != v) continue;
        double px = pix[3 * kp + 1] + 0.5, py = pix[3 * kp + 2] + 0.5;
        const double* gpix = gpix_all + 4 * kp;
        double T = 1.0;
        int64_t n = 0;
        for (int64_t i = 0; i < L.n; ++i) {
          const val_proj* P = &L.P[i];
          double dx = px - P->mean[0], dy = py - P->mean[1];
          double q = P->conic[0] * dx * dx + 2.0 * P->conic[1] * dx * dy + P->conic[2] * dy * dy;
          double Gq = exp(-0.5 * q);
          double a_raw = P->opac * Gq;
          double alpha = a_raw < amax ? a_raw : amax;
          if (alpha < amin) continue;
          double Tn = T * (1.0 - alpha);
          if (Tn < tmin) break;
          ci[n] = i; ca[n] = alpha; cT[n] = T; cG[n] = Gq; cc[n] = (char)(a_raw >= amax);
          ++n;
          T = Tn;
        }
        /* suffix sums S_ch = sum_{j > i} w_j x_j, walked from the back */
        double S[4] = {0, 0, 0, 0};
        for (int64_t k = n - 1; k >= 0; --k) {
          const val_proj* P = &L.P[ci[k]];
          int64_t g = L.id[ci[k]];
          double x[4] = {rgb64[4 * g], rgb64[4 * g + 1], rgb64[4 * g + 2], P->depth};
          double a = ca[k], Ti = cT[k], w = a * Ti;
          double dalpha = 0;
          for (int c = 0; c < 4; ++c) dalpha += gpix[c] * (x[c] * Ti - S[c] / (1.0 - a));
          for (int c = 0; c < 3; ++c) atomic_add(&drgb[4 * g + c], gpix[c] * w);
          atomic_add(&Gv[8 * g + 6], gpix[3] * w);
          for (int c = 0; c < 4; ++c) S[c] += w * x[c];
          if (!cc[k]) {
            double dx = px - P->mean[0], dy = py - P->mean[1];
            atomic_add(&Gv[8 * g + 5], dalpha * cG[k]);
            double dqv = dalpha * (-0.5 * a);
            atomic_add(&Gv[8 * g + 0], dqv * (-2.0) * (P->conic[0] * dx + P->conic[1] * dy));
            atomic_add(&Gv[8 * g + 1], dqv * (-2.0) * (P->conic[1] * dx + P->conic[2] * dy));
            atomic_add(&Gv[8 * g + 2], dqv * dx * dx);
            atomic_add(&Gv[8 * g + 3], dqv * 2.0 * dx * dy);
            atomic_add(&Gv[8 * g + 4], dqv * dy * dy);
          }
        }
      }
      free(ci); free(ca); free(cT); free(cG); free(cc);
    }
    /* projection adjoint for every visible Gaussian of this view */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < L.n; ++i) {
      const val_proj* P = &L.P[i];
      int64_t g = L.id[i];
      const double* gg = Gv + 8 * g;
      double fx = camf[0], fy = camf[1];
      double R[9];
      for (int k = 0; k < 9; ++k) R[k] = camf[4 + k];
      double tx = P->t[0], ty = P->t[1], tz = P->t[2];
      /* conic = inverse(cov): dL/dCov = -C G_C C with symmetric matrix gradients */
      double Cm[2][2] = {{P->conic[0], P->conic[1]}, {P->conic[1], P->conic[2]}};
      double GC[2][2] = {{gg[2], 0.5 * gg[3]}, {0.5 * gg[3], gg[4]}};
      double tmp[2][2], GS[2][2];
      for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) tmp[r][s] = GC[r][0] * Cm[0][s] + GC[r][1] * Cm[1][s];
      for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) GS[r][s] = -(Cm[r][0] * tmp[0][s] + Cm[r][1] * tmp[1][s]);
      double J[2][3] = {{fx / tz, 0.0, -fx * tx / (tz * tz)}, {0.0, fy / tz, -fy * ty / (tz * tz)}};
      double T3[2][3];
      for (int r = 0; r < 2; ++r)
        for (int m = 0; m < 3; ++m) T3[r][m] = J[r][0] * R[3 * m + 0] + J[r][1] * R[3 * m + 1] + J[r][2] * R[3 * m + 2];
      /* dL/dSigma3 = T3^T GS T3 */
      double M3[3][3];
      for (int i3 = 0; i3 < 3; ++i3)
        for (int j3 = 0; j3 < 3; ++j3) {
          double s = 0;
          for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) s += T3[r][i3] * GS[r][c] * T3[c][j3];
          M3[i3][j3] = s;
        }
      /* dL/dT3 = 2 GS T3 Sigma3 */
      double GT3[2][3];
      for (int r = 0; r < 2; ++r)
        for (int m = 0; m < 3; ++m) {
          double s = 0;
          for (int c = 0; c < 2; ++c)
            for (int k = 0; k < 3; ++k) s += GS[r][c] * T3[c][k] * P->S3[3 * k + m];
          GT3[r][m] = 2.0 * s;
        }
      /* dL/dJ = dL/dT3 W^T, W = R^T so W^T = R: GJ[r][k] = sum_m GT3[r][m] * W[k][m] = sum_m GT3[r][m] R[m][k] */
      double GJ[2][3];
      for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) GJ[r][k] = GT3[r][0] * R[0 * 3 + k] + GT3[r][1] * R[1 * 3 + k] + GT3[r][2] * R[2 * 3 + k];
      double iz = 1.0 / tz, iz2 = iz * iz, iz3 = iz2 * iz;
      double gtx = GJ[0][2] * (-fx * iz2) + gg[0] * fx * iz;
      double gty = GJ[1][2] * (-fy * iz2) + gg[1] * fy * iz;
      double gtz = GJ[0][0] * (-fx * iz2) + GJ[0][2] * (2.0 * fx * tx * iz3) + GJ[1][1] * (-fy * iz2) +
                   GJ[1][2] * (2.0 * fy * ty * iz3) + gg[0] * (-fx * tx * iz2) + gg[1] * (-fy * ty * iz2) + gg[6];
      /* t = R^T (mu - T) => dL/dmu = R dL/dt */
      double gmu[3];
      for (int m = 0; m < 3; ++m) gmu[m] = R[3 * m + 0] * gtx + R[3 * m + 1] * gty + R[3 * m + 2] * gtz;
      /* Sigma3 = Rq diag(s2) Rq^T: dL/dRq = 2 M3 Rq diag(s2); dL/ds2_k = (Rq^T M3 Rq)_kk */
      const double* Rq = P->Rq;
      double GR[9], gs2[3];
      for (int i3 = 0; i3 < 3; ++i3)
        for (int k = 0; k < 3; ++k) {
          double s = 0;
          for (int j3 = 0; j3 < 3; ++j3) s += M3[i3][j3] * Rq[3 * j3 + k];
          GR[3 * i3 + k] = 2.0 * s * P->s2[k];
        }
      for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int i3 = 0; i3 < 3; ++i3)
          for (int j3 = 0; j3 < 3; ++j3) s += Rq[3 * i3 + k] * M3[i3][j3] * Rq[3 * j3 + k];
        gs2[k] = s;
      }
      double w = P->qn[0], x = P->qn[1], y = P->qn[2], z = P->qn[3];
      double gw = 2.0 * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
      double gx = 2.0 * (y * GR[1] + z * GR[2] + y * GR[3] - 2.0 * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2.0 * x * GR[8]);
      double gy = 2.0 * (-2.0 * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2.0 * y * GR[8]);
      double gz = 2.0 * (-2.0 * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.0 * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
      double dotq = w * gw + x * gx + y * gy + z * gz;
      double inv = 1.0 / P->qnorm;
      double gqv[4] = {(gw - w * dotq) * inv, (gx - x * dotq) * inv, (gy - y * dotq) * inv, (gz - z * dotq) * inv};
      double o = P->opac;
      /* each Gaussian appears once per view: plain adds are race-free here */
      for (int m = 0; m < 3; ++m) dmo[4 * g + m] += gmu[m];
      dmo[4 * g + 3] += gg[5] * o * (1.0 - o);
      for (int k = 0; k < 3; ++k) dsu[4 * g + k] += gs2[k] * 2.0 * P->s2[k];
      for (int k = 0; k < 4; ++k) dq[4 * g + k] += gqv[k];
    }
    free_view_list(&L);
  }
  if (g2d) memcpy(g2d, G, sizeof(double) * 8 * (size_t)N * (size_t)V);
  free(G);
}

/* ------------------------------------------------------------------------- */
/* tile binning and sort                                                      */
/* Records (in the order given): gaussian id, view, tile rect [x0,x1)x[y0,y1),*/
/* depth key bits.  Emit one pair per covered tile; key = (global tile << 32) */
/* | depth bits, global tile = tile_base[view] + y * tiles_x[view] + x.        */
/* Sorted ascending by (key, record index): the order a stable sort of the    */
/* keys emitted in record order gives.                                        */
/* ------------------------------------------------------------------------- */
int64_t or_bin_count(int64_t R, const int32_t* rect) {
  int64_t P = 0;
  for (int64_t r = 0; r < R; ++r) {
    int64_t w = rect[4 * r + 2] - rect[4 * r + 0], h = rect[4 * r + 3] - rect[4 * r + 1];
    if (w > 0 && h > 0) P += w * h;
  }
  return P;
}

typedef struct { uint64_t key; uint32_t rec; } pair_kr;
static int cmp_pair(const void* A, const void* B) {
  const pair_kr* a = (const pair_kr*)A;
  const pair_kr* b = (const pair_kr*)B;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->rec != b->rec) return a->rec < b->rec ? -1 : 1;
  return 0;
}

void or_bin(int64_t R, const uint32_t* view, const int32_t* rect, const uint32_t* dkey,
            const int32_t* tiles_x, const int64_t* tile_base, int64_t total_tiles,
            uint64_t* keys, uint32_t* vals, int64_t* ranges) {
  int64_t P = or_bin_count(R, rect);
  pair_kr* pr = (pair_kr*)malloc(sizeof(pair_kr) * (size_t)(P > 0 ? P : 1));
  int64_t k = 0;
  for (int64_t r = 0; r < R; ++r) {
    uint32_t v = view[r];
    for (int y = rect[4 * r + 1]; y < rect[4 * r + 3]; ++y)
      for (int x = rect[4 * r + 0]; x < rect[4 * r + 2]; ++x) {
        uint64_t gt = (uint64_t)(tile_base[v] + (int64_t)y * tiles_x[v] + x);
        pr[k].key = (gt << 32) | (uint64_t)dkey[r];
        pr[k].rec = (uint32_t)r;
        ++k;
      }
  }
  qsort(pr, (size_t)P, sizeof(pair_kr), cmp_pair);
  for (int64_t t = 0; t < 2 * total_tiles; ++t) ranges[t] = 0;
  for (int64_t i = 0; i < P; ++i) {
    keys[i] = pr[i].key;
    vals[i] = pr[i].rec;
    int64_t t = (int64_t)(pr[i].key >> 32);
    if (i == 0 || (pr[i - 1].key >> 32) != (uint64_t)t) ranges[2 * t] = i;
    if (i == P - 1 || (pr[i + 1].key >> 32) != (uint64_t)t) ranges[2 * t + 1] = i + 1;
  }
  free(pr);
}
