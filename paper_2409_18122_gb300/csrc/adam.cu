// adam.cu -- the optimiser step of the mapping iterations: Adam (Kingma and Ba) on the
// map tensors in place, one grid-stride float4 pass per tensor (blockIdx.y selects the
// tensor), the step count kept on the device so that a captured graph replays
// successive steps.
#include <math.h>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kAdamThreads = 256;

struct AdamArgs {
  float4* p[GS_ADAM_MAX_TENSORS];
  const float4* g[GS_ADAM_MAX_TENSORS];
  float4* m[GS_ADAM_MAX_TENSORS];
  float4* v[GS_ADAM_MAX_TENSORS];
  int64_t n4[GS_ADAM_MAX_TENSORS];
  int32_t nt;
  float lr, b1, b2, omb1, omb2, lb1, lb2, eps;   // betas, 1 - betas, ln(betas), from doubles on the host
  const uint32_t* step;
};

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, const AdamArgs& a, float step_size,
                                      float c2s) {
  m = a.b1 * m + a.omb1 * g;
  v = a.b2 * v + a.omb2 * g * g;
  p = p - step_size * m / (sqrtf(v) / c2s + a.eps);
}

__global__ void __launch_bounds__(kAdamThreads) k_adam(const __grid_constant__ AdamArgs a) {
  const int ti = blockIdx.y;
  if (ti >= a.nt || !a.g[ti]) return;
  // bias corrections 1 - beta^t = -expm1(t ln beta), accurate also for beta close to 1
  const float t = (float)(*a.step + 1u);
  const float step_size = a.lr / -expm1f(t * a.lb1);
  const float c2s = sqrtf(-expm1f(t * a.lb2));
  float4* P = a.p[ti];
  const float4* G = a.g[ti];
  float4* M = a.m[ti];
  float4* V = a.v[ti];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n4[ti];
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 g = G[i];
    float4 p = P[i], m = M[i], v = V[i];
    adam1(p.x, g.x, m.x, v.x, a, step_size, c2s);
    adam1(p.y, g.y, m.y, v.y, a, step_size, c2s);
    adam1(p.z, g.z, m.z, v.z, a, step_size, c2s);
    adam1(p.w, g.w, m.w, v.w, a, step_size, c2s);
    P[i] = p;
    M[i] = m;
    V[i] = v;
  }
}

__global__ void k_adam_count(uint32_t* step) { *step += 1u; }

}  // namespace

cudaError_t launch_adam(float* const* params, const float* const* grads, float* const* m, float* const* v,
                        const int64_t* sizes, int n_tensors, const gs_adam_params& prm, uint32_t* step,
                        cudaStream_t st) {
  AdamArgs a{};
  int64_t n4_max = 0;
  for (int i = 0; i < n_tensors; ++i) {
    a.p[i] = reinterpret_cast<float4*>(params[i]);
    a.g[i] = reinterpret_cast<const float4*>(grads[i]);
    a.m[i] = reinterpret_cast<float4*>(m[i]);
    a.v[i] = reinterpret_cast<float4*>(v[i]);
    a.n4[i] = sizes[i] / 4;
    if (a.n4[i] > n4_max) n4_max = a.n4[i];
  }
  a.nt = n_tensors;
  a.lr = (float)prm.lr;
  a.b1 = (float)prm.beta1;
  a.b2 = (float)prm.beta2;
  a.omb1 = (float)(1.0 - prm.beta1);
  a.omb2 = (float)(1.0 - prm.beta2);
  a.lb1 = (float)log1p(-(1.0 - prm.beta1));   // ln beta (-inf for beta = 0: no bias correction)
  a.lb2 = (float)log1p(-(1.0 - prm.beta2));
  a.eps = (float)prm.eps;
  a.step = step;
  if (n4_max > 0) {
    int64_t bx = (n4_max + kAdamThreads - 1) / kAdamThreads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (bx > cap) bx = cap;
    k_adam<<<dim3((unsigned)bx, (unsigned)n_tensors), kAdamThreads, 0, st>>>(a);
    note_launch();
  }
  k_adam_count<<<1, 1, 0, st>>>(step);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gs
