// noalloc.cu -- gs_render_bwd_noalloc: the backward pass without a caller
// workspace, for callers that cannot allocate device memory.
//
// gs_render_bwd needs scratch for the per-record screen-space gradients (48
// bytes per record).  Normally the caller provides it as a workspace.  Some
// callers cannot: a process that reserves all its device memory once at start-up
// and forbids allocation afterwards (a robot's real-time mapping loop), a plugin
// that only receives the buffers of its host application and has no allocator of
// its own, or code whose launches are being captured into a CUDA graph by a
// framework that must not see an allocation in the middle of the capture.  This
// entry point keeps that scratch in a fixed-size array that lives in the
// library's device image instead.
//
// The array below is a host-side stand-in when named in host code, not a device
// address, so the host takes the real address with cudaGetSymbolAddress once
// per device and hands that pointer to the kernels.
#include <mutex>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr int64_t kMaxRecords = GS_NOALLOC_MAX_RECORDS;

// 3 float4 per record; every GPU that loads the library holds this until exit.
static __device__ __align__(256) float4 g_bwd_scratch[3 * kMaxRecords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
gs_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bwd_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return GS_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace
}  // namespace gs

extern "C" gs_status gs_render_bwd_noalloc(const gs_map* map, const gs_proj* proj, const gs_bins* bins,
                                           const gs_image* fwd, const gs_image_grad* grad, const gs_camera* cams,
                                           int32_t n_views, const gs_params* prm, gs_map_grad* out, void* stream) {
  using namespace gs;
  if (!map || !proj || !bins || !fwd || !grad || !cams || !prm || !out) return GS_ERR_NULL;
  if (map->n < 0 || n_views < 1 || n_views > (1 << 20)) return GS_ERR_ARG;
  if (proj->capacity < 0 || bins->pair_capacity < 1 || bins->tile_capacity < 1) return GS_ERR_ARG;
  if (proj->capacity > kMaxRecords) return GS_ERR_WORKSPACE;   // the fixed scratch is too small
  if (map->n > 0 && (!map->mo || !map->su || !map->q || !map->rgb)) return GS_ERR_NULL;
  if (!proj->count || !proj->status || !proj->view_info || !proj->grp_mask || !proj->grp_base || !proj->gid ||
      !proj->view || !proj->splat || !proj->color_d || !bins->count || !bins->rec || !bins->ranges || !fwd->T ||
      !fwd->last)
    return GS_ERR_NULL;
  if (map->n > 0 && (!out->dmo || !out->dsu || !out->dq || !out->drgb)) return GS_ERR_NULL;
  if (!aligned(map->mo, 16) || !aligned(map->su, 16) || !aligned(map->q, 16) || !aligned(map->rgb, 16) ||
      !aligned(proj->splat, 32) || !aligned(proj->color_d, 16) ||
      !aligned(out->dmo, 16) || !aligned(out->dsu, 16) ||
      !aligned(out->dq, 16) || !aligned(out->drgb, 16) || !aligned(fwd->T, 4) || !aligned(fwd->last, 4) ||
      !aligned(grad->rgb, 4) || !aligned(grad->depth, 4))
    return GS_ERR_ALIGN;
  const int B = prm->tile_w * prm->tile_h;
  if ((prm->tile_w != 8 && prm->tile_w != 16 && prm->tile_w != 32 && prm->tile_w != 64) || prm->tile_h < 8 ||
      prm->tile_h % 8 != 0 || (B != 64 && B != 128 && B != 256 && B != 512 && B != 1024) || !(prm->alpha_max > 0.f && prm->alpha_max <= 1.f) ||
      !(prm->alpha_min >= 0.f && prm->alpha_min < 1.f))
    return GS_ERR_ARG;
  void* scratch = nullptr;
  gs_status s = scratch_address(&scratch);
  if (s != GS_OK) return s;
  cudaError_t e = launch_render_bwd(*map, *proj, *bins, *fwd, *grad, cams, n_views, *prm, *out, scratch,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
