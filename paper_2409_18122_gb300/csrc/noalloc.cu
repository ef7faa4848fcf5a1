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

}  // namespace
}  // namespace gs

extern "C" gs_status gs_render_bwd_noalloc(const gs_map* map, const gs_proj* proj, const gs_bins* bins,
                                           const gs_image* fwd, const gs_image_grad* grad, const gs_camera* cams,
                                           int32_t n_views, const gs_params* prm, gs_map_grad* out, void* stream) {
  using namespace gs;
  GS_TRACE("gs_render_bwd_noalloc");
  // the same checks as gs_render_bwd, then the bound of the fixed scratch in place of a workspace
  const gs_status v = validate_render_bwd(map, proj, bins, fwd, grad, cams, n_views, prm, out);
  if (v != GS_OK) return v;
  if (proj->capacity > kMaxRecords) return GS_ERR_WORKSPACE;
  void* scratch = nullptr;
  gs_status s = scratch_address(&scratch);
  if (s != GS_OK) return s;
  cudaError_t e = launch_render_bwd(*map, *proj, *bins, *fwd, *grad, cams, n_views, *prm, *out, scratch,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
