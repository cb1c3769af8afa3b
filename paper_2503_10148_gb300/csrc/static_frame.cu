// sss_render_static: forward render of one small frame with no allocation.
//
// Some callers cannot allocate device memory at the time they need a frame:
// a plug-in inside a host application that owns every device byte through
// its own pool or budget, or a real-time thread that must not take the
// allocator's locks or wait for the device synchronisation cudaMalloc can
// imply.  For them this entry point keeps the whole workspace in one
// file-scope __device__ array of fixed size, so a frame needs nothing but the
// caller's parameters and output image.  The call synchronises its stream
// before it returns (it reads the pair-overflow status).
//
// It runs the existing hot-path entry points (sss_project, sss_bin, sss_sort,
// sss_render_fwd) on that array.  In host code `g_static_arena` names only a
// host-side stand-in for the device array, so its device address is fetched
// with cudaGetSymbolAddress once per device (with that device current) and
// cached for the life of the process (a cudaDeviceReset of that device would
// leave the cached address stale; calls after one are not supported).
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

// The workspace of every sss_render_static call on this device (each device
// that loads the library holds its own copy until the process exits).
static __device__ __align__(256) unsigned char g_static_arena[SSS_STATIC_ARENA_BYTES];

namespace sss {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_arena_mutex;
void* g_arena_ptr[kMaxDevices] = {};

// Device address of the arena on the current device (set up on first use).
int arena_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SSS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_arena_mutex);
  if (!g_arena_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_arena) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return SSS_ERR_CUDA;
    }
    g_arena_ptr[dev] = p;
  }
  *out = g_arena_ptr[dev];
  return SSS_OK;
}

}  // namespace
}  // namespace sss

extern "C" int sss_render_static(const sss_params* scene, const sss_camera* cam, const sss_raster_cfg* cfg,
                                 float* out_rgb, sss_stream_t stream) {
  if (!scene || !cam || !cfg || !out_rgb) return SSS_ERR_INVALID_ARG;
  if (scene->n < 0 || scene->n > SSS_STATIC_MAX_COMPONENTS) return SSS_ERR_INVALID_ARG;
  if (cam->width < 1 || cam->height < 1 || (int64_t)cam->width * cam->height > SSS_STATIC_MAX_PIXELS)
    return SSS_ERR_INVALID_ARG;
  const int job_scene = 0;
  // Size the pair capacity to what is left of the arena after every other
  // workspace region (16 bytes per pair: two copies of key and value).
  sss_frame_plan plan;
  int rc = sss_plan_frame(scene, 1, cam, &job_scene, 1, cfg, 1u, &plan);
  if (rc != SSS_OK) return rc;
  if (plan.ws_bytes + 4096 > SSS_STATIC_ARENA_BYTES) return SSS_ERR_CAPACITY;
  const size_t spare = (size_t)SSS_STATIC_ARENA_BYTES - plan.ws_bytes - 4096;
  const uint32_t cap = (uint32_t)(spare / 16 > 0x7fffffffu ? 0x7fffffffu : spare / 16);
  if (cap == 0) return SSS_ERR_CAPACITY;
  rc = sss_plan_frame(scene, 1, cam, &job_scene, 1, cfg, cap, &plan);
  if (rc != SSS_OK) return rc;
  if (plan.ws_bytes > SSS_STATIC_ARENA_BYTES) return SSS_ERR_CAPACITY;
  void* ws = nullptr;
  rc = sss::arena_for_current_device(&ws);
  if (rc != SSS_OK) return rc;
  if ((rc = sss_project(&plan, ws, stream)) != SSS_OK) return rc;
  if ((rc = sss_bin(&plan, ws, stream)) != SSS_OK) return rc;
  if ((rc = sss_sort(&plan, ws, stream)) != SSS_OK) return rc;
  if ((rc = sss_render_fwd(&plan, ws, out_rgb, stream)) != SSS_OK) return rc;
  uint32_t status = 0;
  rc = sss_read_status(&plan, ws, &status, nullptr, nullptr, stream);
  if (rc != SSS_OK) return rc;
  return (status & SSS_STATUS_PAIR_OVERFLOW) ? SSS_ERR_CAPACITY : SSS_OK;
}
