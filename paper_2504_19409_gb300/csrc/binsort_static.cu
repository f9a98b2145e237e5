// gs_bin_sort_static: the tile x depth sort of gs_bin_sort, for callers that
// cannot allocate device memory. Its scratch space is a file-scope device
// array of GS_BIN_SORT_STATIC_SCRATCH_BYTES instead of a caller workspace;
// everything else (inputs, outputs, kernels, launch order) is gs_bin_sort's.
//
// The array is one per device and lives as long as the process. Host code
// cannot use the array's name as a device address, so the entry point looks
// the address up with cudaGetSymbolAddress once per device (on its first call
// on that device, with that device current) and passes it to the kernels.
// The cached address belongs to the device's context at the time of the
// look-up: a call that finds another context current on the device (after a
// cudaDeviceReset, which recreates the primary context and reloads the
// module, so the array may move) looks the address up again before it
// launches anything.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gsff_internal.cuh"

static __device__ __align__(256) unsigned char g_bin_sort_scratch[GS_BIN_SORT_STATIC_SCRATCH_BYTES];

namespace gsff {

size_t bin_sort_workspace_bytes(int P, long long capacity, int num_tiles);
gs_status launch_bin_sort(const CamF& cam, int P, const float* depth, const int32_t* rect, const int32_t* touched,
                          long long capacity, void* workspace, unsigned long long* keys, uint32_t* gids,
                          int32_t* ranges, int64_t* n_out, int32_t* status, cudaStream_t st);

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx_id[kMaxDevices] = {};

// A driver function through the runtime's driver entry point (the library
// does not link the driver library itself); null if unavailable.
void* driver_fn(const char* name, int version) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return f;
}

// Device address of g_bin_sort_scratch on the current device, looked up once
// per (device, context). Contexts are told apart by their unique id
// (cuCtxGetId), which a recreated context never reuses, unlike its handle.
gs_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
  static const auto get_ctx = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(driver_fn("cuCtxGetCurrent", 4000));
  static const auto get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(driver_fn("cuCtxGetId", 12000));
  CUcontext ctx = nullptr;
  if (!get_ctx || !get_id || get_ctx(&ctx) != CUDA_SUCCESS) return GS_ERR_CUDA;
  if (!ctx) {
    // no context bound to this thread yet: cudaSetDevice binds the device's
    // primary context (the one the launches below will use); it allocates nothing
    if (cudaSetDevice(dev) != cudaSuccess || get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return GS_ERR_CUDA;
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev] || g_scratch_ctx_id[dev] != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bin_sort_scratch) != cudaSuccess || p == nullptr) return GS_ERR_CUDA;
    g_scratch_addr[dev] = p;
    g_scratch_ctx_id[dev] = id;
  }
  *out = g_scratch_addr[dev];
  return GS_OK;
}

}  // namespace
}  // namespace gsff

extern "C" gs_status gs_bin_sort_static(const gs_camera* cam, int32_t P, const float* depth, const int32_t* rect,
                                        const int32_t* tiles_touched, int64_t capacity, uint64_t* keys,
                                        uint32_t* gids, int32_t* tile_ranges, int64_t* n_instances,
                                        int32_t* status, void* stream) {
  using namespace gsff;
  if (!cam || cam->width <= 0 || cam->height <= 0 || cam->width > (1 << 15) || cam->height > (1 << 15) ||
      !(cam->fx > 0.f) || !(cam->fy > 0.f) || P < 0 || capacity < 1 || capacity >= (1ll << 31))
    return GS_ERR_INVALID_ARG;
  if (!gids || !tile_ranges || (P > 0 && (!depth || !rect || !tiles_touched))) return GS_ERR_INVALID_ARG;
  if (!aligned(keys, 8) || !aligned(rect, 16) || !aligned(tile_ranges, 8) || !aligned(n_instances, 8))
    return GS_ERR_INVALID_ARG;
  // The sizes must fit the fixed scratch array.
  const CamF k = make_cam(*cam);
  if ((long long)k.tiles_x * k.tiles_y > (1 << 24)) return GS_ERR_INVALID_ARG;
  if (bin_sort_workspace_bytes(P, capacity, k.tiles_x * k.tiles_y) > (size_t)GS_BIN_SORT_STATIC_SCRATCH_BYTES)
    return GS_ERR_INVALID_ARG;
  void* scratch = nullptr;
  const gs_status st = scratch_address(&scratch);
  if (st != GS_OK) return st;
  return launch_bin_sort(k, P, depth, rect, tiles_touched, capacity, scratch,
                         reinterpret_cast<unsigned long long*>(keys), gids, tile_ranges, n_instances, status,
                         static_cast<cudaStream_t>(stream));
}
