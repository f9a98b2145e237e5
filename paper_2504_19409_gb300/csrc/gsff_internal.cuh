// Internal declarations shared by the CUDA translation units of libgsff.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "gsff.h"

namespace gsff {

// Programmatic dependent launch. A kernel started by launch_pdl may be
// scheduled while the previous kernel of its stream is still draining; every
// kernel of the frame's chain calls pdl_wait() before its first global memory
// access (it returns once the previous grid has completed and its writes are
// visible, and at once for a kernel launched without the attribute), then
// pdl_trigger() so that the next kernel can be scheduled in turn.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Clears two device ranges (4-byte aligned, sizes in multiples of 4 bytes; b
// may be null) with one kernel of the programmatic-launch chain.
gs_status launch_zero(void* a, size_t a_bytes, void* b, size_t b_bytes, cudaStream_t st);

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// 3DGS rules the paper's renderer builds on (Sec. 3.1); the paper does not
// print their values.
constexpr float kLowPass = 0.3f;          // added to the 2D covariance diagonal
constexpr float kGuardBand = 1.3f;        // Jacobian clamp, in half-fields of view
constexpr float kSigmas = 3.f;            // footprint radius in standard deviations
constexpr float kEigFloor = 0.1f;         // floor under the eigenvalue discriminant
constexpr float kAlphaMax = 0.99f;        // alpha clamp
constexpr float kAlphaMin = 1.f / 255.f;  // alphas below this are skipped
constexpr float kTStop = 1e-4f;           // walk stops before T falls below this
constexpr int kTile = GS_TILE;
constexpr int kTilePix = kTile * kTile;   // 256 pixels = 256 threads per tile block

struct CamF {
  int W, H, tiles_x, tiles_y;
  float fx, fy, cx, cy;
  float R[9];
  float t[3];
  float near_z;
  const float* pose;  // device (R row-major, t) overriding R, t when not null
};

// The world -> camera rotation and translation a kernel works with: the
// device pose when the caller gave one, else the camera struct's.
__device__ __forceinline__ void cam_pose(const CamF& cam, float (&R)[9], float (&t)[3]) {
  if (cam.pose) {
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = __ldg(cam.pose + i);
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = __ldg(cam.pose + 9 + i);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = cam.R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = cam.t[i];
  }
}

inline CamF make_cam(const gs_camera& c) {
  CamF k;
  k.W = c.width;
  k.H = c.height;
  k.tiles_x = (c.width + kTile - 1) / kTile;
  k.tiles_y = (c.height + kTile - 1) / kTile;
  k.fx = c.fx;
  k.fy = c.fy;
  k.cx = c.cx;
  k.cy = c.cy;
  for (int i = 0; i < 9; ++i) k.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) k.t[i] = c.t[i];
  k.near_z = c.near_z;
  k.pose = c.pose_dev;
  return k;
}

// Device status word: error kinds OR-ed as bits.
__device__ __forceinline__ void flag_status(int32_t* status, gs_status s) {
  if (status) atomicOr(status, 1 << (int)s);
}

// Indices the kernels read from their inputs and then follow: the Gaussian
// ids of the sorted lists and the saved last indices. In the bounds-checked
// build (GS_CHECKED) an id past P flags GS_ERR_BOUNDS and is replaced by 0,
// and a list length past the tile's list is cut to it (flagged the same way),
// so that no gather leaves the caller's arrays; in the normal build both are
// used as given.
__device__ __forceinline__ uint32_t checked_id(uint32_t g, int P, int32_t* status) {
#ifdef GS_CHECKED
  if (g >= (uint32_t)P) {
    flag_status(status, GS_ERR_BOUNDS);
    return 0u;
  }
#endif
  return g;
}

__device__ __forceinline__ int checked_len(int n, int list_len, int32_t* status) {
#ifdef GS_CHECKED
  if (n > list_len || n < 0) {
    flag_status(status, GS_ERR_BOUNDS);
    return n < 0 ? 0 : list_len;
  }
#endif
  return n;
}

// alpha of one (pixel, Gaussian) pair, o exp(-(A dx^2 + 2 B dx dy + C dy^2) / 2)
// clamped to 0.99. It is evaluated in base 2 from the conic scaled by log2(e)
// (conic_q, which a kernel may compute once per Gaussian): the exponent
// dx (qA dx + qB dy) + qC dy^2 takes five multiplies / fused multiply-adds and
// one ex2. The sequence is fixed (explicit roundings and fused multiply-adds),
// and pair_alpha computes conic_q itself with the same operations, so every
// kernel takes identical skip decisions and alphas.
struct PairAlpha {
  float G, alpha;  // G = exp(power)
  bool clamped;
};

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float4 conic_q(float4 co) {
  return make_float4(__fmul_rn(-0.5f * kLog2e, co.x), __fmul_rn(-kLog2e, co.y), __fmul_rn(-0.5f * kLog2e, co.z), co.w);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ bool pair_alpha_q(float4 q, float dx, float dy, PairAlpha& r) {
  const float u = __fmaf_rn(q.y, dy, __fmul_rn(q.x, dx));
  const float p2 = __fmaf_rn(dx, u, __fmul_rn(__fmul_rn(q.z, dy), dy));
  if (p2 > 0.f) return false;
  r.G = ex2_approx(p2);
  const float a = __fmul_rn(q.w, r.G);
  r.clamped = a > kAlphaMax;
  r.alpha = r.clamped ? kAlphaMax : a;
  return r.alpha >= kAlphaMin;
}

__device__ __forceinline__ bool pair_alpha(float4 co, float dx, float dy, PairAlpha& r) {
  return pair_alpha_q(conic_q(co), dx, dy, r);
}

// L1 image loss fused into compositing (class 0 rgb, 1 depth, 2 features).
// The forward evaluates w |pred - target| and stores, per pixel, which
// cotangents w sign(pred - target) are nonzero (word x) and negative (word y),
// bit c for feature c < 16, bits 16, 17, 18 for r, g, b and 19 for depth; the
// adjoint rebuilds the cotangents from those bits and the weights.
constexpr int kL1BitRgb = 16, kL1BitDepth = 19;
struct L1Fwd {
  int on;
  const float* target[3];  // null: the class has no term
  float w[3];
  float* loss;             // device float or null
  uint2* signs;            // [H W]
};
struct L1Bwd {
  int on;
  const uint2* signs;
  float w[3];
};

// ---- tracing (api.cu) -----------------------------------------------------
void trace_begin(const char* name, cudaStream_t s);
void trace_end(cudaStream_t s);

struct TraceScope {
  cudaStream_t s;
  TraceScope(const char* name, cudaStream_t st) : s(st) { trace_begin(name, s); }
  ~TraceScope() { trace_end(s); }
};

#define GS_TRACE(name, stream) ::gsff::TraceScope _gs_trace_scope_(name, stream)

// An NVTX range around an ABI call (seen by profilers that record NVTX; a
// no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
#define GS_NVTX(name) ::gsff::NvtxRange _gs_nvtx_range_(name)

// The decoder trainers' pixel sample s of a step (the ABI's sampling rule):
// splitmix64(seed + (s + 1) * 0x9E3779B97F4A7C15) mod npix, splitmix64 being
// Steele, Lea and Flood's 64-bit finaliser.
__device__ __forceinline__ long long decoder_sample_pixel(unsigned long long seed, long long s, long long npix) {
  unsigned long long z = seed + (unsigned long long)(s + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (long long)(z % (unsigned long long)npix);
}

inline gs_status last_launch_status() {
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---- launchers implemented in the .cu files ---------------------------------
gs_status launch_render_fwd_tc(const CamF& cam, int P, const int32_t* ranges, const int32_t* order,
                               const uint32_t* gids, const uint8_t* masks, const float* uv, const float* co,
                               const __nv_bfloat16* feats, const int32_t* last_idx, int N, float* out_feat,
                               int32_t* status, cudaStream_t st);
gs_status launch_render_bwd_feat_tc(const CamF& cam, int P, const int32_t* ranges, const int32_t* order,
                                    const uint32_t* gids, const uint8_t* masks, const float* uv, const float* co,
                                    const int32_t* last_idx, const float* g_feat, int N, float* d_feats,
                                    int32_t* status, cudaStream_t st);
// Test hook of the tensor-core feature kernels' bounded waits (feat_tc.cu):
// while set, their producer warps issue nothing.
void set_tc_test_hold(int on);

}  // namespace gsff
