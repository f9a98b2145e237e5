// C ABI entry points of libgsff (declared in include/gsff.h): synchronous
// argument checks, workspace carving, and kernel launch sequencing. The
// kernels themselves live in project.cu, binsort.cu and render.cu.

#include <mutex>
#include <vector>

#include "gsff_internal.cuh"

namespace gsff {

void launch_project(const CamF& cam, int P, const float* means, const float* scales, const float* quats,
                    const float* opacity, float* uv, float* co, float* depth, int32_t* rect, int32_t* touched,
                    int64_t* n_inst, cudaStream_t st);
void launch_project_bwd(const CamF& cam, int P, const float* means, const float* scales, const float* quats,
                        const float* d_uv, const float* d_conic, const float* d_depth, float* d_means,
                        float* d_scales, float* d_quats, float* d_pose, cudaStream_t st);
size_t bin_sort_workspace_bytes(int P, long long capacity, int num_tiles);
gs_status launch_bin_sort(const CamF& cam, int P, const float* depth, const int32_t* rect, const int32_t* touched,
                          long long capacity, void* workspace, unsigned long long* keys, uint32_t* gids,
                          int32_t* ranges, int64_t* n_out, int32_t* status, cudaStream_t st);
gs_status launch_tile_order(int T, const int32_t* ranges, int32_t* order, cudaStream_t st);
gs_status launch_render_fwd(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                            uint8_t* masks, const float* uv,
                            const float* co, const float* depth, const float* colors, const void* feats, int N,
                            int bf16, int hwc, const float bg[3], float* out_rgb, float* out_depth,
                            float* out_alpha, float* out_feat, float* T_final, int32_t* last_idx,
                            int32_t* n_contrib, uint8_t* visible, const L1Fwd* l1, int P, int32_t* status,
                            cudaStream_t st);
gs_status launch_render_bwd(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                            const uint8_t* masks, const float* uv,
                            const float* co, const float* depth, const float* colors, const void* feats, int N,
                            int bf16, int hwc, const float bg[3], const float* T_final, const int32_t* last_idx,
                            const float* g_rgb, const float* g_depth, const float* g_alpha, const float* g_feat,
                            int coupled, float* d_uv, float* d_conic, float* d_depth, float* d_opacity,
                            float* d_colors, float* d_feats, const L1Bwd* l1, int P, int32_t* status,
                            cudaStream_t st);

size_t pair_state_workspace_bytes(long long HW);
gs_status launch_store_pairs(const CamF& cam, int P, const int32_t* ranges, const int32_t* order,
                             const uint32_t* gids, const float* uv, const float* co, const int32_t* last_idx,
                             const int32_t* n_contrib, void* workspace, long long capacity, int64_t* pair_off,
                             float* pair_T, int32_t* status, cudaStream_t st);
gs_status launch_render_bwd_pairs(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                                  const float* uv, const float* co, const float* depth, const float* colors,
                                  const void* feats, int N, int bf16, int hwc, const float bg[3],
                                  const float* T_final, const int32_t* last_idx, const float* g_rgb,
                                  const float* g_depth, const float* g_alpha, const float* g_feat, int coupled,
                                  const long long* pair_off, const float* pair_T, float* d_uv, float* d_conic,
                                  float* d_depth, float* d_opacity, float* d_colors, float* d_feats, int P,
                                  int32_t* status, cudaStream_t st);

// ---- tracing -----------------------------------------------------------------
namespace {
struct TraceState {
  std::mutex mu;
  bool on = false;
  int cap = 0;
  int count = 0;
  int open = -1;
  std::vector<cudaEvent_t> ev;  // 2 per launch
  std::vector<const char*> names;
} g_trace;
}  // namespace

void trace_begin(const char* name, cudaStream_t s) {
  if (!g_trace.on) return;
  std::lock_guard<std::mutex> lk(g_trace.mu);
  if (g_trace.count >= g_trace.cap) return;
  const int i = g_trace.count;
  cudaEventRecord(g_trace.ev[2 * i], s);
  g_trace.names[i] = name;
  g_trace.open = i;
}

void trace_end(cudaStream_t s) {
  if (!g_trace.on) return;
  std::lock_guard<std::mutex> lk(g_trace.mu);
  if (g_trace.open < 0) return;
  cudaEventRecord(g_trace.ev[2 * g_trace.open + 1], s);
  g_trace.open = -1;
  ++g_trace.count;
}

namespace {

__device__ __forceinline__ float l1_sign(float d, float scale) { return d > 0.f ? scale : (d < 0.f ? -scale : 0.f); }

// grad = scale * sign(pred - target); loss += scale * sum |pred - target|.
// 16-byte loads and stores over the first 4 * (n / 4) elements when all three
// arrays are 16-byte aligned, scalar otherwise and for the tail.
__global__ void __launch_bounds__(256) k_l1_grad(long long n, const float* __restrict__ pred,
                                                 const float* __restrict__ target, float scale,
                                                 float* __restrict__ grad, float* __restrict__ loss, int vec) {
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long done = 0;
  if (vec) {
    const long long n4 = n >> 2;
    const float4* p4 = reinterpret_cast<const float4*>(pred);
    const float4* q4 = reinterpret_cast<const float4*>(target);
    float4* g4 = reinterpret_cast<float4*>(grad);
    for (long long i = t0; i < n4; i += stride) {
      const float4 a = __ldcs(p4 + i), b = __ldcs(q4 + i);
      const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
      g4[i] = make_float4(l1_sign(d0, scale), l1_sign(d1, scale), l1_sign(d2, scale), l1_sign(d3, scale));
      acc += (fabsf(d0) + fabsf(d1)) + (fabsf(d2) + fabsf(d3));
    }
    done = n4 << 2;
  }
  for (long long i = done + t0; i < n; i += stride) {
    const float d = pred[i] - target[i];
    grad[i] = l1_sign(d, scale);
    acc += fabsf(d);
  }
  if (loss) {
    __shared__ float s_part[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_part[w];
      if (b != 0.f) atomicAdd(loss, b * scale);
    }
  }
}

// The L1 terms of gs_render_fwd_l1's epilogue as a pass over rendered images:
// the same differences pred - target (the images hold the epilogue's values),
// hence the same sign words; the loss adds w |d| per term, summed per block
// and added with one atomic. Four consecutive pixels per thread; with vec
// (every plane 16-byte aligned and a multiple of 4 pixels, or the HWC feature
// rows a multiple of 4 channels) each plane is read with 16-byte loads.
__device__ __forceinline__ void l1_term(float pred, float target, float w, int bit, float& lsum, uint32_t& nz,
                                        uint32_t& ng) {
  const float d = pred - target;
  lsum += w * fabsf(d);
  nz |= (d != 0.f ? 1u : 0u) << bit;
  ng |= (d < 0.f ? 1u : 0u) << bit;
}

// NF > 0: N == NF known at compile time (CHW, vec), so every plane is unrolled.
template <int NF>
__global__ void __launch_bounds__(256) k_l1_signs(long long HW, int N, int hwc, int vec, const float* __restrict__ rgb,
                                                  const float* __restrict__ depth, const float* __restrict__ feat,
                                                  const L1Fwd l1) {
  pdl_wait();
  pdl_trigger();
  const bool V = NF > 0 || vec != 0;  // compile-time true in the specialised kernel
  const long long pix0 = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  float lsum = 0.f;
  if (pix0 < HW) {
    uint32_t nz[4] = {0u, 0u, 0u, 0u}, ng[4] = {0u, 0u, 0u, 0u};
    const int np = HW - pix0 < 4 ? (int)(HW - pix0) : 4;
    // one plane of 4 consecutive pixels (CHW planes, depth): 16-byte loads with vec
    auto plane4 = [&](const float* a, const float* b, long long off, float w, int bit) {
      if (V) {
        const float4 x = __ldcs(reinterpret_cast<const float4*>(a + off));
        const float4 y = __ldcs(reinterpret_cast<const float4*>(b + off));
        l1_term(x.x, y.x, w, bit, lsum, nz[0], ng[0]);
        l1_term(x.y, y.y, w, bit, lsum, nz[1], ng[1]);
        l1_term(x.z, y.z, w, bit, lsum, nz[2], ng[2]);
        l1_term(x.w, y.w, w, bit, lsum, nz[3], ng[3]);
      } else {
        for (int k = 0; k < np; ++k) l1_term(a[off + k], b[off + k], w, bit, lsum, nz[k], ng[k]);
      }
    };
    if (l1.target[0])
      for (int c = 0; c < 3; ++c) plane4(rgb, l1.target[0], c * HW + pix0, l1.w[0], kL1BitRgb + c);
    if (l1.target[1]) plane4(depth, l1.target[1], pix0, l1.w[1], kL1BitDepth);
    if (l1.target[2]) {
      if (NF > 0) {
#pragma unroll
        for (int c = 0; c < NF; ++c) plane4(feat, l1.target[2], c * HW + pix0, l1.w[2], c);
      } else if (!hwc) {
        for (int c = 0; c < N; ++c) plane4(feat, l1.target[2], c * HW + pix0, l1.w[2], c);
      } else if (V) {
        // the 4 pixels' rows are 4 N consecutive floats
        const float4* a = reinterpret_cast<const float4*>(feat + pix0 * N);
        const float4* b = reinterpret_cast<const float4*>(l1.target[2] + pix0 * N);
        for (int v = 0; v < N; ++v) {  // 4 N floats = N float4s
          const float4 x = __ldcs(a + v), y = __ldcs(b + v);
          const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int f = 4 * v + e;  // float index within the 4 rows
            l1_term(xs[e], ys[e], l1.w[2], f % N, lsum, nz[f / N], ng[f / N]);
          }
        }
      } else {
        for (int k = 0; k < np; ++k)
          for (int c = 0; c < N; ++c)
            l1_term(feat[(pix0 + k) * N + c], l1.target[2][(pix0 + k) * N + c], l1.w[2], c, lsum, nz[k], ng[k]);
      }
    }
    if (V) {
      uint4* o = reinterpret_cast<uint4*>(l1.signs + pix0);
      o[0] = make_uint4(nz[0], ng[0], nz[1], ng[1]);
      o[1] = make_uint4(nz[2], ng[2], nz[3], ng[3]);
    } else {
      for (int k = 0; k < np; ++k) l1.signs[pix0 + k] = make_uint2(nz[k], ng[k]);
    }
  }
  if (l1.loss) {
    __shared__ float s_part[8];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = 0.f;
      for (int w = 0; w < 8; ++w) b += s_part[w];
      if (b != 0.f) atomicAdd(l1.loss, b);
    }
  }
}

// Clears one range of 4-byte words: the words before the first 16-byte
// boundary and after the last one singly, the rest with 16-byte stores.
__device__ __forceinline__ void zero_range(uint32_t* __restrict__ a, long long n, long long t, long long stride) {
  const long long head = min(n, (long long)(((16u - ((uintptr_t)a & 15u)) & 15u) >> 2));
  const long long nv = (n - head) >> 2;
  uint4* v = reinterpret_cast<uint4*>(a + head);
  for (long long i = t; i < nv; i += stride) v[i] = make_uint4(0u, 0u, 0u, 0u);
  if (t < head) a[t] = 0u;
  const long long tail = head + 4 * nv;
  if (t < n - tail) a[tail + t] = 0u;
}

__global__ void __launch_bounds__(256) k_zero(uint32_t* __restrict__ a, long long na, uint32_t* __restrict__ b,
                                              long long nb) {
  pdl_wait();
  pdl_trigger();
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  zero_range(a, na, t, stride);
  if (b) zero_range(b, nb, t, stride);
}

// *count += the number of non-finite values among x[0 .. n), 16-byte loads
// where x is 16-byte aligned, one atomic per warp that found any.
__global__ void __launch_bounds__(256) k_count_nonfinite(const float* __restrict__ x, long long n,
                                                         unsigned long long* __restrict__ count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned c = 0;
  const long long head = min(n, (long long)(((16u - ((uintptr_t)x & 15u)) & 15u) >> 2));
  const long long nv = (n - head) >> 2;
  const float4* v = reinterpret_cast<const float4*>(x + head);
  for (long long i = t; i < nv; i += stride) {
    const float4 a = v[i];
    c += !isfinite(a.x) + !isfinite(a.y) + !isfinite(a.z) + !isfinite(a.w);
  }
  if (t < head) c += !isfinite(x[t]);
  const long long tail = head + 4 * nv;
  if (t < n - tail) c += !isfinite(x[tail + t]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// counts[0] += |{g : a_g != 0 and b_g != 0}|, counts[1] += |{g : a_g != 0 or b_g != 0}|.
__global__ void __launch_bounds__(256) k_vis_iou(int P, const uint8_t* __restrict__ a, const uint8_t* __restrict__ b,
                                                 unsigned long long* __restrict__ counts) {
  unsigned both = 0, either = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const bool x = a[i] != 0, y = b[i] != 0;
    both += (x && y) ? 1u : 0u;
    either += (x || y) ? 1u : 0u;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    both += __shfl_xor_sync(0xffffffffu, both, off);
    either += __shfl_xor_sync(0xffffffffu, either, off);
  }
  __shared__ unsigned s_c[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_c[0][wid] = both;
    s_c[1][wid] = either;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_c[threadIdx.x][w];
    if (t) atomicAdd(counts + threadIdx.x, t);
  }
}

bool cam_ok(const gs_camera* cam) {
  return cam && cam->width > 0 && cam->height > 0 && cam->width <= (1 << 15) && cam->height <= (1 << 15) &&
         cam->fx > 0.f && cam->fy > 0.f;
}

int num_tiles(const gs_camera* cam) {
  return ((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
}

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

constexpr float kBlack[3] = {0.f, 0.f, 0.f};

}  // namespace

gs_status launch_zero(void* a, size_t a_bytes, void* b, size_t b_bytes, cudaStream_t st) {
  const long long na = (long long)(a_bytes / 4), nb = b ? (long long)(b_bytes / 4) : 0;
  if (na + nb == 0) return GS_OK;
  long long blocks = (na / 4 + nb / 4 + 255) / 256 + 1;  // one 16-byte store per thread per round
  if (blocks > 152 * 8) blocks = 152 * 8;
  GS_TRACE("k_zero", st);
  launch_pdl(k_zero, (unsigned)blocks, 256, 0, st, static_cast<uint32_t*>(a), na, static_cast<uint32_t*>(b), nb);
  return last_launch_status();
}

}  // namespace gsff

using namespace gsff;

extern "C" {

int32_t gs_version(void) { return 1; }

gs_status gs_test_hold_tc_producer(int32_t on) {
  set_tc_test_hold(on);
  return GS_OK;
}

const char* gs_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "instance capacity exceeded";
    case GS_ERR_TIMEOUT: return "bounded wait timed out";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_UNSUPPORTED: return "unsupported option combination";
    case GS_ERR_BOUNDS: return "index out of range (bounds-checked build)";
  }
  return "unknown status";
}

gs_status gs_project(const gs_camera* cam, int32_t P, const float* means, const float* scales, const float* quats,
                     const float* opacity, float* uv, float* conic_opacity, float* depth, int32_t* rect,
                     int32_t* tiles_touched, int64_t* n_instances, void* stream) {
  GS_NVTX("gs_project");
  if (!cam_ok(cam) || P < 0) return GS_ERR_INVALID_ARG;
  if (P > 0 && (!means || !scales || !quats || !opacity || !uv || !conic_opacity || !depth || !rect ||
                !tiles_touched))
    return GS_ERR_INVALID_ARG;
  if (!aligned(quats, 16) || !aligned(conic_opacity, 16) || !aligned(rect, 16) || !aligned(uv, 8) ||
      !aligned(n_instances, 8))
    return GS_ERR_INVALID_ARG;
  if (n_instances && launch_zero(n_instances, sizeof(int64_t), nullptr, 0, S(stream)) != GS_OK) return GS_ERR_CUDA;
  launch_project(make_cam(*cam), P, means, scales, quats, opacity, uv, conic_opacity, depth, rect, tiles_touched,
                 n_instances, S(stream));
  return last_launch_status();
}

size_t gs_bin_sort_workspace_bytes(int32_t P, int64_t capacity, int32_t num_tiles) {
  if (P < 0 || capacity < 0 || num_tiles < 1 || num_tiles > (1 << 24)) return 0;
  return bin_sort_workspace_bytes(P, capacity, num_tiles);
}

gs_status gs_bin_sort(const gs_camera* cam, int32_t P, const float* depth, const int32_t* rect,
                      const int32_t* tiles_touched, int64_t capacity, void* workspace, size_t workspace_bytes,
                      uint64_t* keys, uint32_t* gids, int32_t* tile_ranges, int64_t* n_instances, int32_t* status,
                      void* stream) {
  GS_NVTX("gs_bin_sort");
  if (!cam_ok(cam) || P < 0 || capacity < 1 || capacity >= (1ll << 31)) return GS_ERR_INVALID_ARG;
  if (num_tiles(cam) > (1 << 24)) return GS_ERR_INVALID_ARG;
  if (!gids || !tile_ranges || !workspace || (P > 0 && (!depth || !rect || !tiles_touched)))
    return GS_ERR_INVALID_ARG;
  if (!aligned(workspace, 256) || !aligned(keys, 8) || !aligned(rect, 16) || !aligned(tile_ranges, 8) ||
      !aligned(n_instances, 8))
    return GS_ERR_INVALID_ARG;
  if (workspace_bytes < bin_sort_workspace_bytes(P, capacity, num_tiles(cam))) return GS_ERR_INVALID_ARG;
  return launch_bin_sort(make_cam(*cam), P, depth, rect, tiles_touched, capacity, workspace,
                         reinterpret_cast<unsigned long long*>(keys), gids, tile_ranges, n_instances, status,
                         S(stream));
}

gs_status gs_count_nonfinite(int64_t n, const float* x, uint64_t* count, void* stream) {
  if (n < 0 || (n > 0 && !x) || !count || !aligned(x, 4) || !aligned(count, 8)) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  long long blocks = (n / 4 + 255) / 256 + 1;
  if (blocks > 152 * 8) blocks = 152 * 8;
  GS_TRACE("k_count_nonfinite", S(stream));
  k_count_nonfinite<<<(unsigned)blocks, 256, 0, S(stream)>>>(x, (long long)n, reinterpret_cast<unsigned long long*>(count));
  return last_launch_status();
}

gs_status gs_zero(void* ptr, size_t bytes, void* stream) {
  GS_NVTX("gs_zero");
  if (bytes == 0) return GS_OK;
  if (!ptr || !aligned(ptr, 4) || bytes % 4 != 0) return GS_ERR_INVALID_ARG;
  return launch_zero(ptr, bytes, nullptr, 0, S(stream));
}

gs_status gs_tile_order(int32_t num_tiles, const int32_t* tile_ranges, int32_t* tile_order, void* stream) {
  GS_NVTX("gs_tile_order");
  if (num_tiles < 0 || (num_tiles > 0 && (!tile_ranges || !tile_order)) || !aligned(tile_ranges, 8))
    return GS_ERR_INVALID_ARG;
  if (num_tiles == 0) return GS_OK;
  return launch_tile_order(num_tiles, tile_ranges, tile_order, S(stream));
}

namespace {
gs_status render_fwd_impl(const gs_camera* cam, int32_t P, const int32_t* tile_ranges, const int32_t* tile_order,
                          const uint32_t* gids, uint8_t* inst_masks,
                          const float* uv, const float* conic_opacity, const float* depth, const float* colors,
                          const void* feats, int32_t N, int32_t feat_dtype, int32_t layout, int32_t flags,
                          const float* bg, float* out_rgb, float* out_depth, float* out_alpha, float* out_feat,
                          float* T_final, int32_t* last_idx, int32_t* n_contrib, uint8_t* visible, const L1Fwd* l1,
                          int32_t* status, void* stream) {
  if (!cam_ok(cam) || P < 0) return GS_ERR_INVALID_ARG;
  if (!tile_ranges || !gids || !out_rgb || !out_depth || !out_alpha || !T_final || !last_idx || !n_contrib)
    return GS_ERR_INVALID_ARG;
  if (P > 0 && (!uv || !conic_opacity || !depth || !colors)) return GS_ERR_INVALID_ARG;
  if (!aligned(conic_opacity, 16) || !aligned(uv, 8) || !aligned(tile_ranges, 8)) return GS_ERR_INVALID_ARG;
  if (feat_dtype != GS_F32 && feat_dtype != GS_BF16) return GS_ERR_INVALID_ARG;
  if (layout != GS_LAYOUT_CHW && layout != GS_LAYOUT_HWC) return GS_ERR_INVALID_ARG;
  const bool feat_on = (flags & GS_FEAT_ON) != 0;
  int n = 0;
  if (feat_on) {
    if (N <= 0 || N > 4096 || !out_feat || (P > 0 && !feats)) return GS_ERR_INVALID_ARG;
    if (!aligned(feats, 16) || !aligned(out_feat, 16)) return GS_ERR_INVALID_ARG;
    n = N;
  }
  const float* b = bg ? bg : kBlack;
  const CamF k = make_cam(*cam);
  if (feat_on && (flags & GS_FEAT_TENSOR_CORE)) {
    if (l1) return GS_ERR_UNSUPPORTED;
    if (feat_dtype != GS_BF16 || layout != GS_LAYOUT_HWC || N % 64 != 0 || N > 512) return GS_ERR_UNSUPPORTED;
    // geometry channels and the saved state on the SIMT kernel, features on tcgen05
    gs_status st = launch_render_fwd(k, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity, depth, colors, nullptr, 0,
                                     0, 1, b,
                                     out_rgb, out_depth, out_alpha, nullptr, T_final, last_idx, n_contrib, visible,
                                     nullptr, P, status, S(stream));
    if (st != GS_OK) return st;
    return launch_render_fwd_tc(k, P, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity,
                                static_cast<const __nv_bfloat16*>(feats), last_idx, N, out_feat, status,
                                S(stream));
  }
  if (l1 && n > 16) return GS_ERR_UNSUPPORTED;
  return launch_render_fwd(k, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity, depth, colors, feats, n,
                           feat_dtype == GS_BF16, layout == GS_LAYOUT_HWC, b, out_rgb, out_depth, out_alpha, out_feat,
                           T_final, last_idx, n_contrib, visible, l1, P, status, S(stream));
}
}  // namespace

gs_status gs_render_fwd(const gs_camera* cam, int32_t P, const int32_t* tile_ranges, const int32_t* tile_order,
                        const uint32_t* gids, uint8_t* inst_masks,
                        const float* uv, const float* conic_opacity, const float* depth, const float* colors,
                        const void* feats, int32_t N, int32_t feat_dtype, int32_t layout, int32_t flags,
                        const float* bg, float* out_rgb, float* out_depth, float* out_alpha, float* out_feat,
                        float* T_final, int32_t* last_idx, int32_t* n_contrib, uint8_t* visible,
                        int32_t* status, void* stream) {
  GS_NVTX("gs_render_fwd");
  return render_fwd_impl(cam, P, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity, depth, colors, feats, N, feat_dtype, layout,
                         flags, bg, out_rgb, out_depth, out_alpha, out_feat, T_final, last_idx, n_contrib, visible,
                         nullptr, status, stream);
}

gs_status gs_render_fwd_l1(const gs_camera* cam, int32_t P, const int32_t* tile_ranges, const int32_t* tile_order,
                           const uint32_t* gids, uint8_t* inst_masks,
                           const float* uv, const float* conic_opacity, const float* depth, const float* colors,
                           const void* feats, int32_t N, int32_t feat_dtype, int32_t layout, int32_t flags,
                           const float* bg, float* out_rgb, float* out_depth, float* out_alpha, float* out_feat,
                           float* T_final, int32_t* last_idx, int32_t* n_contrib, uint8_t* visible,
                           const gs_l1_terms* l1, uint32_t* l1_signs, int32_t* status, void* stream) {
  GS_NVTX("gs_render_fwd_l1");
  if (!l1 || !l1_signs || !aligned(l1_signs, 8)) return GS_ERR_INVALID_ARG;
  const bool feat_on = (flags & GS_FEAT_ON) != 0;
  L1Fwd in{};
  in.on = 1;
  in.target[0] = l1->target_rgb;
  in.target[1] = l1->target_depth;
  in.target[2] = feat_on ? l1->target_feat : nullptr;
  in.w[0] = l1->w_rgb;
  in.w[1] = l1->w_depth;
  in.w[2] = l1->w_feat;
  in.loss = l1->loss;
  in.signs = reinterpret_cast<uint2*>(l1_signs);
  return render_fwd_impl(cam, P, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity, depth, colors, feats, N, feat_dtype, layout,
                         flags, bg, out_rgb, out_depth, out_alpha, out_feat, T_final, last_idx, n_contrib, visible,
                         &in, status, stream);
}

size_t gs_render_bwd_workspace_bytes(int32_t P) {
  if (P < 0) return 0;
  // d_uv [P,2], d_conic [P,3], d_depth [P]
  return align_up((size_t)P * 2 * 4, 256) + align_up((size_t)P * 3 * 4, 256) + align_up((size_t)P * 4, 256);
}

namespace {
gs_status render_bwd_impl(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                          const float* quats, const float* colors, const void* feats, int32_t N, int32_t feat_dtype,
                          int32_t layout, int32_t flags, const float* bg, const int32_t* tile_ranges,
                          const int32_t* tile_order, const uint32_t* gids, const uint8_t* inst_masks,
                          const float* uv, const float* conic_opacity, const float* depth, const float* T_final,
                          const int32_t* last_idx, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dalpha, const float* dL_dfeat, const L1Bwd* l1, int32_t feat_grad_mode,
                          void* workspace, size_t workspace_bytes, float* d_means, float* d_scales, float* d_quats,
                          float* d_opacity, float* d_colors, float* d_feats, float* d_pose, int32_t* status,
                          void* stream) {
  if (!cam_ok(cam) || P < 0) return GS_ERR_INVALID_ARG;
  if (!tile_ranges || !gids || !T_final || !last_idx || !workspace) return GS_ERR_INVALID_ARG;
  if (P > 0 && (!means || !scales || !quats || !colors || !uv || !conic_opacity || !depth)) return GS_ERR_INVALID_ARG;
  if (!d_pose) return GS_ERR_INVALID_ARG;
  if (!aligned(workspace, 256) || !aligned(quats, 16) || !aligned(conic_opacity, 16) || !aligned(uv, 8))
    return GS_ERR_INVALID_ARG;
  if (workspace_bytes < gs_render_bwd_workspace_bytes(P)) return GS_ERR_INVALID_ARG;
  if (feat_dtype != GS_F32 && feat_dtype != GS_BF16) return GS_ERR_INVALID_ARG;
  if (layout != GS_LAYOUT_CHW && layout != GS_LAYOUT_HWC) return GS_ERR_INVALID_ARG;
  if (feat_grad_mode != GS_FEAT_GRAD_DECOUPLED && feat_grad_mode != GS_FEAT_GRAD_COUPLED) return GS_ERR_INVALID_ARG;
  const bool feat_on = (flags & GS_FEAT_ON) != 0;
  int n = 0;
  if (feat_on) {
    if (N <= 0 || N > 4096 || (P > 0 && (!d_feats || !feats))) return GS_ERR_INVALID_ARG;
    if (!aligned(feats, 16)) return GS_ERR_INVALID_ARG;
    n = N;
  }
  const bool coupled = feat_on && feat_grad_mode == GS_FEAT_GRAD_COUPLED && dL_dfeat;
  const bool tc = feat_on && (flags & GS_FEAT_TENSOR_CORE);
  if (tc && (coupled || feat_dtype != GS_BF16 || layout != GS_LAYOUT_HWC || N % 128 != 0 || N > 512))
    return GS_ERR_UNSUPPORTED;
  if (tc && ((dL_dfeat && !aligned(dL_dfeat, 16)) || !aligned(d_feats, 16))) return GS_ERR_INVALID_ARG;
  if (l1 && (tc || coupled || n > 16)) return GS_ERR_UNSUPPORTED;
  const float* b = bg ? bg : kBlack;
  const CamF k = make_cam(*cam);
  char* ws = static_cast<char*>(workspace);
  float* w_uv = reinterpret_cast<float*>(ws);
  float* w_conic = reinterpret_cast<float*>(ws + align_up((size_t)P * 2 * 4, 256));
  float* w_depth = reinterpret_cast<float*>(ws + align_up((size_t)P * 2 * 4, 256) + align_up((size_t)P * 3 * 4, 256));
  if (launch_zero(workspace, gs_render_bwd_workspace_bytes(P), nullptr, 0, S(stream)) != GS_OK) return GS_ERR_CUDA;
  // with the tensor-core form the SIMT adjoint does the geometry only and the
  // feature gradient is a tcgen05 contraction
  gs_status st = launch_render_bwd(k, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity, depth, colors, feats, tc ? 0 : n,
                                   feat_dtype == GS_BF16, layout == GS_LAYOUT_HWC, b, T_final, last_idx, dL_drgb,
                                   dL_ddepth, dL_dalpha, (feat_on && !tc) ? dL_dfeat : nullptr, coupled ? 1 : 0, w_uv,
                                   w_conic, w_depth, d_opacity, d_colors, d_feats, l1, P, status, S(stream));
  if (st != GS_OK) return st;
  if (tc && dL_dfeat) {
    st = launch_render_bwd_feat_tc(k, P, tile_ranges, tile_order, gids, inst_masks, uv, conic_opacity, last_idx, dL_dfeat,
                                   N, d_feats,
                                   status,
                                   S(stream));
    if (st != GS_OK) return st;
  }
  launch_project_bwd(k, P, means, scales, quats, w_uv, w_conic, w_depth, d_means, d_scales, d_quats, d_pose, S(stream));
  return last_launch_status();
}
}  // namespace

size_t gs_pair_state_workspace_bytes(int32_t width, int32_t height) {
  if (width <= 0 || height <= 0) return 0;
  return pair_state_workspace_bytes((long long)width * height);
}

gs_status gs_render_fwd_pairs(const gs_camera* cam, int32_t P, const int32_t* tile_ranges, const int32_t* tile_order,
                              const uint32_t* gids, const float* uv, const float* conic_opacity,
                              const int32_t* last_idx, const int32_t* n_contrib, void* workspace,
                              size_t workspace_bytes, int64_t capacity, int64_t* pair_off, float* pair_T,
                              int32_t* status, void* stream) {
  GS_NVTX("gs_render_fwd_pairs");
  if (!cam_ok(cam) || P < 0 || capacity < 0) return GS_ERR_INVALID_ARG;
  if (!tile_ranges || !gids || !last_idx || !n_contrib || !workspace || !pair_off || (capacity > 0 && !pair_T))
    return GS_ERR_INVALID_ARG;
  if (P > 0 && (!uv || !conic_opacity)) return GS_ERR_INVALID_ARG;
  if (!aligned(conic_opacity, 16) || !aligned(uv, 8) || !aligned(tile_ranges, 8) || !aligned(pair_off, 8) ||
      !aligned(workspace, 256))
    return GS_ERR_INVALID_ARG;
  if (workspace_bytes < gs_pair_state_workspace_bytes(cam->width, cam->height)) return GS_ERR_INVALID_ARG;
  return launch_store_pairs(make_cam(*cam), P, tile_ranges, tile_order, gids, uv, conic_opacity, last_idx, n_contrib,
                            workspace, capacity, pair_off, pair_T, status, S(stream));
}

gs_status gs_render_bwd_pairs(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                              const float* quats, const float* colors, const void* feats, int32_t N,
                              int32_t feat_dtype, int32_t layout, int32_t flags, const float* bg,
                              const int32_t* tile_ranges, const int32_t* tile_order, const uint32_t* gids,
                              const float* uv, const float* conic_opacity, const float* depth, const float* T_final,
                              const int32_t* last_idx, const float* dL_drgb, const float* dL_ddepth,
                              const float* dL_dalpha, const float* dL_dfeat, int32_t feat_grad_mode,
                              const int64_t* pair_off, const float* pair_T, void* workspace,
                              size_t workspace_bytes, float* d_means, float* d_scales, float* d_quats,
                              float* d_opacity, float* d_colors, float* d_feats, float* d_pose, int32_t* status,
                              void* stream) {
  GS_NVTX("gs_render_bwd_pairs");
  if (!cam_ok(cam) || P < 0) return GS_ERR_INVALID_ARG;
  if (!tile_ranges || !gids || !T_final || !last_idx || !workspace || !d_pose) return GS_ERR_INVALID_ARG;
  if (P > 0 && (!means || !scales || !quats || !colors || !uv || !conic_opacity || !depth)) return GS_ERR_INVALID_ARG;
  if (pair_T && !pair_off) return GS_ERR_INVALID_ARG;
  if (!aligned(workspace, 256) || !aligned(quats, 16) || !aligned(conic_opacity, 16) || !aligned(uv, 8) ||
      !aligned(pair_off, 8))
    return GS_ERR_INVALID_ARG;
  if (workspace_bytes < gs_render_bwd_workspace_bytes(P)) return GS_ERR_INVALID_ARG;
  if (feat_dtype != GS_F32 && feat_dtype != GS_BF16) return GS_ERR_INVALID_ARG;
  if (layout != GS_LAYOUT_CHW && layout != GS_LAYOUT_HWC) return GS_ERR_INVALID_ARG;
  if (feat_grad_mode != GS_FEAT_GRAD_DECOUPLED && feat_grad_mode != GS_FEAT_GRAD_COUPLED) return GS_ERR_INVALID_ARG;
  if (flags & GS_FEAT_TENSOR_CORE) return GS_ERR_UNSUPPORTED;
  const bool feat_on = (flags & GS_FEAT_ON) != 0;
  int n = 0;
  if (feat_on) {
    if (N <= 0 || N > 4096 || (P > 0 && (!d_feats || !feats))) return GS_ERR_INVALID_ARG;
    if (!aligned(feats, 16)) return GS_ERR_INVALID_ARG;
    n = N;
  }
  const bool coupled = feat_on && feat_grad_mode == GS_FEAT_GRAD_COUPLED && dL_dfeat;
  const float* b = bg ? bg : kBlack;
  const CamF k = make_cam(*cam);
  char* ws = static_cast<char*>(workspace);
  float* w_uv = reinterpret_cast<float*>(ws);
  float* w_conic = reinterpret_cast<float*>(ws + align_up((size_t)P * 2 * 4, 256));
  float* w_depth = reinterpret_cast<float*>(ws + align_up((size_t)P * 2 * 4, 256) + align_up((size_t)P * 3 * 4, 256));
  if (launch_zero(workspace, gs_render_bwd_workspace_bytes(P), nullptr, 0, S(stream)) != GS_OK) return GS_ERR_CUDA;
  gs_status st = launch_render_bwd_pairs(k, tile_ranges, tile_order, gids, uv, conic_opacity, depth, colors, feats, n,
                                         feat_dtype == GS_BF16, layout == GS_LAYOUT_HWC, b, T_final, last_idx, dL_drgb,
                                         dL_ddepth, dL_dalpha, feat_on ? dL_dfeat : nullptr, coupled ? 1 : 0,
                                         reinterpret_cast<const long long*>(pair_off), pair_T, w_uv, w_conic, w_depth,
                                         d_opacity, d_colors, d_feats, P, status, S(stream));
  if (st != GS_OK) return st;
  launch_project_bwd(k, P, means, scales, quats, w_uv, w_conic, w_depth, d_means, d_scales, d_quats, d_pose, S(stream));
  return last_launch_status();
}

gs_status gs_render_bwd(const gs_camera* cam, int32_t P, const float* means, const float* scales, const float* quats,
                        const float* colors, const void* feats, int32_t N, int32_t feat_dtype, int32_t layout,
                        int32_t flags, const float* bg, const int32_t* tile_ranges, const int32_t* tile_order,
                        const uint32_t* gids, const uint8_t* inst_masks, const float* uv, const float* conic_opacity, const float* depth,
                        const float* T_final,
                        const int32_t* last_idx, const float* dL_drgb, const float* dL_ddepth, const float* dL_dalpha,
                        const float* dL_dfeat, int32_t feat_grad_mode, void* workspace, size_t workspace_bytes,
                        float* d_means, float* d_scales, float* d_quats, float* d_opacity, float* d_colors,
                        float* d_feats, float* d_pose, int32_t* status, void* stream) {
  GS_NVTX("gs_render_bwd");
  return render_bwd_impl(cam, P, means, scales, quats, colors, feats, N, feat_dtype, layout, flags, bg, tile_ranges,
                         tile_order, gids, inst_masks, uv, conic_opacity, depth, T_final, last_idx, dL_drgb, dL_ddepth, dL_dalpha, dL_dfeat,
                         nullptr, feat_grad_mode, workspace, workspace_bytes, d_means, d_scales, d_quats, d_opacity,
                         d_colors, d_feats, d_pose, status, stream);
}

gs_status gs_render_bwd_l1(const gs_camera* cam, int32_t P, const float* means, const float* scales,
                           const float* quats, const float* colors, const void* feats, int32_t N, int32_t feat_dtype,
                           int32_t layout, int32_t flags, const float* bg, const int32_t* tile_ranges,
                           const int32_t* tile_order, const uint32_t* gids, const uint8_t* inst_masks,
                           const float* uv, const float* conic_opacity, const float* depth,
                           const float* T_final, const int32_t* last_idx, const gs_l1_terms* l1,
                           const uint32_t* l1_signs, void* workspace, size_t workspace_bytes, float* d_means,
                           float* d_scales, float* d_quats, float* d_opacity, float* d_colors, float* d_feats,
                           float* d_pose, int32_t* status, void* stream) {
  GS_NVTX("gs_render_bwd_l1");
  if (!l1 || !l1_signs || !aligned(l1_signs, 8)) return GS_ERR_INVALID_ARG;
  L1Bwd in{};
  in.on = 1;
  in.signs = reinterpret_cast<const uint2*>(l1_signs);
  in.w[0] = l1->w_rgb;
  in.w[1] = l1->w_depth;
  in.w[2] = l1->w_feat;
  return render_bwd_impl(cam, P, means, scales, quats, colors, feats, N, feat_dtype, layout, flags, bg, tile_ranges,
                         tile_order, gids, inst_masks, uv, conic_opacity, depth, T_final, last_idx, nullptr, nullptr, nullptr, nullptr, &in,
                         GS_FEAT_GRAD_DECOUPLED, workspace, workspace_bytes, d_means, d_scales, d_quats, d_opacity,
                         d_colors, d_feats, d_pose, status, stream);
}

gs_status gs_l1_loss_grad(int64_t n, const float* pred, const float* target, float scale, float* grad,
                          float* loss_sum, void* stream) {
  if (n < 0 || (n > 0 && (!pred || !target || !grad))) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  const int vec = aligned(pred, 16) && aligned(target, 16) && aligned(grad, 16);
  long long blocks = (n + 1023) / 1024;  // about one float4 per thread
  if (blocks > 152 * 16) blocks = 152 * 16;
  GS_TRACE("k_l1_grad", S(stream));
  k_l1_grad<<<(unsigned)blocks, 256, 0, S(stream)>>>(n, pred, target, scale, grad, loss_sum, vec);
  return last_launch_status();
}

gs_status gs_l1_signs(int32_t width, int32_t height, int32_t N, int32_t layout, const float* rgb, const float* depth,
                      const float* feat, const gs_l1_terms* l1, uint32_t* l1_signs, void* stream) {
  GS_NVTX("gs_l1_signs");
  if (width <= 0 || height <= 0 || N < 0 || !l1 || !l1_signs || !aligned(l1_signs, 8)) return GS_ERR_INVALID_ARG;
  if (layout != GS_LAYOUT_CHW && layout != GS_LAYOUT_HWC) return GS_ERR_INVALID_ARG;
  if (N > 16) return GS_ERR_UNSUPPORTED;
  if ((l1->target_rgb && !rgb) || (l1->target_depth && !depth) || (N > 0 && l1->target_feat && !feat))
    return GS_ERR_INVALID_ARG;
  L1Fwd in{};
  in.on = 1;
  in.target[0] = l1->target_rgb;
  in.target[1] = l1->target_depth;
  in.target[2] = N > 0 ? l1->target_feat : nullptr;
  in.w[0] = l1->w_rgb;
  in.w[1] = l1->w_depth;
  in.w[2] = l1->w_feat;
  in.loss = l1->loss;
  in.signs = reinterpret_cast<uint2*>(l1_signs);
  const long long HW = (long long)width * height;
  const bool hwc = layout == GS_LAYOUT_HWC;
  // 16-byte loads: every plane base aligned and HW % 4 == 0 (CHW planes, and
  // the rgb and depth planes in either layout), and for HWC N % 4 == 0
  bool vec = HW % 4 == 0 && aligned(l1_signs, 16) && (!hwc || N % 4 == 0);
  for (const float* q : {rgb, depth, feat, l1->target_rgb, l1->target_depth, in.target[2]})
    if (q && !aligned(q, 16)) vec = false;
  const long long quads = (HW + 3) / 4;
  GS_TRACE("k_l1_signs", S(stream));
  const unsigned grid = (unsigned)((quads + 255) / 256);
  if (vec && !hwc && N == 16 && in.target[2])
    launch_pdl(k_l1_signs<16>, grid, 256, 0, S(stream), HW, N, 0, 1, rgb, depth, feat, in);
  else
    launch_pdl(k_l1_signs<0>, grid, 256, 0, S(stream), HW, N, hwc ? 1 : 0, vec ? 1 : 0, rgb, depth, feat, in);
  return last_launch_status();
}

gs_status gs_visibility_iou(int32_t P, const uint8_t* vis_a, const uint8_t* vis_b, int64_t* counts, void* stream) {
  if (P < 0 || !counts || !aligned(counts, 8) || (P > 0 && (!vis_a || !vis_b))) return GS_ERR_INVALID_ARG;
  if (cudaMemsetAsync(counts, 0, 2 * sizeof(int64_t), S(stream)) != cudaSuccess) return GS_ERR_CUDA;
  if (P == 0) return GS_OK;
  int blocks = (P + 1023) / 1024;
  if (blocks > 152 * 4) blocks = 152 * 4;
  GS_TRACE("k_vis_iou", S(stream));
  k_vis_iou<<<blocks, 256, 0, S(stream)>>>(P, vis_a, vis_b, reinterpret_cast<unsigned long long*>(counts));
  return last_launch_status();
}

gs_status gs_trace_enable(int32_t capacity) {
  std::lock_guard<std::mutex> lk(g_trace.mu);
  for (cudaEvent_t e : g_trace.ev) cudaEventDestroy(e);
  g_trace.ev.clear();
  g_trace.names.clear();
  g_trace.count = 0;
  g_trace.open = -1;
  g_trace.on = false;
  g_trace.cap = 0;
  if (capacity <= 0) return GS_OK;
  g_trace.ev.resize(2 * (size_t)capacity);
  for (auto& e : g_trace.ev)
    if (cudaEventCreate(&e) != cudaSuccess) return GS_ERR_CUDA;
  g_trace.names.assign(capacity, nullptr);
  g_trace.cap = capacity;
  g_trace.on = true;
  return GS_OK;
}

void gs_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_trace.mu);
  g_trace.count = 0;
  g_trace.open = -1;
}

int32_t gs_trace_count(void) { return g_trace.count; }

gs_status gs_trace_get(int32_t i, const char** name, float* ms) {
  if (i < 0 || i >= g_trace.count || !name || !ms) return GS_ERR_INVALID_ARG;
  if (cudaEventSynchronize(g_trace.ev[2 * i + 1]) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaEventElapsedTime(ms, g_trace.ev[2 * i], g_trace.ev[2 * i + 1]) != cudaSuccess) return GS_ERR_CUDA;
  *name = g_trace.names[i];
  return GS_OK;
}

}  // extern "C"
