// Per-pair saved state for the adjoint (the alternative to the saved
// T_final / last index that the paper's renderer builds on, Sec. 3.1): for
// every blended (pixel, Gaussian) pair the transmittance T_i in front of the
// Gaussian, as the forward computed it, so that the adjoint reads T_i instead
// of recovering it by division, T_i = T_{i+1} / (1 - alpha_i).
//
// Storage is per pixel, contiguous in list order: the pairs of pixel q (row
// major) occupy [pair_off[q], pair_off[q + 1]), pair_off being the exclusive
// scan of the forward's contributor counts (HW + 1 entries). The scan is three
// kernels (1024-pixel block sums, one block over the sums, per-block scans);
// the store pass walks each tile's list like the forward (the same alpha and
// transmittance operations in the same order, so the values equal the
// forward's bit for bit), bounded by the pixel's last index.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kPsBlock = 1024;  // pixels per block of the offset scan
constexpr int kPsBatch = 256;   // Gaussians per shared-memory batch of the store pass

__device__ __forceinline__ long long block_scan_ll(long long v, long long* s_warp, long long& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[nw - 1];
  const long long before = wid > 0 ? s_warp[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kPsBlock) k_pair_block_sums(const int32_t* __restrict__ n_contrib, long long HW,
                                                              long long* __restrict__ bsum) {
  __shared__ long long s_warp[32];
  const long long i = (long long)blockIdx.x * kPsBlock + threadIdx.x;
  const long long v = i < HW ? n_contrib[i] : 0;
  long long total;
  block_scan_ll(v, s_warp, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums in place; the total into
// pair_off[HW]; more pairs than the capacity flags GS_ERR_CAPACITY.
__global__ void __launch_bounds__(kPsBlock) k_pair_scan_sums(long long* __restrict__ bsum, int nb, long long HW,
                                                             long long capacity, long long* __restrict__ pair_off,
                                                             int32_t* __restrict__ status) {
  __shared__ long long s_warp[32];
  __shared__ long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kPsBlock) {
    const int i = base + threadIdx.x;
    const long long v = i < nb ? bsum[i] : 0;
    long long total;
    const long long ex = block_scan_ll(v, s_warp, total);
    const long long carry = s_carry;
    if (i < nb) bsum[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pair_off[HW] = s_carry;
    if (s_carry > capacity) flag_status(status, GS_ERR_CAPACITY);
  }
}

__global__ void __launch_bounds__(kPsBlock) k_pair_offsets(const int32_t* __restrict__ n_contrib, long long HW,
                                                           const long long* __restrict__ bsum,
                                                           long long* __restrict__ pair_off) {
  __shared__ long long s_warp[32];
  const long long i = (long long)blockIdx.x * kPsBlock + threadIdx.x;
  const long long v = i < HW ? n_contrib[i] : 0;
  long long total;
  const long long ex = block_scan_ll(v, s_warp, total);
  if (i < HW) pair_off[i] = bsum[blockIdx.x] + ex;
}

struct PairParams {
  CamF cam;
  const int2* ranges;
  const int* order;
  const uint32_t* gids;
  const float2* uv;
  const float4* co;
  const int32_t* last_idx;
  const long long* pair_off;
  long long capacity;
  float* pair_T;
  int P;
  int32_t* status;
};

// One 256-thread block per tile, one thread per pixel (row major in the tile).
__global__ void __launch_bounds__(kTilePix) k_store_pair_T(const PairParams p) {
  __shared__ float2 s_uv[kPsBatch];
  __shared__ float4 s_co[kPsBatch];
  __shared__ int s_maxlast;
  const int tile = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  const int px = tx * kTile + (threadIdx.x & 15), py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < p.cam.W && py < p.cam.H;
  const size_t pix = inside ? (size_t)py * p.cam.W + px : 0;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const int2 rg = p.ranges[tile];
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  const int last = inside ? p.last_idx[pix] : 0;
  if (last > 0) atomicMax(&s_maxlast, last);
  long long o = inside ? p.pair_off[pix] : 0;
  __syncthreads();
  const int maxlast = checked_len(s_maxlast, rg.y - rg.x, p.status);
  float T = 1.f;
  for (int start = 0; start < maxlast; start += kPsBatch) {
    const int n = min(kPsBatch, maxlast - start);
    if ((int)threadIdx.x < n) {
      const uint32_t g = checked_id(p.gids[rg.x + start + threadIdx.x], p.P, p.status);
      s_uv[threadIdx.x] = p.uv[g];
      s_co[threadIdx.x] = p.co[g];
    }
    __syncthreads();
    const int lim = min(n, last - start);
    for (int j = 0; j < lim; ++j) {
      PairAlpha pa;
      if (!pair_alpha(s_co[j], s_uv[j].x - pxc, s_uv[j].y - pyc, pa)) continue;
      // below the last index every pair that passes the alpha rules is blended
      if (o < p.capacity) p.pair_T[o] = T;
      ++o;
      T = __fmul_rn(T, __fsub_rn(1.f, pa.alpha));
    }
    __syncthreads();
  }
}

}  // namespace

size_t pair_state_workspace_bytes(long long HW) {
  return align_up((size_t)((HW + kPsBlock - 1) / kPsBlock + 1) * sizeof(long long), 256);
}

gs_status launch_store_pairs(const CamF& cam, int P, const int32_t* ranges, const int32_t* order,
                             const uint32_t* gids, const float* uv, const float* co, const int32_t* last_idx,
                             const int32_t* n_contrib, void* workspace, long long capacity, int64_t* pair_off,
                             float* pair_T, int32_t* status, cudaStream_t st) {
  const long long HW = (long long)cam.W * cam.H;
  const int nb = (int)((HW + kPsBlock - 1) / kPsBlock);
  long long* bsum = static_cast<long long*>(workspace);
  long long* off = reinterpret_cast<long long*>(pair_off);
  {
    GS_TRACE("k_pair_block_sums", st);
    k_pair_block_sums<<<nb, kPsBlock, 0, st>>>(n_contrib, HW, bsum);
  }
  {
    GS_TRACE("k_pair_scan_sums", st);
    k_pair_scan_sums<<<1, kPsBlock, 0, st>>>(bsum, nb, HW, capacity, off, status);
  }
  {
    GS_TRACE("k_pair_offsets", st);
    k_pair_offsets<<<nb, kPsBlock, 0, st>>>(n_contrib, HW, bsum, off);
  }
  PairParams p;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.gids = gids;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.last_idx = last_idx;
  p.pair_off = off;
  p.capacity = capacity;
  p.pair_T = pair_T;
  p.P = P;
  p.status = status;
  GS_TRACE("k_store_pair_T", st);
  k_store_pair_T<<<(unsigned)(cam.tiles_x * cam.tiles_y), kTilePix, 0, st>>>(p);
  return last_launch_status();
}

}  // namespace gsff
