// Tile x depth keys and a stable LSD radix sort (Sec. 3.1: Gaussians are
// sorted front-to-back per tile).
//
// Every kernel reads the instance count I from device memory, so one frame
// can be enqueued (and captured in a CUDA graph) without a host round trip;
// the grids are sized from the caller's capacity and idle blocks exit.
//
// Steps (all integer work, bit-exact):
//   1. k_scan_partials  : per-chunk sums of tiles_touched (4096 Gaussians a chunk)
//   2. k_scan_top       : exclusive scan of the chunk sums, I, capacity check
//   3. k_emit           : per-chunk exclusive scan + emission of (tile<<32 | depth bits, id)
//   4. per 8-bit digit  : k_digit_count -> k_digit_scan -> k_digit_scatter
//                         (ping-pong between the caller's buffers and the workspace)
//   5. k_tile_ranges    : [start, end) of every tile in the sorted keys
// Stability of the scatter: within a chunk each warp owns 512 consecutive
// keys, ranks equal digits with __match_any_sync in index order, and warps
// and chunks are offset by exclusive prefix sums in index order.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kScanChunk = 4096;  // Gaussians per chunk of the touched-count scan
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;    // keys per thread
constexpr int kSortChunk = kSortThreads * kSortItems;  // 4096 keys per block
constexpr int kRadix = 256;

struct SortCtrl {
  long long n_total;   // I (may exceed capacity)
  long long n_eff;     // min(I, capacity)
};

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total) {
  // 256 threads; returns the exclusive prefix of v over the block.
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  const int before = wid > 0 ? s_warp[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(256) k_scan_partials(int P, const int* __restrict__ touched, long long* __restrict__ partial) {
  __shared__ int s_warp[8];
  const int base = blockIdx.x * kScanChunk;
  int sum = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x) {
    const int g = base + i;
    if (g < P) sum += touched[g];
  }
  int total;
  block_exclusive_scan(sum, s_warp, total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Single block: exclusive scan of the chunk sums (in place), I, capacity check.
__global__ void __launch_bounds__(1024) k_scan_top(int nchunks, long long* __restrict__ partial, long long capacity,
                                                   SortCtrl* __restrict__ ctrl, long long* __restrict__ n_out,
                                                   int32_t* __restrict__ status) {
  __shared__ long long s_carry;
  __shared__ long long s_warp[32];
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < nchunks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const long long v = i < nchunks ? partial[i] : 0;
    long long x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
      long long w = s_warp[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const long long before = (wid > 0 ? s_warp[wid - 1] : 0) + s_carry;
    if (i < nchunks) partial[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long I = s_carry;
    ctrl->n_total = I;
    ctrl->n_eff = I < capacity ? I : capacity;
    if (n_out) *n_out = I;
    if (I > capacity) flag_status(status, GS_ERR_CAPACITY);
  }
}

// Each block: 4096 consecutive Gaussians, 16 per thread in order.
__global__ void __launch_bounds__(256) k_emit(int P, const int* __restrict__ touched, const int4* __restrict__ rect,
                                              const float* __restrict__ depth, const long long* __restrict__ partial,
                                              int tiles_x, long long capacity,
                                              unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
  __shared__ int s_cnt[kScanChunk];
  __shared__ int s_warp[8];
  const int base = blockIdx.x * kScanChunk;
  for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x) {
    const int g = base + i;
    s_cnt[i] = g < P ? touched[g] : 0;
  }
  __syncthreads();
  constexpr int per = kScanChunk / 256;
  int mine = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) mine += s_cnt[threadIdx.x * per + k];
  int total;
  long long off = partial[blockIdx.x] + block_exclusive_scan(mine, s_warp, total);
  for (int k = 0; k < per; ++k) {
    const int g = base + threadIdx.x * per + k;
    const int n = s_cnt[threadIdx.x * per + k];
    if (n > 0) {
      const int4 r = rect[g];
      const unsigned long long dbits = (unsigned long long)__float_as_uint(depth[g]);
      long long o = off;
      for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx) {
          if (o < capacity) {
            keys[o] = ((unsigned long long)(ty * tiles_x + tx) << 32) | dbits;
            vals[o] = (uint32_t)g;
          }
          ++o;
        }
    }
    off += n;
  }
}

// Count the digit occurrences of one 4096-key chunk per warp (512 keys each,
// 16 rounds of 32 in index order). Keys stay in registers for the scatter.
__device__ __forceinline__ void chunk_warp_counts(const unsigned long long* __restrict__ keys_in, long long n, int shift,
                                                  long long base, unsigned long long (&k)[kSortItems],
                                                  int (&d)[kSortItems], uint32_t (*s_hist)[kRadix]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 8 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long idx = base + wid * (kSortItems * 32) + r * 32 + lane;
    const bool valid = idx < n;
    k[r] = valid ? keys_in[idx] : 0ull;
    d[r] = valid ? (int)((k[r] >> shift) & (kRadix - 1)) : kRadix;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    const int leader = __ffs(peers) - 1;
    if (lane == leader && d[r] < kRadix) s_hist[wid][d[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSortThreads) k_digit_count(const unsigned long long* __restrict__ keys_in,
                                                              const SortCtrl* __restrict__ ctrl, int shift, int nblk,
                                                              uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[8][kRadix];
  const long long n = ctrl->n_eff;
  const long long base = (long long)blockIdx.x * kSortChunk;
  if (base >= n) return;
  unsigned long long k[kSortItems];
  int d[kSortItems];
  chunk_warp_counts(keys_in, n, shift, base, k, d, s_hist);
  const int dg = threadIdx.x;  // 256 threads = 256 digits
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) tot += s_hist[w][dg];
  hist[(size_t)dg * nblk + blockIdx.x] = tot;
}

// Exclusive scan over (digit, chunk) in digit-major order, in place.
__global__ void __launch_bounds__(1024) k_digit_scan(const SortCtrl* __restrict__ ctrl, int nblk, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_warp[32];
  const long long n = ctrl->n_eff;
  const int nact = (int)((n + kSortChunk - 1) / kSortChunk);
  if (nact == 0) return;
  const long long L = (long long)kRadix * nact;
  const long long per = (L + blockDim.x - 1) / blockDim.x;
  const long long lo = threadIdx.x * per;
  const long long hi = lo + per < L ? lo + per : L;
  auto at = [&](long long i) -> uint32_t& { return hist[(size_t)(i / nact) * nblk + (i % nact)]; };
  uint32_t sum = 0;
  for (long long i = lo; i < hi; ++i) sum += at(i);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = s_warp[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t run = (wid > 0 ? s_warp[wid - 1] : 0) + x - sum;
  for (long long i = lo; i < hi; ++i) {
    uint32_t& h = at(i);
    const uint32_t c = h;
    h = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(
    const unsigned long long* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    unsigned long long* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const SortCtrl* __restrict__ ctrl,
    int shift, int nblk, const uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[8][kRadix];
  const long long n = ctrl->n_eff;
  const long long base = (long long)blockIdx.x * kSortChunk;
  if (base >= n) return;
  unsigned long long k[kSortItems];
  int d[kSortItems];
  chunk_warp_counts(keys_in, n, shift, base, k, d, s_hist);
  {
    // exclusive prefix over warps, offset by the chunk's global digit base
    const int dg = threadIdx.x;
    uint32_t run = hist[(size_t)dg * nblk + blockIdx.x];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t c = s_hist[w][dg];
      s_hist[w][dg] = run;
      run += c;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long idx = base + wid * (kSortItems * 32) + r * 32 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    uint32_t pos = 0;
    if (d[r] < kRadix) {
      pos = s_hist[wid][d[r]] + __popc(peers & lt);
      if ((long long)pos < n) {
        keys_out[pos] = k[r];
        vals_out[pos] = vals_in[idx];
      }
    }
    __syncwarp();
    if (d[r] < kRadix && lane == __ffs(peers) - 1) s_hist[wid][d[r]] += __popc(peers);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) k_tile_ranges(const unsigned long long* __restrict__ keys,
                                                     const SortCtrl* __restrict__ ctrl, int num_tiles,
                                                     int2* __restrict__ ranges) {
  const long long n = ctrl->n_eff;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(keys[i] >> 32);
    if (t < 0 || t >= num_tiles) continue;
    if (i == 0 || (int)(keys[i - 1] >> 32) != t) ranges[t].x = (int)i;
    if (i == n - 1 || (int)(keys[i + 1] >> 32) != t) ranges[t].y = (int)(i + 1);
  }
}

struct SortLayout {
  size_t keys_alt, vals_alt, partial, hist, ctrl, total;
  int nscan, nblk;
};

SortLayout sort_layout(int P, long long capacity) {
  SortLayout L;
  L.nscan = (P + kScanChunk - 1) / kScanChunk;
  if (L.nscan < 1) L.nscan = 1;
  L.nblk = (int)((capacity + kSortChunk - 1) / kSortChunk);
  if (L.nblk < 1) L.nblk = 1;
  size_t o = 0;
  L.keys_alt = o;
  o = align_up(o + (size_t)capacity * 8, 256);
  L.vals_alt = o;
  o = align_up(o + (size_t)capacity * 4, 256);
  L.partial = o;
  o = align_up(o + (size_t)L.nscan * 8, 256);
  L.hist = o;
  o = align_up(o + (size_t)kRadix * L.nblk * 4, 256);
  L.ctrl = o;
  o = align_up(o + sizeof(SortCtrl), 256);
  L.total = o;
  return L;
}

int tile_bits(int num_tiles) {
  int b = 1;
  while ((1 << b) < num_tiles) ++b;
  return b;
}

}  // namespace

size_t bin_sort_workspace_bytes(int P, long long capacity) { return sort_layout(P, capacity).total; }

// Enqueues the whole sort on `st`. The workspace base must be 256-aligned.
gs_status launch_bin_sort(const CamF& cam, int P, const float* depth, const int32_t* rect, const int32_t* touched,
                          long long capacity, void* workspace, unsigned long long* keys, uint32_t* gids,
                          int32_t* ranges, int64_t* n_out, int32_t* status, cudaStream_t st) {
  const SortLayout L = sort_layout(P, capacity);
  char* ws = static_cast<char*>(workspace);
  auto* keys_alt = reinterpret_cast<unsigned long long*>(ws + L.keys_alt);
  auto* vals_alt = reinterpret_cast<uint32_t*>(ws + L.vals_alt);
  auto* partial = reinterpret_cast<long long*>(ws + L.partial);
  auto* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  auto* ctrl = reinterpret_cast<SortCtrl*>(ws + L.ctrl);
  const int num_tiles = cam.tiles_x * cam.tiles_y;
  const int bits = 32 + tile_bits(num_tiles);
  const int npass = (bits + 7) / 8;
  // Ping-pong so that the last pass lands in the caller's buffers.
  unsigned long long* kb[2];
  uint32_t* vb[2];
  if (npass % 2 == 0) {
    kb[0] = keys; vb[0] = gids; kb[1] = keys_alt; vb[1] = vals_alt;
  } else {
    kb[0] = keys_alt; vb[0] = vals_alt; kb[1] = keys; vb[1] = gids;
  }
  if (cudaMemsetAsync(ranges, 0, (size_t)num_tiles * 2 * sizeof(int32_t), st) != cudaSuccess) return GS_ERR_CUDA;
  {
    GS_TRACE("k_scan_partials", st);
    k_scan_partials<<<L.nscan, 256, 0, st>>>(P, touched, partial);
  }
  {
    GS_TRACE("k_scan_top", st);
    k_scan_top<<<1, 1024, 0, st>>>(L.nscan, partial, capacity, ctrl, reinterpret_cast<long long*>(n_out), status);
  }
  {
    GS_TRACE("k_emit", st);
    k_emit<<<L.nscan, 256, 0, st>>>(P, touched, reinterpret_cast<const int4*>(rect), depth, partial, cam.tiles_x,
                                    capacity, kb[0], vb[0]);
  }
  for (int p = 0; p < npass; ++p) {
    const int shift = 8 * p;
    {
      GS_TRACE("k_digit_count", st);
      k_digit_count<<<L.nblk, kSortThreads, 0, st>>>(kb[p & 1], ctrl, shift, L.nblk, hist);
    }
    {
      GS_TRACE("k_digit_scan", st);
      k_digit_scan<<<1, 1024, 0, st>>>(ctrl, L.nblk, hist);
    }
    {
      GS_TRACE("k_digit_scatter", st);
      k_digit_scatter<<<L.nblk, kSortThreads, 0, st>>>(kb[p & 1], vb[p & 1], kb[(p + 1) & 1], vb[(p + 1) & 1], ctrl,
                                                       shift, L.nblk, hist);
    }
  }
  {
    GS_TRACE("k_tile_ranges", st);
    int nb = (int)((capacity + 255) / 256);
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    k_tile_ranges<<<nb, 256, 0, st>>>(keys, ctrl, num_tiles, reinterpret_cast<int2*>(ranges));
  }
  return last_launch_status();
}

}  // namespace gsff
