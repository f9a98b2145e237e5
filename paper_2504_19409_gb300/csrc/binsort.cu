// Tile x depth binning and sorting (Sec. 3.1: projected Gaussians are sorted
// front-to-back per 16x16 tile).
//
// The result equals a stable sort of all (tile, Gaussian) instances by the
// 64-bit key (tile << 32 | depth bits) with ties in ascending Gaussian id,
// but it is computed in two much smaller stable sorts:
//   1. the P Gaussians by depth (32-bit keys, 4 passes over P pairs);
//      culled Gaussians get the largest key;
//   2. instances are emitted in that depth order (an exclusive scan of the
//      touched counts taken in sorted order, then a load-balanced expansion
//      of each 256-Gaussian chunk), each carrying its tile id;
//   3. the instances are sorted stably by tile id alone (ceil(bits/8) passes,
//      2 for up to 65,536 tiles), which keeps the depth order inside a tile.
// Every kernel reads its item count from device memory, so one frame is
// enqueued without a host round trip (grids are sized from P and the
// caller's capacity; idle blocks exit).
//
// One LSD pass over (u32 key, u32 value) pairs = three kernels:
//   k_rs_count   per 2048-key chunk, digit counts (per warp, then per chunk)
//   k_rs_scan    exclusive offsets for (chunk, digit), coalesced, one block
//   k_rs_scatter stable scatter: each warp owns 256 consecutive keys, ranks
//                equal digits with __match_any_sync in index order; warps and
//                chunks are offset by the exclusive prefix sums.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kScanChunk = 256;   // Gaussians per chunk of the touched-count scan / emission
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;       // keys per thread
constexpr int kRsChunk = kRsThreads * kRsItems;  // 2048 keys per block
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRadix = 256;

struct SortCtrl {
  long long n_total;    // I (may exceed capacity)
  long long n_eff;      // min(I, capacity)
  long long n_gauss;    // P
};

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total) {
  // blockDim.x threads (a multiple of 32, <= 1024); returns the exclusive prefix of v.
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[nw - 1];
  const int before = wid > 0 ? s_warp[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// ---- step 1: depth keys ------------------------------------------------------
__global__ void __launch_bounds__(256) k_depth_keys(int P, const float* __restrict__ depth,
                                                    const int* __restrict__ touched, uint32_t* __restrict__ dk,
                                                    uint32_t* __restrict__ dv, SortCtrl* __restrict__ ctrl) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) ctrl->n_gauss = P;
  if (g < P) {
    dk[g] = touched[g] > 0 ? __float_as_uint(depth[g]) : 0xFFFFFFFFu;
    dv[g] = (uint32_t)g;
  }
}

// ---- step 2: scan of touched counts in depth order, emission -------------------
__global__ void __launch_bounds__(256) k_scan_partials(int P, const uint32_t* __restrict__ order,
                                                       const int* __restrict__ touched,
                                                       long long* __restrict__ partial) {
  __shared__ int s_warp[32];
  const int r = blockIdx.x * kScanChunk + threadIdx.x;
  const int v = r < P ? touched[order[r]] : 0;
  int total;
  block_exclusive_scan(v, s_warp, total);
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

// Each block: 256 consecutive depth-ordered Gaussians (one per thread). The
// block's instances [0, total) are spread evenly over its threads; instance
// i belongs to the Gaussian k with off[k] <= i < off[k+1] (binary search in
// shared memory) and is tile (i - off[k]) of its rectangle, row-major.
// Writes are contiguous.
__global__ void __launch_bounds__(256) k_emit(int P, const uint32_t* __restrict__ order,
                                              const int* __restrict__ touched, const int4* __restrict__ rect,
                                              const long long* __restrict__ partial, int tiles_x, long long capacity,
                                              uint32_t* __restrict__ tkeys, uint32_t* __restrict__ vals) {
  __shared__ int s_off[kScanChunk + 1];
  __shared__ uint32_t s_g[kScanChunk];
  __shared__ int4 s_rc[kScanChunk];
  __shared__ int s_warp[32];
  const int r = blockIdx.x * kScanChunk + threadIdx.x;
  uint32_t g = 0;
  int n = 0;
  if (r < P) {
    g = order[r];
    n = touched[g];
  }
  s_g[threadIdx.x] = g;
  if (n > 0) s_rc[threadIdx.x] = rect[g];
  int total;
  const int ex = block_exclusive_scan(n, s_warp, total);
  s_off[threadIdx.x] = ex;
  if (threadIdx.x == 0) s_off[kScanChunk] = total;
  __syncthreads();
  const long long base = partial[blockIdx.x];
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    int lo = 0, hi = kScanChunk - 1;  // largest k with s_off[k] <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int4 rc = s_rc[lo];
    const int li = i - s_off[lo];
    const int rw = rc.z - rc.x;
    const int ty = rc.y + li / rw, tx = rc.x + li % rw;
    const long long o = base + i;
    if (o < capacity) {
      tkeys[o] = (uint32_t)(ty * tiles_x + tx);
      vals[o] = s_g[lo];
    }
  }
}

// ---- one LSD radix pass over (u32 key, u32 value) ------------------------------
// The count of items is *n (device); each block owns kRsChunk consecutive
// items; warp w of a block owns items [w*256, (w+1)*256) of the chunk, in 8
// rounds of 32 consecutive items.
__device__ __forceinline__ void rs_load_and_count(const uint32_t* __restrict__ keys_in, long long n, int shift,
                                                  long long base, uint32_t (&k)[kRsItems], int (&d)[kRsItems],
                                                  uint32_t (*s_hist)[kRadix]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const long long idx = base + wid * (kRsItems * 32) + r * 32 + lane;
    const bool valid = idx < n;
    k[r] = valid ? keys_in[idx] : 0u;
    d[r] = valid ? (int)((k[r] >> shift) & (kRadix - 1)) : kRadix;
  }
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    if (lane == __ffs(peers) - 1 && d[r] < kRadix) s_hist[wid][d[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kRsThreads) k_rs_count(const uint32_t* __restrict__ keys_in,
                                                         const long long* __restrict__ n_ptr, int shift,
                                                         uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[kRsWarps][kRadix];
  const long long n = *n_ptr;
  const long long base = (long long)blockIdx.x * kRsChunk;
  if (base >= n) return;
  uint32_t k[kRsItems];
  int d[kRsItems];
  rs_load_and_count(keys_in, n, shift, base, k, d, s_hist);
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) tot += s_hist[w][threadIdx.x];
  hist[(size_t)blockIdx.x * kRadix + threadIdx.x] = tot;  // block-major [chunk][digit]
}

// Exclusive offsets over (digit, chunk) in digit-major order, written back in
// place into the block-major table. 1024 threads = 4 groups x 256 digits; a
// group walks a contiguous quarter of the chunks (loads coalesced over digits).
__global__ void __launch_bounds__(1024) k_rs_scan(const long long* __restrict__ n_ptr, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_part[4][kRadix];
  __shared__ uint32_t s_warp[32];
  const long long n = *n_ptr;
  const int nact = (int)((n + kRsChunk - 1) / kRsChunk);
  if (nact == 0) return;
  const int d = threadIdx.x & (kRadix - 1), q = threadIdx.x >> 8;
  const int per = (nact + 3) / 4;
  const int b0 = min(nact, q * per), b1 = min(nact, b0 + per);
  uint32_t sum = 0;
#pragma unroll 8
  for (int b = b0; b < b1; ++b) sum += hist[(size_t)b * kRadix + d];
  s_part[q][d] = sum;
  __syncthreads();
  // digit totals and their exclusive scan (threads 0..255)
  uint32_t total = 0;
  if (threadIdx.x < kRadix) total = s_part[0][d] + s_part[1][d] + s_part[2][d] + s_part[3][d];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = total;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31 && wid < 8) s_warp[wid] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t w = lane < 8 ? s_warp[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < 8) s_warp[lane] = w;
  }
  __syncthreads();
  __shared__ uint32_t s_base[kRadix];
  if (threadIdx.x < kRadix) s_base[d] = (wid > 0 ? s_warp[wid - 1] : 0) + x - total;
  __syncthreads();
  uint32_t run = s_base[d];
  for (int qq = 0; qq < q; ++qq) run += s_part[qq][d];
  int b = b0;
  for (; b + 8 <= b1; b += 8) {
    uint32_t c[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) c[e] = hist[(size_t)(b + e) * kRadix + d];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      hist[(size_t)(b + e) * kRadix + d] = run;
      run += c[e];
    }
  }
  for (; b < b1; ++b) {
    uint32_t* h = hist + (size_t)b * kRadix + d;
    const uint32_t c = *h;
    *h = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           uint32_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out,
                                                           const long long* __restrict__ n_ptr, int shift,
                                                           const uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[kRsWarps][kRadix];
  const long long n = *n_ptr;
  const long long base = (long long)blockIdx.x * kRsChunk;
  if (base >= n) return;
  uint32_t k[kRsItems];
  int d[kRsItems];
  rs_load_and_count(keys_in, n, shift, base, k, d, s_hist);
  {
    const int dg = threadIdx.x;
    uint32_t run = hist[(size_t)blockIdx.x * kRadix + dg];
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t c = s_hist[w][dg];
      s_hist[w][dg] = run;
      run += c;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const long long idx = base + wid * (kRsItems * 32) + r * 32 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    if (d[r] < kRadix) {
      const uint32_t pos = s_hist[wid][d[r]] + __popc(peers & lt);
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

// ---- step 3 output: tile ranges and the 64-bit keys ------------------------------
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ gids,
                                                     const float* __restrict__ depth, const SortCtrl* __restrict__ ctrl,
                                                     int num_tiles, int2* __restrict__ ranges,
                                                     unsigned long long* __restrict__ keys64) {
  const long long n = ctrl->n_eff;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t t = tkeys[i];
    if (keys64) keys64[i] = ((unsigned long long)t << 32) | (unsigned long long)__float_as_uint(depth[gids[i]]);
    if (t >= (uint32_t)num_tiles) continue;
    if (i == 0 || tkeys[i - 1] != t) ranges[t].x = (int)i;
    if (i == n - 1 || tkeys[i + 1] != t) ranges[t].y = (int)(i + 1);
  }
}

struct SortLayout {
  size_t dk, dv, dk2, dv2, partial, hist, ctrl, tk_alt, tv_alt, tk, total;
  int nscan, nblk_p, nblk_i;
};

SortLayout sort_layout(int P, long long capacity) {
  SortLayout L;
  L.nscan = (P + kScanChunk - 1) / kScanChunk;
  if (L.nscan < 1) L.nscan = 1;
  L.nblk_p = (P + kRsChunk - 1) / kRsChunk;
  if (L.nblk_p < 1) L.nblk_p = 1;
  L.nblk_i = (int)((capacity + kRsChunk - 1) / kRsChunk);
  if (L.nblk_i < 1) L.nblk_i = 1;
  const int nblk = L.nblk_p > L.nblk_i ? L.nblk_p : L.nblk_i;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.dk = take((size_t)P * 4);
  L.dv = take((size_t)P * 4);
  L.dk2 = take((size_t)P * 4);
  L.dv2 = take((size_t)P * 4);
  L.partial = take((size_t)L.nscan * 8);
  L.hist = take((size_t)kRadix * nblk * 4);
  L.ctrl = take(sizeof(SortCtrl));
  L.tk = take((size_t)capacity * 4);
  L.tk_alt = take((size_t)capacity * 4);
  L.tv_alt = take((size_t)capacity * 4);
  L.total = o;
  return L;
}

int tile_bits(int num_tiles) {
  int b = 1;
  while ((1 << b) < num_tiles) ++b;
  return b;
}

void radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, const long long* n_ptr,
                int shift, int nblk, uint32_t* hist, cudaStream_t st) {
  {
    GS_TRACE("k_rs_count", st);
    k_rs_count<<<nblk, kRsThreads, 0, st>>>(kin, n_ptr, shift, hist);
  }
  {
    GS_TRACE("k_rs_scan", st);
    k_rs_scan<<<1, 1024, 0, st>>>(n_ptr, hist);
  }
  {
    GS_TRACE("k_rs_scatter", st);
    k_rs_scatter<<<nblk, kRsThreads, 0, st>>>(kin, vin, kout, vout, n_ptr, shift, hist);
  }
}

}  // namespace

size_t bin_sort_workspace_bytes(int P, long long capacity) { return sort_layout(P, capacity).total; }

// Enqueues the whole binning on `st`. The workspace base must be 256-aligned.
// keys64 may be null (the 64-bit keys are then not written).
gs_status launch_bin_sort(const CamF& cam, int P, const float* depth, const int32_t* rect, const int32_t* touched,
                          long long capacity, void* workspace, unsigned long long* keys64, uint32_t* gids,
                          int32_t* ranges, int64_t* n_out, int32_t* status, cudaStream_t st) {
  const SortLayout L = sort_layout(P, capacity);
  char* ws = static_cast<char*>(workspace);
  auto* dk = reinterpret_cast<uint32_t*>(ws + L.dk);
  auto* dv = reinterpret_cast<uint32_t*>(ws + L.dv);
  auto* dk2 = reinterpret_cast<uint32_t*>(ws + L.dk2);
  auto* dv2 = reinterpret_cast<uint32_t*>(ws + L.dv2);
  auto* partial = reinterpret_cast<long long*>(ws + L.partial);
  auto* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  auto* ctrl = reinterpret_cast<SortCtrl*>(ws + L.ctrl);
  auto* tk = reinterpret_cast<uint32_t*>(ws + L.tk);
  auto* tk_alt = reinterpret_cast<uint32_t*>(ws + L.tk_alt);
  auto* tv_alt = reinterpret_cast<uint32_t*>(ws + L.tv_alt);
  const int num_tiles = cam.tiles_x * cam.tiles_y;
  const long long* n_gauss = &ctrl->n_gauss;
  const long long* n_inst = &ctrl->n_eff;

  if (cudaMemsetAsync(ranges, 0, (size_t)num_tiles * 2 * sizeof(int32_t), st) != cudaSuccess) return GS_ERR_CUDA;
  {
    GS_TRACE("k_depth_keys", st);
    k_depth_keys<<<(P + 255) / 256 > 0 ? (P + 255) / 256 : 1, 256, 0, st>>>(P, depth, touched, dk, dv, ctrl);
  }
  // 1. depth sort: 4 passes, ending in (dk, dv)
  radix_pass(dk, dv, dk2, dv2, n_gauss, 0, L.nblk_p, hist, st);
  radix_pass(dk2, dv2, dk, dv, n_gauss, 8, L.nblk_p, hist, st);
  radix_pass(dk, dv, dk2, dv2, n_gauss, 16, L.nblk_p, hist, st);
  radix_pass(dk2, dv2, dk, dv, n_gauss, 24, L.nblk_p, hist, st);
  // 2. scan + emission in depth order
  {
    GS_TRACE("k_scan_partials", st);
    k_scan_partials<<<L.nscan, 256, 0, st>>>(P, dv, touched, partial);
  }
  {
    GS_TRACE("k_scan_top", st);
    k_scan_top<<<1, 1024, 0, st>>>(L.nscan, partial, capacity, ctrl, reinterpret_cast<long long*>(n_out), status);
  }
  // 3. tile sort: passes ping-pong so that the last one lands in (tk, gids)
  const int npass = (tile_bits(num_tiles) + 7) / 8;
  uint32_t* kb[2];
  uint32_t* vb[2];
  if (npass % 2 == 0) {
    kb[0] = tk; vb[0] = gids; kb[1] = tk_alt; vb[1] = tv_alt;
  } else {
    kb[0] = tk_alt; vb[0] = tv_alt; kb[1] = tk; vb[1] = gids;
  }
  {
    GS_TRACE("k_emit", st);
    k_emit<<<L.nscan, 256, 0, st>>>(P, dv, touched, reinterpret_cast<const int4*>(rect), partial, cam.tiles_x,
                                    capacity, kb[0], vb[0]);
  }
  for (int p = 0; p < npass; ++p)
    radix_pass(kb[p & 1], vb[p & 1], kb[(p + 1) & 1], vb[(p + 1) & 1], n_inst, 8 * p, L.nblk_i, hist, st);
  {
    GS_TRACE("k_tile_ranges", st);
    int nb = (int)((capacity + 255) / 256);
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    k_tile_ranges<<<nb, 256, 0, st>>>(tk, gids, depth, ctrl, num_tiles, reinterpret_cast<int2*>(ranges), keys64);
  }
  return last_launch_status();
}

}  // namespace gsff
