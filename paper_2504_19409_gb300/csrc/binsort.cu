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
// One LSD pass over (u32 key, u32 value) pairs is a single kernel in the
// one-sweep style (a decoupled look-back across chunks):
//   - the digit counts of every pass are accumulated up front by the kernel
//     that writes the keys (k_depth_keys for the depth passes, k_emit for the
//     tile passes), so a pass knows where each digit starts globally;
//   - k_os_scatter: a block takes the next chunk of 2048 items by an atomic
//     ticket (chunks start in order), counts its digits, publishes the counts,
//     and sums its predecessors' counts per digit by walking back until a
//     chunk that has published its inclusive prefix; then scatters stably
//     (each warp owns 256 consecutive items and ranks equal digits with
//     __match_any_sync in index order). A block only waits on chunks with
//     earlier tickets, which are already running; every wait is bounded and
//     a timeout flags GS_ERR_TIMEOUT instead of hanging. After a timeout the
//     pass's output may have unwritten slots: the kernels after it treat ids
//     >= P as absent and the tile ranges stay empty, so nothing downstream
//     reads through a stale id.
// The look-back words and the counters are cleared by one zeroing kernel per
// frame.

#include <atomic>

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kScanChunk = 256;   // Gaussians per chunk of the touched-count scan / emission
constexpr int kEmitThreads = 1024;  // threads sharing a chunk's instances in k_emit
constexpr int kDkThreads = 1024;    // threads of k_depth_keys (kRsChunk keys per block)
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;       // keys per thread
constexpr int kRsChunk = kRsThreads * kRsItems;  // 2048 keys per block
static_assert(kRsChunk % kDkThreads == 0, "k_depth_keys covers a chunk in whole rounds of its threads");
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRadix = 256;

struct SortCtrl {
  long long n_total;    // I (may exceed capacity)
  long long n_eff;      // min(I, capacity)
  long long n_gauss;    // P
};

constexpr int kDepthPasses = 4;
constexpr int kMaxTilePasses = 3;  // tile ids < 2^24
constexpr int kMaxPasses = kDepthPasses + kMaxTilePasses;

// Per-frame one-sweep state (cleared by the zeroing kernel before the first
// kernel of the sort).
struct OsCtrl {
  uint32_t hist[kMaxPasses][kRadix];  // digit counts of each pass over all items
  uint32_t ticket[kMaxPasses];        // next chunk of each pass
  uint32_t timed_out;                 // set by a pass whose look-back gave up
};

// Look-back word of (chunk, digit): state in the top two bits, count below.
constexpr unsigned long long kLbAggregate = 1ull << 62;  // this chunk's own count
constexpr unsigned long long kLbPrefix = 2ull << 62;     // count of this and all earlier chunks
constexpr unsigned long long kLbCount = (1ull << 62) - 1;
constexpr int kLbWindow = 8;  // look-back words loaded per round trip

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

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
// One block per kRsChunk Gaussians. Culled Gaussians get the largest key. The
// block also adds its digit counts for the four depth passes to the frame's
// histograms (culled keys are 0xFFFFFFFF: digit 255 in every pass).
__global__ void __launch_bounds__(kDkThreads) k_depth_keys(int P, const float* __restrict__ depth,
                                                           const int* __restrict__ touched, uint32_t* __restrict__ dk,
                                                           uint32_t* __restrict__ dv, SortCtrl* __restrict__ ctrl,
                                                           OsCtrl* __restrict__ os) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_h[kDepthPasses][kRadix];
  __shared__ uint32_t s_cull;
  for (int i = threadIdx.x; i < kDepthPasses * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
  if (threadIdx.x == 0) s_cull = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->n_gauss = P;
  __syncthreads();
  const int base = blockIdx.x * kRsChunk;
  uint32_t ncull = 0;
#pragma unroll
  for (int r = 0; r < kRsChunk / kDkThreads; ++r) {
    const int g = base + r * kDkThreads + threadIdx.x;
    bool culled = false;
    if (g < P) {
      const bool vis = touched[g] > 0;
      const uint32_t key = vis ? __float_as_uint(depth[g]) : 0xFFFFFFFFu;
      dk[g] = key;
      dv[g] = (uint32_t)g;
      if (vis) {
#pragma unroll
        for (int p = 0; p < kDepthPasses; ++p) atomicAdd(&s_h[p][(key >> (8 * p)) & (kRadix - 1)], 1u);
      }
      culled = !vis;
    }
    ncull += __popc(__ballot_sync(0xffffffffu, culled));
  }
  if ((threadIdx.x & 31) == 0 && ncull) atomicAdd(&s_cull, ncull);
  __syncthreads();
  const int d = threadIdx.x;
  if (d < kRadix) {
#pragma unroll
    for (int p = 0; p < kDepthPasses; ++p) {
      const uint32_t v = s_h[p][d] + (d == kRadix - 1 ? s_cull : 0u);
      if (v) atomicAdd(&os->hist[p][d], v);
    }
  }
}

// ---- step 2: scan of touched counts in depth order, emission -------------------
__global__ void __launch_bounds__(256) k_scan_partials(int P, const uint32_t* __restrict__ order,
                                                       const int* __restrict__ touched,
                                                       long long* __restrict__ partial) {
  pdl_wait();
  pdl_trigger();
  __shared__ int s_warp[32];
  const int r = blockIdx.x * kScanChunk + threadIdx.x;
  // ids >= P can only come from a depth pass whose look-back timed out (its
  // output slots are then not all written): they count as culled
  const uint32_t g = r < P ? order[r] : 0xFFFFFFFFu;
  const int v = g < (uint32_t)P ? touched[g] : 0;
  int total;
  block_exclusive_scan(v, s_warp, total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Single block: exclusive scan of the chunk sums (in place), I, capacity check.
__global__ void __launch_bounds__(1024) k_scan_top(int nchunks, long long* __restrict__ partial, long long capacity,
                                                   SortCtrl* __restrict__ ctrl, long long* __restrict__ n_out,
                                                   int32_t* __restrict__ status) {
  pdl_wait();
  pdl_trigger();
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

// Each block: 256 consecutive depth-ordered Gaussians (one per thread of the
// first eight warps). The block's instances [0, total) are spread evenly over
// all 1024 of its threads (culled Gaussians sort last, so only a few chunks
// hold instances and each needs many threads); instance
// i belongs to the Gaussian k with off[k] <= i < off[k+1] (binary search in
// shared memory) and is tile (i - off[k]) of its rectangle, row-major.
// Writes are contiguous.
__global__ void __launch_bounds__(kEmitThreads) k_emit(int P, const uint32_t* __restrict__ order,
                                              const int* __restrict__ touched, const int4* __restrict__ rect,
                                              const long long* __restrict__ partial, int tiles_x, long long capacity,
                                              int npass, uint32_t* __restrict__ tkeys, uint32_t* __restrict__ vals,
                                              OsCtrl* __restrict__ os) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_th[kMaxTilePasses][kRadix];  // digit counts of the written tile keys
  __shared__ int s_off[kScanChunk + 1];
  __shared__ uint32_t s_g[kScanChunk];
  __shared__ int4 s_rc[kScanChunk];
  __shared__ int s_warp[32];
  const int r = blockIdx.x * kScanChunk + threadIdx.x;
  uint32_t g = 0;
  int n = 0;
  if (threadIdx.x < kScanChunk && r < P) {
    g = order[r];
    n = g < (uint32_t)P ? touched[g] : 0;  // as in k_scan_partials
  }
  for (int i = threadIdx.x; i < kMaxTilePasses * kRadix; i += blockDim.x) (&s_th[0][0])[i] = 0;
  if (threadIdx.x < kScanChunk) {
    s_g[threadIdx.x] = g;
    if (n > 0) s_rc[threadIdx.x] = rect[g];
  }
  int total;
  const int ex = block_exclusive_scan(n, s_warp, total);  // threads past the chunk add 0
  if (threadIdx.x < kScanChunk) s_off[threadIdx.x] = ex;
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
      const uint32_t t = (uint32_t)(ty * tiles_x + tx);
      tkeys[o] = t;
      vals[o] = s_g[lo];
      for (int p = 0; p < npass; ++p) atomicAdd(&s_th[p][(t >> (8 * p)) & (kRadix - 1)], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < kRadix)
    for (int p = 0; p < npass; ++p) {
      const uint32_t v = s_th[p][threadIdx.x];
      if (v) atomicAdd(&os->hist[kDepthPasses + p][threadIdx.x], v);
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

// One pass: see the file comment. `hist` = this pass's digit counts over all
// items, `ticket` its chunk counter, `lb` its look-back words [chunks][256].
__global__ void __launch_bounds__(kRsThreads) k_os_scatter(const uint32_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           uint32_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out,
                                                           const long long* __restrict__ n_ptr, int shift,
                                                           const uint32_t* __restrict__ hist, uint32_t* ticket,
                                                           unsigned long long* lb, uint32_t* timed_out,
                                                           unsigned long long wait_ns, int32_t* __restrict__ status) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_hist[kRsWarps][kRadix];
  __shared__ int s_warp[32];
  __shared__ uint32_t s_chunk;
  if (threadIdx.x == 0) s_chunk = atomicAdd(ticket, 1u);
  __syncthreads();
  const long long c = s_chunk;
  const long long n = *n_ptr;
  const long long base = c * kRsChunk;
  if (base >= n) return;
  uint32_t k[kRsItems];
  int d[kRsItems];
  rs_load_and_count(keys_in, n, shift, base, k, d, s_hist);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t v[kRsItems];  // values loaded before the look-back, so their latency overlaps it
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const long long idx = base + wid * (kRsItems * 32) + r * 32 + lane;
    v[r] = idx < n ? vals_in[idx] : 0u;
  }
  const int dg = threadIdx.x;
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) tot += s_hist[w][dg];
  unsigned long long* mine = lb + c * kRadix + dg;
  lb_store(mine, (c == 0 ? kLbPrefix : kLbAggregate) | tot);
  // where digit dg starts in the output: exclusive scan of the digit counts
  int all;
  const uint32_t start = (uint32_t)block_exclusive_scan((int)hist[dg], s_warp, all);
  unsigned long long before = 0;  // items of digit dg in chunks 0..c-1
  if (c > 0 && wait_ns == 0) {
    // a bound of 0 gives up before the first look-back (the timeout path,
    // taken deterministically)
    flag_status(status, GS_ERR_TIMEOUT);
    *timed_out = 1u;
    lb_store(mine, kLbPrefix | tot);
  } else if (c > 0) {
    // Walk back kLbWindow chunks per round trip: the words of chunks
    // j, j-1, .. are loaded together and consumed newest first until a
    // prefix; a chunk that has published nothing yet restarts the window
    // at that chunk.
    const unsigned long long t0 = globaltimer_ns();
    long long j = c - 1;
    while (true) {
      unsigned long long w[kLbWindow];
#pragma unroll
      for (int e = 0; e < kLbWindow; ++e) w[e] = j - e >= 0 ? lb_load(lb + (j - e) * kRadix + dg) : kLbPrefix;
      int e = 0;
      bool done = false;
#pragma unroll
      for (; e < kLbWindow; ++e) {
        const unsigned long long state = w[e] & ~kLbCount;
        if (state == 0) break;
        before += w[e] & kLbCount;
        if (state == kLbPrefix) {
          done = true;
          break;
        }
      }
      if (done) break;
      j -= e;
      if (e < kLbWindow && globaltimer_ns() - t0 > wait_ns) {
        flag_status(status, GS_ERR_TIMEOUT);
        *timed_out = 1u;
        break;
      }
    }
    lb_store(mine, kLbPrefix | (before + tot));
  }
  {
    uint32_t run = start + (uint32_t)before;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t cnt = s_hist[w][dg];
      s_hist[w][dg] = run;
      run += cnt;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    const unsigned peers = __match_any_sync(0xffffffffu, d[r]);
    if (d[r] < kRadix) {
      const uint32_t pos = s_hist[wid][d[r]] + __popc(peers & lt);
      if ((long long)pos < n) {
        keys_out[pos] = k[r];
        vals_out[pos] = v[r];
      }
    }
    __syncwarp();
    if (d[r] < kRadix && lane == __ffs(peers) - 1) s_hist[wid][d[r]] += __popc(peers);
    __syncwarp();
  }
}

// ---- step 3 output: tile ranges and the 64-bit keys ------------------------------
// After a pass of this frame timed out (its outputs are then unspecified and
// may hold unwritten slots), every tile range stays (0, 0) as the zeroing
// kernel left it, so no consumer of the lists reads a stale id.
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ gids,
                                                     const float* __restrict__ depth, const SortCtrl* __restrict__ ctrl,
                                                     const OsCtrl* __restrict__ os, int P, int num_tiles,
                                                     int2* __restrict__ ranges, unsigned long long* __restrict__ keys64) {
  pdl_wait();
  pdl_trigger();
  if (os->timed_out) return;
  const long long n = ctrl->n_eff;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t t = tkeys[i];
    if (keys64) {
      const uint32_t g = gids[i];
      keys64[i] = ((unsigned long long)t << 32) | (g < (uint32_t)P ? (unsigned long long)__float_as_uint(depth[g]) : 0ull);
    }
    if (t >= (uint32_t)num_tiles) continue;
    if (i == 0 || tkeys[i - 1] != t) ranges[t].x = (int)i;
    if (i == n - 1 || tkeys[i + 1] != t) ranges[t].y = (int)(i + 1);
  }
}

struct SortLayout {
  size_t dk, dv, dk2, dv2, partial, os, lb, ctrl, tk_alt, tv_alt, tk, total;
  size_t lb_bytes;   // look-back words of all passes (zeroed each frame with os)
  int nscan, nblk_p, nblk_i, npass_t;
};

int tile_bits(int num_tiles) {
  int b = 1;
  while ((1 << b) < num_tiles) ++b;
  return b;
}

SortLayout sort_layout(int P, long long capacity, int num_tiles) {
  SortLayout L;
  L.nscan = (P + kScanChunk - 1) / kScanChunk;
  if (L.nscan < 1) L.nscan = 1;
  L.nblk_p = (P + kRsChunk - 1) / kRsChunk;
  if (L.nblk_p < 1) L.nblk_p = 1;
  L.nblk_i = (int)((capacity + kRsChunk - 1) / kRsChunk);
  if (L.nblk_i < 1) L.nblk_i = 1;
  L.npass_t = (tile_bits(num_tiles) + 7) / 8;
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
  L.ctrl = take(sizeof(SortCtrl));
  // os and lb are adjacent: one memset clears both
  L.lb_bytes = ((size_t)kDepthPasses * L.nblk_p + (size_t)L.npass_t * L.nblk_i) * kRadix * 8;
  L.os = take(sizeof(OsCtrl));
  L.lb = take(L.lb_bytes);
  L.tk = take((size_t)capacity * 4);
  L.tk_alt = take((size_t)capacity * 4);
  L.tv_alt = take((size_t)capacity * 4);
  L.total = o;
  return L;
}

std::atomic<unsigned long long> g_lookback_wait_ns{1000000000ull};  // 1 s

void os_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, const long long* n_ptr,
             int shift, int pass, int nblk, OsCtrl* os, unsigned long long* lb, int32_t* status, cudaStream_t st) {
  GS_TRACE("k_os_scatter", st);
  launch_pdl(k_os_scatter, nblk, kRsThreads, 0, st, kin, vin, kout, vout, n_ptr, shift, os->hist[pass], &os->ticket[pass],
             lb, &os->timed_out, g_lookback_wait_ns.load(std::memory_order_relaxed), status);
}

}  // namespace

void set_lookback_wait_ns(unsigned long long ns) { g_lookback_wait_ns.store(ns, std::memory_order_relaxed); }

size_t bin_sort_workspace_bytes(int P, long long capacity, int num_tiles) {
  return sort_layout(P, capacity, num_tiles).total;
}

// Enqueues the whole binning on `st`. The workspace base must be 256-aligned.
// keys64 may be null (the 64-bit keys are then not written).
gs_status launch_bin_sort(const CamF& cam, int P, const float* depth, const int32_t* rect, const int32_t* touched,
                          long long capacity, void* workspace, unsigned long long* keys64, uint32_t* gids,
                          int32_t* ranges, int64_t* n_out, int32_t* status, cudaStream_t st) {
  const int num_tiles = cam.tiles_x * cam.tiles_y;
  const SortLayout L = sort_layout(P, capacity, num_tiles);
  if (L.npass_t > kMaxTilePasses) return GS_ERR_INVALID_ARG;
  char* ws = static_cast<char*>(workspace);
  auto* dk = reinterpret_cast<uint32_t*>(ws + L.dk);
  auto* dv = reinterpret_cast<uint32_t*>(ws + L.dv);
  auto* dk2 = reinterpret_cast<uint32_t*>(ws + L.dk2);
  auto* dv2 = reinterpret_cast<uint32_t*>(ws + L.dv2);
  auto* partial = reinterpret_cast<long long*>(ws + L.partial);
  auto* ctrl = reinterpret_cast<SortCtrl*>(ws + L.ctrl);
  auto* os = reinterpret_cast<OsCtrl*>(ws + L.os);
  auto* lb = reinterpret_cast<unsigned long long*>(ws + L.lb);
  auto* tk = reinterpret_cast<uint32_t*>(ws + L.tk);
  auto* tk_alt = reinterpret_cast<uint32_t*>(ws + L.tk_alt);
  auto* tv_alt = reinterpret_cast<uint32_t*>(ws + L.tv_alt);
  const long long* n_gauss = &ctrl->n_gauss;
  const long long* n_inst = &ctrl->n_eff;
  const size_t lb_pass_p = (size_t)L.nblk_p * kRadix, lb_pass_i = (size_t)L.nblk_i * kRadix;

  // the tile ranges and the passes' counters and look-back words, in one
  // kernel of the programmatic-launch chain
  static_assert(sizeof(OsCtrl) % 4 == 0, "cleared in 4-byte words");
  if (launch_zero(ranges, (size_t)num_tiles * 2 * sizeof(int32_t), os, (L.lb - L.os) + L.lb_bytes, st) != GS_OK)
    return GS_ERR_CUDA;
  {
    GS_TRACE("k_depth_keys", st);
    launch_pdl(k_depth_keys, L.nblk_p, kDkThreads, 0, st, P, depth, touched, dk, dv, ctrl, os);
  }
  // 1. depth sort: 4 passes, ending in (dk, dv)
  os_pass(dk, dv, dk2, dv2, n_gauss, 0, 0, L.nblk_p, os, lb, status, st);
  os_pass(dk2, dv2, dk, dv, n_gauss, 8, 1, L.nblk_p, os, lb + lb_pass_p, status, st);
  os_pass(dk, dv, dk2, dv2, n_gauss, 16, 2, L.nblk_p, os, lb + 2 * lb_pass_p, status, st);
  os_pass(dk2, dv2, dk, dv, n_gauss, 24, 3, L.nblk_p, os, lb + 3 * lb_pass_p, status, st);
  // 2. scan + emission in depth order
  {
    GS_TRACE("k_scan_partials", st);
    launch_pdl(k_scan_partials, L.nscan, 256, 0, st, P, dv, touched, partial);
  }
  {
    GS_TRACE("k_scan_top", st);
    launch_pdl(k_scan_top, 1, 1024, 0, st, L.nscan, partial, capacity, ctrl, reinterpret_cast<long long*>(n_out), status);
  }
  // 3. tile sort: passes ping-pong so that the last one lands in (tk, gids)
  const int npass = L.npass_t;
  uint32_t* kb[2];
  uint32_t* vb[2];
  if (npass % 2 == 0) {
    kb[0] = tk; vb[0] = gids; kb[1] = tk_alt; vb[1] = tv_alt;
  } else {
    kb[0] = tk_alt; vb[0] = tv_alt; kb[1] = tk; vb[1] = gids;
  }
  {
    GS_TRACE("k_emit", st);
    launch_pdl(k_emit, L.nscan, kEmitThreads, 0, st, P, dv, touched, reinterpret_cast<const int4*>(rect), partial, cam.tiles_x,
                                    capacity, npass, kb[0], vb[0], os);
  }
  unsigned long long* lb_t = lb + kDepthPasses * lb_pass_p;
  for (int p = 0; p < npass; ++p)
    os_pass(kb[p & 1], vb[p & 1], kb[(p + 1) & 1], vb[(p + 1) & 1], n_inst, 8 * p, kDepthPasses + p, L.nblk_i, os,
            lb_t + p * lb_pass_i, status, st);
  {
    GS_TRACE("k_tile_ranges", st);
    int nb = (int)((capacity + 255) / 256);
    if (nb > 8 * 152) nb = 8 * 152;  // one wave; the kernel strides over the instances
    if (nb < 1) nb = 1;
    launch_pdl(k_tile_ranges, nb, 256, 0, st, tk, gids, depth, ctrl, os, P, num_tiles, reinterpret_cast<int2*>(ranges),
               keys64);
  }
  return last_launch_status();
}

// ---------------------------------------------------------------------------
// Launch order of the compositing kernels' tile blocks: tiles by descending
// list length, as a counting sort over buckets of 8 instances in one block
// (a histogram in shared memory, a block scan, then a scatter through one
// cursor per bucket, whose order within a bucket follows the atomics).
namespace {
constexpr int kToThreads = 1024;
constexpr int kToBuckets = 1024;  // one per thread
constexpr int kToShift = 3;       // 8 instances per bucket
static_assert(kToBuckets == kToThreads, "one bucket per thread in the scan");

__device__ __forceinline__ int tile_bucket(int2 r) {
  return (kToBuckets - 1) - min((r.y - r.x) >> kToShift, kToBuckets - 1);
}

__global__ void __launch_bounds__(kToThreads) k_tile_order(const int2* __restrict__ ranges, int T,
                                                          int32_t* __restrict__ order) {
  pdl_wait();
  pdl_trigger();
  __shared__ int s_h[kToBuckets];
  __shared__ int s_w[kToThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  s_h[threadIdx.x] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += kToThreads) atomicAdd(&s_h[tile_bucket(ranges[t])], 1);
  __syncthreads();
  // exclusive scan of the bucket counts: warps, then the warp totals
  const int v = s_h[threadIdx.x];
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int w = s_w[lane];
    int xw = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, xw, o);
      if (lane >= o) xw += y;
    }
    s_w[lane] = xw - w;
  }
  __syncthreads();
  s_h[threadIdx.x] = s_w[wid] + x - v;
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += kToThreads) order[atomicAdd(&s_h[tile_bucket(ranges[t])], 1)] = t;
}
}  // namespace

gs_status launch_tile_order(int T, const int32_t* ranges, int32_t* order, cudaStream_t st) {
  GS_TRACE("k_tile_order", st);
  launch_pdl(k_tile_order, 1, kToThreads, 0, st, reinterpret_cast<const int2*>(ranges), T, order);
  return last_launch_status();
}

}  // namespace gsff
