// Tile x depth binning and sorting (Sec. 3.1: projected Gaussians are sorted
// front-to-back per 16x16 tile).
//
// The result equals a sort of all (tile, Gaussian) instances by the 64-bit key
// (tile << 32 | depth bits) with ties in ascending Gaussian id. It is computed
// per tile, with no global sort:
//   1. k_bin_count: every instance adds one to its tile's count; then
//      k_bin_ranges (one block) turns the counts into the tile ranges (an
//      exclusive scan), the instance total I and the capacity check;
//   2. k_bin_scatter: every instance takes a free slot of its tile (an atomic
//      count-down of the tile's count) and writes (depth bits << 32 | g) there;
//      the order of the slots inside a tile is arbitrary;
//   3. k_bin_tile_sort: one block per tile sorts the tile's keys ascending.
//      (depth bits, g) is unique inside a tile, so the sorted order, and with
//      it the result, does not depend on the slot order of step 2. Lists of up
//      to 2048 keys are sorted by a bitonic network held in registers
//      (partners less than 32 apart through warp shuffles, 32..255 apart
//      through shared memory, further apart inside a thread); longer lists
//      are cut into 2048-key runs sorted that way and then merged pairwise in
//      global memory (merge path) until one run remains.
// Steps 1 and 2 share each block's 512 Gaussians' instances evenly over its
// threads (a block scan of the tile counts, then each thread finds its
// instance's Gaussian by a binary search over the scan in shared memory). The
// sort has no wait on other blocks. Every kernel reads its item counts from device memory, so one frame
// is enqueued without a host round trip.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kBinThreads = 512;    // threads of steps 1 and 2 (one Gaussian each)
constexpr int kTsThreads = 256;     // threads of a tile-sort block
constexpr int kTsMaxE = 8;          // keys per thread of the register sort
constexpr int kTsRun = kTsThreads * kTsMaxE;  // 2048: the longest list sorted in one piece
constexpr unsigned long long kPadKey = ~0ull;  // sorts after every real key (depth bits < 0x7f800000)
constexpr int kRgThreads = 1024;    // threads of the one-block range scan

// The block's Gaussians [g0, g0 + 512) in shared memory: their exclusive
// instance offsets, rectangles and 64-bit keys (depth bits << 32 | g).
struct BinStage {
  int off[kBinThreads + 1];
  int4 rc[kBinThreads];
  unsigned long long key[kBinThreads];
  long long warp[kBinThreads / 32];
};

// Stages the block's Gaussians and returns its instance count. With KEYS the
// Gaussians' depths are read for the keys.
template <bool KEYS>
__device__ __forceinline__ int stage_gaussians(long long g0, int P, const int* __restrict__ touched,
                                               const int4* __restrict__ rect, const float* __restrict__ depth,
                                               BinStage& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long g = g0 + threadIdx.x;
  const int n = g < P ? max(touched[g], 0) : 0;
  if (n > 0) {
    S.rc[threadIdx.x] = rect[g];
    if (KEYS) S.key[threadIdx.x] = ((unsigned long long)__float_as_uint(depth[g]) << 32) | (unsigned long long)g;
  }
  int x = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) S.warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < kBinThreads / 32 ? S.warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kBinThreads / 32) S.warp[lane] = w;
  }
  __syncthreads();
  const int ex = (wid > 0 ? (int)S.warp[wid - 1] : 0) + x - n;
  S.off[threadIdx.x] = ex;
  if (threadIdx.x == kBinThreads - 1) S.off[kBinThreads] = ex + n;
  __syncthreads();
  return S.off[kBinThreads];
}

// The tile and Gaussian slot k of the block's instance i: k is the last slot
// with off[k] <= i (slots without instances share the next slot's offset and
// lose to it). False for a tile outside the grid.
__device__ __forceinline__ bool locate(const BinStage& S, int i, int tiles_x, int num_tiles, int& t, int& k) {
  k = 0;
#pragma unroll
  for (int step = kBinThreads / 2; step > 0; step >>= 1)
    if (S.off[k + step] <= i) k += step;
  const int4 rc = S.rc[k];
  const int li = i - S.off[k];
  const int rw = max(rc.z - rc.x, 1);
  t = (rc.y + li / rw) * tiles_x + rc.x + li % rw;
  return (unsigned)t < (unsigned)num_tiles;
}

// Instances per thread and round in steps 1 and 2: their searches and memory
// operations are independent, so four are in flight at a time.
constexpr int kBinIlp = 4;

// ---- step 1: counts, then the ranges ---------------------------------------------
__global__ void __launch_bounds__(kBinThreads) k_bin_count(int P, const int* __restrict__ touched,
                                                           const int4* __restrict__ rect, int tiles_x, int num_tiles,
                                                           unsigned int* __restrict__ cnt) {
  pdl_wait();
  pdl_trigger();
  __shared__ BinStage S;
  const int total = stage_gaussians<false>((long long)blockIdx.x * kBinThreads, P, touched, rect, nullptr, S);
  for (int i0 = threadIdx.x; i0 < total; i0 += kBinIlp * kBinThreads) {
    int t[kBinIlp], k[kBinIlp];
    bool v[kBinIlp];
#pragma unroll
    for (int u = 0; u < kBinIlp; ++u) {
      const int i = i0 + u * kBinThreads;
      v[u] = i < total && locate(S, i, tiles_x, num_tiles, t[u], k[u]);
    }
#pragma unroll
    for (int u = 0; u < kBinIlp; ++u)
      if (v[u]) atomicAdd(&cnt[t[u]], 1u);
  }
}

// One block: each thread a contiguous run of tiles (its sum, a block scan,
// then the ranges); empty tiles and tiles past the capacity keep (0, 0) and a
// tile across the capacity is cut to it.
__global__ void __launch_bounds__(kRgThreads) k_bin_ranges(int num_tiles, long long capacity,
                                                           const unsigned int* __restrict__ cnt,
                                                           int2* __restrict__ ranges, long long* __restrict__ n_out,
                                                           int32_t* __restrict__ status) {
  pdl_wait();
  pdl_trigger();
  __shared__ long long s_warp[32];
  const int per = (num_tiles + kRgThreads - 1) / kRgThreads;
  const int t0 = min((int)threadIdx.x * per, num_tiles), t1 = min(t0 + per, num_tiles);
  long long sum = 0;
  for (int t = t0; t < t1; t += 8) {
    unsigned int c[8];  // eight loads in flight at a time
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = t + u < t1 ? cnt[t + u] : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += c[u];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  long long run = (wid > 0 ? s_warp[wid - 1] : 0) + x - sum;
  for (int t = t0; t < t1; t += 8) {
    unsigned int c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = t + u < t1 ? cnt[t + u] : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (c[u] > 0 && run < capacity) ranges[t + u] = make_int2((int)run, (int)min(run + (long long)c[u], capacity));
      run += c[u];
    }
  }
  if (threadIdx.x == kRgThreads - 1) {
    if (n_out) *n_out = run;
    if (run > capacity) flag_status(status, GS_ERR_CAPACITY);
  }
}

// ---- step 2: the keys into their tiles' slots -------------------------------------
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(int P, const int* __restrict__ touched,
                                                             const int4* __restrict__ rect,
                                                             const float* __restrict__ depth, int tiles_x,
                                                             int num_tiles, const int2* __restrict__ ranges,
                                                             unsigned int* __restrict__ cnt,
                                                             unsigned long long* __restrict__ keys) {
  pdl_wait();
  pdl_trigger();
  __shared__ BinStage S;
  const int total = stage_gaussians<true>((long long)blockIdx.x * kBinThreads, P, touched, rect, depth, S);
  for (int i0 = threadIdx.x; i0 < total; i0 += kBinIlp * kBinThreads) {
    int t[kBinIlp], k[kBinIlp];
    bool v[kBinIlp];
#pragma unroll
    for (int u = 0; u < kBinIlp; ++u) {
      const int i = i0 + u * kBinThreads;
      v[u] = i < total && locate(S, i, tiles_x, num_tiles, t[u], k[u]);
    }
    int2 r[kBinIlp];
    int slot[kBinIlp];
#pragma unroll
    for (int u = 0; u < kBinIlp; ++u)
      if (v[u]) {
        r[u] = ranges[t[u]];
        slot[u] = (int)atomicSub(&cnt[t[u]], 1u) - 1;
      }
#pragma unroll
    for (int u = 0; u < kBinIlp; ++u)
      if (v[u] && slot[u] < r[u].y - r[u].x) keys[r[u].x + slot[u]] = S.key[k[u]];
  }
}

// ---- step 3: per-tile sort --------------------------------------------------------
// One compare-exchange stage between the thread's own elements e and e + JE
// (partners 256 JE apart).
template <int E, int JE>
__device__ __forceinline__ void stage_in_thread(unsigned long long (&r)[E], int k) {
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (e & JE) continue;
    const bool asc = (((e * kTsThreads + (int)threadIdx.x) & k) == 0);
    const unsigned long long a = r[e], b = r[e + JE];
    const bool swap = (b < a) == asc;
    r[e] = swap ? b : a;
    r[e + JE] = swap ? a : b;
  }
}

// Bitonic sort, ascending, of the block's 256 E keys: thread t holds element
// e * 256 + t in r[e]. For a stage (k, j), element i meets partner i ^ j and
// keeps the smaller key if (i & j) == 0 equals (i & k) == 0, else the larger.
// s: shared scratch of 256 E keys. UNROLL unrolls the stage loops (for
// E <= 2; a fully unrolled network of E = 8 needs over 200 registers).
template <int E, bool UNROLL>
__device__ __forceinline__ void bitonic_regs(unsigned long long (&r)[E], unsigned long long* s) {
  constexpr int LOG_M = 8 + (E == 1 ? 0 : E == 2 ? 1 : E == 4 ? 2 : 3);
  const int t = threadIdx.x;
#pragma unroll(UNROLL ? LOG_M : 1)
  for (int lk = 1; lk <= LOG_M; ++lk) {
    const int k = 1 << lk;
#pragma unroll(UNROLL ? LOG_M : 1)
    for (int lj = lk - 1; lj >= 0; --lj) {
      const int j = 1 << lj;
      if (j >= kTsThreads) {
        if (E >= 2 && j == kTsThreads) stage_in_thread<E, 1>(r, k);
        else if (E >= 4 && j == 2 * kTsThreads) stage_in_thread<E, (E >= 4 ? 2 : 1)>(r, k);
        else if (E >= 8) stage_in_thread<E, (E >= 8 ? 4 : 1)>(r, k);
      } else if (j >= 32) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) s[e * kTsThreads + t] = r[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const unsigned long long o = s[e * kTsThreads + (t ^ j)];
          const int i = e * kTsThreads + t;
          // keep the smaller key iff (i & j) == 0 equals (i & k) == 0
          const bool take = (o < r[e]) == (((i & j) == 0) == ((i & k) == 0));
          r[e] = take ? o : r[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, r[e], j);
          const int i = e * kTsThreads + t;
          const bool take = (o < r[e]) == (((i & j) == 0) == ((i & k) == 0));
          r[e] = take ? o : r[e];
        }
      }
    }
  }
}

// Where a tile's sorted keys go: its ids (and 64-bit keys) from list
// position `at` on, or, for a run of a long list, back into the key buffer.
struct TileOut {
  uint32_t* gids;
  unsigned long long* keys64;
  unsigned long long tile_hi;  // tile << 32
  long long at;
  __device__ __forceinline__ void put(int i, unsigned long long k) const {
    gids[at + i] = (uint32_t)k;
    if (keys64) keys64[at + i] = tile_hi | (k >> 32);
  }
};

// Sorts src[0, n), n <= 256 E: to o (FINAL) or back into src.
template <int E, bool FINAL>
__device__ __forceinline__ void sort_piece(unsigned long long* src, int n, const TileOut& o, unsigned long long* s) {
  unsigned long long r[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * kTsThreads + threadIdx.x;
    r[e] = i < n ? src[i] : kPadKey;
  }
  bitonic_regs<E, (E <= 2)>(r, s);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * kTsThreads + threadIdx.x;
    if (i < n) {
      if (FINAL) o.put(i, r[e]);
      else src[i] = r[e];
    }
  }
}

// Merges the sorted runs a[0, la) and b[0, lb) into out[0, la + lb); each
// thread writes one contiguous share, located by a binary search on its
// first output's diagonal (keys are distinct).
__device__ void merge_pair(const unsigned long long* a, int la, const unsigned long long* b, int lb,
                           unsigned long long* out) {
  const int total = la + lb;
  const int per = (total + kTsThreads - 1) / kTsThreads;
  const int d0 = min((int)threadIdx.x * per, total), d1 = min(d0 + per, total);
  int lo = max(0, d0 - lb), hi = min(d0, la);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < b[d0 - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  int i = lo, j = d0 - lo;
  for (int d = d0; d < d1; ++d) {
    const bool take_a = j >= lb || (i < la && a[i] < b[j]);
    out[d] = take_a ? a[i++] : b[j++];
  }
}

__global__ void __launch_bounds__(kTsThreads, 5) k_bin_tile_sort(const int2* __restrict__ ranges,
                                                              unsigned long long* __restrict__ keys,
                                                              unsigned long long* __restrict__ alt,
                                                              uint32_t* __restrict__ gids,
                                                              unsigned long long* __restrict__ keys64) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned long long s[kTsRun];
  const int t = blockIdx.x;
  const int2 r = ranges[t];
  const int n = r.y - r.x;
  if (n <= 0) return;
  const TileOut o{gids, keys64, (unsigned long long)t << 32, r.x};
  unsigned long long* src = keys + r.x;
  if (n <= kTsThreads) return sort_piece<1, true>(src, n, o, s);
  if (n <= 2 * kTsThreads) return sort_piece<2, true>(src, n, o, s);
  if (n <= 4 * kTsThreads) return sort_piece<4, true>(src, n, o, s);
  if (n <= kTsRun) return sort_piece<kTsMaxE, true>(src, n, o, s);
  // a long list: sorted runs, then pairwise merges (ping-pong with alt)
  for (int c = 0; c < n; c += kTsRun) {
    sort_piece<kTsMaxE, false>(src + c, min(kTsRun, n - c), o, s);
    __syncthreads();  // s is reused by the next run
  }
  unsigned long long* dst = alt + r.x;
  for (int len = kTsRun; len < n; len *= 2) {
    __syncthreads();  // the previous round's writes are visible to the block
    for (int c = 0; c < n; c += 2 * len) {
      const int la = min(len, n - c), lb = min(len, n - c - la);
      merge_pair(src + c, la, src + c + la, lb, dst + c);
    }
    unsigned long long* tmp = src;
    src = dst;
    dst = tmp;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kTsThreads) o.put(i, src[i]);
}

struct SortLayout {
  size_t keys, alt, cnt, total;
};

SortLayout sort_layout(long long capacity, int num_tiles) {
  SortLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.keys = take((size_t)capacity * 8);
  L.alt = take((size_t)capacity * 8);
  L.cnt = take((size_t)num_tiles * 4);
  L.total = o;
  return L;
}

}  // namespace

size_t bin_sort_workspace_bytes(int P, long long capacity, int num_tiles) {
  (void)P;
  return sort_layout(capacity, num_tiles).total;
}

// Enqueues the whole binning on `st`. The workspace base must be 256-aligned.
// keys64 may be null (the 64-bit keys are then not written).
gs_status launch_bin_sort(const CamF& cam, int P, const float* depth, const int32_t* rect, const int32_t* touched,
                          long long capacity, void* workspace, unsigned long long* keys64, uint32_t* gids,
                          int32_t* ranges, int64_t* n_out, int32_t* status, cudaStream_t st) {
  const int num_tiles = cam.tiles_x * cam.tiles_y;
  const SortLayout L = sort_layout(capacity, num_tiles);
  char* ws = static_cast<char*>(workspace);
  auto* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  auto* alt = reinterpret_cast<unsigned long long*>(ws + L.alt);
  auto* cnt = reinterpret_cast<unsigned int*>(ws + L.cnt);
  auto* rg = reinterpret_cast<int2*>(ranges);
  const auto* rc = reinterpret_cast<const int4*>(rect);
  // the tile ranges and the counts, in one kernel of the programmatic-launch chain
  if (launch_zero(ranges, (size_t)num_tiles * 2 * sizeof(int32_t), cnt, (size_t)num_tiles * 4, st) != GS_OK)
    return GS_ERR_CUDA;
  const long long nbl = ((long long)P + kBinThreads - 1) / kBinThreads;
  const unsigned nb = (unsigned)(nbl > 0 ? nbl : 1);
  {
    GS_TRACE("k_bin_count", st);
    launch_pdl(k_bin_count, nb, kBinThreads, 0, st, P, touched, rc, cam.tiles_x, num_tiles, cnt);
  }
  {
    GS_TRACE("k_bin_ranges", st);
    launch_pdl(k_bin_ranges, 1u, kRgThreads, 0, st, num_tiles, capacity, (const unsigned int*)cnt, rg,
               reinterpret_cast<long long*>(n_out), status);
  }
  {
    GS_TRACE("k_bin_scatter", st);
    launch_pdl(k_bin_scatter, nb, kBinThreads, 0, st, P, touched, rc, depth, cam.tiles_x, num_tiles,
               (const int2*)rg, cnt, keys);
  }
  {
    GS_TRACE("k_bin_tile_sort", st);
    launch_pdl(k_bin_tile_sort, (unsigned)num_tiles, kTsThreads, 0, st, (const int2*)rg, keys, alt, gids, keys64);
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
