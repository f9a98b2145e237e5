// Tensor-core (tcgen05) form of the feature channels of Eq. 3.
//
// Per half tile (16 x 8 = 128 pixels, the M = 128 rows of a tcgen05 tile)
// the N feature channels are a dense contraction over the tile's
// depth-sorted list:
//     F[p, :] = sum_k w[p, k] f[g_k, :],   w[p, k] = alpha_k(p) T_k(p)
// (w = 0 where pixel p skips or has stopped). Below a pixel's last index
// (from the SIMT forward) no pixel has stopped, so T_k is the product of
// (1 - alpha_j) over the blended j < k. A Gaussian whose footprint does not
// reach the half tile (the SIMT forward's per-instance skip mask) has w = 0
// at all its pixels and is left out of the contraction. The weights are
// rounded to bf16 (A operand, K-major), the features are bf16 (B operand,
// channels contiguous), and the products accumulate in fp32 in tensor
// memory. The forward kernel is persistent and warp-specialised (its
// comment below has the roles); RGB, depth, alpha, T_final and last_idx come
// from the SIMT forward launched before it.
//
// Shared-memory operand layouts (no swizzle; 16-byte core-matrix rows):
//   A: element (m, k) at (m/8)*512 + (k/8)*128 + (m%8)*16 + (k%8)*2
//      descriptor LBO = 128 (K direction), SBO = 512 (M direction)
//   B: element (k, n) at (n/8)*128 + (k/8)*SK + (k%8)*16 + (n%8)*2, SK = N*16
//      descriptor LBO = SK (K direction), SBO = 128 (N direction)
// Every wait is bounded (1 s of %globaltimer); a timeout flags
// GS_ERR_TIMEOUT, waits (bounded) for the tensor core, frees tensor memory
// and returns.

#include <atomic>

#include "tc_util.cuh"

namespace gsff {
namespace {

constexpr int kTcPix = 128;      // pixels per half tile = MMA M
constexpr int kTcMaxN = 512;
// ---------------------------------------------------------------------------
// Forward of the feature channels (persistent, warp-specialised).
//
// One CTA per SM walks a fixed list of half tiles (128 pixels each; the
// tiles in the launch order, half tiles dealt to the CTAs round by round,
// alternating direction). The whole N-channel accumulator of a half tile
// lives in tensor memory (128 lanes x N fp32 columns). Roles:
//   warp 0 (producer): per half tile, the largest last index of its pixels
//     bounds the list; the list is compacted to the Gaussians whose skip
//     mask (from the SIMT forward) reaches the half tile, which are the only
//     ones with a nonzero weight there (ids and masks read 128 positions at
//     a time, one batch ahead; the next half tile's range and last indices
//     one half tile ahead); every 32 entries fill one stage of a 4-deep
//     ring: the records (uv, conic and opacity) by cp.async and the id list;
//   warps 22-29 (loaders): the stage's bf16 feature rows (B operand,
//     channels contiguous) by 16-byte cp.async, each instruction whole core
//     matrices (4 chunks of 8 rows); the stage's "full" barrier completes
//     when every copy has landed;
//   warps 6-21 (weight builders, 4 threads per pixel, 8 entries each):
//     alpha of each entry (exact skip test; 0 at or past the pixel's last
//     index), w = alpha T with T the product of (1 - alpha) over the entries
//     in front (a width-4 shuffle scan joins the quarters), rounded to bf16
//     into the A operand (K-major), then the stage's "weights ready" barrier;
//   warp 1 (one thread): per stage, tcgen05.mma M=128, N<=256 per
//     instruction, K=16 x 2, accumulating in tensor memory; commits free the
//     stage, and after the last stage of a half tile signal the epilogue. The
//     first stage of a half tile waits for the epilogue to have read the
//     previous accumulator, channel half by channel half;
//   warps 2-5 (epilogue; warp w reads tensor-memory lanes 32 (w % 4)..):
//     32 columns at a time into registers, into a 4 KB box of shared memory
//     in the 128-byte swizzled order, then one TMA tensor store of the box
//     (32 channels x 16 pixels x 2 rows of the HWC map; the tensor map clips
//     the image edge) with an L2 evict-first hint (the map is not read again
//     here; the feature rows that later half tiles reuse stay in L2); two
//     boxes per warp alternate. Each channel half of
//     tensor memory is released as soon as every warp has read it.
// Every wait is bounded (1 s of %globaltimer): a role that gives up flags
// GS_ERR_TIMEOUT and raises the CTA's abort word, on which every other wait
// returns, and the CTA drains its copies and tensor-core work before it frees
// tensor memory.
constexpr int kFwThreads = 960;
constexpr int kFwStages = 4;
constexpr int kFwK = 32;
constexpr int kFwWarpMma = 1, kFwWarpEpi = 2, kFwWarpBuild = 6, kFwWarpLoad = 22, kFwLoaders = 8;
constexpr int kFwBuilders = kFwWarpLoad - kFwWarpBuild;  // 16 warps: 4 threads per pixel

struct alignas(1024) FwStage {
  uint8_t A[kTcPix * kFwK * 2];   // 8 KB: element (m, k) at (m/8)*512 + (k/8)*128 + (m%8)*16 + (k%8)*2
  uint8_t B[kFwK * kTcMaxN * 2];  // 32 KB: element (k, n) at (n/8)*128 + (k/8)*(16 N) + (k%8)*16 + (n%8)*2
  float2 uv[kFwK];                // entry k at slot (k % 8) * 4 + k / 8
  float4 co[kFwK];                // conic and opacity
  int pos[kFwK];                  // list position (from the tile's start); INT_MAX past the stage's entries
  uint32_t gid[kFwK];             // Gaussian of entry k (0 past the stage's entries)
  int nvalid, flags;              // flags: 1 first stage of its half tile, 2 last
};
static_assert(sizeof(FwStage) % 1024 == 0, "stages keep 1024-byte alignment");

struct FwSmem {
  FwStage st[kFwStages];
  uint8_t box[4][2][4096];  // epilogue boxes (1024-aligned: 128-byte swizzle)
  uint32_t cgid[64];        // the producer's compaction queue
  int cpos[64];
  unsigned long long ids[kFwStages], full[kFwStages], ready[kFwStages], empty[kFwStages];
  unsigned long long acc_full, acc_empty[2], drain;
  uint32_t tmem;
  int abort;
};

static_assert(sizeof(FwSmem) + 1024 <= 227 * 1024, "shared memory of the forward");
static_assert(kFwWarpBuild * 32 + 4 * kTcPix == kFwWarpLoad * 32, "four builder threads per pixel");
static_assert((kFwWarpLoad + kFwLoaders) * 32 == kFwThreads && kFwK % kFwLoaders == 0, "loader warps");

struct FwParams {
  CamF cam;
  const int2* ranges;
  const int* order;  // launch order of the tiles, or null
  const uint32_t* gids;
  const uint8_t* masks;  // per instance: 8x8-block skip mask of the SIMT forward (bits 0,1: rows 0-7), or null
  const float2* uv;
  const float4* co;
  const __nv_bfloat16* feats;
  const int* last_idx;
  int N, tmem_cols, nhalf;
  int P;  // Gaussians (bound of the checked build's id checks)
  int hold;  // test hook: the producer issues nothing, so the other roles' waits run out
  int32_t* status;
};

__device__ __forceinline__ int fw_slot(int k) { return ((k & 7) << 2) | (k >> 3); }

// Half tile number r of this CTA's list (-1 past the end): round r deals
// half tiles [r G, r G + G) to the G CTAs, in alternating direction.
__device__ __forceinline__ int fw_half_tile(int r, int nhalf) {
  const int G = gridDim.x;
  const int b = (r & 1) ? (G - 1 - (int)blockIdx.x) : (int)blockIdx.x;
  const int h = r * G + b;
  return h < nhalf ? h : -1;
}

// Bounded wait for the phase of the given parity; false (and the abort word
// raised, GS_ERR_TIMEOUT flagged) after 1 s, false at once if another role
// has raised the abort word.
__device__ __forceinline__ bool fw_wait(uint32_t bar, uint32_t parity, volatile int* abort, int32_t* status) {
  const unsigned long long t0 = gtime();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort) return false;
    if (gtime() - t0 > kWaitNs) {
      *abort = 1;
      flag_status(status, GS_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tile_of(const FwParams& p, int h, int& tx, int& ty, int& half) {
  const int t = p.order ? p.order[h >> 1] : (h >> 1);
  tx = t % p.cam.tiles_x;
  ty = t / p.cam.tiles_x;
  half = h & 1;
}

// warp 0: compaction, records and the stages' id lists
__device__ void fw_producer(const FwParams& p, FwSmem& S) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  volatile int* abort = &S.abort;
  int s = 0;
  uint32_t ph = 0;  // parity of the ring's current round
  // the next half tile's range and its pixels' last indices are loaded one
  // half tile ahead, the ids and masks of the list one batch of 128 ahead
  auto fetch_meta = [&](int r, int2& rg, int (&li)[4], int& half) {
    const int h = fw_half_tile(r, p.nhalf);
    rg = make_int2(0, 0);
    half = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) li[i] = 0;
    if (h < 0) return;
    int tx, ty;
    tile_of(p, h, tx, ty, half);
    rg = p.ranges[ty * p.cam.tiles_x + tx];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = lane + 32 * i;
      const int px = tx * kTile + (m & 15), py = ty * kTile + half * 8 + (m >> 4);
      if (px < p.cam.W && py < p.cam.H) li[i] = p.last_idx[(size_t)py * p.cam.W + px];
    }
  };
  auto fetch_batch = [&](int2 rg, int maxlast, int base, uint32_t (&gb)[4], uint32_t (&mb)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int pos = base + 32 * i + lane;
      gb[i] = pos < maxlast ? checked_id(p.gids[rg.x + pos], p.P, p.status) : 0u;
      mb[i] = pos < maxlast ? (p.masks ? (uint32_t)p.masks[rg.x + pos] : 0xFu) : 0u;
    }
  };
  int2 nrg;
  int nli[4], nhalf_;
  fetch_meta(0, nrg, nli, nhalf_);
  for (int r = 0;; ++r) {
    if (fw_half_tile(r, p.nhalf) < 0) break;
    const int2 rg = nrg;
    const int half = nhalf_;
    int maxlast = max(max(nli[0], nli[1]), max(nli[2], nli[3]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxlast = max(maxlast, __shfl_xor_sync(0xffffffffu, maxlast, o));
    maxlast = checked_len(maxlast, rg.y - rg.x, p.status);
    fetch_meta(r + 1, nrg, nli, nhalf_);
    int fill = 0;
    bool first = true;
    // emits queue entries [0, n) as one stage: records by cp.async, then the
    // id list for the loader warps
    auto emit = [&](int n, bool last) -> bool {
      FwStage& st = S.st[s];
      if (!fw_wait(smem_u32(&S.empty[s]), ph ^ 1u, abort, p.status)) return false;
      const uint32_t g = lane < n ? S.cgid[lane] : 0u;
      const int slot = fw_slot(lane);
      cp_async8(smem_u32(&st.uv[slot]), p.uv + g, lane < n);
      cp_async16(smem_u32(&st.co[slot]), p.co + g, lane < n);
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.full[s])) : "memory");
      st.pos[slot] = lane < n ? S.cpos[lane] : 0x7fffffff;
      st.gid[lane] = g;
      if (lane == 0) {
        st.nvalid = n;
        st.flags = (first ? 1 : 0) | (last ? 2 : 0);
      }
      mbar_arrive(smem_u32(&S.full[s]));
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&S.ids[s]));
      first = false;
      if (++s == kFwStages) {
        s = 0;
        ph ^= 1u;
      }
      return true;
    };
    uint32_t gb[4], mb[4];
    if (maxlast > 0) fetch_batch(rg, maxlast, 0, gb, mb);
    for (int base = 0; base < maxlast; base += 128) {
      uint32_t gc[4], mc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        gc[i] = gb[i];
        mc[i] = mb[i];
      }
      if (base + 128 < maxlast) fetch_batch(rg, maxlast, base + 128, gb, mb);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int pos = base + 32 * i + lane;
        const bool hit = ((mc[i] >> (2 * half)) & 3u) != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int idx = fill + __popc(bal & lt);
          S.cgid[idx] = gc[i];
          S.cpos[idx] = pos;
        }
        fill += __popc(bal);
        __syncwarp();
        if (fill > 32) {
          // a full stage, and more entries follow
          if (!emit(32, false)) return;
          const bool mv = lane < fill - 32;
          const uint32_t mg = mv ? S.cgid[32 + lane] : 0u;
          const int mp = mv ? S.cpos[32 + lane] : 0;
          __syncwarp();
          if (mv) {
            S.cgid[lane] = mg;
            S.cpos[lane] = mp;
          }
          fill -= 32;
          __syncwarp();
        }
      }
    }
    // the last stage of the half tile (also the one stage of an empty half
    // tile, whose weights and rows are all zero)
    if (!emit(fill, true)) return;
  }
}

// warps 22-29: the bf16 feature rows of each stage (B operand) by 16-byte
// cp.async; warp L copies rows 8 (L / 2) .. 8 (L / 2) + 7 and half of their
// chunks, each instruction 4 chunks of 8 rows, which are whole 128-byte core
// matrices in shared memory (no bank conflicts); each lane's copies complete
// an arrival on the stage's "full" barrier
__device__ void fw_loader(const FwParams& p, FwSmem& S) {
  const int lane = threadIdx.x & 31, L = (threadIdx.x >> 5) - kFwWarpLoad;
  volatile int* abort = &S.abort;
  const int cpr = p.N / 8;  // 16-byte chunks per feature row
  const uint32_t SK = (uint32_t)p.N * 16;
  static_assert(kFwLoaders == 2 * (kFwK / 8), "two loader warps per group of 8 rows");
  const int k = 8 * (L >> 1) + (lane & 7);    // this lane's row
  const int c_begin = (L & 1) * (cpr / 2) + (lane >> 3), c_end = (L & 1) ? cpr : cpr / 2;
  int s = 0;
  uint32_t ph = 0;
  for (int r = 0;; ++r) {
    if (fw_half_tile(r, p.nhalf) < 0) break;
    while (true) {
      if (!fw_wait(smem_u32(&S.ids[s]), ph, abort, p.status)) return;
      FwStage& st = S.st[s];
      const int n = st.nvalid, flags = st.flags;
      const bool valid = k < n;
      const __nv_bfloat16* row = p.feats + (size_t)st.gid[k] * p.N;
      const uint32_t dk = smem_u32(st.B) + (uint32_t)(k >> 3) * SK + (uint32_t)(k & 7) * 16u;
      for (int c = c_begin; c < c_end; c += 4) cp_async16(dk + (uint32_t)c * 128u, row + 8 * c, valid);
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.full[s])) : "memory");
      if (++s == kFwStages) {
        s = 0;
        ph ^= 1u;
      }
      if (flags & 2) break;
    }
  }
}

// warps 6-21: weights, four threads per pixel (entries 8 q .. 8 q + 7 of each
// stage); T in front of a thread's entries is the product over the quarters
// before it (width-4 shuffle scan), so the four threads of a pixel carry the
// same T from stage to stage
__device__ void fw_builder(const FwParams& p, FwSmem& S) {
  const int b = threadIdx.x - kFwWarpBuild * 32;
  const int m = b >> 2, q = b & 3, lane = threadIdx.x & 31;
  volatile int* abort = &S.abort;
  int s = 0;
  uint32_t ph = 0;
  for (int r = 0;; ++r) {
    const int h = fw_half_tile(r, p.nhalf);
    if (h < 0) break;
    int tx, ty, half;
    tile_of(p, h, tx, ty, half);
    const int px = tx * kTile + (m & 15), py = ty * kTile + half * 8 + (m >> 4);
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const int last = (px < p.cam.W && py < p.cam.H) ? p.last_idx[(size_t)py * p.cam.W + px] : 0;
    float T = 1.f;
    while (true) {
      if (!fw_wait(smem_u32(&S.full[s]), ph, abort, p.status)) return;
      FwStage& st = S.st[s];
      float a[8];
      float prod = 1.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int sl = 4 * j + q;  // slot of entry 8 q + j
        a[j] = 0.f;
        PairAlpha pa;
        if (st.pos[sl] < last && pair_alpha(st.co[sl], st.uv[sl].x - pxc, st.uv[sl].y - pyc, pa)) {
          a[j] = pa.alpha;
          prod = __fmul_rn(prod, __fsub_rn(1.f, pa.alpha));
        }
      }
      // exclusive product over the quarters before mine (lanes 4m .. 4m+3)
      float incl = prod;
      float y = __shfl_up_sync(0xffffffffu, incl, 1, 4);
      if (q >= 1) incl = __fmul_rn(incl, y);
      y = __shfl_up_sync(0xffffffffu, incl, 2, 4);
      if (q >= 2) incl = __fmul_rn(incl, y);
      float excl = __shfl_up_sync(0xffffffffu, incl, 1, 4);
      if (q == 0) excl = 1.f;
      const float total = __shfl_sync(0xffffffffu, incl, 3, 4);
      float Tj = __fmul_rn(T, excl);
      uint32_t packed[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const float w0 = __fmul_rn(a[j], Tj);
        if (a[j] > 0.f) Tj = __fmul_rn(Tj, __fsub_rn(1.f, a[j]));
        const float w1 = __fmul_rn(a[j + 1], Tj);
        if (a[j + 1] > 0.f) Tj = __fmul_rn(Tj, __fsub_rn(1.f, a[j + 1]));
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(w0, w1);
        packed[j / 2] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      T = __fmul_rn(T, total);
      *reinterpret_cast<uint4*>(st.A + (m >> 3) * 512 + q * 128 + (m & 7) * 16) =
          make_uint4(packed[0], packed[1], packed[2], packed[3]);
      const int flags = st.flags;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&S.ready[s]));
      if (++s == kFwStages) {
        s = 0;
        ph ^= 1u;
      }
      if (flags & 2) break;
    }
  }
}

// warp 1, one thread: the tensor-core products
__device__ void fw_mma(const FwParams& p, FwSmem& S, uint32_t tmem) {
  volatile int* abort = &S.abort;
  const uint32_t SK = (uint32_t)p.N * 16;
  int s = 0;
  uint32_t ph = 0;
  for (int r = 0;; ++r) {
    if (fw_half_tile(r, p.nhalf) < 0) break;
    const uint32_t acc_par = ((uint32_t)r & 1u) ^ 1u;  // the epilogue's release of the previous accumulator
    while (true) {
      if (!fw_wait(smem_u32(&S.full[s]), ph, abort, p.status)) return;
      if (!fw_wait(smem_u32(&S.ready[s]), ph, abort, p.status)) return;
      FwStage& st = S.st[s];
      const int flags = st.flags;
      const bool first = flags & 1;
      const uint32_t a0 = smem_u32(st.A), b0 = smem_u32(st.B);
      for (int n0 = 0, hb = 0; n0 < p.N; n0 += 256, ++hb) {
        if (first && !fw_wait(smem_u32(&S.acc_empty[hb]), acc_par, abort, p.status)) return;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int nn = min(256, p.N - n0);
        const uint32_t idesc = idesc_bf16(kTcPix, nn, 1);
#pragma unroll
        for (int k16 = 0; k16 < kFwK / 16; ++k16) {
          const uint64_t ad = smem_desc(a0 + (uint32_t)k16 * 256u, 128, 512);
          const uint64_t bd = smem_desc(b0 + (uint32_t)(n0 / 8) * 128u + (uint32_t)k16 * 2u * SK, SK, 128);
          const uint32_t acc = (!first || k16 > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)n0),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.empty[s])));
      if (flags & 2)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&S.acc_full)));
      if (++s == kFwStages) {
        s = 0;
        ph ^= 1u;
      }
      if (flags & 2) break;
    }
  }
}

// warps 2-5: tensor memory -> swizzled boxes -> TMA tensor stores
__device__ void fw_epilogue(const FwParams& p, FwSmem& S, uint32_t tmem, const CUtensorMap* omap) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qd = warp & 3;  // tensor-memory lanes 32 qd .. 32 qd + 31 = pixel rows 2 qd, 2 qd + 1 of the half tile
  volatile int* abort = &S.abort;
  const int nbox = p.N / 32;
  const int half0 = min(p.N, 256) / 32;  // boxes of the first channel half
  int used = 0;  // boxes this warp has stored so far
  for (int r = 0;; ++r) {
    const int h = fw_half_tile(r, p.nhalf);
    if (h < 0) break;
    int tx, ty, half;
    tile_of(p, h, tx, ty, half);
    if (!fw_wait(smem_u32(&S.acc_full), (uint32_t)r & 1u, abort, p.status)) return;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int x0 = tx * kTile, y0 = ty * kTile + half * 8 + 2 * qd;
    for (int c = 0; c < nbox; ++c, ++used) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(32 * c), v);
      if (c + 1 == half0 || c + 1 == nbox) {
        // this warp has read every column of the channel half: release it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&S.acc_empty[c + 1 == half0 ? 0 : 1]));
      }
      uint8_t* box = S.box[qd][used & 1];
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");  // the box's last store has read it
      __syncwarp();
#pragma unroll
      for (int ch = 0; ch < 8; ++ch)
        *reinterpret_cast<float4*>(box + lane * 128 + ((ch ^ (lane & 7)) << 4)) =
            make_float4(v[4 * ch], v[4 * ch + 1], v[4 * ch + 2], v[4 * ch + 3]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        asm volatile(
            "{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
            "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3, %4}], [%1], pol;"
            "\n\t}\n" ::"l"(omap),
            "r"(smem_u32(box)), "r"(32 * c), "r"(x0), "r"(y0)
            : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
  }
}

__global__ void __launch_bounds__(kFwThreads, 1) k_render_feat_tc(const FwParams p,
                                                                  const __grid_constant__ CUtensorMap omap) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
  FwSmem& S = *reinterpret_cast<FwSmem*>(smem_raw + pad);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_wait();
  pdl_trigger();
  if (tid == 0) {
    for (int s = 0; s < kFwStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.ids[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.full[s])), "r"(64 + 32 * kFwLoaders));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.ready[s])), "r"(kFwBuilders));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.acc_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&S.acc_empty[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&S.acc_empty[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.drain)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    S.abort = 0;
  }
  if (warp == kFwWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(p.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = S.tmem;

  if (warp == 0) {
    if (!p.hold) fw_producer(p, S);
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == kFwWarpMma) {
    if (lane == 0) {
      fw_mma(p, S, tmem);
      // every product issued has completed before tensor memory is freed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.drain)));
      volatile int never = 0;
      fw_wait(smem_u32(&S.drain), 0u, &never, p.status);
    }
  } else if (warp >= kFwWarpEpi && warp < kFwWarpBuild) {
    fw_epilogue(p, S, tmem, &omap);
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  } else if (warp < kFwWarpLoad) {
    fw_builder(p, S);
  } else {
    fw_loader(p, S);
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == kFwWarpMma) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
  }
}

std::atomic<int> g_tc_hold{0};

}  // namespace

void set_tc_test_hold(int on) { g_tc_hold.store(on ? 1 : 0); }

gs_status launch_render_fwd_tc(const CamF& cam, int P, const int32_t* ranges, const int32_t* order,
                               const uint32_t* gids, const uint8_t* masks, const float* uv, const float* co,
                               const __nv_bfloat16* feats, const int32_t* last_idx, int N, float* out_feat,
                               int32_t* status, cudaStream_t st) {
  if (N <= 0 || N % 64 != 0 || N > kTcMaxN) return GS_ERR_UNSUPPORTED;
  FwParams p;
  p.P = P;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.gids = gids;
  p.masks = masks;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.feats = feats;
  p.last_idx = last_idx;
  p.N = N;
  int cols = 32;
  while (cols < N) cols *= 2;
  p.tmem_cols = cols;
  p.nhalf = 2 * cam.tiles_x * cam.tiles_y;
  p.hold = g_tc_hold.load();
  p.status = status;
  // the HWC feature map as a 3D tensor (channels, x, y) for the epilogue's
  // TMA stores of 32 x 16 x 2 boxes with 128-byte swizzle
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return GS_ERR_CUDA;
  CUtensorMap omap;
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)cam.W, (cuuint64_t)cam.H};
  const cuuint64_t strides[2] = {(cuuint64_t)N * sizeof(float), (cuuint64_t)cam.W * N * sizeof(float)};
  const cuuint32_t boxdim[3] = {32, 16, 2};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode(&omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, out_feat, dims, strides, boxdim, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GS_ERR_CUDA;
  const size_t smem = sizeof(FwSmem) + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_render_feat_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned blocks = (unsigned)(p.nhalf < sms ? p.nhalf : sms);
  GS_TRACE("k_render_feat_tc", st);
  launch_pdl(k_render_feat_tc, blocks, kFwThreads, smem, st, p, omap);
  return last_launch_status();
}


// ===========================================================================
// Adjoint of the feature channels in the paper's decoupled mode (Sec. 3.1:
// the feature cotangent reaches only f): dL/df_g = sum_p w_g(p) dL/dF(p, :).
// Per half tile and block of 32 Gaussians, transposed so that every operand
// keeps a validated layout:
//     D [N channels x 32 Gaussians] = dF^T [N x 128 px] * W [128 px x 32]
//   A = dF^T, bf16, NMB = N/128 M-blocks; channel c sits in M-block c % NMB,
//       row r = c / NMB, so that a tensor-memory lane r holds the NMB
//       contiguous channels NMB r .. and the epilogue adds them with one
//       vector atomic. Staged in shared memory, K-major:
//       element (mb, r, p) at mb*32768 + (r/8)*2048 + (p/8)*128 + (r%8)*16 + (p%8)*2
//       and copied from there into tensor memory (tcgen05.cp, 128 rows x 32
//       bytes per M-block and 16 pixels; descriptor LBO = 128, SBO = 2048):
//       row r in lane r, pixels p, p + 1 in column A0 + 64 mb + p / 2, where
//       the products read it (A0 = 64 NMB, after the accumulators);
//   B = W, MN-major (Gaussians contiguous for a pixel):
//       element (p, g) at (g/8)*128 + (p/8)*512 + (p%8)*16 + (g%8)*2
//       descriptor LBO = 512 (K = pixels), SBO = 128 (N = Gaussians)
// The kernel is persistent (one CTA per SM, the forward's list of half
// tiles). Each half tile's dF^T is staged in shared memory: the first one by
// every warp from global memory (the fp32 cotangents of its 128 pixels,
// eight 16-byte loads in flight per thread, rounded to bf16), every later
// one by the epilogue warps while the previous half tile ran (see below).
// At the start of a half tile the MMA thread copies it into tensor memory
// (its products are ordered after the copies) and the copies' commit frees
// shared memory for the next staging. The roles run over the blocks of the
// compacted lists (the Gaussians whose skip mask reaches the half tile) of
// all the CTA's half tiles without a CTA-wide barrier between half tiles, so
// the producer and builders run up to the ring's depth ahead across them:
//   warp 0 (producer): the compaction and the records of each block by
//     cp.async into a 3-deep ring;
//   warps 10-25 (builders, 4 threads per pixel): W as in the forward, and
//     the bits of the block's Gaussians that weigh something here;
//   warp 1 (one thread): per half tile the copies of A, then per block
//     NMB x 8 tcgen05.mma (M=128, N=32, K=16, A from tensor memory) into one
//     of two tensor-memory accumulators;
//   warps 2-9 (epilogue; lanes 32 (w % 4).., Gaussians 16 (w >= 6)..+15):
//     the accumulator into registers, then one vector atomic per (Gaussian,
//     lane) into d_feats for the Gaussians that weigh something. While they
//     wait for the products they stage the NEXT half tile's cotangents: 16
//     chunks of 8 pixels (one row segment, all N channels, fp32) arrive in a
//     4-slot shared-memory ring, and per chunk one set of four warps (rows
//     32 (w % 4) ..) rounds it to bf16 into A once the copy of the current
//     half tile's A has completed. After a half tile's last block (whose
//     completion implies every product of the half tile has read A) they
//     signal the MMA thread, which copies the staged A in before the next
//     half tile's first product;
//   warp 26 (one thread, the copier): each chunk (8 consecutive pixels of a
//     row, contiguous in the HWC map) by one bulk copy into its slot as soon
//     as the slot's previous chunk has been converted; the copy's bytes
//     complete the slot's barrier.
// Every wait is bounded (1 s); a timeout flags GS_ERR_TIMEOUT and raises the
// abort word, on which every role stops.
namespace {

constexpr int kTbG = 32;  // Gaussians per block (MMA N)
constexpr int kBwThreads = 864;
constexpr int kBwStages = 3;
constexpr int kBwWarpMma = 1, kBwWarpEpi = 2, kBwEpi = 8, kBwWarpBuild = 10, kBwBuilders = 16, kBwWarpCopy = 26;
static_assert(kBwWarpBuild * 32 + 4 * kTcPix == kBwWarpCopy * 32, "four builder threads per pixel");
static_assert((kBwWarpCopy + 1) * 32 == kBwThreads, "one copier warp after the builders");

struct alignas(16) BwStage {
  uint8_t W[kTcPix * kTbG * 2];  // 8 KB, B operand
  float2 uv[kTbG];               // entry k at slot (k % 8) * 4 + k / 8
  float4 co[kTbG];
  int pos[kTbG];
  uint32_t gid[kTbG];            // by entry
  uint32_t nz;                   // bit k: entry k weighs something in this half tile
  int nvalid, flags;             // flags: 1 first block of its half tile, 2 last
};

constexpr int kStgSlots = 4;   // cotangent staging ring (chunks of 8 pixels)
constexpr int kStgChunks = 16;  // chunks per half tile
// The two converting warp sets take alternate chunks (and kStgChunks is
// even), so with an even slot count every slot is converted by one set, in
// order: a converter never tests a slot's barrier one use ahead of a copy
// still in flight, which would alias its phase parity.
static_assert(kStgSlots % 2 == 0 && kStgChunks % 2 == 0, "each staging slot belongs to one converting set");

struct BwSmem {
  uint8_t A[kTcMaxN * kTcPix * 2];  // dF^T, 128 KB for N = 512
  BwStage st[kBwStages];
  float stg[kStgSlots][8 * kTcMaxN];  // 16 KB per slot: pixel e's N channels at e * N
  unsigned long long stg_full[kStgSlots], stg_empty[kStgSlots];
  uint32_t cgid[64];
  int cpos[64];
  unsigned long long full[kBwStages], ready[kBwStages], empty[kBwStages];
  unsigned long long done[2], dfree[2], drain;
  unsigned long long a_full;  // the epilogue warps have staged the next half tile's dF^T in A (shared)
  unsigned long long a_free;  // the tensor core has copied A into tensor memory (A may be overwritten)
  uint32_t tmem;
  int abort;
};
// the structure is placed at the first 128-byte boundary of the dynamic shared
// memory (no operand here is swizzled: 16-byte alignment is what they need)
static_assert(sizeof(BwSmem) + 128 <= 227 * 1024, "shared memory of the adjoint");

struct BwParams {
  CamF cam;
  const int2* ranges;
  const int* order;
  const uint32_t* gids;
  const uint8_t* masks;
  const float2* uv;
  const float4* co;
  const int* last_idx;
  const float* g_feat;  // [H, W, N]
  int N, tmem_cols, nhalf;
  int P;  // Gaussians (bound of the checked build's id checks)
  float* d_feats;  // [P, N]
  int hold;  // test hook: the producer issues nothing, so the other roles' waits run out
  int32_t* status;
};

__device__ __forceinline__ void bw_tile(const BwParams& p, int h, int& tx, int& ty, int& half) {
  const int t = p.order ? p.order[h >> 1] : (h >> 1);
  tx = t % p.cam.tiles_x;
  ty = t / p.cam.tiles_x;
  half = h & 1;
}

// All threads: dF^T of half tile (tx, ty, half) into A. Item (i, pg): channel
// quad i (4 i .. 4 i + 3) of the 8 pixels m = 8 pg .. 8 pg + 7 (one row
// segment of the image); a warp reads 32 consecutive quads of a pixel and
// writes 16-byte rows of 8 pixels.
template <int NMB>
__device__ __forceinline__ void bw_stage_cotangents(const BwParams& p, BwSmem& S, int tx, int ty, int half) {
  constexpr int N = NMB * 128, nq = N / 4;
  const int ry0 = ty * kTile + half * 8, rx0 = tx * kTile;
  for (int it = threadIdx.x; it < nq * 16; it += kBwThreads) {
    const int i = it % nq, pg = it / nq;
    const int ry = ry0 + (pg >> 1), rx = rx0 + (pg & 1) * 8;
    float4 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ry < p.cam.H && rx + e < p.cam.W)
        v[e] = __ldg(reinterpret_cast<const float4*>(p.g_feat + ((size_t)ry * p.cam.W + rx + e) * N) + i);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int c = 4 * i + s, mb = c % NMB, r = c / NMB;
      uint32_t w4[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float f0 = s == 0 ? v[2 * e].x : s == 1 ? v[2 * e].y : s == 2 ? v[2 * e].z : v[2 * e].w;
        const float f1 = s == 0 ? v[2 * e + 1].x : s == 1 ? v[2 * e + 1].y : s == 2 ? v[2 * e + 1].z : v[2 * e + 1].w;
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(f0, f1);
        w4[e] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      *reinterpret_cast<uint4*>(S.A + mb * 32768 + (r >> 3) * 2048 + pg * 128 + (r & 7) * 16) =
          make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
  }
}

// Non-blocking test of an mbarrier phase.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// The epilogue warps' staging of the next half tile (see the kernel comment).
// Chunk c of the half tile is the CTA's chunk number g = g0 + c: ring slot
// g % kStgSlots, its use number u = g / kStgSlots picks the barrier phases.
struct BwStg {
  bool on;
  int tx, ty, half;  // the next half tile
  int cc;            // next chunk this warp converts (its set's chunks: cc = set, set + 2, ..)
  uint32_t g0;
  bool afree;        // the current half tile's A has been copied out of shared memory
  uint32_t apar;     // parity of that copy's a_free phase
};

// Pixels of chunk c of a half tile that lie in the image (the chunk's first
// nv pixels; 0 for a row below the image).
__device__ __forceinline__ int bw_chunk_pixels(const BwParams& p, int tx, int ty, int half, int c) {
  const int ry = ty * kTile + half * 8 + (c >> 1), rx0 = tx * kTile + (c & 1) * 8;
  return ry < p.cam.H ? max(0, min(8, p.cam.W - rx0)) : 0;
}

// chunk -> bf16 -> A in shared memory (the next half tile's dF^T), by the
// warp of lane quarter (warp % 4), rows r = 32 (warp % 4) + lane; chunk c
// holds the half tile's pixels 8 c .. 8 c + 7, one 16-byte core-matrix row per
// (M-block, r); pixels past the chunk's nv valid ones are zero
template <int NMB>
__device__ __forceinline__ void bw_stg_convert(BwSmem& S, int chunk, uint32_t slot, int nv) {
  constexpr int N = NMB * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = 32 * (warp & 3) + lane;  // row: channels NMB r .. NMB r + NMB - 1
  const float* src = S.stg[slot];
  float v[8][NMB];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const float* q = src + e * N + NMB * r;  // lanes read consecutive NMB-float groups
    if (e >= nv) {
#pragma unroll
      for (int mb = 0; mb < NMB; ++mb) v[e][mb] = 0.f;
    } else if constexpr (NMB == 4) {
      const float4 x = *reinterpret_cast<const float4*>(q);
      v[e][0] = x.x, v[e][1] = x.y, v[e][2] = x.z, v[e][3] = x.w;
    } else if constexpr (NMB == 2) {
      const float2 x = *reinterpret_cast<const float2*>(q);
      v[e][0] = x.x, v[e][1] = x.y;
    } else {
#pragma unroll
      for (int mb = 0; mb < NMB; ++mb) v[e][mb] = q[mb];
    }
  }
  uint8_t* dst = S.A + (r >> 3) * 2048 + chunk * 128 + (r & 7) * 16;
#pragma unroll
  for (int mb = 0; mb < NMB; ++mb) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * k][mb], v[2 * k + 1][mb]);
      w[k] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(dst + mb * 32768) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// One round of staging work that needs no waiting: convert this warp's next
// chunk if it has landed.
template <int NMB>
__device__ bool bw_stg_step(const BwParams& p, BwSmem& S, uint32_t tmem, BwStg& c) {
  if (!c.on || c.cc >= kStgChunks) return false;
  // A is overwritten only after the tensor core has copied the current half tile's out
  if (!c.afree) {
    if (!mbar_test(smem_u32(&S.a_free), c.apar)) return false;
    c.afree = true;
  }
  const uint32_t g = c.g0 + (uint32_t)c.cc, slot = g % kStgSlots, u = g / kStgSlots;
  if (!mbar_test(smem_u32(&S.stg_full[slot]), u & 1u)) return false;
  bw_stg_convert<NMB>(S, c.cc, slot, bw_chunk_pixels(p, c.tx, c.ty, c.half, c.cc));
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(smem_u32(&S.stg_empty[slot]));
  c.cc += 2;
  return true;
}

// Bounded wait for a barrier phase that stages while it waits; false on
// timeout (the abort word raised, GS_ERR_TIMEOUT flagged) or another role's abort.
template <int NMB>
__device__ bool bw_wait_staging(const BwParams& p, BwSmem& S, uint32_t tmem, BwStg& c, uint32_t bar,
                                uint32_t parity) {
  volatile int* abort = &S.abort;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (bw_stg_step<NMB>(p, S, tmem, c)) continue;
    if (*abort) return false;
    if (gtime() - t0 > kWaitNs) {
      *abort = 1;
      flag_status(p.status, GS_ERR_TIMEOUT);
      return false;
    }
  }
}

// The rest of the next half tile's staging after the current one's last block.
template <int NMB>
__device__ bool bw_stg_finish(const BwParams& p, BwSmem& S, uint32_t tmem, BwStg& c) {
  volatile int* abort = &S.abort;
  const unsigned long long t0 = gtime();
  while (c.on && c.cc < kStgChunks) {
    if (bw_stg_step<NMB>(p, S, tmem, c)) continue;
    if (*abort) return false;
    if (gtime() - t0 > kWaitNs) {
      *abort = 1;
      flag_status(p.status, GS_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// warp 0: compaction and records of one half tile's blocks; returns false on abort
__device__ bool bw_producer(const BwParams& p, BwSmem& S, int tx, int ty, int half, int& s, uint32_t& ph) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  volatile int* abort = &S.abort;
  const int2 rg = p.ranges[ty * p.cam.tiles_x + tx];
  int maxlast = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = lane + 32 * i;
    const int px = tx * kTile + (m & 15), py = ty * kTile + half * 8 + (m >> 4);
    if (px < p.cam.W && py < p.cam.H) maxlast = max(maxlast, p.last_idx[(size_t)py * p.cam.W + px]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxlast = max(maxlast, __shfl_xor_sync(0xffffffffu, maxlast, o));
  maxlast = checked_len(maxlast, rg.y - rg.x, p.status);
  int fill = 0;
  bool first = true;
  auto emit = [&](int n, bool last) -> bool {
    BwStage& st = S.st[s];
    if (!fw_wait(smem_u32(&S.empty[s]), ph ^ 1u, abort, p.status)) return false;
    const uint32_t g = lane < n ? S.cgid[lane] : 0u;
    const int slot = fw_slot(lane);
    cp_async8(smem_u32(&st.uv[slot]), p.uv + g, lane < n);
    cp_async16(smem_u32(&st.co[slot]), p.co + g, lane < n);
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.full[s])) : "memory");
    st.pos[slot] = lane < n ? S.cpos[lane] : 0x7fffffff;
    st.gid[lane] = g;
    if (lane == 0) {
      st.nvalid = n;
      st.flags = (first ? 1 : 0) | (last ? 2 : 0);
      st.nz = 0u;
    }
    mbar_arrive(smem_u32(&S.full[s]));
    first = false;
    if (++s == kBwStages) {
      s = 0;
      ph ^= 1u;
    }
    return true;
  };
  uint32_t gb[4], mb[4];
  auto fetch_batch = [&](int base) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int pos = base + 32 * i + lane;
      gb[i] = pos < maxlast ? checked_id(p.gids[rg.x + pos], p.P, p.status) : 0u;
      mb[i] = pos < maxlast ? (p.masks ? (uint32_t)p.masks[rg.x + pos] : 0xFu) : 0u;
    }
  };
  if (maxlast > 0) fetch_batch(0);
  for (int base = 0; base < maxlast; base += 128) {
    uint32_t gc[4], mc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      gc[i] = gb[i];
      mc[i] = mb[i];
    }
    if (base + 128 < maxlast) fetch_batch(base + 128);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int pos = base + 32 * i + lane;
      const bool hit = ((mc[i] >> (2 * half)) & 3u) != 0;
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int idx = fill + __popc(bal & lt);
        S.cgid[idx] = gc[i];
        S.cpos[idx] = pos;
      }
      fill += __popc(bal);
      __syncwarp();
      if (fill > 32) {
        if (!emit(32, false)) return false;
        const bool mv = lane < fill - 32;
        const uint32_t mg = mv ? S.cgid[32 + lane] : 0u;
        const int mp = mv ? S.cpos[32 + lane] : 0;
        __syncwarp();
        if (mv) {
          S.cgid[lane] = mg;
          S.cpos[lane] = mp;
        }
        fill -= 32;
        __syncwarp();
      }
    }
  }
  return emit(fill, true);
}

// warps 10-25: W of each block of one half tile (as the forward's weights)
__device__ bool bw_builder(const BwParams& p, BwSmem& S, int tx, int ty, int half, int& s, uint32_t& ph) {
  const int b = threadIdx.x - kBwWarpBuild * 32;
  const int m = b >> 2, q = b & 3, lane = threadIdx.x & 31;
  volatile int* abort = &S.abort;
  const int px = tx * kTile + (m & 15), py = ty * kTile + half * 8 + (m >> 4);
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const int last = (px < p.cam.W && py < p.cam.H) ? p.last_idx[(size_t)py * p.cam.W + px] : 0;
  float T = 1.f;
  while (true) {
    if (!fw_wait(smem_u32(&S.full[s]), ph, abort, p.status)) return false;
    BwStage& st = S.st[s];
    float a[8];
    float prod = 1.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int sl = 4 * j + q;
      a[j] = 0.f;
      PairAlpha pa;
      if (st.pos[sl] < last && pair_alpha(st.co[sl], st.uv[sl].x - pxc, st.uv[sl].y - pyc, pa)) {
        a[j] = pa.alpha;
        prod = __fmul_rn(prod, __fsub_rn(1.f, pa.alpha));
      }
    }
    float incl = prod;
    float y = __shfl_up_sync(0xffffffffu, incl, 1, 4);
    if (q >= 1) incl = __fmul_rn(incl, y);
    y = __shfl_up_sync(0xffffffffu, incl, 2, 4);
    if (q >= 2) incl = __fmul_rn(incl, y);
    float excl = __shfl_up_sync(0xffffffffu, incl, 1, 4);
    if (q == 0) excl = 1.f;
    const float total = __shfl_sync(0xffffffffu, incl, 3, 4);
    float Tj = __fmul_rn(T, excl);
    uint32_t packed[4];
    uint32_t mine = 0u;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const float w0 = __fmul_rn(a[j], Tj);
      if (a[j] > 0.f) Tj = __fmul_rn(Tj, __fsub_rn(1.f, a[j]));
      const float w1 = __fmul_rn(a[j + 1], Tj);
      if (a[j + 1] > 0.f) Tj = __fmul_rn(Tj, __fsub_rn(1.f, a[j + 1]));
      if (w0 != 0.f) mine |= 1u << (8 * q + j);
      if (w1 != 0.f) mine |= 1u << (8 * q + j + 1);
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(w0, w1);
      packed[j / 2] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    T = __fmul_rn(T, total);
    *reinterpret_cast<uint4*>(st.W + q * 128 + (m >> 3) * 512 + (m & 7) * 16) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
    const uint32_t wmask = __reduce_or_sync(0xffffffffu, mine);
    if (lane == 0 && wmask) atomicOr(&st.nz, wmask);
    const int flags = st.flags;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&S.ready[s]));
    if (++s == kBwStages) {
      s = 0;
      ph ^= 1u;
    }
    if (flags & 2) return true;
  }
}

// warp 1, one thread: the products of one half tile's blocks
template <int NMB>
__device__ bool bw_mma(const BwParams& p, BwSmem& S, uint32_t tmem, int& s, uint32_t& ph, uint32_t& nblk) {
  volatile int* abort = &S.abort;
  constexpr uint32_t dcols = (uint32_t)(NMB * kTbG);
  const uint32_t a0 = tmem + (uint32_t)(NMB * 64);  // A in tensor memory
  while (true) {
    if (!fw_wait(smem_u32(&S.ready[s]), ph, abort, p.status)) return false;
    BwStage& st = S.st[s];
    const int flags = st.flags;
    const uint32_t buf = nblk & 1u, use = nblk >> 1;
    if (!fw_wait(smem_u32(&S.dfree[buf]), (use & 1u) ^ 1u, abort, p.status)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t b0 = smem_u32(st.W);
    const uint32_t idesc = idesc_bf16(kTcPix, kTbG, 1);
#pragma unroll
    for (int mb = 0; mb < NMB; ++mb) {
#pragma unroll
      for (int k16 = 0; k16 < kTcPix / 16; ++k16) {
        const uint32_t at = a0 + (uint32_t)(mb * 64 + k16 * 8);
        const uint64_t bd = smem_desc(b0 + (uint32_t)k16 * 1024u, 512, 128);
        const uint32_t acc = k16 > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(
                tmem + buf * dcols + (uint32_t)(mb * kTbG)),
            "r"(at), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&S.done[buf])));
    ++nblk;
    if (++s == kBwStages) {
      s = 0;
      ph ^= 1u;
    }
    if (flags & 2) return true;
  }
}

// warp 26, one thread: the staging ring's copies. Chunk g of the CTA (the
// chunks of its half tiles after the first, in order) goes to slot
// g % kStgSlots once the chunk kStgSlots before it there has been converted:
// one bulk copy of the chunk's valid pixels (8 consecutive pixels of a row,
// contiguous in the HWC map), completing the slot's barrier with its bytes.
// The copies carry an L2 evict-first policy: the cotangents are read once, and
// the feature-gradient rows that the epilogue's atomics keep updating should
// stay in L2. Before returning it waits (bounded, whatever the abort word
// says) until every copy it issued has landed.
__device__ void bw_copier(const BwParams& p, BwSmem& S) {
  volatile int* abort = &S.abort;
  const int N = p.N;
  uint32_t g = 0;
  for (int rr = 1;; ++rr) {
    const int h = fw_half_tile(rr, p.nhalf);
    if (h < 0) break;
    int tx, ty, half;
    bw_tile(p, h, tx, ty, half);
    bool ok = true;
    for (int c = 0; c < kStgChunks && ok; ++c, ++g) {
      const uint32_t slot = g % kStgSlots, u = g / kStgSlots;
      if (u > 0 && !fw_wait(smem_u32(&S.stg_empty[slot]), (u - 1) & 1u, abort, p.status)) {
        ok = false;
        break;
      }
      const uint32_t bar = smem_u32(&S.stg_full[slot]);
      const uint32_t bytes = (uint32_t)bw_chunk_pixels(p, tx, ty, half, c) * (uint32_t)N * 4u;
      if (bytes) {
        const int ry = ty * kTile + half * 8 + (c >> 1), rx0 = tx * kTile + (c & 1) * 8;
        const float* src = p.g_feat + ((size_t)ry * p.cam.W + rx0) * N;
        asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        asm volatile(
            "{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], pol;"
            "\n\t}\n" ::"r"(smem_u32(S.stg[slot])),
            "l"(src), "r"(bytes), "r"(bar)
            : "memory");
      } else {
        mbar_arrive(bar);
      }
    }
    if (!ok) break;
  }
  // the last use of each slot this thread filled has landed
  volatile int never = 0;
  for (uint32_t k = 0; k < kStgSlots && k < g; ++k) {
    const uint32_t last = g - 1 - k, slot = last % kStgSlots, u = last / kStgSlots;
    fw_wait(smem_u32(&S.stg_full[slot]), u & 1u, &never, p.status);
  }
}

// warps 2-9: accumulators into the feature gradient
template <int NMB>
__device__ bool bw_epilogue(const BwParams& p, BwSmem& S, uint32_t tmem, int& s, uint32_t& ph, uint32_t& nblk,
                            BwStg& stg) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qd = warp & 3, gh = (warp - kBwWarpEpi) >> 2;  // lane quarter, Gaussians 16 gh .. 16 gh + 15
  volatile int* abort = &S.abort;
  constexpr uint32_t dcols = (uint32_t)(NMB * kTbG);
  constexpr int N = NMB * 128;
  const int r = 32 * qd + lane;  // channel row: channels NMB r .. NMB r + NMB - 1
  while (true) {
    const uint32_t buf = nblk & 1u, use = nblk >> 1;
    if (!bw_wait_staging<NMB>(p, S, tmem, stg, smem_u32(&S.done[buf]), use & 1u)) return false;
    // the builders' release of this block (its gids, bits and flags)
    if (!fw_wait(smem_u32(&S.ready[s]), ph, abort, p.status)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    BwStage& st = S.st[s];
    const int flags = st.flags;
    const uint32_t nzm = st.nz >> (16 * gh);
    const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + buf * dcols + (uint32_t)(16 * gh);
    // two groups of 8 Gaussians: the accumulator is released after the
    // second group's load, the stage after the last atomic is issued
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float v[NMB][8];
#pragma unroll
      for (int mb = 0; mb < NMB; ++mb) tmem_ld8(ta + (uint32_t)(mb * kTbG + 8 * i), v[mb]);
      tmem_wait_ld<NMB>(v);
      if (i == 1) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&S.dfree[buf]));
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (!((nzm >> (8 * i + j)) & 1u)) continue;
        float* dst = p.d_feats + (size_t)st.gid[16 * gh + 8 * i + j] * N + NMB * r;
        if constexpr (NMB == 4) {
          atomicAdd(reinterpret_cast<float4*>(dst), make_float4(v[0][j], v[1][j], v[2][j], v[3][j]));
        } else if constexpr (NMB == 2) {
          atomicAdd(reinterpret_cast<float2*>(dst), make_float2(v[0][j], v[1][j]));
        } else {
#pragma unroll
          for (int mb = 0; mb < NMB; ++mb) atomicAdd(dst + mb, v[mb][j]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&S.empty[s]));
    ++nblk;
    if (++s == kBwStages) {
      s = 0;
      ph ^= 1u;
    }
    if (flags & 2) return true;
  }
}

template <int NMB>
__global__ void __launch_bounds__(kBwThreads, 1) k_render_feat_tc_bwd(const BwParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;
  BwSmem& S = *reinterpret_cast<BwSmem*>(smem_raw + pad);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pdl_wait();
  pdl_trigger();
  if (tid == 0) {
    for (int s = 0; s < kBwStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 64;" ::"r"(smem_u32(&S.full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.ready[s])), "r"(kBwBuilders));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.empty[s])), "r"(kBwEpi));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.done[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.dfree[b])), "r"(kBwEpi));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.drain)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.a_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.a_free)));
    for (int k = 0; k < kStgSlots; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.stg_full[k])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.stg_empty[k])), "r"(kBwEpi / 2));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    S.abort = 0;
  }
  if (warp == kBwWarpMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(p.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = S.tmem;
  int s = 0;
  uint32_t ph = 0, nblk = 0;
  // the first half tile's dF^T, by every warp from global memory
  {
    const int h0 = fw_half_tile(0, p.nhalf);
    if (h0 >= 0) {
      int tx, ty, half;
      bw_tile(p, h0, tx, ty, half);
      bw_stage_cotangents<NMB>(p, S, tx, ty, half);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    for (int rr = 0; !p.hold; ++rr) {
      const int h = fw_half_tile(rr, p.nhalf);
      if (h < 0) break;
      int tx, ty, half;
      bw_tile(p, h, tx, ty, half);
      if (!bw_producer(p, S, tx, ty, half, s, ph)) break;
    }
  } else if (warp == kBwWarpMma) {
    if (lane == 0) {
      volatile int* abort = &S.abort;
      for (int rr = 0;; ++rr) {
        if (fw_half_tile(rr, p.nhalf) < 0) break;
        // this half tile's dF^T is in A (shared memory); the previous half
        // tile's products, which read A in tensor memory, have completed (the
        // epilogue signals a_full after its last block's completion)
        if (rr > 0 && !fw_wait(smem_u32(&S.a_full), (uint32_t)(rr - 1) & 1u, abort, p.status)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // A -> tensor memory: per M-block and 16 pixels, 128 rows x 32 bytes;
        // the products that follow are ordered after these copies
        const uint32_t as = smem_u32(S.A);
#pragma unroll 1
        for (int mb = 0; mb < NMB; ++mb)
#pragma unroll
          for (int k16 = 0; k16 < kTcPix / 16; ++k16)
            asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" ::"r"(tmem + (uint32_t)(NMB * 64 + mb * 64 +
                                                                                            k16 * 8)),
                         "l"(smem_desc(as + (uint32_t)mb * 32768u + (uint32_t)k16 * 256u, 128, 2048)));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&S.a_free)));
        if (!bw_mma<NMB>(p, S, tmem, s, ph, nblk)) break;
      }
    }
  } else if (warp < kBwWarpBuild) {
    uint32_t gchunks = 0;  // staging chunks this CTA has used (ring slot phases)
    for (int rr = 0;; ++rr) {
      if (fw_half_tile(rr, p.nhalf) < 0) break;
      const int hn = fw_half_tile(rr + 1, p.nhalf);
      BwStg stg;
      stg.on = hn >= 0;
      if (stg.on) bw_tile(p, hn, stg.tx, stg.ty, stg.half);
      stg.cc = (warp - kBwWarpEpi) >> 2;
      stg.g0 = gchunks;
      stg.afree = false;
      stg.apar = (uint32_t)rr & 1u;
      bool ok = bw_epilogue<NMB>(p, S, tmem, s, ph, nblk, stg);
      if (ok) ok = bw_stg_finish<NMB>(p, S, tmem, stg);
      // every epilogue warp has staged its chunks into A and read its
      // accumulators; the last block's completion means every product of this
      // half tile has completed. This thread's writes to A are made visible to
      // the tensor core's copy; the decision to stop is taken together (a
      // barrier reduction, which also joins the warps before a_full).
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      int stop;
      asm volatile(
          "{\n\t.reg .pred q, r;\n\tsetp.ne.b32 q, %1, 0;\n\tbar.red.or.pred r, 1, %2, q;\n\tselp.u32 %0, 1, 0, r;\n\t}\n"
          : "=r"(stop)
          : "r"((int)(!ok || S.abort || hn < 0)), "n"(kBwEpi * 32)
          : "memory");
      if (stop) break;
      if (warp == kBwWarpEpi && lane == 0) mbar_arrive(smem_u32(&S.a_full));
      gchunks += kStgChunks;
    }
  } else if (warp < kBwWarpCopy) {
    for (int rr = 0;; ++rr) {
      const int h = fw_half_tile(rr, p.nhalf);
      if (h < 0) break;
      int tx, ty, half;
      bw_tile(p, h, tx, ty, half);
      if (!bw_builder(p, S, tx, ty, half, s, ph)) break;
    }
  } else if (lane == 0) {
    bw_copier(p, S);
  }
  // every thread's copies have landed (warp 0's records; the copier waited for its own)
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (warp == kBwWarpMma && lane == 0) {
    // every product issued has completed before tensor memory is freed
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&S.drain)));
    volatile int never = 0;
    fw_wait(smem_u32(&S.drain), 0u, &never, p.status);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == kBwWarpMma) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
  }
}

template <int NMB>
gs_status launch_bwd_nmb(const BwParams& p, cudaStream_t st) {
  const size_t smem = sizeof(BwSmem) + 128;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_render_feat_tc_bwd<NMB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned blocks = (unsigned)(p.nhalf < sms ? p.nhalf : sms);
  GS_TRACE("k_render_feat_tc_bwd", st);
  launch_pdl(k_render_feat_tc_bwd<NMB>, blocks, kBwThreads, smem, st, p);
  return last_launch_status();
}

}  // namespace

gs_status launch_render_bwd_feat_tc(const CamF& cam, int P, const int32_t* ranges, const int32_t* order,
                                    const uint32_t* gids, const uint8_t* masks, const float* uv, const float* co,
                                    const int32_t* last_idx, const float* g_feat, int N, float* d_feats,
                                    int32_t* status, cudaStream_t st) {
  if (N <= 0 || N % 128 != 0 || N > kTcMaxN) return GS_ERR_UNSUPPORTED;
  // the vector atomics of the epilogue need NMB * 4-byte alignment of every row
  if ((reinterpret_cast<uintptr_t>(d_feats) & 15u) != 0) return GS_ERR_INVALID_ARG;
  // the staging's bulk copies start on 16-byte boundaries
  if ((reinterpret_cast<uintptr_t>(g_feat) & 15u) != 0) return GS_ERR_INVALID_ARG;
  BwParams p;
  p.P = P;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.gids = gids;
  p.masks = masks;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.last_idx = last_idx;
  p.g_feat = g_feat;
  p.N = N;
  // two accumulators (NMB x 32 columns each) and the staged next dF^T (NMB x 64)
  int cols = 32;
  while (cols < 4 * (N / 128) * kTbG) cols *= 2;
  p.tmem_cols = cols;
  p.nhalf = 2 * cam.tiles_x * cam.tiles_y;
  p.d_feats = d_feats;
  p.hold = g_tc_hold.load();
  p.status = status;
  switch (N / 128) {
    case 1: return launch_bwd_nmb<1>(p, st);
    case 2: return launch_bwd_nmb<2>(p, st);
    case 3: return launch_bwd_nmb<3>(p, st);
    default: return launch_bwd_nmb<4>(p, st);
  }
}


// ===========================================================================
// Decoder inference on tcgen05 (the learned-decoder form): per 128-pixel tile
//   D1 [128 x 128] = z [128 x 16] * W1 [16 x 128]        (one K=16 MMA)
//   h = gelu(D1 + b1) -> bf16 -> shared memory (A operand of the next product)
//   D2 [128 x 512] = h [128 x 128] * W2 [128 x 512]      (2 x 8 MMAs, N = 256)
//   y = D2 + b2 -> fp32 rows [128 x 512]
// Persistent CTAs (one per SM) keep W1 and W2 in shared memory as bf16.
// Layouts (validated rule: LBO along K, SBO along M/N):
//   A1 z  : (m/8)*256  + (k/8)*128 + (m%8)*16 + (k%8)*2   LBO 128, SBO 256
//   B1 W1 : (n/8)*128  + (k/8)*2048 + (k%8)*16 + (n%8)*2  LBO 2048, SBO 128
//   A2 h  : (m/8)*2048 + (k/8)*128 + (m%8)*16 + (k%8)*2   LBO 128, SBO 2048
//   B2 W2 : (n/8)*128  + (k/8)*8192 + (k%8)*16 + (n%8)*2  LBO 8192, SBO 128
// Tensor memory: D1 in columns [0, 128), then D2 in [0, 512): half a
// (outputs 0-255) in [0, 256), half b in [256, 512). Roles, so that a tile's
// drain overlaps the next tile's work:
//   warps 0-7 (group A): the gather of z, the GELU into H, then the drain of
//     half a; then, with half a free, the next tile's gather and GELU while
//     group B still drains half b;
//   warps 8-15 (group B): the drain of half b;
//   warp 16 (one thread): the products: G1 when z is in, G2a when H is, G2b
//     once group B has released half b of the previous tile.
// A drain warp (lanes 32 (w % 4).., 128 columns of its group's half) adds b2
// to 16 columns at a time and writes them into its own 2 KB box in the 64-byte
// swizzled order (16-byte chunk q of box row r at chunk q ^ ((r / 2) % 4):
// conflict-free stores), then stores the box with one TMA tensor store (the
// tensor map clips rows past npix). Every wait is bounded (1 s); a group takes
// each decision to stop together (a barrier reduction).
namespace {

struct DecSmem {
  uint8_t W2[128 * 512 * 2];            // 128 KB
  uint8_t H[128 * 128 * 2];             // 32 KB
  uint8_t Ybox[16 * 2048 + 1024];       // one 2 KB output box per drain warp (+ room to align them)
  uint8_t W1[16 * 128 * 2];             // 4 KB
  uint8_t Z[128 * 16 * 2];              // 4 KB
  float b1[128];
  float b2[512];
  unsigned long long z_ready, d1_full, h_ready, d2a_full, d2b_full, b_free, drain;
  uint32_t tmem;
};
constexpr int kDecThreads = 32 * 17;  // two drain groups of 8 warps and the MMA warp

struct DecTcParams {
  long long npix;
  const float* z;
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  float* y;
  int32_t* status;
};

// All 256 threads of drain group g (named barrier 1 + g) agree on v.
__device__ __forceinline__ bool dec_group_and(bool v, int g) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, r;\n\tsetp.ne.b32 q, %1, 0;\n\tbar.red.and.pred r, %2, 256, q;\n\tselp.u32 %0, 1, 0, r;\n\t}\n"
      : "=r"(r)
      : "r"((int)v), "r"(1 + g)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kDecThreads, 1) k_decoder_fwd_tc(const DecTcParams p,
                                                                   const __grid_constant__ CUtensorMap ymap) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  DecSmem& S = *reinterpret_cast<DecSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights -> bf16 operands (once per CTA)
  for (int e = tid; e < 128 * 512; e += kDecThreads) {
    const int k = e / 512, n = e % 512;
    *reinterpret_cast<__nv_bfloat16*>(S.W2 + (n >> 3) * 128 + (k >> 3) * 8192 + (k & 7) * 16 + (n & 7) * 2) =
        __float2bfloat16_rn(p.W2[e]);
  }
  for (int e = tid; e < 16 * 128; e += kDecThreads) {
    const int k = e / 128, n = e % 128;
    *reinterpret_cast<__nv_bfloat16*>(S.W1 + (n >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (n & 7) * 2) =
        __float2bfloat16_rn(p.W1[e]);
  }
  for (int e = tid; e < 128; e += kDecThreads) S.b1[e] = p.b1[e];
  for (int e = tid; e < 512; e += kDecThreads) S.b2[e] = p.b2[e];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    unsigned long long* bars[7] = {&S.z_ready, &S.d1_full, &S.h_ready, &S.d2a_full, &S.d2b_full, &S.b_free, &S.drain};
    for (int b = 0; b < 7; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars[b])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = S.tmem;
  const long long ntiles = (p.npix + 127) / 128;

  if (warp == 16) {
    // the products
    if (lane == 0) {
      const uint32_t idesc1 = idesc_bf16(128, 128, 1), idesc2 = idesc_bf16(128, 256, 1);
      const uint32_t a0 = smem_u32(S.H), b0 = smem_u32(S.W2);
      bool ok = true;
      int n = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++n) {
        const uint32_t par = (uint32_t)n & 1u;
        if (!mbar_wait(smem_u32(&S.z_ready), par)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        mma_bf16(tmem, smem_desc(smem_u32(S.Z), 128, 256), smem_desc(smem_u32(S.W1), 2048, 128), idesc1, 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&S.d1_full)));
        if (!mbar_wait(smem_u32(&S.h_ready), par)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int k16 = 0; k16 < 8; ++k16)
          mma_bf16(tmem, smem_desc(a0 + k16 * 256, 128, 2048), smem_desc(b0 + (uint32_t)k16 * 16384u, 8192, 128),
                   idesc2, k16 > 0 ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&S.d2a_full)));
        // half b of the previous tile has been read out
        if (n > 0 && !mbar_wait(smem_u32(&S.b_free), par ^ 1u)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int k16 = 0; k16 < 8; ++k16)
          mma_bf16(tmem + 256u, smem_desc(a0 + k16 * 256, 128, 2048),
                   smem_desc(b0 + 4096u + (uint32_t)k16 * 16384u, 8192, 128), idesc2, k16 > 0 ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&S.d2b_full)));
      }
      if (!ok) flag_status(p.status, GS_ERR_TIMEOUT);
      // every product issued has completed before tensor memory is freed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.drain)));
      mbar_wait(smem_u32(&S.drain), 0u);
    }
  } else {
    const int g = warp >> 3, gw = warp & 7;  // group (0: A, 1: B), warp in the group
    const int lq = warp & 3, cb = gw >> 2;   // tensor-memory lane quarter, column block of the group's half
    const int row = 32 * lq + lane;          // pixel row of the tile this thread reads back
    const uint32_t lane_off = (uint32_t)(32 * lq) << 16;
    const uint32_t box = ((smem_u32(S.Ybox) + 1023u) & ~1023u) + (uint32_t)warp * 2048u;
    const uint32_t rowa = box + (uint32_t)lane * 64u;
    bool ok = true;
    int n = 0;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++n) {
      const uint32_t par = (uint32_t)n & 1u;
      const long long base = t * 128;
      if (g == 0) {
        // z rows -> A1: two threads per row, 8 latents each (Z was last read by
        // the previous tile's G1, complete before its D1 was read)
        {
          const int r = tid >> 1, h8 = tid & 1;
          const long long pix = base + r;
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = 0.f;
          if (pix < p.npix) {
            const float4 a = *reinterpret_cast<const float4*>(p.z + pix * 16 + 8 * h8);
            const float4 b = *reinterpret_cast<const float4*>(p.z + pix * 16 + 8 * h8 + 4);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
          }
          uint32_t pk[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
          }
          *reinterpret_cast<uint4*>(S.Z + (r >> 3) * 256 + h8 * 128 + (r & 7) * 16) =
              make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        // the previous tile's half a has been read out (its loads waited for)
        // and z is in: the products may overwrite half a
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (tid == 0) mbar_arrive(smem_u32(&S.z_ready));
        ok = dec_group_and(mbar_wait(smem_u32(&S.d1_full), par), 0);
        // H is overwritten only after the previous tile's G2b has read it
        if (ok && n > 0) ok = dec_group_and(mbar_wait(smem_u32(&S.d2b_full), par ^ 1u), 0);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // hidden layer: columns [64 cb, 64 cb + 64) of D1 for pixel row `row`
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
          const int c0 = 64 * cb + 32 * k;
          float v[32];
          tmem_ld32(tmem + lane_off + (uint32_t)c0, v);
          uint32_t pk[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float h0 = gelu_exact(v[2 * i] + S.b1[c0 + 2 * i]);
            const float h1 = gelu_exact(v[2 * i + 1] + S.b1[c0 + 2 * i + 1]);
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(h0, h1);
            pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4*>(S.H + (row >> 3) * 2048 + (c0 / 8 + c) * 128 + (row & 7) * 16) =
                make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (tid == 0) mbar_arrive(smem_u32(&S.h_ready));
        ok = dec_group_and(mbar_wait(smem_u32(&S.d2a_full), par), 0);
      } else {
        ok = dec_group_and(mbar_wait(smem_u32(&S.d2b_full), par), 1);
      }
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // drain: this warp's 128 columns of its group's half, 16 at a time
      const int colbase = 256 * g + 128 * cb;
      const int row0 = (int)(base + 32 * lq);
#pragma unroll 1
      for (int s8 = 0; s8 < 8; ++s8) {
        const int c = colbase + 16 * s8;
        float v[2][8];
        tmem_ld8(tmem + lane_off + (uint32_t)c, v[0]);
        tmem_ld8(tmem + lane_off + (uint32_t)(c + 8), v[1]);
        tmem_wait_ld<2>(v);
        // the box's previous store has read it
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 b = *reinterpret_cast<const float4*>(&S.b2[c + 4 * q]);
          const float* x = &v[q >> 1][4 * (q & 1)];
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + (uint32_t)((q ^ ((lane >> 1) & 3)) << 4)),
                       "f"(x[0] + b.x), "f"(x[1] + b.y), "f"(x[2] + b.z), "f"(x[3] + b.w)
                       : "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(&ymap),
                       "r"(c), "r"(row0), "r"(box)
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      // this half of the tile's tensor memory has been read out
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (g == 1) {
        asm volatile("bar.sync 2, 256;" ::: "memory");
        if (tid == 256) mbar_arrive(smem_u32(&S.b_free));
      }
    }
    if (!ok && lane == 0) flag_status(p.status, GS_ERR_TIMEOUT);
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // this warp's stores complete
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

}  // namespace

// Label read-out straight from the latent render (Eq. 11 composed with
// Eq. 12): with y = W2^T h + b2, the logit of label l is
//   y . q(l) = h . G(:, l) + c(l),   G = W2 q^T [128 x L],   c = b2 . q^T,
// so the 512-d features never have to be formed. Per 128-pixel tile:
//   D1 [128 x 128] = z W1 (one K=16 MMA), h = gelu(D1 + b1) -> bf16 -> H,
//   D3 [128 x Lp] = H G   (8 K=16 MMAs, Lp = L rounded up to 16, G in bf16),
//   then per pixel row: logits D3 + c over the first L columns, argmax and
//   softmax. Each CTA folds G and c once (fp32 dot products over the 512
//   channels, from the queries staged in shared memory).
// Layouts (validated rule: LBO along K, SBO along M/N):
//   G : (n/8)*128 + (k/8)*(Lp*16) + (k%8)*16 + (n%8)*2   LBO Lp*16, SBO 128
// D3 reuses tensor-memory columns [0, Lp) of D1 once the GELU has read D1.
namespace {

constexpr int kDecLabMax = 64;

struct DecLabSmem {
  uint8_t H[128 * 128 * 2];          // 32 KB
  uint8_t W1[16 * 128 * 2];          // 4 KB
  uint8_t Z[128 * 16 * 2];           // 4 KB
  uint8_t G[128 * kDecLabMax * 2];   // 16 KB
  float qs[kDecLabMax * 512];        // 128 KB: the queries, fp32
  float b1[128];
  float b2[512];
  float cq[kDecLabMax];
  unsigned long long mbar;
  uint32_t tmem;
};

struct DecLabParams {
  long long npix;
  int L, Lp;
  const float* z;
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  const float* q;
  float* probs;
  int32_t* labels;
  int32_t* status;
};

__global__ void __launch_bounds__(512, 1) k_decoder_labels_tc(const DecLabParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  DecLabSmem& S = *reinterpret_cast<DecLabSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = warp & 3, cq = warp >> 2;
  const int row = 32 * lg + lane;
  const int L = p.L, Lp = p.Lp;

  for (int e = tid; e < 16 * 128; e += 512) {
    const int k = e / 128, n = e % 128;
    *reinterpret_cast<__nv_bfloat16*>(S.W1 + (n >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (n & 7) * 2) =
        __float2bfloat16_rn(p.W1[e]);
  }
  for (int e = tid; e < 128; e += 512) S.b1[e] = p.b1[e];
  for (int e = tid; e < 512; e += 512) S.b2[e] = p.b2[e];
  for (int e = tid; e < L * 512; e += 512) S.qs[e] = p.q[e];
  __syncthreads();
  // fold: G[k][l] = W2[k, :] . q[l, :] (0 for padded columns), c[l] = b2 . q[l, :].
  // Thread (k = tid % 128, group g = tid / 128) takes labels g, g + 4, ...: it
  // streams its W2 row once and reuses it for all of them (the label index is
  // the same across a warp, so the query reads are broadcasts).
  {
    constexpr int PER = kDecLabMax / 4;
    const int k = tid & 127, g4 = tid >> 7;
    float acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0.f;
    const float4* w = reinterpret_cast<const float4*>(p.W2 + (size_t)k * 512);
#pragma unroll 4
    for (int j = 0; j < 128; ++j) {
      const float4 a = __ldg(w + j);
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int l = g4 + 4 * i;
        if (l < L) {
          const float4 b = *reinterpret_cast<const float4*>(S.qs + (size_t)l * 512 + 4 * j);
          acc[i] = fmaf(a.x, b.x, acc[i]);
          acc[i] = fmaf(a.y, b.y, acc[i]);
          acc[i] = fmaf(a.z, b.z, acc[i]);
          acc[i] = fmaf(a.w, b.w, acc[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int l = g4 + 4 * i;
      if (l < Lp)
        *reinterpret_cast<__nv_bfloat16*>(S.G + (l >> 3) * 128 + (k >> 3) * (Lp * 16) + (k & 7) * 16 + (l & 7) * 2) =
            __float2bfloat16_rn(l < L ? acc[i] : 0.f);
    }
  }
  for (int l = tid; l < L; l += 512) {
    float acc = 0.f;
    for (int j = 0; j < 512; ++j) acc = fmaf(S.b2[j], S.qs[l * 512 + j], acc);
    S.cq[l] = acc;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = S.tmem;
  const uint32_t idesc1 = idesc_bf16(128, 128, 1), idesc3 = idesc_bf16(128, Lp, 1);
  const long long ntiles = (p.npix + 127) / 128;
  uint32_t phase = 0;
  bool ok = true;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const long long base = t * 128;
    if (cq < 2) {
      const long long pix = base + row;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = 0.f;
      if (pix < p.npix) {
        const float4 a = *reinterpret_cast<const float4*>(p.z + pix * 16 + 8 * cq);
        const float4 b = *reinterpret_cast<const float4*>(p.z + pix * 16 + 8 * cq + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      }
      uint32_t pk[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      *reinterpret_cast<uint4*>(S.Z + (row >> 3) * 256 + cq * 128 + (row & 7) * 16) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      mma_bf16(tmem, smem_desc(smem_u32(S.Z), 128, 256), smem_desc(smem_u32(S.W1), 2048, 128), idesc1, 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.mbar)));
    }
    ok = __syncthreads_and(mbar_wait(smem_u32(&S.mbar), phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(32 * cq), v);
      uint32_t pk[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float h0 = gelu_exact(v[2 * i] + S.b1[32 * cq + 2 * i]);
        const float h1 = gelu_exact(v[2 * i + 1] + S.b1[32 * cq + 2 * i + 1]);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(h0, h1);
        pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(S.H + (row >> 3) * 2048 + (4 * cq + c) * 128 + (row & 7) * 16) =
            make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(S.H), g0 = smem_u32(S.G);
#pragma unroll
      for (int k16 = 0; k16 < 8; ++k16)
        mma_bf16(tmem, smem_desc(a0 + k16 * 256, 128, 2048),
                 smem_desc(g0 + (uint32_t)k16 * 2u * (uint32_t)(Lp * 16), (uint32_t)(Lp * 16), 128), idesc3,
                 k16 > 0 ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.mbar)));
    }
    ok = __syncthreads_and(mbar_wait(smem_u32(&S.mbar), phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (cq == 0) {
      // warps 0-3: one pixel row each, all L logits
      float zl[kDecLabMax];
      tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16), *reinterpret_cast<float(*)[32]>(zl));
      if (Lp > 32) tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + 32u, *reinterpret_cast<float(*)[32]>(zl + 32));
      const long long pix = base + row;
      float mx = -INFINITY;
      int arg = 0;
#pragma unroll
      for (int l = 0; l < kDecLabMax; ++l)
        if (l < L) {
          zl[l] += S.cq[l];
          if (zl[l] > mx) {
            mx = zl[l];
            arg = l;
          }
        }
      if (pix < p.npix) {
        if (p.labels) p.labels[pix] = arg;
        if (p.probs) {
          float sum = 0.f;
#pragma unroll
          for (int l = 0; l < kDecLabMax; ++l)
            if (l < L) {
              zl[l] = expf(zl[l] - mx);
              sum += zl[l];
            }
          const float is = 1.f / sum;
#pragma unroll
          for (int l = 0; l < kDecLabMax; ++l)
            if (l < L) p.probs[pix * L + l] = zl[l] * is;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (!ok && tid == 0) flag_status(p.status, GS_ERR_TIMEOUT);
  if (!ok) mbar_wait(smem_u32(&S.mbar), phase ^ 1u);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

}  // namespace
}  // namespace gsff

extern "C" gs_status gs_decoder_fwd_tc(const gs_decoder* dec, int64_t npix, const float* z, float* y, int32_t* status,
                                       void* stream) {
  using namespace gsff;
  if (!dec || dec->din != 16 || dec->dh != 128 || dec->dout != 512 || !dec->W1 || !dec->b1 || !dec->W2 || !dec->b2)
    return GS_ERR_UNSUPPORTED;
  if (npix < 0 || (npix > 0 && (!z || !y)) || !aligned(z, 16) || !aligned(y, 16)) return GS_ERR_INVALID_ARG;
  if (npix == 0) return GS_OK;
  if (npix >= (1ll << 31)) return GS_ERR_UNSUPPORTED;  // row coordinates of the output tensor map are int32
  // output y [npix, 512] fp32 as a 2D tensor for TMA stores of 16-column x 32-row boxes, 64-byte swizzle
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return GS_ERR_CUDA;
  CUtensorMap ymap;
  const cuuint64_t dims[2] = {512, (cuuint64_t)npix};
  const cuuint64_t strides[1] = {512 * sizeof(float)};
  const cuuint32_t boxdim[2] = {16, 32};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, y, dims, strides, boxdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GS_ERR_CUDA;
  DecTcParams p;
  p.npix = npix;
  p.z = z;
  p.W1 = dec->W1;
  p.b1 = dec->b1;
  p.W2 = dec->W2;
  p.b2 = dec->b2;
  p.y = y;
  p.status = status;
  const size_t smem = sizeof(DecSmem) + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_decoder_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (npix + 127) / 128;
  const unsigned blocks = (unsigned)(ntiles < sms ? ntiles : sms);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GS_TRACE("k_decoder_fwd_tc", st);
  k_decoder_fwd_tc<<<blocks, kDecThreads, smem, st>>>(p, ymap);
  return last_launch_status();
}

extern "C" gs_status gs_decoder_labels_tc(const gs_decoder* dec, int64_t npix, const float* z, int32_t L,
                                          const float* queries, float* probs, int32_t* labels, int32_t* status,
                                          void* stream) {
  using namespace gsff;
  if (!dec || dec->din != 16 || dec->dh != 128 || dec->dout != 512 || !dec->W1 || !dec->b1 || !dec->W2 || !dec->b2)
    return GS_ERR_UNSUPPORTED;
  if (npix < 0 || L <= 0 || L > kDecLabMax || !queries || (!probs && !labels) || (npix > 0 && !z) ||
      !aligned(z, 16) || !aligned(dec->W2, 16))
    return GS_ERR_INVALID_ARG;
  if (npix == 0) return GS_OK;
  DecLabParams p;
  p.npix = npix;
  p.L = L;
  p.Lp = (L + 15) / 16 * 16;
  p.z = z;
  p.W1 = dec->W1;
  p.b1 = dec->b1;
  p.W2 = dec->W2;
  p.b2 = dec->b2;
  p.q = queries;
  p.probs = probs;
  p.labels = labels;
  p.status = status;
  const size_t smem = sizeof(DecLabSmem) + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_decoder_labels_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (npix + 127) / 128;
  const unsigned blocks = (unsigned)(ntiles < sms ? ntiles : sms);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GS_TRACE("k_decoder_labels_tc", st);
  k_decoder_labels_tc<<<blocks, 512, smem, st>>>(p);
  return last_launch_status();
}
