// Tensor-core (tcgen05) form of the feature channels of Eq. 3.
//
// Per tile the N feature channels are a dense contraction: with the tile's
// depth-sorted list as the contraction index k,
//     F[p, :] = sum_k w[p, k] f[g_k, :],   w[p, k] = alpha_k(p) T_k(p)
// (w = 0 where pixel p skips or has stopped). One CTA owns half a tile
// (16 x 8 = 128 pixels = the 128 rows of a tcgen05 M=128 tile) and up to 256
// of the channels (a 256-column accumulator, so two CTAs share an SM's tensor
// memory and overlap one's epilogue with the other's main loop), and walks
// the list in K-steps of 32 Gaussians:
//   - 4 threads per pixel (512 threads) each evaluate alpha for 8 of the 32
//     Gaussians with the SIMT kernel's exact skip test; below last_idx no
//     pixel has stopped, so T_k is the product of (1 - alpha_j) over the
//     blended j < k, combined across the 4 threads by a width-4 shuffle
//     scan; each thread stores its 8 weights (bf16) as one 16-byte row of a
//     core matrix of the A operand [128 x 32] (K-major);
//   - the 32 feature rows (bf16) are copied with cp.async into the B operand
//     [32 x N] (MN-major: channels contiguous);
//   - one thread issues tcgen05.mma kind::f16 (M=128, N<=256 per
//     instruction, K=16) accumulating F in fp32 in tensor memory (N columns);
//   - a 3-stage shared-memory ring lets the next step's loads and weights
//     proceed while the tensor core consumes the current step
//     (tcgen05.commit -> mbarrier per stage).
// The epilogue reads F from tensor memory (tcgen05.ld 32x32b), stages it in
// shared memory and writes it in HWC layout with bulk asynchronous copies. RGB, depth, alpha, T_final and last_idx come from the SIMT
// forward kernel launched before this one (its last_idx bounds each pixel).
//
// Shared-memory operand layouts (no swizzle; 16-byte core-matrix rows):
//   A: element (m, k) at (m/8)*512 + (k/8)*128 + (m%8)*16 + (k%8)*2
//      descriptor LBO = 128 (K direction), SBO = 512 (M direction)
//   B: element (k, n) at (n/8)*128 + (k/8)*SK + (k%8)*16 + (n%8)*2, SK = Nc*16
//      (Nc <= 256 channels of this CTA)
//      descriptor LBO = SK (K direction), SBO = 128 (N direction)
// Every wait is bounded (1 s of %globaltimer); a timeout flags
// GS_ERR_TIMEOUT, waits (bounded) for the tensor core, frees tensor memory
// and returns.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kTcPix = 128;    // pixels per CTA = MMA M
constexpr int kTcThreads = 512;  // 4 threads per pixel
constexpr int kTcK = 32;       // Gaussians per K-step
constexpr int kTcStages = 3;
constexpr int kTcMaxN = 512;
constexpr int kTcNC = 256;     // channels per CTA (tensor-memory columns of one accumulator)
constexpr unsigned long long kWaitNs = 1000000000ull;

struct TcStage {
  uint8_t A[kTcPix * kTcK * 2];       // 8 KB
  uint8_t B[kTcK * kTcNC * 2];        // 16 KB (256 channels)
  float2 uv[kTcK];
  float4 co[kTcK];
};

struct TcSmem {
  TcStage st[kTcStages];  // also the epilogue's staging area (128 rows x 528 B)
  unsigned long long mbar[kTcStages];
  uint32_t tmem;
  int maxlast;
};

static_assert(sizeof(TcStage) * kTcStages >= (kTcPix - 1) * 528 + 512, "epilogue staging does not fit the ring");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: f32 accumulate, bf16 A and B, A K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N, int b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn_major << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the given phase parity of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = gtime();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtime() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Record slot of the k-th Gaussian of a 32-Gaussian step: thread quarter q
// reads Gaussians 8q..8q+7, so slot 4 (k % 8) + k / 8 puts the four quarters'
// j-th records side by side (one bank group, no conflicts).
__device__ __forceinline__ int rec_slot(int k) { return ((k & 7) << 2) | (k >> 3); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Waits for this thread's outstanding tensor-memory loads; the values pass
// through the barrier so that no use of them is scheduled before it.
template <int G>
__device__ __forceinline__ void tmem_wait_ld(float (&v)[G][8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int g = 0; g < G; ++g)
    asm volatile("" : "+f"(v[g][0]), "+f"(v[g][1]), "+f"(v[g][2]), "+f"(v[g][3]), "+f"(v[g][4]), "+f"(v[g][5]),
                 "+f"(v[g][6]), "+f"(v[g][7]));
}

struct TcFwdParams {
  CamF cam;
  const int2* ranges;
  const int* order;  // launch order of the tiles, or null
  const uint32_t* gids;
  const float2* uv;
  const float4* co;
  const __nv_bfloat16* feats;
  const int* last_idx;
  int N;          // feature channels in total
  int nsplit;     // CTAs per half tile, each owning kTcNC channels (the last may own fewer)
  float* out_feat;
  int32_t* status;
};

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool valid) {
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

// Gaussian ids a thread needs to issue the copies of one K-step: the record
// id (threads 0..31) and the ids of its feature rows (16-byte chunks tid and
// tid + 512). They are fetched one step before use, so no id load stalls the
// step that issues the copies.
struct TcIds {
  uint32_t rec;
  uint32_t row[2];
};
static_assert(kTcK * kTcNC / 8 <= 2 * kTcThreads, "two feature chunks per thread per K-step");

__device__ __forceinline__ TcIds tc_fetch_ids(const TcFwdParams& p, int t, int2 rg, int maxlast, int cpr) {
  const int tid = threadIdx.x;
  const int base = rg.x + t * kTcK, lim = rg.x + maxlast;
  TcIds ids{0u, {0u, 0u}};
  if (tid < kTcK && base + tid < lim) ids.rec = p.gids[base + tid];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int e = tid + i * kTcThreads;
    if (e < kTcK * cpr) {
      const int k = e / cpr;
      if (base + k < lim) ids.row[i] = p.gids[base + k];
    }
  }
  return ids;
}

// Asynchronous copies of K-step t into stage `st`: the Gaussian records
// (threads 0..31) and the feature rows (16-byte chunks), zero-filled past the
// list; one commit group per step.
__device__ __forceinline__ void tc_issue_loads(const TcFwdParams& p, TcStage& st, int t, int2 rg, int maxlast, int c0,
                                               int Nc, const TcIds& ids) {
  const int tid = threadIdx.x;
  const int base = rg.x + t * kTcK;
  const int lim = rg.x + maxlast;
  if (tid < kTcK) {
    const bool valid = base + tid < lim;
    cp_async8(smem_u32(&st.uv[rec_slot(tid)]), p.uv + ids.rec, valid);
    cp_async16(smem_u32(&st.co[rec_slot(tid)]), p.co + ids.rec, valid);
  }
  const int cpr = Nc / 8;  // 16-byte chunks of this CTA's channels per feature row
  const uint32_t SK = (uint32_t)Nc * 16;
  const uint32_t b0 = smem_u32(st.B);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int e = tid + i * kTcThreads;
    if (e < kTcK * cpr) {
      const int k = e / cpr, c = e - k * cpr;
      const bool valid = base + k < lim;
      const __nv_bfloat16* src = p.feats + (size_t)ids.row[i] * p.N + c0 + 8 * c;
      const uint32_t dst = b0 + (uint32_t)c * 128u + (uint32_t)(k >> 3) * SK + (uint32_t)(k & 7) * 16u;
      cp_async16(dst, src, valid);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 2) k_render_feat_tc(const TcFwdParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = tid >> 2, q = tid & 3;  // pixel row of the MMA tile, quarter of the K-step
  const int split = blockIdx.x % p.nsplit;
  const int lt = (blockIdx.x / p.nsplit) >> 1, half = (blockIdx.x / p.nsplit) & 1;
  const int tile = p.order ? p.order[lt] : lt;
  const int c0 = split * kTcNC, Nc = min(kTcNC, p.N - c0);
  int tmem_cols = 32;
  while (tmem_cols < Nc) tmem_cols *= 2;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  const int px = tx * kTile + (m & 15);
  const int py = ty * kTile + half * 8 + (m >> 4);
  const bool inside = px < p.cam.W && py < p.cam.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const int2 rg = p.ranges[tile];
  const int last = inside ? p.last_idx[(size_t)py * p.cam.W + px] : 0;

  if (tid == 0) S.maxlast = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (q == 0 && last > 0) atomicMax(&S.maxlast, last);
  __syncthreads();
  const int maxlast = S.maxlast;
  const uint32_t tmem = S.tmem;
  const int nsteps = (maxlast + kTcK - 1) / kTcK;
  const uint32_t SK = (uint32_t)Nc * 16;
  bool ok = true;

  const int cpr = Nc / 8;
  if (nsteps > 0) tc_issue_loads(p, S.st[0], 0, rg, maxlast, c0, Nc, tc_fetch_ids(p, 0, rg, maxlast, cpr));
  if (nsteps > 1) tc_issue_loads(p, S.st[1], 1, rg, maxlast, c0, Nc, tc_fetch_ids(p, 1, rg, maxlast, cpr));
  TcIds next_ids = tc_fetch_ids(p, 2, rg, maxlast, cpr);  // ids of the next K-step to issue
  float T = 1.f;  // transmittance in front of this K-step (same in the 4 threads of a pixel)
  int last_issued = -1;  // last K-step whose MMAs were issued (block-uniform)
  for (int t = 0; t < nsteps && ok; ++t) {
    const int s = t % kTcStages;
    TcStage& st = S.st[s];
    if (t + 1 < nsteps) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // alphas of my 8 Gaussians (0 where skipped or past last_idx)
    float a[8];
    float prod = 1.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] = 0.f;
      const int k = 8 * q + j, ks = rec_slot(k);
      PairAlpha pa;
      if (t * kTcK + k < last && pair_alpha(st.co[ks], st.uv[ks].x - pxc, st.uv[ks].y - pyc, pa)) {
        a[j] = pa.alpha;
        prod = __fmul_rn(prod, __fsub_rn(1.f, pa.alpha));
      }
    }
    // exclusive product over the quarters before mine (lanes 4m..4m+3)
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
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(st.A), b0 = smem_u32(st.B);
      for (int n0 = 0; n0 < Nc; n0 += 256) {
        const int nn = min(256, Nc - n0);
        const uint32_t idesc = idesc_bf16(kTcPix, nn, 1);
#pragma unroll
        for (int k16 = 0; k16 < kTcK / 16; ++k16) {
          const uint64_t ad = smem_desc(a0 + k16 * 256, 128, 512);
          const uint64_t bd = smem_desc(b0 + (uint32_t)(n0 / 8) * 128u + (uint32_t)k16 * 2u * SK, SK, 128);
          const uint32_t acc = (t > 0 || k16 > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)n0),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.mbar[s])));
    }
    last_issued = t;
    if (t + 2 < nsteps) {
      // stage (t+2)%3 was last read by the MMAs of step t-1
      bool w_ok = true;
      if (t >= 1) w_ok = mbar_wait(smem_u32(&S.mbar[(t - 1) % kTcStages]), (uint32_t)(((t - 1) / kTcStages) & 1));
      ok = __syncthreads_and(w_ok) != 0;
      if (ok) {
        tc_issue_loads(p, S.st[(t + 2) % kTcStages], t + 2, rg, maxlast, c0, Nc, next_ids);
        next_ids = tc_fetch_ids(p, t + 3, rg, maxlast, cpr);
      }
    }
  }
  if (nsteps > 0 && ok) {
    const int tl = nsteps - 1;
    ok = __syncthreads_and(mbar_wait(smem_u32(&S.mbar[tl % kTcStages]), (uint32_t)((tl / kTcStages) & 1))) != 0;
  }
  if (!ok) {
    if (tid == 0) flag_status(p.status, GS_ERR_TIMEOUT);
    // bounded drain of the last issued commit before freeing tensor memory
    if (last_issued >= 0)
      mbar_wait(smem_u32(&S.mbar[last_issued % kTcStages]), (uint32_t)((last_issued / kTcStages) & 1));
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // Epilogue through shared memory and the bulk-copy engine: for each slab
    // of pw <= 128 columns (the last slab of a 192-channel share is 64 wide),
    // warp w (tensor-memory lanes 32*(w%4).., column quarter w/4) stages its
    // 32 x 32 block into the idle operand ring with rows padded to 528 B
    // (conflict-free 16-byte stores), then one thread per pixel row issues a
    // bulk copy of its pw * 4 contiguous bytes into the HWC output.
    uint8_t* stage = S.st[0].A;  // >= 128 * 528 bytes of the idle ring
    const uint32_t stage_u32 = smem_u32(stage);
    const int row = 32 * (warp & 3) + (tid & 31);
    const int PW = Nc < 128 ? Nc : 128;
    for (int p0 = 0; p0 < Nc; p0 += PW) {
      const int pw = min(PW, Nc - p0);  // columns in this slab: a multiple of 32 (Nc % 64 == 0)
      const int cbase = 32 * (warp >> 2);
      if (cbase < pw) {
        float v[32];
        if (nsteps > 0) {
          tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(p0 + cbase), v);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
        uint8_t* dst = stage + row * 528 + cbase * 4;
#pragma unroll
        for (int i = 0; i < 32; i += 4)
          *reinterpret_cast<float4*>(dst + i * 4) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid < kTcPix) {
        const int ex = tx * kTile + (tid & 15), ey = ty * kTile + half * 8 + (tid >> 4);
        if (ex < p.cam.W && ey < p.cam.H) {
          float* g = p.out_feat + ((size_t)ey * p.cam.W + ex) * p.N + c0 + p0;
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g),
                       "r"(stage_u32 + (uint32_t)tid * 528u), "r"(pw * 4)
                       : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      }
      __syncthreads();
    }
    if (tid < kTcPix) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

}  // namespace

gs_status launch_render_fwd_tc(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                               const float* uv,
                               const float* co, const __nv_bfloat16* feats, const int32_t* last_idx, int N,
                               float* out_feat, int32_t* status, cudaStream_t st) {
  if (N <= 0 || N % 64 != 0 || N > kTcMaxN) return GS_ERR_UNSUPPORTED;
  TcFwdParams p;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.gids = gids;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.feats = feats;
  p.last_idx = last_idx;
  p.N = N;
  p.nsplit = (N + kTcNC - 1) / kTcNC;
  p.out_feat = out_feat;
  p.status = status;
  const size_t smem = sizeof(TcSmem) + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_render_feat_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_render_feat_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  const unsigned blocks = (unsigned)(cam.tiles_x * cam.tiles_y * 2 * p.nsplit);
  GS_TRACE("k_render_feat_tc", st);
  k_render_feat_tc<<<blocks, kTcThreads, smem, st>>>(p);
  return last_launch_status();
}


// ===========================================================================
// Adjoint of the feature channels in the paper's decoupled mode (Sec. 3.1:
// the feature cotangent reaches only f): dL/df_g = sum_p w_g(p) dL/dF(p, :).
// Per half tile, transposed so that every operand keeps a validated layout:
//     D [N channels x 32 Gaussians] = dF^T [N x 128 px] * W [128 px x 32]
//   A = dF^T, K-major, converted to bf16 once per CTA, NMB = N/128 M-blocks.
//       Channel c sits in M-block c % NMB, row r = c / NMB, so that a
//       tensor-memory lane r holds the NMB contiguous channels NMB r .. and
//       the epilogue adds them with one vector atomic:
//       element (mb, r, p) at mb*32768 + (r/8)*2048 + (p/8)*128 + (r%8)*16 + (p%8)*2
//       descriptor LBO = 128 (K = pixels), SBO = 2048 (M = channel rows)
//   B = W, MN-major (Gaussians contiguous for a pixel), one 16-byte row per
//       thread exactly as in the forward:
//       element (p, g) at (g/8)*128 + (p/8)*512 + (p%8)*16 + (g%8)*2
//       descriptor LBO = 512 (K = pixels), SBO = 128 (N = Gaussians)
// D is double-buffered in tensor memory (2 x NMB x 32 columns), so the MMAs
// of a Gaussian block overlap the epilogue of the previous one. In the
// epilogue warp w takes lanes 32 (w % 4).. and Gaussians 8 (w / 4)..+7 of the
// block and skips Gaussians that weigh nothing in this half tile (a bit mask
// built with one warp reduction per warp).
namespace {

constexpr int kTbG = 32;  // Gaussians per block (MMA N)

struct TbSmem {
  uint8_t A[kTcMaxN * kTcPix * 2];  // dF^T, 128 KB for N = 512
  uint8_t B[2][kTcPix * kTbG * 2];  // W, 8 KB per buffer
  float2 uv[3][kTbG];  // record ring: block b uses slot b % 3, Gaussian k at rec_slot(k)
  float4 co[3][kTbG];
  uint32_t gid[3][kTbG];  // by position k in the block
  uint32_t nz[3];         // bit k: Gaussian k has a nonzero weight in this half tile
  unsigned long long mbar[2];
  uint32_t tmem;
  int maxlast;
};

struct TcBwdParams {
  CamF cam;
  const int2* ranges;
  const int* order;  // launch order of the tiles, or null
  const uint32_t* gids;
  const float2* uv;
  const float4* co;
  const int* last_idx;
  const float* g_feat;  // [H, W, N]
  int N;
  int tmem_cols;
  float* d_feats;  // [P, N]
  int32_t* status;
};

__device__ __forceinline__ uint32_t tb_fetch_id(const TcBwdParams& p, int b, int2 rg, int maxlast) {
  const int pos = rg.x + b * kTbG + (int)threadIdx.x;
  return pos < rg.x + maxlast ? p.gids[pos] : 0u;
}

// Records of Gaussian block b into ring slot `slot` (threads 0..31): id from
// registers, uv and conic/opacity by asynchronous copy (zero past the list).
__device__ __forceinline__ void tb_issue(const TcBwdParams& p, TbSmem& S, int slot, int b, int2 rg, int maxlast,
                                         uint32_t g) {
  const int tid = threadIdx.x;
  const bool valid = rg.x + b * kTbG + tid < rg.x + maxlast;
  const int k = rec_slot(tid);
  cp_async8(smem_u32(&S.uv[slot][k]), p.uv + g, valid);
  cp_async16(smem_u32(&S.co[slot][k]), p.co + g, valid);
  asm volatile("cp.async.commit_group;" ::: "memory");
  S.gid[slot][tid] = g;
  if (tid == 0) S.nz[slot] = 0u;
}

template <int NMB>
__global__ void __launch_bounds__(kTcThreads, 1) k_render_feat_tc_bwd(const TcBwdParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TbSmem& S = *reinterpret_cast<TbSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = tid >> 2, q = tid & 3;
  const int tile = p.order ? p.order[blockIdx.x >> 1] : (int)(blockIdx.x >> 1), half = blockIdx.x & 1;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  const int px = tx * kTile + (m & 15);
  const int py = ty * kTile + half * 8 + (m >> 4);
  const bool inside = px < p.cam.W && py < p.cam.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const int2 rg = p.ranges[tile];
  const int last = inside ? p.last_idx[(size_t)py * p.cam.W + px] : 0;
  constexpr uint32_t dcols = (uint32_t)(NMB * kTbG);  // tensor-memory columns per D buffer
  const int N = NMB * 128;

  if (tid == 0) S.maxlast = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(p.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // dF^T for this half tile. Item (i, pg): channel quad i (4 i .. 4 i + 3) of
  // the 8 pixels m = 8 pg .. 8 pg + 7 (one row segment of the image); the 32
  // lanes of a warp read 32 consecutive quads of a pixel (coalesced) and write
  // 16-byte rows of 8 pixels (distinct bank groups for NMB = 4).
  {
    const int nq = N / 4;
    const int ry0 = ty * kTile + half * 8;
    const int rx0 = tx * kTile;
    for (int it = tid; it < nq * 16; it += kTcThreads) {
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
        float f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = s == 0 ? v[e].x : s == 1 ? v[e].y : s == 2 ? v[e].z : v[e].w;
        uint32_t w4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
          w4[e] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        *reinterpret_cast<uint4*>(S.A + mb * 32768 + (r >> 3) * 2048 + pg * 128 + (r & 7) * 16) =
            make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (q == 0 && last > 0) atomicMax(&S.maxlast, last);
  __syncthreads();
  const int maxlast = S.maxlast;
  const uint32_t tmem = S.tmem;
  const int nb = (maxlast + kTbG - 1) / kTbG;
  bool ok = true;
  uint32_t next_id = 0;  // id of this thread's Gaussian in the next block to stage (threads 0..31)
  if (nb > 0 && tid < kTbG) {
    tb_issue(p, S, 0, 0, rg, maxlast, tb_fetch_id(p, 0, rg, maxlast));
    if (nb > 1) next_id = tb_fetch_id(p, 1, rg, maxlast);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  __syncthreads();

  float T = 1.f;
  int last_issued = -1;
  auto epilogue = [&](int b) -> bool {
    const int buf = b & 1, slot = b % 3;
    const bool w_ok =
        __syncthreads_and(mbar_wait(smem_u32(&S.mbar[buf]), (uint32_t)((b >> 1) & 1))) != 0;
    if (!w_ok) return false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int r = 32 * (warp & 3) + lane;  // channel row: channels NMB r .. NMB r + NMB - 1
    const int g0 = 8 * (warp >> 2);
    float v[NMB][8];
    const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)buf * dcols + (uint32_t)g0;
#pragma unroll
    for (int mb = 0; mb < NMB; ++mb) tmem_ld8(ta + (uint32_t)(mb * kTbG), v[mb]);
    tmem_wait_ld<NMB>(v);
    const uint32_t msk = S.nz[slot] >> g0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!((msk >> j) & 1u)) continue;
      float* dst = p.d_feats + (size_t)S.gid[slot][g0 + j] * N + NMB * r;
      if constexpr (NMB == 4) {
        atomicAdd(reinterpret_cast<float4*>(dst), make_float4(v[0][j], v[1][j], v[2][j], v[3][j]));
      } else if constexpr (NMB == 2) {
        atomicAdd(reinterpret_cast<float2*>(dst), make_float2(v[0][j], v[1][j]));
      } else {
#pragma unroll
        for (int mb = 0; mb < NMB; ++mb) atomicAdd(dst + mb, v[mb][j]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    return true;
  };

  for (int b = 0; b < nb && ok; ++b) {
    const int buf = b & 1, slot = b % 3;
    // stage block b+1's records (slot (b+1)%3 was last read by the epilogue of
    // block b-2, which finished in the previous iteration); fetch the ids of b+2
    if (b + 1 < nb && tid < kTbG) {
      tb_issue(p, S, (b + 1) % 3, b + 1, rg, maxlast, next_id);
      if (b + 2 < nb) next_id = tb_fetch_id(p, b + 2, rg, maxlast);
    }
    // weights of my 8 Gaussians (one 16-byte row of B)
    float a[8];
    float prod = 1.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] = 0.f;
      const int k = 8 * q + j, ks = rec_slot(k);
      PairAlpha pa;
      if (b * kTbG + k < last && pair_alpha(S.co[slot][ks], S.uv[slot][ks].x - pxc, S.uv[slot][ks].y - pyc, pa)) {
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
    const uint32_t wmask = __reduce_or_sync(0xffffffffu, mine);
    if (lane == 0 && wmask) atomicOr(&S.nz[slot], wmask);
    *reinterpret_cast<uint4*>(S.B[buf] + q * 128 + (m >> 3) * 512 + (m & 7) * 16) =
        make_uint4(packed[0], packed[1], packed[2], packed[3]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(S.A), b0 = smem_u32(S.B[buf]);
      const uint32_t idesc = idesc_bf16(kTcPix, kTbG, 1);
#pragma unroll
      for (int mb = 0; mb < NMB; ++mb) {
#pragma unroll
        for (int k16 = 0; k16 < kTcPix / 16; ++k16) {
          const uint64_t ad = smem_desc(a0 + (uint32_t)mb * 16u * 2048u + (uint32_t)k16 * 256u, 128, 2048);
          const uint64_t bd = smem_desc(b0 + (uint32_t)k16 * 1024u, 512, 128);
          const uint32_t acc = k16 > 0 ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                  tmem + (uint32_t)buf * dcols + (uint32_t)(mb * kTbG)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.mbar[buf])));
    }
    last_issued = b;
    if (b >= 1) ok = epilogue(b - 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }
  if (ok && nb > 0) ok = epilogue(nb - 1);
  if (!ok) {
    if (tid == 0) flag_status(p.status, GS_ERR_TIMEOUT);
    if (last_issued >= 0) mbar_wait(smem_u32(&S.mbar[last_issued & 1]), (uint32_t)((last_issued >> 1) & 1));
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
}

template <int NMB>
gs_status launch_bwd_nmb(const TcBwdParams& p, const CamF& cam, cudaStream_t st) {
  const size_t smem = sizeof(TbSmem) + 1024;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_render_feat_tc_bwd<NMB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  const unsigned blocks = (unsigned)(cam.tiles_x * cam.tiles_y * 2);
  GS_TRACE("k_render_feat_tc_bwd", st);
  k_render_feat_tc_bwd<NMB><<<blocks, kTcThreads, smem, st>>>(p);
  return last_launch_status();
}

}  // namespace

gs_status launch_render_bwd_feat_tc(const CamF& cam, const int32_t* ranges, const int32_t* order,
                                    const uint32_t* gids, const float* uv,
                                    const float* co, const int32_t* last_idx, const float* g_feat, int N,
                                    float* d_feats, int32_t* status, cudaStream_t st) {
  if (N <= 0 || N % 128 != 0 || N > kTcMaxN) return GS_ERR_UNSUPPORTED;
  // the vector atomics of the epilogue need NMB * 4-byte alignment of every row
  if ((reinterpret_cast<uintptr_t>(d_feats) & 15u) != 0) return GS_ERR_INVALID_ARG;
  TcBwdParams p;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.gids = gids;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.last_idx = last_idx;
  p.g_feat = g_feat;
  p.N = N;
  int cols = 32;
  while (cols < 2 * (N / 128) * kTbG) cols *= 2;
  p.tmem_cols = cols;
  p.d_feats = d_feats;
  p.status = status;
  switch (N / 128) {
    case 1: return launch_bwd_nmb<1>(p, cam, st);
    case 2: return launch_bwd_nmb<2>(p, cam, st);
    case 3: return launch_bwd_nmb<3>(p, cam, st);
    default: return launch_bwd_nmb<4>(p, cam, st);
  }
}


// ===========================================================================
// Decoder inference on tcgen05 (the learned-decoder form): per 128-pixel tile
//   D1 [128 x 128] = z [128 x 16] * W1 [16 x 128]        (one K=16 MMA)
//   h = gelu(D1 + b1) -> bf16 -> shared memory (A operand of the next product)
//   D2 [128 x 512] = h [128 x 128] * W2 [128 x 512]      (2 x 8 MMAs, N = 256)
//   y = D2 + b2 -> fp32 rows [128 x 512]
// Persistent CTAs (one per SM, 512 threads) keep W1 and W2 in shared memory
// as bf16. Layouts (validated rule: LBO along K, SBO along M/N):
//   A1 z  : (m/8)*256  + (k/8)*128 + (m%8)*16 + (k%8)*2   LBO 128, SBO 256
//   B1 W1 : (n/8)*128  + (k/8)*2048 + (k%8)*16 + (n%8)*2  LBO 2048, SBO 128
//   A2 h  : (m/8)*2048 + (k/8)*128 + (m%8)*16 + (k%8)*2   LBO 128, SBO 2048
//   B2 W2 : (n/8)*128  + (k/8)*8192 + (k%8)*16 + (n%8)*2  LBO 8192, SBO 128
// D1 occupies tensor-memory columns [0, 128) and is overwritten by D2
// (columns [0, 512)) once read.
// Epilogue: warp w (tensor-memory lanes 32 (w % 4).., columns 128 (w / 4)..)
// adds b2 to 32 x 32 blocks of D2 and writes each into its own 4 KB box in
// shared memory in the 128-byte swizzled order (16-byte chunk q of box row r
// at chunk q ^ (r % 8): conflict-free stores), then stores the box with one
// TMA tensor store. The tensor map clips rows past npix. The 16 boxes reuse
// H (free once D2 is complete) and the 32 KB after it, from a 1024-byte
// boundary.
namespace {

struct DecSmem {
  uint8_t W2[128 * 512 * 2];   // 128 KB
  uint8_t H[128 * 128 * 2];    // 32 KB; also the first half of the output boxes
  uint8_t Ybox[128 * 128 * 2 + 1024];  // second half of the boxes (+ room to align them)
  uint8_t W1[16 * 128 * 2];    // 4 KB
  uint8_t Z[128 * 16 * 2];     // 4 KB
  float b1[128];
  float b2[512];
  unsigned long long mbar;
  uint32_t tmem;
};

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

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__global__ void __launch_bounds__(512, 1) k_decoder_fwd_tc(const DecTcParams p,
                                                           const __grid_constant__ CUtensorMap ymap) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  DecSmem& S = *reinterpret_cast<DecSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = warp & 3, cq = warp >> 2;  // tensor-memory lane group, column quarter
  const int row = 32 * lg + lane;           // pixel row of the tile this thread reads back

  // weights -> bf16 operands (once per CTA)
  for (int e = tid; e < 128 * 512; e += 512) {
    const int k = e / 512, n = e % 512;
    *reinterpret_cast<__nv_bfloat16*>(S.W2 + (n >> 3) * 128 + (k >> 3) * 8192 + (k & 7) * 16 + (n & 7) * 2) =
        __float2bfloat16_rn(p.W2[e]);
  }
  for (int e = tid; e < 16 * 128; e += 512) {
    const int k = e / 128, n = e % 128;
    *reinterpret_cast<__nv_bfloat16*>(S.W1 + (n >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 + (n & 7) * 2) =
        __float2bfloat16_rn(p.W1[e]);
  }
  for (int e = tid; e < 128; e += 512) S.b1[e] = p.b1[e];
  for (int e = tid; e < 512; e += 512) S.b2[e] = p.b2[e];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(512));
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
  const uint32_t idesc1 = idesc_bf16(128, 128, 1), idesc2 = idesc_bf16(128, 256, 1);
  const long long ntiles = (p.npix + 127) / 128;
  uint32_t phase = 0;
  bool ok = true;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const long long base = t * 128;
    // z rows -> A1 (threads with cq < 2 write chunk cq of row `row`)
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
      *reinterpret_cast<uint4*>(S.Z + (row >> 3) * 256 + cq * 128 + (row & 7) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
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
      // hidden layer: columns [32 cq, 32 cq + 32) of D1 for pixel row `row`
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
      const uint32_t a0 = smem_u32(S.H), b0 = smem_u32(S.W2);
      for (int nh = 0; nh < 2; ++nh)
#pragma unroll
        for (int k16 = 0; k16 < 8; ++k16)
          mma_bf16(tmem + (uint32_t)(256 * nh), smem_desc(a0 + k16 * 256, 128, 2048),
                   smem_desc(b0 + (uint32_t)nh * 4096u + (uint32_t)k16 * 16384u, 8192, 128), idesc2,
                   k16 > 0 ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&S.mbar)));
    }
    ok = __syncthreads_and(mbar_wait(smem_u32(&S.mbar), phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    {
      const uint32_t box = ((smem_u32(S.H) + 1023u) & ~1023u) + (uint32_t)warp * 4096u;
      const uint32_t rowa = box + (uint32_t)lane * 128u;
      const int row0 = (int)(base + 32 * lg);
      for (int s4 = 0; s4 < 4; ++s4) {
        const int c = 128 * cq + 32 * s4;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)c, v);
        if (s4 > 0) {
          // the previous box must have been read out before it is overwritten
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 b = *reinterpret_cast<const float4*>(&S.b2[c + 4 * q]);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(rowa + (uint32_t)((q ^ (lane & 7)) << 4)),
                       "f"(v[4 * q] + b.x), "f"(v[4 * q + 1] + b.y), "f"(v[4 * q + 2] + b.z),
                       "f"(v[4 * q + 3] + b.w)
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
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (!ok && tid == 0) flag_status(p.status, GS_ERR_TIMEOUT);
  if (!ok) mbar_wait(smem_u32(&S.mbar), phase ^ 1u);  // bounded drain of the outstanding commit
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // this warp's stores complete
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

}  // namespace

// Label read-out straight from the latent render (Eq. 9 composed with
// Eq. 11): with y = W2^T h + b2, the logit of label l is
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
  // output y [npix, 512] fp32 as a 2D tensor for TMA stores of 32 x 32 boxes, 128-byte swizzle
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return GS_ERR_CUDA;
  CUtensorMap ymap;
  const cuuint64_t dims[2] = {512, (cuuint64_t)npix};
  const cuuint64_t strides[1] = {512 * sizeof(float)};
  const cuuint32_t boxdim[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, y, dims, strides, boxdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
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
  k_decoder_fwd_tc<<<blocks, 512, smem, st>>>(p, ymap);
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
