// Decoder training on tcgen05: one evaluation of the MSE loss of Eq. 11's
// o(.) against the full-width target on sampled pixels, with its gradients
// (the same step as gs_decoder_train: y = W2^T gelu(W1^T z + b1) + b2,
// L = scale sum (y - t)^2), in two kernels over tiles of 128 samples.
//
// k_decoder_train_tc (persistent, 512 threads, one CTA per SM), per tile:
//   G1  D1[s, h]   = Z[s, d] W1[d, h]                 (M = s, N = h, K = 16)
//   E1  H = gelu(D1 + b1) -> bf16, transposed: HT[h, s]
//   for each quarter q of the 512 outputs (o = 128 q + o'):
//   G2  D2T[o', s] = W2T[o', h] HT[h, s]              (M = o', N = s, K = 128)
//   E2  dY[s, o'] = 2 scale (D2T + b2 - target) -> bf16; loss and db2 in fp32
//   G3  dH[s, h]  += dY[s, o'] W2T[o', h]             (M = s, N = h, K = 128)
//   E3  dPRE[s, h] = dH gelu'(D1 + b1) -> bf16
//   G4  dZ[s, d]   = dPRE[s, h] W1T[h, d]             (M = s, N = 16, K = 128)
//   G5  dW1x[d', h] = ZT1[d', s] dPRE[s, h]           (M = 128, N = h, K = s)
//   E4  dZ added to dz_map at the sampled pixels; rows 0-15 of dW1x added to
//       dW1, row 16 (a row of ones in ZT1) to db1 (vector atomics).
// Each product keeps A K-major and B MN-major (the two validated layouts):
// W2T serves as G2's A and G3's B, dPRE as G4's A and G5's B. The
// transposed operands (HT, dY, ZT1) are written with 2-byte stores at a
// column-group stride of 144 bytes, so that 8 consecutive groups fall in
// different banks. ZT1's rows 17-127 are not data: G5 computes them into
// tensor-memory lanes that are never read, from shared memory inside the
// allocation.
// The CTA writes HT and dY of every tile to a workspace (bf16, coalesced);
// k_decoder_dw2_tc then forms dW2[h, o] = sum_s HT[h, s] dY[s, o] (M = h,
// N = 256, K = s), each CTA one half of the outputs over a share of the
// tiles, and adds it with vector atomics. dW2 needs all 512 tensor-memory
// columns for the whole sample set, so it cannot share the first kernel's.
//
// Rounding: z, H, dY and dPRE enter the products as bf16 (unit roundoff
// 2^-8), the weights are bf16-exact by contract, every sum is fp32. GELU and
// its derivative take erf from Abramowitz & Stegun 7.1.26 (absolute error at
// most 1.5e-7) with one exponential shared with the normal density.

#include <atomic>
#include <cstddef>

#include "tc_util.cuh"

namespace gsff {
namespace {

constexpr int kDtThreads = 512;
constexpr int kDtS = 128;             // samples per tile
constexpr uint32_t kCs = 144;         // bytes between 8-column groups of the transposed operands
constexpr uint32_t kRs = 16 * kCs;    // bytes between 8-row groups of a 128-column transposed operand
static_assert(kDtThreads == 4 * kDtS, "the gather takes four threads per sample");

struct DtSmem {
  uint8_t W2T[512 * 128 * 2];  // (o, h) at (o/8)*2048 + (h/8)*128 + (o%8)*16 + (h%8)*2
  uint8_t ZT1[3 * kRs];        // (d', s) at (d'/8)*kRs + (s/8)*kCs + (d'%8)*16 + (s%8)*2: z, a row of ones, zeros
  uint8_t HT[16 * kRs];        // (h, s) like ZT1; from E3 on, dPRE (s, h) at (s/8)*2048 + (h/8)*128 + ...
  uint8_t DY[16 * kRs];        // (s, o') at (s/8)*kRs + (o'/8)*kCs + (s%8)*16 + (o'%8)*2
  uint8_t Z[128 * 16 * 2];     // (s, d) at (s/8)*256 + (d/8)*128 + (s%8)*16 + (d%8)*2
  uint8_t W1[16 * 128 * 2];    // (d, h) at (h/8)*128 + (d/8)*2048 + (d%8)*16 + (h%8)*2
  uint8_t W1T[128 * 16 * 2];   // (h, d) at (h/8)*256 + (d/8)*128 + (h%8)*16 + (d%8)*2
  float b1[128];
  float b2[512];
  long long pix[kDtS];         // sampled pixel of each row of the tile, -1 past the sample count
  float red[kDtThreads / 32];
  unsigned long long mbar;
  uint32_t tmem;
};
// G5 reads ZT1 rows up to 127 (15 row groups past its start); they must stay
// inside the structure
static_assert(offsetof(DtSmem, ZT1) + 16 * kRs <= offsetof(DtSmem, Z), "ZT1 garbage rows inside shared memory");

struct DtParams {
  long long nsample, npix, s_pad;
  unsigned long long seed;
  float scale;
  const float* z;
  const float* target;
  const float* W1;
  const float* b1;
  const float* W2;
  const float* b2;
  float* dW1;
  float* db1;
  float* db2;
  float* dz;
  float* loss;
  __nv_bfloat16* HTg;  // [128][s_pad]
  __nv_bfloat16* DYg;  // [s_pad][512]
  int32_t* status;
};

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

__device__ __forceinline__ void before_sync() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
}

__device__ __forceinline__ void after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }

__global__ void __launch_bounds__(kDtThreads, 1) k_decoder_train_tc(const DtParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  DtSmem& S = *reinterpret_cast<DtSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lg = warp & 3, cq = warp >> 2;  // tensor-memory lane group, column quarter
  const int row = 32 * lg + lane;           // tensor-memory lane this thread reads

  // weights -> bf16 operands, once per CTA (the values are bf16-exact)
  for (int e = tid; e < 128 * 512; e += kDtThreads) {
    const int h = e >> 9, o = e & 511;
    st_bf16(S.W2T, (uint32_t)((o >> 3) * 2048 + (h >> 3) * 128 + (o & 7) * 16 + (h & 7) * 2), p.W2[e]);
  }
  for (int e = tid; e < 16 * 128; e += kDtThreads) {
    const int d = e >> 7, h = e & 127;
    st_bf16(S.W1, (uint32_t)((h >> 3) * 128 + (d >> 3) * 2048 + (d & 7) * 16 + (h & 7) * 2), p.W1[e]);
    st_bf16(S.W1T, (uint32_t)((h >> 3) * 256 + (d >> 3) * 128 + (h & 7) * 16 + (d & 7) * 2), p.W1[e]);
  }
  for (int e = tid; e < 128; e += kDtThreads) S.b1[e] = p.b1[e];
  for (int e = tid; e < 512; e += kDtThreads) S.b2[e] = p.b2[e];
  // ZT1 rows 16 (ones) .. 23 (zeros)
  for (int e = tid; e < 8 * kDtS; e += kDtThreads) {
    const int d = 16 + (e >> 7), s = e & 127;
    st_bf16(S.ZT1, (uint32_t)(2 * kRs + (s >> 3) * kCs + (d & 7) * 16 + (s & 7) * 2), d == 16 ? 1.f : 0.f);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  before_sync();
  __syncthreads();
  after_sync();
  const uint32_t tmem = S.tmem, mbar = smem_u32(&S.mbar);
  const uint32_t lane_off = (uint32_t)(32 * lg) << 16;
  const uint32_t id128 = idesc_bf16(128, 128, 1), id16 = idesc_bf16(128, 16, 1);
  const uint32_t aZ = smem_u32(S.Z), aW1 = smem_u32(S.W1), aW1T = smem_u32(S.W1T), aW2T = smem_u32(S.W2T);
  const uint32_t aHT = smem_u32(S.HT), aDY = smem_u32(S.DY), aZT = smem_u32(S.ZT1);
  // tensor-memory columns: D1 [0, 128), D2T buffers [128, 256) and [256, 384),
  // dH [384, 512); then dZ [128, 144) and dW1x [256, 384)
  constexpr uint32_t cD1 = 0, cD2 = 128, cDH = 384, cDZ = 128, cDW1 = 256;

  float acc_db2[4] = {0.f, 0.f, 0.f, 0.f};  // output 128 q + row, over this thread's columns
  float acc_loss = 0.f;

  const long long ntiles = (p.nsample + kDtS - 1) / kDtS;
  uint32_t phase = 0;
  bool ok = true;
  auto wait_mma = [&]() {
    ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
    phase ^= 1u;
    if (ok) after_sync();
    return ok;
  };
  // gather: sample row s of tile tt -> its pixel and latents 4 c .. 4 c + 3,
  // four threads per sample; issued one tile ahead (under the previous tile's
  // last products), with the sample's 2 KB target row prefetched into L2 for
  // the loss epilogues
  const int gs_s = tid >> 2, gs_c = tid & 3;
  auto fetch = [&](long long tt, long long& pix, float4& a) {
    const long long gs = tt * kDtS + gs_s;
    pix = (tt < ntiles && gs < p.nsample) ? decoder_sample_pixel(p.seed, gs, p.npix) : -1;
    a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pix >= 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.target + pix * 512 + 32 * (4 * gs_c + k)));
      a = *reinterpret_cast<const float4*>(p.z + pix * 16 + 4 * gs_c);
    }
  };
  long long pix_n;
  float4 a_n;
  fetch(blockIdx.x, pix_n, a_n);
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const long long s0 = t * kDtS;
    // the fetched sample rows -> Z (s, d) and ZT1 (d, s)
    {
      const int s = gs_s, c = gs_c;
      if (c == 0) S.pix[s] = pix_n;
      const float4 a = a_n;
      const __nv_bfloat162 lo = __floats2bfloat162_rn(a.x, a.y), hi = __floats2bfloat162_rn(a.z, a.w);
      *reinterpret_cast<uint2*>(S.Z + (s >> 3) * 256 + (c >> 1) * 128 + (s & 7) * 16 + (c & 1) * 8) =
          make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
      const float v[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int d = 4 * c + k;
        st_bf16(S.ZT1, (uint32_t)((d >> 3) * kRs + (s >> 3) * kCs + (d & 7) * 16 + (s & 7) * 2), v[k]);
      }
    }
    before_sync();
    __syncthreads();
    if (tid == 0) {
      after_sync();
      mma_bf16(tmem + cD1, smem_desc(aZ, 128, 256), smem_desc(aW1, 2048, 128), id128, 0u);
      mma_commit(mbar);
    }
    if (!wait_mma()) break;
    // E1: H = gelu(D1 + b1) for row s, columns h = 32 cq .., into HT (h, s) and HTg
    {
      const int s = row;
      float v[32];
      tmem_ld32(tmem + lane_off + cD1 + 32 * cq, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int h = 32 * cq + i;
        const __nv_bfloat16 hb = __float2bfloat16_rn(gelu_as(v[i] + S.b1[h]));
        *reinterpret_cast<__nv_bfloat16*>(S.HT + (h >> 3) * kRs + (s >> 3) * kCs + (h & 7) * 16 + (s & 7) * 2) = hb;
        p.HTg[(size_t)h * p.s_pad + s0 + s] = hb;
      }
    }
    before_sync();
    __syncthreads();
    if (tid == 0) {
      after_sync();
#pragma unroll
      for (int k = 0; k < 8; ++k)
        mma_bf16(tmem + cD2, smem_desc(aW2T + k * 256, 128, 2048), smem_desc(aHT + k * 2 * kRs, kRs, kCs), id128,
                 k > 0 ? 1u : 0u);
      mma_commit(mbar);
    }
    for (int q = 0; q < 4; ++q) {
      // E2: row = output o' of quarter q, columns s = 32 cq ..; the targets
      // are loaded before the wait for the products, under it
      const int o = 128 * q + row;
      float tg[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const long long pix = S.pix[32 * cq + i];
        tg[i] = pix >= 0 ? __ldg(p.target + pix * 512 + o) : 0.f;
      }
      if (!wait_mma()) break;
      {
        float v[32];
        tmem_ld32(tmem + lane_off + cD2 + 128 * (q & 1) + 32 * cq, v);
        const float b = S.b2[o];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int s = 32 * cq + i;
          const bool valid = S.pix[s] >= 0;
          const float dlt = valid ? (v[i] + b) - tg[i] : 0.f;
          acc_loss = fmaf(dlt, dlt, acc_loss);
          const float g = 2.f * p.scale * dlt;
          acc_db2[q] += g;
          const __nv_bfloat16 gb = __float2bfloat16_rn(g);
          *reinterpret_cast<__nv_bfloat16*>(S.DY + (s >> 3) * kRs + (row >> 3) * kCs + (s & 7) * 16 + (row & 7) * 2) =
              gb;
          p.DYg[(size_t)(s0 + s) * 512 + o] = gb;
        }
      }
      before_sync();
      __syncthreads();
      if (tid == 0) {
        after_sync();
        // G3: dH += dY W2T over this quarter's outputs
#pragma unroll
        for (int k = 0; k < 8; ++k)
          mma_bf16(tmem + cDH, smem_desc(aDY + k * 2 * kCs, kCs, kRs),
                   smem_desc(aW2T + (uint32_t)q * 32768u + k * 4096, 2048, 128), id128, (q > 0 || k > 0) ? 1u : 0u);
        // G2 of the next quarter into the other buffer (read by E2 of the previous one)
        if (q < 3) {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            mma_bf16(tmem + cD2 + 128 * ((q + 1) & 1), smem_desc(aW2T + (uint32_t)(q + 1) * 32768u + k * 256, 128, 2048),
                     smem_desc(aHT + k * 2 * kRs, kRs, kCs), id128, k > 0 ? 1u : 0u);
        }
        mma_commit(mbar);
      }
    }
    if (!ok || !wait_mma()) break;
    // E3: dPRE = dH gelu'(D1 + b1) for row s, columns h = 32 cq .., into HT's space as (s, h)
    {
      const int s = row;
      float dh[32], pre[32];
      tmem_ld32(tmem + lane_off + cDH + 32 * cq, dh);
      tmem_ld32(tmem + lane_off + cD1 + 32 * cq, pre);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t pk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = 8 * c + 2 * i, h = 32 * cq + j;
          const float x0 = dh[j] * gelu_grad_as(pre[j] + S.b1[h]);
          const float x1 = dh[j + 1] * gelu_grad_as(pre[j + 1] + S.b1[h + 1]);
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
          pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(S.HT + (s >> 3) * 2048 + (4 * cq + c) * 128 + (s & 7) * 16) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    before_sync();
    __syncthreads();
    if (tid == 0) {
      after_sync();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        // G4: dZ = dPRE W1T
        mma_bf16(tmem + cDZ, smem_desc(aHT + k * 256, 128, 2048), smem_desc(aW1T + k * 512, 256, 128), id16,
                 k > 0 ? 1u : 0u);
        // G5: dW1x = ZT1 dPRE
        mma_bf16(tmem + cDW1, smem_desc(aZT + k * 2 * kCs, kCs, kRs), smem_desc(aHT + k * 4096, 2048, 128), id128,
                 k > 0 ? 1u : 0u);
      }
      mma_commit(mbar);
    }
    // the next tile's sample rows, under these products (Z and ZT1 are
    // rewritten only after them)
    fetch(t + gridDim.x, pix_n, a_n);
    if (!wait_mma()) break;
    // E4: dZ to the sampled pixels (column quarter 0 holds its 16 columns);
    // dW1x rows 0-16 (lane group 0) to dW1 and db1
    if (cq == 0) {
      float v[32];
      tmem_ld32(tmem + lane_off + cDZ, v);
      const long long pix = S.pix[row];
      if (p.dz && pix >= 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          atomicAdd(reinterpret_cast<float4*>(p.dz + pix * 16 + 4 * c),
                    make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]));
      }
    }
    if (lg == 0) {
      float v[32];
      tmem_ld32(tmem + cDW1 + 32 * cq, v);
      if (lane <= 16) {
        float* dst = lane < 16 ? p.dW1 + lane * 128 + 32 * cq : p.db1 + 32 * cq;
#pragma unroll
        for (int c = 0; c < 8; ++c)
          atomicAdd(reinterpret_cast<float4*>(dst + 4 * c), make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (!ok && tid == 0) flag_status(p.status, GS_ERR_TIMEOUT);
  if (!ok) mbar_wait(mbar, phase ^ 1u);  // bounded drain of the outstanding commit
  // the CTA's sums: db2, the loss
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (acc_db2[q] != 0.f) atomicAdd(p.db2 + 128 * q + row, acc_db2[q]);
  if (p.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_loss += __shfl_xor_sync(0xffffffffu, acc_loss, o);
    if (lane == 0) S.red[warp] = acc_loss;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (p.loss && tid == 0) {
    float b = 0.f;
    for (int w = 0; w < kDtThreads / 32; ++w) b += S.red[w];
    if (b != 0.f) atomicAdd(p.loss, b * p.scale);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// dW2[h, o] += sum_s HT[h, s] dY[s, o]: CTA (half, split) accumulates outputs
// [256 half, 256 half + 256) over the tiles t = split, split + nsplit, ... in
// tensor memory (128 lanes x 256 columns), the operands copied in with
// 16-byte cp.async into two buffers (the next tile's copies run under the
// current tile's products), then adds its sums with vector atomics.
//   A = HT tile (h, s) at (h/8)*2048 + (s/8)*128 + (h%8)*16 + (s%8)*2   LBO 128, SBO 2048
//   B = dY tile (s, o) at (s/8)*4096 + (o/8)*128 + (s%8)*16 + (o%8)*2   LBO 4096, SBO 128
constexpr int kD2Threads = 256;

struct D2Buf {
  uint8_t A[128 * 128 * 2];  // 32 KB
  uint8_t B[128 * 256 * 2];  // 64 KB
};

struct D2Smem {
  D2Buf buf[2];
  unsigned long long mbar;
  uint32_t tmem;
};

struct D2Params {
  long long ntiles, s_pad;
  int nsplit;
  const __nv_bfloat16* HTg;
  const __nv_bfloat16* DYg;
  float* dW2;
  int32_t* status;
};

__device__ __forceinline__ void d2_load(const D2Params& p, D2Buf& b, long long t, int half) {
  const long long s0 = t * kDtS;
  const uint32_t aA = smem_u32(b.A), aB = smem_u32(b.B);
  for (int c = threadIdx.x; c < 128 * 16; c += kD2Threads) {  // A: 8 samples of one h per chunk
    const int h = c >> 4, j = c & 15;
    cp_async16(aA + (h >> 3) * 2048 + j * 128 + (h & 7) * 16, p.HTg + (size_t)h * p.s_pad + s0 + 8 * j, true);
  }
  for (int c = threadIdx.x; c < 128 * 32; c += kD2Threads) {  // B: 8 outputs of one sample per chunk
    const int s = c >> 5, j = c & 31;
    cp_async16(aB + (s >> 3) * 4096 + j * 128 + (s & 7) * 16, p.DYg + (size_t)(s0 + s) * 512 + 256 * half + 8 * j,
               true);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kD2Threads, 1) k_decoder_dw2_tc(const D2Params p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  D2Smem& S = *reinterpret_cast<D2Smem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = blockIdx.x & 1, split = blockIdx.x >> 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  after_sync();
  const uint32_t tmem = S.tmem, mbar = smem_u32(&S.mbar);
  const uint32_t idesc = idesc_bf16(128, 256, 1);
  // this CTA's tiles: split, split + nsplit, ...
  const long long n_mine = split < p.ntiles ? (p.ntiles - 1 - split) / p.nsplit + 1 : 0;
  if (n_mine > 0) d2_load(p, S.buf[0], split, half);
  if (n_mine > 1) d2_load(p, S.buf[1], split + p.nsplit, half);
  uint32_t phase = 0;
  bool ok = true;
  for (long long i = 0; i < n_mine; ++i) {
    if (i + 1 < n_mine) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    before_sync();
    __syncthreads();
    const D2Buf& b = S.buf[i & 1];
    if (tid == 0) {
      after_sync();
#pragma unroll
      for (int k = 0; k < 8; ++k)
        mma_bf16(tmem, smem_desc(smem_u32(b.A) + k * 256, 128, 2048), smem_desc(smem_u32(b.B) + k * 8192, 4096, 128),
                 idesc, (i > 0 || k > 0) ? 1u : 0u);
      mma_commit(mbar);
    }
    ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
    after_sync();
    if (i + 2 < n_mine) d2_load(p, S.buf[i & 1], split + (i + 2) * p.nsplit, half);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok && tid == 0) flag_status(p.status, GS_ERR_TIMEOUT);
  if (ok && n_mine > 0) {
    // row h = 32 (warp % 4) + lane, columns 128 (warp / 4) ..
    const int h = 32 * (warp & 3) + lane, c0 = 128 * (warp >> 2);
    float* dst = p.dW2 + (size_t)h * 512 + 256 * half + c0;
#pragma unroll 1
    for (int c = 0; c < 128; c += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + c), v);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        atomicAdd(reinterpret_cast<float4*>(dst + c + 4 * j), make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

struct DtLayout {
  size_t ht, dy, total;
  long long s_pad;
};

DtLayout dt_layout(long long nsample) {
  DtLayout L;
  L.s_pad = (nsample + kDtS - 1) / kDtS * kDtS;
  L.ht = 0;
  L.dy = align_up((size_t)128 * L.s_pad * 2, 256);
  L.total = L.dy + align_up((size_t)L.s_pad * 512 * 2, 256);
  return L;
}

}  // namespace
}  // namespace gsff

using namespace gsff;

extern "C" size_t gs_decoder_train_tc_workspace_bytes(int64_t nsample) {
  if (nsample <= 0 || nsample > (1ll << 31) / 8) return 0;
  return dt_layout(nsample).total;
}

extern "C" gs_status gs_decoder_train_tc(const gs_decoder* dec, int64_t nsample, int64_t npix, uint64_t seed,
                                         const float* z_map, const float* target, float loss_scale, void* workspace,
                                         size_t workspace_bytes, float* dW1, float* db1, float* dW2, float* db2,
                                         float* dz_map, float* loss_sum, int32_t* status, void* stream) {
  GS_NVTX("gs_decoder_train_tc");
  if (!dec || dec->din != 16 || dec->dh != 128 || dec->dout != 512 || !dec->W1 || !dec->b1 || !dec->W2 || !dec->b2)
    return GS_ERR_UNSUPPORTED;
  if (nsample <= 0 || nsample > (1ll << 31) / 8 || npix <= 0 || npix >= (1ll << 31)) return GS_ERR_INVALID_ARG;
  if (!z_map || !target || !workspace || !dW1 || !db1 || !dW2 || !db2) return GS_ERR_INVALID_ARG;
  if (!aligned(z_map, 16) || !aligned(dz_map, 16) || !aligned(dW1, 16) || !aligned(db1, 16) || !aligned(dW2, 16) ||
      !aligned(workspace, 256))
    return GS_ERR_INVALID_ARG;
  const DtLayout L = dt_layout(nsample);
  if (workspace_bytes < L.total) return GS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem1 = sizeof(DtSmem), smem2 = sizeof(D2Smem);
  static std::atomic<uint64_t> attr_done{0};
  const uint64_t bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    if (cudaFuncSetAttribute(k_decoder_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_decoder_dw2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) != cudaSuccess)
      return GS_ERR_CUDA;
    attr_done.fetch_or(bit);
  }
  char* ws = static_cast<char*>(workspace);
  DtParams p;
  p.nsample = nsample;
  p.npix = npix;
  p.s_pad = L.s_pad;
  p.seed = seed;
  p.scale = loss_scale;
  p.z = z_map;
  p.target = target;
  p.W1 = dec->W1;
  p.b1 = dec->b1;
  p.W2 = dec->W2;
  p.b2 = dec->b2;
  p.dW1 = dW1;
  p.db1 = db1;
  p.db2 = db2;
  p.dz = dz_map;
  p.loss = loss_sum;
  p.HTg = reinterpret_cast<__nv_bfloat16*>(ws + L.ht);
  p.DYg = reinterpret_cast<__nv_bfloat16*>(ws + L.dy);
  p.status = status;
  const long long ntiles = L.s_pad / kDtS;
  {
    GS_TRACE("k_decoder_train_tc", st);
    k_decoder_train_tc<<<(unsigned)(ntiles < sms ? ntiles : sms), kDtThreads, smem1, st>>>(p);
  }
  D2Params q;
  q.ntiles = ntiles;
  q.s_pad = L.s_pad;
  q.nsplit = (int)(ntiles < sms / 2 ? ntiles : sms / 2);
  if (q.nsplit < 1) q.nsplit = 1;
  q.HTg = p.HTg;
  q.DYg = p.DYg;
  q.dW2 = dW2;
  q.status = status;
  {
    GS_TRACE("k_decoder_dw2_tc", st);
    k_decoder_dw2_tc<<<(unsigned)(2 * q.nsplit), kD2Threads, smem2, st>>>(q);
  }
  return last_launch_status();
}
