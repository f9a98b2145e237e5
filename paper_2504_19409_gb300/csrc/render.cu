// Tile compositing (Sec. 3.1, Eq. 2-3) and its reverse-order adjoint.
//
// Both kernels run one 256-thread block per 16x16 tile (one thread per
// pixel) and blockIdx.y over chunks of NC feature channels (chunk 0 also does
// RGB, depth and alpha). Gaussian records of the tile's depth-sorted list
// are staged in shared memory in batches; per-pixel work is SIMT fp32.
//
// Each warp owns an 8x4 (forward) or 8x8 (backward, two pixels per thread)
// block of the tile. A warp skips a Gaussian as a whole when its block lies
// outside a conservative box around the region where that Gaussian's alpha
// can reach 1/255 (warp_skip_extent): the per-pixel decisions are unchanged,
// only work that would be discarded is avoided. The test is taken for all
// warp blocks by the thread that loads the Gaussian into shared memory; a
// warp then walks only the Gaussians whose bit it holds, 32 at a time
// through one ballot.
//
// Forward: early termination is tracked per pixel; a block leaves its list
// as soon as __syncthreads_count sees every pixel done.
//
// Backward: each pixel walks its list from last_idx down, recovers T_i =
// T_{i+1} / (1 - alpha_i) from the saved T_final, and forms the per-pair
// partials of (u, v, A, B, C, opacity, colour, depth, features). With at most
// 16 feature channels each thread owns two pixels (rows r and r+4 of its
// warp's 8x8 block) and sums their partials first, which halves the warp
// reductions per pixel. The per-pixel partials of each Gaussian are then
// summed in two stages before one global atomic per (Gaussian, channel, tile):
//   (1) within a warp by a transpose-reduction -- 32 channel values per lane
//       are halved five times with xor-shuffles (16+8+4+2+1 = 31 shuffles)
//       so that lane l ends up owning the warp sum of channel l;
//   (2) across the warps through shared memory after each batch.

#include <atomic>

#include "gsff_internal.cuh"

namespace gsff {
namespace {

struct FwdParams {
  CamF cam;
  const int2* ranges;
  const int* order;  // launch order of the tiles, or null
  const uint32_t* gids;
  uint8_t* masks;    // per loaded instance: its 8x8-block skip mask (see k_render_bwd_mma), or null
  const float2* uv;
  const float4* co;
  const float* depth;
  const float* colors;
  const void* feats;
  int N, bf16, hwc;
  float bg[3];
  float* out_rgb;
  float* out_depth;
  float* out_alpha;
  float* out_feat;
  float* T_final;
  int* last_idx;
  int* n_contrib;
  uint8_t* visible;  // [P] or null: set to 1 when blended with T > 0.5 in front (Sec. 3.2)
  L1Fwd l1;          // L1 loss against targets, evaluated in the epilogue (N <= 16)
  int P;             // Gaussians (bound of the checked build's id checks)
  int32_t* status;
};


// Pixel layout: each warp owns an 8-wide block of the 16x16 tile, 4*PPT
// rows tall (PPT = pixels per thread, stacked 4 rows apart); warps tile the
// tile 2 across. Compact blocks make the per-warp skip test effective.
template <int PPT>
__device__ __forceinline__ void thread_pixels(int tx, int ty, int (&px)[PPT], int (&py)[PPT]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    px[q] = tx * kTile + (w & 1) * 8 + (lane & 7);
    py[q] = ty * kTile + (w >> 1) * (4 * PPT) + (lane >> 3) + 4 * q;
  }
}

// Half-extents, around (u, v), of a box that holds every pixel centre of a
// warp block that can reach alpha >= 1/255 for this Gaussian. alpha = o G
// with G = exp(power) needs power >= -ln(255 o); at vertical offset dy the
// largest power over dx is -dy^2 det / (2 A) (det = A C - B^2), so the
// region is |dy| <= sqrt(2 ln(255 o) A / det), and |dx| alike with C. The
// extents are widened by 2% + 0.05 px (far beyond fp32 error, so no skip
// decision the exact test would keep is dropped) and by the warp block's
// half-size (hx, hy); nearly singular conics (det < 1e-3 A C) are never
// skipped. A warp block of 8 x 4 PPT pixels has its centre at (4, 2 PPT)
// from its corner, its pixel centres within +-3.5 and +-(2 PPT - 0.5) of it;
// the test of all warp blocks of a tile is taken once per Gaussian when a
// batch is loaded and kept as a bit mask (bit w = warp w's block passes).
__device__ __forceinline__ float2 warp_skip_extent(float4 co, float hx, float hy) {
  const float t = logf(255.f * co.w);
  if (t < 0.f) return make_float2(-1.f, -1.f);  // o < 1/255: never blended
  const float ac = co.x * co.z;
  const float det = ac - co.y * co.y;
  if (!(det > 1e-3f * ac)) return make_float2(3.0e38f, 3.0e38f);
  const float ex = sqrtf(2.f * t * co.z / det), ey = sqrtf(2.f * t * co.x / det);
  return make_float2(ex * 1.02f + 0.05f + hx, ey * 1.02f + 0.05f + hy);
}

// Exact companion of the box test: the smallest value of the quadratic form
// q(dx, dy) = A dx^2 + 2 B dx dy + C dy^2 (= -2 power) over the rectangle
// [x0, x1] x [y0, y1] of offsets (uv minus pixel centre). q is convex, so the
// minimum is 0 when the rectangle holds the origin and otherwise lies on an
// edge, where it is the clamped stationary point of a 1-D parabola.
__device__ __forceinline__ float quad_min_box(float A, float B, float C, float x0, float x1, float y0, float y1) {
  if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return 0.f;
  const float iA = 1.f / A, iC = 1.f / C;
  auto q = [&](float x, float y) { return A * x * x + 2.f * B * x * y + C * y * y; };
  float m = q(x0, fminf(fmaxf(-B * x0 * iC, y0), y1));
  m = fminf(m, q(x1, fminf(fmaxf(-B * x1 * iC, y0), y1)));
  m = fminf(m, q(fminf(fmaxf(-B * y0 * iA, x0), x1), y0));
  m = fminf(m, q(fminf(fmaxf(-B * y1 * iA, x0), x1), y1));
  return m;
}

// Bit mask (bit w = block w may blend the Gaussian) of the NW warp blocks of
// a tile (2 columns x NW/2 rows of 8 x RH pixels) for a Gaussian at u with
// conic/opacity co: the box test, then (EXACT) for blocks that pass it the
// exact test q_min <= 2 ln(255 o) widened by 5 % + 0.1 (far beyond fp32
// error in q and in the exponential, so no pixel that the per-pixel rule
// blends is ever skipped). Nearly singular conics pass (as in the box test).
// The adjoint takes the exact test (a measured 1.8 % gain); in the forward
// its registers cost more occupancy than it saves.
template <int NW, int RH, bool EXACT>
__device__ __forceinline__ uint32_t warp_block_mask(float2 u, float4 co, int tx, int ty) {
  const float2 ext = warp_skip_extent(co, 3.5f, 0.5f * RH - 0.5f);
  const float x0 = (float)(tx * kTile) + 4.f, y0 = (float)(ty * kTile) + 0.5f * RH;
  uint32_t xok = 0, yok = 0;
#pragma unroll
  for (int c = 0; c < 2; ++c) xok |= (fabsf(u.x - (x0 + 8.f * c)) > ext.x ? 0u : 1u) << c;
#pragma unroll
  for (int r = 0; r < NW / 2; ++r) yok |= (fabsf(u.y - (y0 + (float)RH * r)) > ext.y ? 0u : 1u) << r;
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) m |= ((xok >> (w & 1)) & (yok >> (w >> 1)) & 1u) << w;
  if (!EXACT) return m;
  const float ac = co.x * co.z;
  if (m == 0 || !(ac - co.y * co.y > 1e-3f * ac)) return m;
  const float thr = 2.f * logf(255.f * co.w) * 1.05f + 0.1f;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    if (!((m >> w) & 1u)) continue;
    // pixel centres of block w: x in [xb + 0.5, xb + 7.5], y in [yb + 0.5, yb + RH - 0.5]
    const float xb = (float)(tx * kTile + (w & 1) * 8), yb = (float)(ty * kTile + (w >> 1) * RH);
    const float qmin = quad_min_box(co.x, co.y, co.z, u.x - (xb + 7.5f), u.x - (xb + 0.5f), u.y - (yb + RH - 0.5f),
                                    u.y - (yb + 0.5f));
    if (qmin > thr) m &= ~(1u << w);
  }
  return m;
}


template <int NC>
__device__ __forceinline__ void load_feat_row(const void* feats, int bf16, int N, uint32_t g, int c0,
                                              float* __restrict__ dst) {
  const int nch = min(NC, N - c0);
  if (!bf16) {
    const float* src = static_cast<const float*>(feats) + (size_t)g * N + c0;
    if ((N & 3) == 0 && nch == NC) {
#pragma unroll
      for (int c = 0; c < NC; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(src + c);
        dst[c] = v.x; dst[c + 1] = v.y; dst[c + 2] = v.z; dst[c + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) dst[c] = c < nch ? src[c] : 0.f;
    }
  } else {
    const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(feats) + (size_t)g * N + c0;
    if ((N & 7) == 0 && nch == NC) {
#pragma unroll
      for (int c = 0; c < NC; c += 8) {
        const uint4 raw = *reinterpret_cast<const uint4*>(src + c);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(h[e]);
          dst[c + 2 * e] = f.x;
          dst[c + 2 * e + 1] = f.y;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) dst[c] = c < nch ? __bfloat162float(src[c]) : 0.f;
    }
  }
}

template <int NC, bool VIS>
__global__ void __launch_bounds__(kTilePix) k_render_fwd(const FwdParams p) {
  pdl_wait();
  pdl_trigger();
  constexpr int NCs = NC > 0 ? NC : 1;
  static_assert(NC % 2 == 0, "channels are blended in pairs");
  __shared__ float2 s_uv[kTilePix];
  __shared__ uint8_t s_wmask[kTilePix];  // bit w: warp w's pixel block passes the skip test
  __shared__ float4 s_co[kTilePix];
  __shared__ float4 s_cd[kTilePix];
  __shared__ float s_f[kTilePix][NCs];
  __shared__ uint32_t s_gid[VIS ? kTilePix : 1];
  __shared__ float s_lsum;

  const int tile = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const int chunk = blockIdx.y;
  const bool geom = chunk == 0;
  const bool mark = VIS && geom;
  if (threadIdx.x == 0) s_lsum = 0.f;
  const unsigned lanes_below = (1u << (threadIdx.x & 31)) - 1u;
  const int c0 = chunk * NC;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  int pxa[1], pya[1];
  thread_pixels<1>(tx, ty, pxa, pya);
  const int px = pxa[0], py = pya[0];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool inside = px < p.cam.W && py < p.cam.H;
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const int2 rg = p.ranges[tile];

  float T = 1.f;
  float ac0 = 0.f, ac1 = 0.f, ac2 = 0.f, ad = 0.f;
  float af[NCs];
#pragma unroll
  for (int c = 0; c < NCs; ++c) af[c] = 0.f;
  int last = 0, cnt = 0;
  bool done = !inside;

  for (int start = rg.x; start < rg.y; start += kTilePix) {
    if (__syncthreads_count(done) == kTilePix) break;
    const int idx = start + threadIdx.x;
    if (idx < rg.y) {
      const uint32_t g = checked_id(p.gids[idx], p.P, p.status);
      const float4 co = p.co[g];
      const float2 u = p.uv[g];
      s_uv[threadIdx.x] = u;
      s_co[threadIdx.x] = conic_q(co);  // the walk's alphas take the base-2 form
      // the skip tests of all 8 warp blocks (2 columns x 4 rows of 8x4 pixels)
      s_wmask[threadIdx.x] = (uint8_t)warp_block_mask<8, 4, false>(u, co, tx, ty);
      if (geom && p.masks) p.masks[idx] = (uint8_t)warp_block_mask<4, 8, true>(u, co, tx, ty);
      if (VIS) s_gid[threadIdx.x] = g;
      if (geom) s_cd[threadIdx.x] = make_float4(p.colors[3 * g], p.colors[3 * g + 1], p.colors[3 * g + 2], p.depth[g]);
      if (NC > 0) load_feat_row<NCs>(p.feats, p.bf16, p.N, g, c0, s_f[threadIdx.x]);
    }
    __syncthreads();
    const int n = min(kTilePix, rg.y - start);
    // this warp's Gaussians of the batch, 32 at a time, in list order
    for (int base = 0; base < n; base += 32) {
      if (__all_sync(0xffffffffu, done)) break;
      const int jj = base + lane;
      uint32_t bits = __ballot_sync(0xffffffffu, jj < n && ((s_wmask[jj] >> wid) & 1u));
      while (bits) {
        const int j = base + __ffs(bits) - 1;
        bits &= bits - 1u;
        if (done) continue;
        const float2 uj = s_uv[j];
        PairAlpha pa;
        if (!pair_alpha_q(s_co[j], uj.x - pxc, uj.y - pyc, pa)) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, pa.alpha));
        if (Tn < kTStop) {
          done = true;
          continue;
        }
        const float w = __fmul_rn(pa.alpha, T);
        if (mark && T > 0.5f) {
          // visible (T in front > 0.5): the lowest lane of those here writes
          if ((__activemask() & lanes_below) == 0) p.visible[s_gid[j]] = 1;
        }
        // packed two-lane FMAs (each lane rounds as fmaf): half the issue slots
        const float2 w2 = make_float2(w, w);
        if (geom) {
          const float4 cd = s_cd[j];
          const float2 a01 = __ffma2_rn(w2, make_float2(cd.x, cd.y), make_float2(ac0, ac1));
          const float2 a23 = __ffma2_rn(w2, make_float2(cd.z, cd.w), make_float2(ac2, ad));
          ac0 = a01.x, ac1 = a01.y, ac2 = a23.x, ad = a23.y;
        }
#pragma unroll
        for (int c = 0; c < NC; c += 2) {
          const float2 f = __ffma2_rn(w2, make_float2(s_f[j][c], s_f[j][c + 1]), make_float2(af[c], af[c + 1]));
          af[c] = f.x, af[c + 1] = f.y;
        }
        T = Tn;
        last = start + j + 1 - rg.x;
        ++cnt;
      }
    }
  }
  const size_t HW = (size_t)p.cam.W * p.cam.H;
  const size_t pix = inside ? (size_t)py * p.cam.W + px : 0;
  float lsum = 0.f;
  if (inside) {
    const float r0 = ac0 + T * p.bg[0], r1 = ac1 + T * p.bg[1], r2 = ac2 + T * p.bg[2];
    if (geom) {
      p.out_rgb[pix] = r0;
      p.out_rgb[HW + pix] = r1;
      p.out_rgb[2 * HW + pix] = r2;
      p.out_depth[pix] = ad;
      p.out_alpha[pix] = 1.f - T;
      p.T_final[pix] = T;
      p.last_idx[pix] = last;
      p.n_contrib[pix] = cnt;
    }
    if (NC > 0) {
      const int nch = min(NC, p.N - c0);
      if (p.hwc) {
        float* dst = p.out_feat + pix * p.N + c0;
        if ((p.N & 3) == 0 && nch == NC) {
#pragma unroll
          for (int c = 0; c < NCs; c += 4) *reinterpret_cast<float4*>(dst + c) = make_float4(af[c], af[c + 1], af[c + 2], af[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < NCs; ++c)
            if (c < nch) dst[c] = af[c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < NCs; ++c)
          if (c < nch) p.out_feat[(size_t)(c0 + c) * HW + pix] = af[c];
      }
    }
    if (p.l1.on) {
      // L1 terms of this pixel; cotangent signs as bits (see L1Fwd)
      uint32_t nz = 0, ng = 0;
      auto term = [&](float pred, float target, float w, int bit) {
        const float d = pred - target;
        lsum += w * fabsf(d);
        nz |= (d != 0.f ? 1u : 0u) << bit;
        ng |= (d < 0.f ? 1u : 0u) << bit;
      };
      if (p.l1.target[0]) {
        term(r0, p.l1.target[0][pix], p.l1.w[0], kL1BitRgb);
        term(r1, p.l1.target[0][HW + pix], p.l1.w[0], kL1BitRgb + 1);
        term(r2, p.l1.target[0][2 * HW + pix], p.l1.w[0], kL1BitRgb + 2);
      }
      if (p.l1.target[1]) term(ad, p.l1.target[1][pix], p.l1.w[1], kL1BitDepth);
      if (NC > 0 && p.l1.target[2]) {
        const int nch = min(NC, p.N);
#pragma unroll
        for (int c = 0; c < NCs; ++c)
          if (c < nch) term(af[c], p.l1.target[2][p.hwc ? pix * p.N + c : (size_t)c * HW + pix], p.l1.w[2], c);
      }
      p.l1.signs[pix] = make_uint2(nz, ng);
    }
  }
  if (p.l1.on && p.l1.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(&s_lsum, lsum);
    __syncthreads();
    if (threadIdx.x == 0 && s_lsum != 0.f) atomicAdd(p.l1.loss, s_lsum);
  }
}

// ---------------------------------------------------------------------------
// Forward compositing with two pixels per thread (N <= 16): 128 threads per
// tile, each warp owning an 8 x 8 pixel block and each thread two pixels of
// one column, 4 rows apart. Per pixel the operations and their order are
// those of k_render_fwd (identical bits); what the two pixels share is done
// once: the Gaussian's records, its skip bit, its dx and q.x dx, and the
// alpha arithmetic runs on packed two-lane fp32 operands.
constexpr int kFwd2Threads = kTilePix / 2;

template <int NC, bool VIS>
__global__ void __launch_bounds__(kFwd2Threads, 5) k_render_fwd2(const FwdParams p) {
  pdl_wait();
  pdl_trigger();
  constexpr int NCs = NC > 0 ? NC : 2;
  constexpr int kB = 2 * kFwd2Threads;  // Gaussians per shared-memory batch
  static_assert(NC % 2 == 0 && NC <= 16, "channels are blended in pairs; one 16-channel chunk");
  __shared__ float2 s_uv[kB];
  __shared__ uint8_t s_wmask[kB];  // bit w: warp w's pixel block passes the skip test
  __shared__ float4 s_co[kB];
  __shared__ float4 s_cd[kB];
  __shared__ __align__(16) float s_f[kB][NCs];
  __shared__ uint32_t s_gid[VIS ? kB : 1];
  __shared__ float s_lsum;

  const int tile = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  if (threadIdx.x == 0) s_lsum = 0.f;
  const unsigned lanes_below = (1u << (threadIdx.x & 31)) - 1u;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  int px[2], py[2];
  thread_pixels<2>(tx, ty, px, py);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float pxc = (float)px[0] + 0.5f;  // both pixels lie in one column
  const float2 npy2 = make_float2(-((float)py[0] + 0.5f), -((float)py[1] + 0.5f));
  const int2 rg = p.ranges[tile];

  float T[2] = {1.f, 1.f};
  float ac[2][4];
  float af[2][NCs];
  int last[2] = {0, 0}, cnt[2] = {0, 0};
  bool done[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    done[q] = !(px[q] < p.cam.W && py[q] < p.cam.H);
    ac[q][0] = ac[q][1] = ac[q][2] = ac[q][3] = 0.f;
#pragma unroll
    for (int c = 0; c < NCs; ++c) af[q][c] = 0.f;
  }

  for (int start = rg.x; start < rg.y; start += kB) {
    if (__syncthreads_count(done[0] && done[1]) == kFwd2Threads) break;
#pragma unroll
    for (int i = threadIdx.x; i < kB; i += kFwd2Threads) {
      const int idx = start + i;
      if (idx < rg.y) {
        const uint32_t g = checked_id(p.gids[idx], p.P, p.status);
        const float4 co = p.co[g];
        const float2 u = p.uv[g];
        s_uv[i] = u;
        s_co[i] = conic_q(co);
        s_wmask[i] = (uint8_t)warp_block_mask<4, 8, true>(u, co, tx, ty);
        if (p.masks) p.masks[idx] = s_wmask[i];
        if (VIS) s_gid[i] = g;
        s_cd[i] = make_float4(p.colors[3 * g], p.colors[3 * g + 1], p.colors[3 * g + 2], p.depth[g]);
        if (NC > 0) load_feat_row<NCs>(p.feats, p.bf16, p.N, g, 0, s_f[i]);
      }
    }
    __syncthreads();
    const int n = min(kB, rg.y - start);
    for (int base = 0; base < n; base += 32) {
      if (__all_sync(0xffffffffu, done[0] && done[1])) break;
      const int jj = base + lane;
      uint32_t bits = __ballot_sync(0xffffffffu, jj < n && ((s_wmask[jj] >> wid) & 1u));
      // two Gaussians per iteration: their alphas first (four independent
      // chains), then the blends in list order
      while (bits) {
        const int j1 = base + __ffs(bits) - 1;
        bits &= bits - 1u;
        const bool two = bits != 0;
        const int j2 = two ? base + __ffs(bits) - 1 : j1;
        if (two) bits &= bits - 1u;
        if (done[0] && done[1]) continue;
        const int jg[2] = {j1, j2};
        float2 ea[2], aa[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          // pair_alpha_q for both pixels (dx is shared)
          const float2 uj = s_uv[jg[k]];
          const float4 qc = s_co[jg[k]];
          const float dx = __fsub_rn(uj.x, pxc);
          const float2 dy = __fadd2_rn(make_float2(uj.y, uj.y), npy2);
          const float qxdx = __fmul_rn(qc.x, dx);
          const float2 u = __ffma2_rn(make_float2(qc.y, qc.y), dy, make_float2(qxdx, qxdx));
          ea[k] = __ffma2_rn(make_float2(dx, dx), u, __fmul2_rn(__fmul2_rn(make_float2(qc.z, qc.z), dy), dy));
          aa[k] = __fmul2_rn(make_float2(qc.w, qc.w), make_float2(ex2_approx(ea[k].x), ex2_approx(ea[k].y)));
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (k == 1 && !two) break;
          const int j = jg[k];
          const float ev[2] = {ea[k].x, ea[k].y}, av[2] = {aa[k].x, aa[k].y};
          bool bl[2];
          float w[2], Tn[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float alpha = av[q] > kAlphaMax ? kAlphaMax : av[q];
            bl[q] = !done[q] && !(ev[q] > 0.f) && alpha >= kAlphaMin;
            Tn[q] = __fmul_rn(T[q], __fsub_rn(1.f, alpha));
            if (bl[q] && Tn[q] < kTStop) {
              done[q] = true;
              bl[q] = false;
            }
            w[q] = __fmul_rn(alpha, T[q]);
          }
          if (!(bl[0] || bl[1])) continue;
          if (VIS && ((bl[0] && T[0] > 0.5f) || (bl[1] && T[1] > 0.5f))) {
            // visible (T in front > 0.5): the lowest lane of those here writes
            if ((__activemask() & lanes_below) == 0) p.visible[s_gid[j]] = 1;
          }
          // packed two-lane FMAs over channel pairs (each lane rounds as
          // fmaf); a pixel that does not blend this Gaussian skips its updates
          const float2 w20 = make_float2(w[0], w[0]), w21 = make_float2(w[1], w[1]);
          {
            const float4 cd = s_cd[j];
            if (bl[0]) {
              const float2 a01 = __ffma2_rn(w20, make_float2(cd.x, cd.y), make_float2(ac[0][0], ac[0][1]));
              const float2 a23 = __ffma2_rn(w20, make_float2(cd.z, cd.w), make_float2(ac[0][2], ac[0][3]));
              ac[0][0] = a01.x, ac[0][1] = a01.y, ac[0][2] = a23.x, ac[0][3] = a23.y;
            }
            if (bl[1]) {
              const float2 a01 = __ffma2_rn(w21, make_float2(cd.x, cd.y), make_float2(ac[1][0], ac[1][1]));
              const float2 a23 = __ffma2_rn(w21, make_float2(cd.z, cd.w), make_float2(ac[1][2], ac[1][3]));
              ac[1][0] = a01.x, ac[1][1] = a01.y, ac[1][2] = a23.x, ac[1][3] = a23.y;
            }
          }
#pragma unroll
          for (int c = 0; c < NC; c += 4) {
            const float4 v = *reinterpret_cast<const float4*>(&s_f[j][c]);
            if (bl[0]) {
              const float2 r0 = __ffma2_rn(w20, make_float2(v.x, v.y), make_float2(af[0][c], af[0][c + 1]));
              const float2 r1 = __ffma2_rn(w20, make_float2(v.z, v.w), make_float2(af[0][c + 2], af[0][c + 3]));
              af[0][c] = r0.x, af[0][c + 1] = r0.y, af[0][c + 2] = r1.x, af[0][c + 3] = r1.y;
            }
            if (bl[1]) {
              const float2 r0 = __ffma2_rn(w21, make_float2(v.x, v.y), make_float2(af[1][c], af[1][c + 1]));
              const float2 r1 = __ffma2_rn(w21, make_float2(v.z, v.w), make_float2(af[1][c + 2], af[1][c + 3]));
              af[1][c] = r0.x, af[1][c + 1] = r0.y, af[1][c + 2] = r1.x, af[1][c + 3] = r1.y;
            }
          }
          const int pos = start + j + 1 - rg.x;
#pragma unroll
          for (int q = 0; q < 2; ++q)
            if (bl[q]) {
              T[q] = Tn[q];
              last[q] = pos;
              ++cnt[q];
            }
        }
      }
    }
  }
  const size_t HW = (size_t)p.cam.W * p.cam.H;
  float lsum = 0.f;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!(px[q] < p.cam.W && py[q] < p.cam.H)) continue;
    const size_t pix = (size_t)py[q] * p.cam.W + px[q];
    const float r0 = ac[q][0] + T[q] * p.bg[0], r1 = ac[q][1] + T[q] * p.bg[1], r2 = ac[q][2] + T[q] * p.bg[2];
    p.out_rgb[pix] = r0;
    p.out_rgb[HW + pix] = r1;
    p.out_rgb[2 * HW + pix] = r2;
    p.out_depth[pix] = ac[q][3];
    p.out_alpha[pix] = 1.f - T[q];
    p.T_final[pix] = T[q];
    p.last_idx[pix] = last[q];
    p.n_contrib[pix] = cnt[q];
    if (NC > 0) {
      const int nch = min(NC, p.N);
      if (p.hwc) {
        float* dst = p.out_feat + pix * p.N;
        if ((p.N & 3) == 0 && nch == NC) {
#pragma unroll
          for (int c = 0; c < NCs; c += 4)
            *reinterpret_cast<float4*>(dst + c) = make_float4(af[q][c], af[q][c + 1], af[q][c + 2], af[q][c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < NCs; ++c)
            if (c < nch) dst[c] = af[q][c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < NCs; ++c)
          if (c < nch) p.out_feat[(size_t)c * HW + pix] = af[q][c];
      }
    }
    if (p.l1.on) {
      uint32_t nz = 0, ng = 0;
      auto term = [&](float pred, float target, float wt, int bit) {
        const float d = pred - target;
        lsum += wt * fabsf(d);
        nz |= (d != 0.f ? 1u : 0u) << bit;
        ng |= (d < 0.f ? 1u : 0u) << bit;
      };
      if (p.l1.target[0]) {
        term(r0, p.l1.target[0][pix], p.l1.w[0], kL1BitRgb);
        term(r1, p.l1.target[0][HW + pix], p.l1.w[0], kL1BitRgb + 1);
        term(r2, p.l1.target[0][2 * HW + pix], p.l1.w[0], kL1BitRgb + 2);
      }
      if (p.l1.target[1]) term(ac[q][3], p.l1.target[1][pix], p.l1.w[1], kL1BitDepth);
      if (NC > 0 && p.l1.target[2]) {
        const int nch = min(NC, p.N);
#pragma unroll
        for (int c = 0; c < NCs; ++c)
          if (c < nch) term(af[q][c], p.l1.target[2][p.hwc ? pix * p.N + c : (size_t)c * HW + pix], p.l1.w[2], c);
      }
      p.l1.signs[pix] = make_uint2(nz, ng);
    }
  }
  if (p.l1.on && p.l1.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(&s_lsum, lsum);
    __syncthreads();
    if (threadIdx.x == 0 && s_lsum != 0.f) atomicAdd(p.l1.loss, s_lsum);
  }
}

// ---------------------------------------------------------------------------
struct BwdParams {
  CamF cam;
  const int2* ranges;
  const int* order;  // launch order of the tiles, or null
  const uint32_t* gids;
  const uint8_t* masks;  // the forward's per-instance 8x8-block skip masks, or null (recomputed)
  const float2* uv;
  const float4* co;
  const float* depth;
  const float* colors;
  const void* feats;
  int N, bf16, hwc;
  float bg[3];
  const float* T_final;
  const int* last_idx;
  const float* g_rgb;
  const float* g_depth;
  const float* g_alpha;
  const float* g_feat;
  float* d_uv;
  float* d_conic;
  float* d_depth;
  float* d_opacity;
  float* d_colors;
  float* d_feats;
  L1Bwd l1;  // cotangents rebuilt from the forward's L1 sign bits (tensor-core adjoint only)
  int P;     // Gaussians (bound of the checked build's id checks)
  int32_t* status;
  // per-pair saved state (k_render_bwd<..., STORED>): pixel q's pairs are
  // [pair_off[q], pair_off[q + 1]) of pair_T, the transmittance in front of
  // each blended Gaussian in list order
  const long long* pair_off;
  const float* pair_T;
};

// Lane l ends up with the warp-wide sum of v[l] (see the file comment).
__device__ __forceinline__ float transpose_reduce32(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const float send = upper ? v[k] : v[k + s];
      const float keep = upper ? v[k + s] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

constexpr int kGeomCh = 10;  // u, v, A, B, C, opacity, r, g, b, depth

template <int NC>
struct BwdShape {
  static constexpr int CH = kGeomCh + NC;
  static constexpr int CHP = (CH + 31) / 32 * 32;
};

// PPT pixels per thread (1 or 2); kTilePix / PPT threads per tile block.
// STORED: the transmittance in front of each blended Gaussian is read from the
// per-pair saved state instead of being recovered as T_{i+1} / (1 - alpha_i).
template <int NC, bool COUPLED, int PPT, bool STORED = false>
__global__ void __launch_bounds__(kTilePix / PPT, (PPT == 2) ? 4 : ((NC > 16 || COUPLED) ? 2 : 3))
    k_render_bwd(const BwdParams p) {
  using S = BwdShape<NC>;
  constexpr int CH = S::CH, CHP = S::CHP;
  constexpr int NT = kTilePix / PPT, NW = NT / 32;
  constexpr int BB = (8192 / (NW * CHP)) < 64 ? (8192 / (NW * CHP)) : 64;  // batch: 32 KB of partials
  constexpr int NCs = NC > 0 ? NC : 1;
  constexpr int NFs = (COUPLED && NC > 0) ? NC : 1;
  __shared__ float s_red[NW][BB][CHP];
  __shared__ float2 s_uv[BB];
  __shared__ uint8_t s_wmask[BB];  // bit w: warp w's pixel block passes the skip test
  __shared__ float4 s_co[BB];
  __shared__ float4 s_cd[BB];
  __shared__ float s_f[BB][NFs];
  __shared__ uint32_t s_gid[BB];
  __shared__ int s_maxlast;

  const int tile = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const int chunk = blockIdx.y;
  const bool geom = chunk == 0;
  const int c0 = chunk * NC;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  int px[PPT], py[PPT];
  thread_pixels<PPT>(tx, ty, px, py);
  const int2 rg = p.ranges[tile];
  const size_t HW = (size_t)p.cam.W * p.cam.H;

  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  float T[PPT], pxc[PPT], pyc[PPT], gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], gA[PPT], bgdot[PPT];
  float Bc0[PPT], Bc1[PPT], Bc2[PPT], Bd[PPT], Sx[PPT];
  float gF[PPT][NCs], Bf[PPT][NFs];
  int last[PPT];
  long long pt[PPT];  // STORED: the pixel's next saved pair, walking backwards
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const bool inside = px[q] < p.cam.W && py[q] < p.cam.H;
    const size_t pix = inside ? (size_t)py[q] * p.cam.W + px[q] : 0;
    pxc[q] = (float)px[q] + 0.5f;
    pyc[q] = (float)py[q] + 0.5f;
    T[q] = 1.f;
    last[q] = 0;
    gC0[q] = gC1[q] = gC2[q] = gD[q] = gA[q] = 0.f;
    Bc0[q] = Bc1[q] = Bc2[q] = Bd[q] = 0.f;
    Sx[q] = 1.f;
#pragma unroll
    for (int c = 0; c < NCs; ++c) gF[q][c] = 0.f;
#pragma unroll
    for (int c = 0; c < NFs; ++c) Bf[q][c] = 0.f;
    pt[q] = 0;
    if (inside) {
      T[q] = p.T_final[pix];
      last[q] = p.last_idx[pix];
      if (STORED) pt[q] = p.pair_off[pix + 1] - 1;
      if (p.g_rgb) {
        gC0[q] = p.g_rgb[pix];
        gC1[q] = p.g_rgb[HW + pix];
        gC2[q] = p.g_rgb[2 * HW + pix];
      }
      if (p.g_depth) gD[q] = p.g_depth[pix];
      if (p.g_alpha) gA[q] = p.g_alpha[pix];
      if (NC > 0 && p.g_feat) {
        const int nch = min(NC, p.N - c0);
#pragma unroll
        for (int c = 0; c < NCs; ++c)
          if (c < nch) gF[q][c] = p.hwc ? p.g_feat[pix * p.N + c0 + c] : p.g_feat[(size_t)(c0 + c) * HW + pix];
      }
      if (last[q] > 0) atomicMax(&s_maxlast, last[q]);
    }
    bgdot[q] = p.bg[0] * gC0[q] + p.bg[1] * gC1[q] + p.bg[2] * gC2[q];
  }
  __syncthreads();
  const int maxlast = checked_len(s_maxlast, rg.y - rg.x, p.status);

  for (int hi = rg.x + maxlast; hi > rg.x; hi -= BB) {
    const int lo = max(rg.x, hi - BB);
    const int n = hi - lo;
    if ((int)threadIdx.x < n) {
      const uint32_t g = checked_id(p.gids[lo + threadIdx.x], p.P, p.status);
      const float4 co = p.co[g];
      const float2 u = p.uv[g];
      s_gid[threadIdx.x] = g;
      s_uv[threadIdx.x] = u;
      s_co[threadIdx.x] = co;
      // the skip tests of all NW warp blocks (2 columns x NW/2 rows of 8 x 4 PPT pixels)
      s_wmask[threadIdx.x] = (uint8_t)warp_block_mask<NW, 4 * PPT, true>(u, co, tx, ty);
      if (geom) s_cd[threadIdx.x] = make_float4(p.colors[3 * g], p.colors[3 * g + 1], p.colors[3 * g + 2], p.depth[g]);
      if (COUPLED && NC > 0) load_feat_row<NFs>(p.feats, p.bf16, p.N, g, c0, s_f[threadIdx.x]);
    }
    __syncthreads();
    // this warp's Gaussians of the batch, 32 at a time, in reverse list order
    for (int base = ((n - 1) >> 5) << 5; base >= 0; base -= 32) {
    const int jj = base + lane;
    uint32_t bits = __ballot_sync(0xffffffffu, jj < n && ((s_wmask[jj] >> wid) & 1u));
    while (bits) {
      const int jb = 31 - __clz(bits);
      bits &= ~(1u << jb);
      const int j = base + jb;
      const int pos = lo + j - rg.x;
      const float2 uj = s_uv[j];
      const float4 cj = s_co[j];
      float v[CHP];
#pragma unroll
      for (int c = 0; c < CHP; ++c) v[c] = 0.f;
      bool any = false;
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        PairAlpha pa;
        const float dx = uj.x - pxc[q], dy = uj.y - pyc[q];
        if (!(pos < last[q] && pair_alpha(cj, dx, dy, pa))) continue;
        any = true;
        const float om = 1.f - pa.alpha;
        if (STORED) T[q] = p.pair_T[pt[q]--];
        else T[q] = __fdividef(T[q], om);
        const float w = pa.alpha * T[q];
        float da = 0.f;
        if (geom) {
          const float4 cd = s_cd[j];
          da = T[q] * ((cd.x - Bc0[q]) * gC0[q] + (cd.y - Bc1[q]) * gC1[q] + (cd.z - Bc2[q]) * gC2[q] +
                       (cd.w - Bd[q]) * gD[q]) +
               T[q] * Sx[q] * (gA[q] - bgdot[q]);
          Bc0[q] = pa.alpha * cd.x + om * Bc0[q];
          Bc1[q] = pa.alpha * cd.y + om * Bc1[q];
          Bc2[q] = pa.alpha * cd.z + om * Bc2[q];
          Bd[q] = pa.alpha * cd.w + om * Bd[q];
          Sx[q] *= om;
          v[6] += w * gC0[q];
          v[7] += w * gC1[q];
          v[8] += w * gC2[q];
          v[9] += w * gD[q];
        }
        if (COUPLED && NC > 0) {
          float daf = 0.f;
#pragma unroll
          for (int c = 0; c < NFs; ++c) {
            daf += (s_f[j][c] - Bf[q][c]) * gF[q][c];
            Bf[q][c] = pa.alpha * s_f[j][c] + om * Bf[q][c];
          }
          da += T[q] * daf;
        }
        if ((geom || COUPLED) && !pa.clamped) {
          v[5] += da * pa.G;
          const float dp = da * pa.alpha;
          v[2] += -0.5f * dx * dx * dp;
          v[3] += -dx * dy * dp;
          v[4] += -0.5f * dy * dy * dp;
          v[0] += -(cj.x * dx + cj.y * dy) * dp;
          v[1] += -(cj.y * dx + cj.z * dy) * dp;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) v[kGeomCh + c] += w * gF[q][c];
      }
      if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int r = 0; r < CHP / 32; ++r) {
          float part[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) part[c] = v[32 * r + c];
          s_red[wid][j][32 * r + lane] = transpose_reduce32(part);
        }
      } else {
#pragma unroll
        for (int r = 0; r < CHP / 32; ++r) s_red[wid][j][32 * r + lane] = 0.f;
      }
    }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * CH; e += NT) {
      const int j = e / CH, ch = e - j * CH;
      const uint32_t wm = s_wmask[j];  // rows of warps that skipped j were not written
      float sum = 0.f;
#pragma unroll
      for (int w8 = 0; w8 < NW; ++w8)
        if ((wm >> w8) & 1u) sum += s_red[w8][j][ch];
      if (sum == 0.f) continue;
      const uint32_t g = s_gid[j];
      float* dst;
      if (ch < 2) dst = p.d_uv + 2 * (size_t)g + ch;
      else if (ch < 5) dst = p.d_conic + 3 * (size_t)g + (ch - 2);
      else if (ch == 5) {
        if (!p.d_opacity) continue;
        dst = p.d_opacity + g;
      } else if (ch < 9) {
        if (!p.d_colors) continue;
        dst = p.d_colors + 3 * (size_t)g + (ch - 6);
      } else if (ch == 9) dst = p.d_depth + g;
      else {
        const int c = c0 + ch - kGeomCh;
        if (c >= p.N) continue;
        dst = p.d_feats + (size_t)g * p.N + c;
      }
      atomicAdd(dst, sum);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Adjoint with the pixel sums on tensor cores (decoupled features, N <= 64:
// above 16 channels one block per tile and 16-channel chunk, chunk 0 also
// doing the geometry; the coupled and wider forms use k_render_bwd above).
//
// A Gaussian's colour, depth and feature gradients over a tile are
// sum_p w_p g_p[c] (w = alpha T, g the pixel's cotangent): for a warp, a
// [Gaussians x 64 pixels] . [64 pixels x channels] contraction. Its u, v,
// conic and opacity gradients need sum_p dp m(x, y) for the pixel monomials
// m = 1, x, y, x^2, xy, y^2 relative to the warp block's centre (dp =
// dL/dalpha alpha): the same contraction of dp against a constant monomial
// operand, exact in bf16. The walk stores w (rows 0-7) and dp (rows 8-15) of
// 8 Gaussians in a 16 x 64 tile, and then the warp multiplies it with
// mma.sync (bf16; W and dp split into hi + lo, G into hi + lo, or G = the
// exact signs +-1 with the L1 weight applied after the sum). This replaces,
// per Gaussian and warp, 20 multiply-adds per pixel, the per-pixel partial
// products of the geometry and a 32-channel transposition.
namespace mma_bwd {
constexpr int kBB = 32;           // Gaussians per shared-memory batch
constexpr int kRows = 16;         // rows of a warp's contraction tile (MMA M)
constexpr int kGRows = 8;         // Gaussians per contraction: w in rows 0..7, dp in rows 8..15
constexpr int kWStride = 72;      // bf16 per W row: 64 pixels + 8 (rows 144 B apart: conflict-free ldmatrix)
constexpr int kNW = 4;            // warps (8 x 8 pixel blocks) per tile
constexpr int kThreads = 32 * kNW;
constexpr int kGeo = 6;           // geometric sums: dp, dx dp, dy dp, dx^2 dp, dx dy dp, dy^2 dp
constexpr int kNBuf = 3;          // batch buffers: walked, being staged, still named by the last batch's sums
}  // namespace mma_bwd

// One batch of a tile's list in shared memory.
struct BwdBatch {
  float4 co[mma_bwd::kBB];  // conic A, B, C and opacity
  float4 q[mma_bwd::kBB];   // the same in base-2 form (conic_q)
  float4 cd[mma_bwd::kBB];  // colour r, g, b and depth
  float2 uv[mma_bwd::kBB];
  uint32_t gid[mma_bwd::kBB];
  uint8_t wmask[mma_bwd::kBB];  // bit w: warp w's pixel block passes the skip test
};

template <int NC>
struct MmaBwdShape {
  static constexpr int NCH = NC + 4;          // contracted channels: features, r, g, b, depth
  static constexpr int NT = (NCH + 7) / 8;    // n-tiles of 8 channels
  static constexpr int NG = NC / 4 + 1;       // output groups: features by 4, then r, g, b, depth
  static constexpr int SR = NCH + mma_bwd::kGeo + 2;  // per (warp, Gaussian) sums: NCH channels, the six geometric, pad
  static constexpr size_t kWBytes = (size_t)mma_bwd::kNW * mma_bwd::kRows * mma_bwd::kWStride * 2;
  static constexpr size_t kRedBytes = (size_t)2 * mma_bwd::kNW * mma_bwd::kBB * SR * 4;
  static constexpr size_t kSmem = 2 * kWBytes + kRedBytes;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void mma_bf16_m16n8k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// L1 cotangent w sign(...) of bit b of a pixel's sign words (see L1Fwd).
__device__ __forceinline__ float l1_cot(uint2 sg, int b, float w) {
  return ((sg.x >> b) & 1u) ? (((sg.y >> b) & 1u) ? -w : w) : 0.f;
}

// (x0, x1) -> bf16x2 hi and lo parts (x0 in the low half): x = hi + lo + O(2^-16 x).
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Starts the copies of Gaussian g's record into slot i of a batch.
__device__ __forceinline__ void stage_batch(const BwdParams& p, BwdBatch& b, int i, uint32_t g) {
  b.gid[i] = g;
  cp_async16(&b.co[i], p.co + g);
  cp_async8(&b.uv[i], p.uv + g);
  float* cd = reinterpret_cast<float*>(&b.cd[i]);
  cp_async4(cd + 0, p.colors + 3 * (size_t)g);
  cp_async4(cd + 1, p.colors + 3 * (size_t)g + 1);
  cp_async4(cd + 2, p.colors + 3 * (size_t)g + 2);
  cp_async4(cd + 3, p.depth + g);
}

// After the slot's copies landed: the base-2 conic and, without the forward's
// stored masks, the warp skip tests of its Gaussian.
__device__ __forceinline__ void finish_batch(BwdBatch& b, int i, int tx, int ty, bool stored) {
  if (!stored) b.wmask[i] = (uint8_t)warp_block_mask<mma_bwd::kNW, 8, true>(b.uv[i], b.co[i], tx, ty);
  b.q[i] = conic_q(b.co[i]);
}

// L1: the cotangents are w sign(...) from the forward's sign words (p.l1); the
// cotangent operand is then the exact signs (bf16 +-1, 0) and each sum is
// scaled by its class weight at the end, so W . G takes two products.
template <int NC, bool L1>
__global__ void __launch_bounds__(mma_bwd::kThreads, 4) k_render_bwd_mma(const BwdParams p) {
  pdl_wait();
  pdl_trigger();
  using namespace mma_bwd;
  using S = MmaBwdShape<NC>;
  constexpr int NT = S::NT, SR = S::SR, NCH = S::NCH, NG = S::NG;
  static_assert(NC % 4 == 0 && SR % 4 == 0, "16-byte groups of per-warp sums");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __nv_bfloat16* s_wh = reinterpret_cast<__nv_bfloat16*>(smem_raw);                   // [kNW][kRows][kWStride]
  __nv_bfloat16* s_wl = reinterpret_cast<__nv_bfloat16*>(smem_raw + S::kWBytes);      // same
  float* s_red = reinterpret_cast<float*>(smem_raw + 2 * S::kWBytes);                   // [2][kNW][kBB][SR]
  __shared__ BwdBatch s_b[kNBuf];
  __shared__ int s_maxlast;

  const int tile = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;  // MMA fragment row group and column pair
  // feature channels c0 .. c0 + NC - 1 of this block's chunk (blockIdx.y); the
  // colour, depth and geometric sums belong to chunk 0 alone
  // (one chunk with the L1 cotangents, which take N <= 16)
  const int c0 = L1 ? 0 : (int)blockIdx.y * NC;
  const bool geom = L1 || blockIdx.y == 0;
  const int tx = tile % p.cam.tiles_x, ty = tile / p.cam.tiles_x;
  int px[2], py[2];
  thread_pixels<2>(tx, ty, px, py);
  const int2 rg = p.ranges[tile];
  const size_t HW = (size_t)p.cam.W * p.cam.H;

  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  // Per pixel: T recovered backwards, the colour / depth cotangent g and
  // J = sum_c B_c g_c - S gAb, where B_c are the suffix sums of the channels
  // behind the current Gaussian, S the transmittance product behind it and
  // gAb = dL/dA - bg . g. Then dL/dalpha_i = T_i (c_i . g - J) and
  // J <- alpha c_i . g + (1 - alpha) J (both B_c and S follow that recurrence).
  float T[2], pxc[2], pyc[2], gC0[2], gC1[2], gC2[2], gD[2], J[2];
  int last[2];
  uint2 sgo[2] = {make_uint2(0u, 0u), make_uint2(0u, 0u)};  // L1: this thread's pixels' sign words
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool inside = px[q] < p.cam.W && py[q] < p.cam.H;
    const size_t pix = inside ? (size_t)py[q] * p.cam.W + px[q] : 0;
    pxc[q] = (float)px[q] + 0.5f;
    pyc[q] = (float)py[q] + 0.5f;
    T[q] = 1.f;
    last[q] = 0;
    gC0[q] = gC1[q] = gC2[q] = gD[q] = 0.f;
    float gA = 0.f;
    if (inside) {
      T[q] = p.T_final[pix];
      last[q] = p.last_idx[pix];
      if constexpr (L1) {
        const uint2 sg = p.l1.signs[pix];
        sgo[q] = sg;
        gC0[q] = l1_cot(sg, kL1BitRgb, p.l1.w[0]);
        gC1[q] = l1_cot(sg, kL1BitRgb + 1, p.l1.w[0]);
        gC2[q] = l1_cot(sg, kL1BitRgb + 2, p.l1.w[0]);
        gD[q] = l1_cot(sg, kL1BitDepth, p.l1.w[1]);
      } else {
        if (p.g_rgb) {
          gC0[q] = p.g_rgb[pix];
          gC1[q] = p.g_rgb[HW + pix];
          gC2[q] = p.g_rgb[2 * HW + pix];
        }
        if (p.g_depth) gD[q] = p.g_depth[pix];
        if (p.g_alpha) gA = p.g_alpha[pix];
      }
      if (last[q] > 0) atomicMax(&s_maxlast, last[q]);
    }
    J[q] = -(gA - (p.bg[0] * gC0[q] + p.bg[1] * gC1[q] + p.bg[2] * gC2[q]));  // B_c = 0, S = 1
  }
  // B fragments of the cotangent matrix (k = this warp's 64 pixels, n = channels),
  // held for the whole tile. Row k = 16 s + 2 t + 8 hf + q of step s is the
  // pixel at column t + 4 hf, row s + 4 q of the warp block.
  uint32_t bh[NT][4][2], bl[L1 ? 1 : NT][4][2];
  {
    const int bx = tx * kTile + (wid & 1) * 8, by = ty * kTile + (wid >> 1) * 8;
    if constexpr (L1) {
      // the signs of w sign(...) from the forward's sign words as exact bf16
      // (+1 = 0x3f80); the 16 pixels of this lane's fragments lie in the warp's
      // own block: pixel (column t + 4 hf, row s + 4 q) is pixel q of lane
      // t + 4 hf + 8 s, whose word comes by shuffle
      int bit[NT];
      uint32_t on[NT];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int c = 8 * nt + g8;
        bit[nt] = 0;
        on[nt] = 0u;
        if (c < NC) {
          if (c < p.N) bit[nt] = c, on[nt] = 0xffffu;
        } else if (c < NC + 3) {
          bit[nt] = kL1BitRgb + (c - NC), on[nt] = 0xffffu;
        } else if (c == NC + 3) {
          bit[nt] = kL1BitDepth, on[nt] = 0xffffu;
        }
      }
      auto half = [](uint2 sg, int b, uint32_t en) -> uint32_t {
        const uint32_t nz = (sg.x >> b) & 1u, ng = (sg.y >> b) & 1u;
        return (0x3f80u ^ (ng << 15)) & (0u - nz) & en;
      };
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int src = t4 + 4 * hf + 8 * s;
          uint2 sg[2];
#pragma unroll
          for (int q = 0; q < 2; ++q)
            sg[q] = make_uint2(__shfl_sync(0xffffffffu, sgo[q].x, src), __shfl_sync(0xffffffffu, sgo[q].y, src));
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
            bh[nt][s][hf] = half(sg[0], bit[nt], on[nt]) | (half(sg[1], bit[nt], on[nt]) << 16);
        }
    } else {
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int c = 8 * nt + g8;
        const float* plane = nullptr;  // channel c of the cotangent, indexed by pixel * pstride
        size_t pstride = 1;
        if (c < NC) {
          if (p.g_feat && c0 + c < p.N) {
            plane = p.hwc ? p.g_feat + c0 + c : p.g_feat + (size_t)(c0 + c) * HW;
            pstride = p.hwc ? (size_t)p.N : 1;
          }
        } else if (c < NC + 3) {
          if (geom && p.g_rgb) plane = p.g_rgb + (size_t)(c - NC) * HW;
        } else if (c == NC + 3) {
          if (geom) plane = p.g_depth;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            const int qx = bx + t4 + 4 * hf;
            float v[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int qy = by + s + 4 * q;
              v[q] = (plane && qx < p.cam.W && qy < p.cam.H) ? plane[((size_t)qy * p.cam.W + qx) * pstride] : 0.f;
            }
            if constexpr (!L1) split_bf16x2(v[0], v[1], bh[nt][s][hf], bl[L1 ? 0 : nt][s][hf]);
          }
      }
    }
  }
  // B fragment of the pixel monomials 1, x, y, x^2, x y, y^2 (n = 0..5; 6, 7
  // are zero), x and y the pixel centre minus the warp block's centre:
  // half-integers in [-3.5, 3.5], so all six are exact in bf16. The walk's dp
  // rows contracted against it give the block's geometric moments.
  uint32_t bm[4][2];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const float x = (float)(t4 + 4 * hf) - 3.5f;
      float m[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float y = (float)(s + 4 * q) - 3.5f;
        m[q] = g8 == 0 ? 1.f : g8 == 1 ? x : g8 == 2 ? y : g8 == 3 ? x * x : g8 == 4 ? x * y : g8 == 5 ? y * y : 0.f;
      }
      const __nv_bfloat162 v = __floats2bfloat162_rn(m[0], m[1]);
      bm[s][hf] = *reinterpret_cast<const uint32_t*>(&v);
    }
  __syncthreads();
  const int maxlast = checked_len(s_maxlast, rg.y - rg.x, p.status);
  // the walk's per-pixel state, pixel q in lane q of packed operands
  float2 T2 = make_float2(T[0], T[1]), J2 = make_float2(J[0], J[1]);
  const float2 gC02 = make_float2(gC0[0], gC0[1]), gC12 = make_float2(gC1[0], gC1[1]);
  const float2 gC22 = make_float2(gC2[0], gC2[1]), gD2 = make_float2(gD[0], gD[1]);
  const float2 npx2 = make_float2(-pxc[0], -pxc[1]), npy2 = make_float2(-pyc[0], -pyc[1]);
  const float2 one2 = make_float2(1.f, 1.f);
  // batches of the list, back to front: batch b holds positions [lo_b, hi_b)
  const int nb = (maxlast + kBB - 1) / kBB;
  auto batch_hi = [&](int b) { return rg.x + maxlast - b * kBB; };
  auto batch_lo = [&](int b) { return max(rg.x, batch_hi(b) - kBB); };
  // Batches are staged by warp 0 one batch ahead with cp.async (ids read two
  // batches ahead), so each batch costs the block a single barrier.
  // With the forward's stored skip masks (p.masks, one byte per instance) the
  // staging warp reads each mask with its id instead of testing the ellipse.
  const bool stored = p.masks != nullptr;
  uint32_t g_next = 0, m_next = 0;
  if (wid == 0 && nb > 0) {
    const int lo0 = batch_lo(0);
    if (lane < batch_hi(0) - lo0) {
      stage_batch(p, s_b[0], lane, checked_id(p.gids[lo0 + lane], p.P, p.status));
      if (stored) s_b[0].wmask[lane] = p.masks[lo0 + lane];
      cp_async_wait_all();
      finish_batch(s_b[0], lane, tx, ty, stored);
    }
    if (nb > 1 && lane < batch_hi(1) - batch_lo(1)) {
      g_next = checked_id(p.gids[batch_lo(1) + lane], p.P, p.status);
      if (stored) m_next = p.masks[batch_lo(1) + lane];
    }
  }
  __syncthreads();

  __nv_bfloat16* wh_w = s_wh + wid * kRows * kWStride;
  __nv_bfloat16* wl_w = s_wl + wid * kRows * kWStride;
  // ldmatrix row addresses: lane i supplies row (i & 7) + 8 ((i >> 3) & 1) of
  // the 16-row tile, at column block (i >> 4)
  const int lrow = (lane & 7) + 8 * ((lane >> 3) & 1), lcol = lane >> 4;
  const uint32_t a_wh = smem_u32(wh_w + lrow * kWStride + 8 * lcol);
  const uint32_t a_wl = smem_u32(wl_w + lrow * kWStride + 8 * lcol);

  for (int b = 0; b < nb; ++b) {
    const BwdBatch& B = s_b[b % kNBuf];
    float* red = s_red + (b & 1) * kNW * kBB * SR;  // [kNW][kBB][SR] of this batch
    const int lo = batch_lo(b), n = batch_hi(b) - lo;
    const bool stage = wid == 0 && b + 1 < nb && lane < batch_hi(b + 1) - batch_lo(b + 1);
    if (stage) {
      stage_batch(p, s_b[(b + 1) % kNBuf], lane, g_next);
      if (stored) s_b[(b + 1) % kNBuf].wmask[lane] = (uint8_t)m_next;
    }
    if (wid == 0 && b + 2 < nb && lane < batch_hi(b + 2) - batch_lo(b + 2)) {
      g_next = checked_id(p.gids[batch_lo(b + 2) + lane], p.P, p.status);
      if (stored) m_next = p.masks[batch_lo(b + 2) + lane];
    }

    // Contraction of the warp's tile: rows r < 8 hold w of the r-th Gaussian
    // walked since the last contraction and rows 8 + r its dp. The cotangent
    // n-tiles take rows r (W . G), the monomial n-tile rows 8 + r (dp . m);
    // the other products and rows past `rows` (stale values) are not stored.
    int rows = 0, row_j = 0;  // lane r: batch index of the Gaussian in rows r and 8 + r
    auto flush = [&]() {
      __syncwarp();
      float dW[NT][4], dM[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) dW[nt][0] = dW[nt][1] = dW[nt][2] = dW[nt][3] = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        uint32_t ah[4], al4[4];
        ldsm_x4(ah, a_wh + 32 * s);
        ldsm_x4(al4, a_wl + 32 * s);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_bf16_m16n8k16(dW[nt], al4, bh[nt][s][0], bh[nt][s][1]);
          if constexpr (!L1) mma_bf16_m16n8k16(dW[nt], ah, bl[L1 ? 0 : nt][s][0], bl[L1 ? 0 : nt][s][1]);
          mma_bf16_m16n8k16(dW[nt], ah, bh[nt][s][0], bh[nt][s][1]);
        }
        mma_bf16_m16n8k16(dM, al4, bm[s][0], bm[s][1]);
        mma_bf16_m16n8k16(dM, ah, bm[s][0], bm[s][1]);
      }
      // D rows g8 (W . G, columns 2 t4 and 2 t4 + 1) and g8 + 8 (dp . m)
      const int j0 = __shfl_sync(0xffffffffu, row_j, g8);
      if (g8 < rows) {
        float* r = red + ((size_t)wid * kBB + j0) * SR;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
          if (8 * nt + 2 * t4 < NCH) *reinterpret_cast<float2*>(r + 8 * nt + 2 * t4) = make_float2(dW[nt][0], dW[nt][1]);
        if (2 * t4 < kGeo) *reinterpret_cast<float2*>(r + NCH + 2 * t4) = make_float2(dM[2], dM[3]);
      }
      __syncwarp();
      rows = 0;
    };

    // walk: this warp's Gaussians of the batch in reverse list order, two at a
    // time. Both pairs' alphas are formed first (four independent chains); a
    // pair that does not blend takes alpha = 0, for which every update below
    // is an exact identity (T / 1, 0 cg + 1 J) and w = dp = 0. After every
    // eight Gaussians the tile is contracted (pairs never straddle: rows stay
    // even until the last, single Gaussian).
    uint32_t bits = __ballot_sync(0xffffffffu, lane < n && ((B.wmask[lane] >> wid) & 1u));
    while (bits) {
      const int j1 = 31 - __clz(bits);
      bits &= ~(1u << j1);
      const bool two = bits != 0;
      const int j2 = two ? 31 - __clz(bits) : j1;
      bits &= ~(1u << j2);
      const int jg[2] = {j1, j2};
      // the two pixels of this thread ride in the two lanes of packed
      // fp32 operations (each lane rounds as the scalar operation does)
      float2 al[2];
      bool cl[2][2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float2 uj = B.uv[jg[k]];
        const float4 cj = B.q[jg[k]];
        const int pos = lo + jg[k] - rg.x;
        // pair_alpha_q for both pixels
        const float2 dx2 = __fadd2_rn(make_float2(uj.x, uj.x), npx2);
        const float2 dy2 = __fadd2_rn(make_float2(uj.y, uj.y), npy2);
        const float2 u = __ffma2_rn(make_float2(cj.y, cj.y), dy2, __fmul2_rn(make_float2(cj.x, cj.x), dx2));
        const float2 e = __ffma2_rn(dx2, u, __fmul2_rn(__fmul2_rn(make_float2(cj.z, cj.z), dy2), dy2));
        const float2 a = __fmul2_rn(make_float2(cj.w, cj.w), make_float2(ex2_approx(e.x), ex2_approx(e.y)));
        const bool live = k == 0 || two;
        const bool ok0 = live && pos < last[0] && !(e.x > 0.f), ok1 = live && pos < last[1] && !(e.y > 0.f);
        cl[k][0] = a.x > kAlphaMax;
        cl[k][1] = a.y > kAlphaMax;
        const float a0 = cl[k][0] ? kAlphaMax : a.x, a1 = cl[k][1] ? kAlphaMax : a.y;
        const bool b0 = ok0 && a0 >= kAlphaMin, b1 = ok1 && a1 >= kAlphaMin;
        al[k] = make_float2(b0 ? a0 : 0.f, b1 ? a1 : 0.f);
        cl[k][0] = b0 && cl[k][0];
        cl[k][1] = b1 && cl[k][1];
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (k == 1 && !two) break;
        const float4 cd = B.cd[jg[k]];
        const float2 a = al[k], om = __fadd2_rn(one2, make_float2(-a.x, -a.y));
        T2 = make_float2(__fdividef(T2.x, om.x), __fdividef(T2.y, om.y));
        const float2 wq = __fmul2_rn(a, T2);
        const float2 cg = __ffma2_rn(make_float2(cd.w, cd.w), gD2,
                                     __ffma2_rn(make_float2(cd.z, cd.z), gC22,
                                                __ffma2_rn(make_float2(cd.y, cd.y), gC12,
                                                           __fmul2_rn(make_float2(cd.x, cd.x), gC02))));
        const float2 da = __fmul2_rn(T2, __fadd2_rn(cg, make_float2(-J2.x, -J2.y)));
        J2 = __ffma2_rn(a, cg, __fmul2_rn(om, J2));
        const float2 dp = __fmul2_rn(da, a);
        uint32_t hi, lo2;
        split_bf16x2(wq.x, wq.y, hi, lo2);
        reinterpret_cast<uint32_t*>(wh_w + rows * kWStride)[lane] = hi;
        reinterpret_cast<uint32_t*>(wl_w + rows * kWStride)[lane] = lo2;
        split_bf16x2(cl[k][0] ? 0.f : dp.x, cl[k][1] ? 0.f : dp.y, hi, lo2);
        reinterpret_cast<uint32_t*>(wh_w + (rows + kGRows) * kWStride)[lane] = hi;
        reinterpret_cast<uint32_t*>(wl_w + (rows + kGRows) * kWStride)[lane] = lo2;
        if (lane == rows) row_j = jg[k];
        ++rows;
      }
      if (rows == kGRows) flush();
    }
    if (rows > 0) flush();
    if (stage) {
      cp_async_wait_all();
      finish_batch(s_b[(b + 1) % kNBuf], lane, tx, ty, stored);
    }
    __syncthreads();
    // the block's sums of the batch: rows of warps that did not walk Gaussian j
    // are stale and skipped; one global atomic per (Gaussian, output)
    if (wid < kNW - 1) {
      // groups of 4 outputs: 16-byte loads of the warps' sums and, for the
      // features, one vector atomic per group
      const bool vec = NC > 0 && p.d_feats && (p.N & 3) == 0 && ((uintptr_t)p.d_feats & 15u) == 0;
      for (int e = threadIdx.x; e < n * NG; e += kThreads - 32) {
        const int j = e / NG, gq = e - j * NG;
        const uint32_t wm = B.wmask[j];
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 0; w < kNW; ++w)
          if ((wm >> w) & 1u) {
            const float4 v = *reinterpret_cast<const float4*>(red + ((size_t)w * kBB + j) * SR + 4 * gq);
            sum.x += v.x;
            sum.y += v.y;
            sum.z += v.z;
            sum.w += v.w;
          }
        const uint32_t g = B.gid[j];
        if (gq < NC / 4) {
          if (!p.d_feats) continue;
          if (L1) sum = make_float4(sum.x * p.l1.w[2], sum.y * p.l1.w[2], sum.z * p.l1.w[2], sum.w * p.l1.w[2]);
          const int c = c0 + 4 * gq;
          if (vec && c + 4 <= p.N) {
            if (sum.x != 0.f || sum.y != 0.f || sum.z != 0.f || sum.w != 0.f)
              atomicAdd(reinterpret_cast<float4*>(p.d_feats + (size_t)g * p.N + c), sum);
          } else {
            const float sv[4] = {sum.x, sum.y, sum.z, sum.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (c + k < p.N && sv[k] != 0.f) atomicAdd(p.d_feats + (size_t)g * p.N + c + k, sv[k]);
          }
        } else if (geom) {
          const float wc = L1 ? p.l1.w[0] : 1.f, wd = L1 ? p.l1.w[1] : 1.f;
          if (p.d_colors) {
            if (sum.x != 0.f) atomicAdd(p.d_colors + 3 * (size_t)g, sum.x * wc);
            if (sum.y != 0.f) atomicAdd(p.d_colors + 3 * (size_t)g + 1, sum.y * wc);
            if (sum.z != 0.f) atomicAdd(p.d_colors + 3 * (size_t)g + 2, sum.z * wc);
          }
          if (sum.w != 0.f) atomicAdd(p.d_depth + g, sum.w * wd);
        }
      }
    } else if (geom && lane < n) {
      // u, v, conic and opacity of Gaussian `lane`: v_u = -sum (A dx + B dy) dp,
      // v_v = -sum (B dx + C dy) dp, v_A = -sum dx^2 dp / 2, v_B = -sum dx dy dp,
      // v_C = -sum dy^2 dp / 2 (dx = u - pixel centre), v_o = sum dp / o
      // from each warp's moments m = sum dp (1, x, y, x^2, x y, y^2), x, y
      // relative to its block's centre c: with (du, dv) = u - c, dx = du - x
      const int j = lane;
      const uint32_t wm = B.wmask[j];
      const float2 uj = B.uv[j];
      float sdp = 0.f, sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
      for (int w = 0; w < kNW; ++w) {
        if (!((wm >> w) & 1u)) continue;
        const float* M = red + ((size_t)w * kBB + j) * SR + NCH;
        const float du = uj.x - (float)(tx * kTile + (w & 1) * 8 + 4);
        const float dv = uj.y - (float)(ty * kTile + (w >> 1) * 8 + 4);
        sdp += M[0];
        sx += du * M[0] - M[1];
        sy += dv * M[0] - M[2];
        sxx += du * (du * M[0] - 2.f * M[1]) + M[3];
        sxy += du * (dv * M[0] - M[2]) - dv * M[1] + M[4];
        syy += dv * (dv * M[0] - 2.f * M[2]) + M[5];
      }
      const float4 co = B.co[j];
      const uint32_t g = B.gid[j];
      const float out[6] = {-(co.x * sx + co.y * sy), -(co.y * sx + co.z * sy), -0.5f * sxx, -sxy, -0.5f * syy,
                            sdp / co.w};
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (out[k] != 0.f) atomicAdd(p.d_uv + 2 * (size_t)g + k, out[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (out[2 + k] != 0.f) atomicAdd(p.d_conic + 3 * (size_t)g + k, out[2 + k]);
      if (p.d_opacity && out[5] != 0.f) atomicAdd(p.d_opacity + g, out[5]);
    }
  }
}

}  // namespace

gs_status launch_render_fwd(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                            uint8_t* masks, const float* uv,
                            const float* co, const float* depth, const float* colors, const void* feats, int N,
                            int bf16, int hwc, const float bg[3], float* out_rgb, float* out_depth,
                            float* out_alpha, float* out_feat, float* T_final, int32_t* last_idx,
                            int32_t* n_contrib, uint8_t* visible, const L1Fwd* l1, int P, int32_t* status,
                            cudaStream_t st) {
  FwdParams p;
  p.P = P;
  p.status = status;
  p.l1 = l1 ? *l1 : L1Fwd{};
  if (p.l1.on && N > 16) return GS_ERR_UNSUPPORTED;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.masks = masks;
  p.gids = gids;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.depth = depth;
  p.colors = colors;
  p.feats = feats;
  p.N = N;
  p.bf16 = bf16;
  p.hwc = hwc;
  for (int i = 0; i < 3; ++i) p.bg[i] = bg[i];
  p.out_rgb = out_rgb;
  p.out_depth = out_depth;
  p.out_alpha = out_alpha;
  p.out_feat = out_feat;
  p.T_final = T_final;
  p.last_idx = last_idx;
  p.n_contrib = n_contrib;
  p.visible = visible;
  const unsigned tiles = (unsigned)(cam.tiles_x * cam.tiles_y);
  GS_TRACE("k_render_fwd", st);
  const dim3 grid(tiles, N <= 16 ? 1 : (N + 31) / 32);
  if (visible) {
    if (N <= 0) launch_pdl(k_render_fwd2<0, true>, grid, kFwd2Threads, 0, st, p);
    else if (N <= 16) launch_pdl(k_render_fwd2<16, true>, grid, kFwd2Threads, 0, st, p);
    else launch_pdl(k_render_fwd<32, true>, grid, kTilePix, 0, st, p);
  } else {
    if (N <= 0) launch_pdl(k_render_fwd2<0, false>, grid, kFwd2Threads, 0, st, p);
    else if (N <= 16) launch_pdl(k_render_fwd2<16, false>, grid, kFwd2Threads, 0, st, p);
    else launch_pdl(k_render_fwd<32, false>, grid, kTilePix, 0, st, p);
  }
  return last_launch_status();
}

// The tensor-core adjoint takes its tiles (48 KB) in dynamic shared memory; the
// limit is raised once per device.
template <int NC, bool L1>
gs_status launch_bwd_mma(const BwdParams& p, unsigned tiles, cudaStream_t st) {
  constexpr size_t smem = MmaBwdShape<NC>::kSmem;
  static std::atomic<uint64_t> attr_done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  const uint64_t bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    if (cudaFuncSetAttribute(k_render_bwd_mma<NC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GS_ERR_CUDA;
    attr_done.fetch_or(bit);
  }
  const int chunks = NC > 0 && p.N > NC ? (p.N + NC - 1) / NC : 1;
  launch_pdl(k_render_bwd_mma<NC, L1>, dim3(tiles, chunks), dim3(mma_bwd::kThreads), smem, st, p);
  return last_launch_status();
}

gs_status launch_render_bwd(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                            const uint8_t* masks, const float* uv,
                            const float* co, const float* depth, const float* colors, const void* feats, int N,
                            int bf16, int hwc, const float bg[3], const float* T_final, const int32_t* last_idx,
                            const float* g_rgb, const float* g_depth, const float* g_alpha, const float* g_feat,
                            int coupled, float* d_uv, float* d_conic, float* d_depth, float* d_opacity,
                            float* d_colors, float* d_feats, const L1Bwd* l1, int P, int32_t* status,
                            cudaStream_t st) {
  BwdParams p;
  p.P = P;
  p.status = status;
  p.pair_off = nullptr;
  p.pair_T = nullptr;
  p.l1 = l1 ? *l1 : L1Bwd{};
  if (p.l1.on && (N > 16 || coupled)) return GS_ERR_UNSUPPORTED;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.masks = masks;
  p.gids = gids;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.depth = depth;
  p.colors = colors;
  p.feats = feats;
  p.N = N;
  p.bf16 = bf16;
  p.hwc = hwc;
  for (int i = 0; i < 3; ++i) p.bg[i] = bg[i];
  p.T_final = T_final;
  p.last_idx = last_idx;
  p.g_rgb = g_rgb;
  p.g_depth = g_depth;
  p.g_alpha = g_alpha;
  p.g_feat = g_feat;
  p.d_uv = d_uv;
  p.d_conic = d_conic;
  p.d_depth = d_depth;
  p.d_opacity = d_opacity;
  p.d_colors = d_colors;
  p.d_feats = d_feats;
  const unsigned tiles = (unsigned)(cam.tiles_x * cam.tiles_y);
  // decoupled features up to 64 channels: the tensor-core adjoint, in chunks of
  // 16 channels above 16 (chunk 0 also does the geometry)
  if (N <= 64 && !coupled) {
    GS_TRACE("k_render_bwd_mma", st);
    if (p.l1.on) return N <= 0 ? launch_bwd_mma<0, true>(p, tiles, st) : launch_bwd_mma<16, true>(p, tiles, st);
    return N <= 0 ? launch_bwd_mma<0, false>(p, tiles, st) : launch_bwd_mma<16, false>(p, tiles, st);
  }
  GS_TRACE("k_render_bwd", st);
  if (N <= 16) {
    k_render_bwd<16, true, 1><<<dim3(tiles, 1), kTilePix, 0, st>>>(p);
  } else {
    const dim3 grid(tiles, (N + 31) / 32);
    if (coupled) k_render_bwd<32, true, 1><<<grid, kTilePix, 0, st>>>(p);
    else k_render_bwd<32, false, 1><<<grid, kTilePix, 0, st>>>(p);
  }
  return last_launch_status();
}

// The SIMT adjoint in 32-channel chunks with the transmittance either
// recovered by division (pair_T null) or read from the per-pair saved state.
gs_status launch_render_bwd_pairs(const CamF& cam, const int32_t* ranges, const int32_t* order, const uint32_t* gids,
                                  const float* uv, const float* co, const float* depth, const float* colors,
                                  const void* feats, int N, int bf16, int hwc, const float bg[3],
                                  const float* T_final, const int32_t* last_idx, const float* g_rgb,
                                  const float* g_depth, const float* g_alpha, const float* g_feat, int coupled,
                                  const long long* pair_off, const float* pair_T, float* d_uv, float* d_conic,
                                  float* d_depth, float* d_opacity, float* d_colors, float* d_feats, int P,
                                  int32_t* status, cudaStream_t st) {
  BwdParams p;
  p.l1 = L1Bwd{};
  p.P = P;
  p.status = status;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
  p.order = order;
  p.masks = nullptr;
  p.gids = gids;
  p.uv = reinterpret_cast<const float2*>(uv);
  p.co = reinterpret_cast<const float4*>(co);
  p.depth = depth;
  p.colors = colors;
  p.feats = feats;
  p.N = N;
  p.bf16 = bf16;
  p.hwc = hwc;
  for (int i = 0; i < 3; ++i) p.bg[i] = bg[i];
  p.T_final = T_final;
  p.last_idx = last_idx;
  p.g_rgb = g_rgb;
  p.g_depth = g_depth;
  p.g_alpha = g_alpha;
  p.g_feat = g_feat;
  p.d_uv = d_uv;
  p.d_conic = d_conic;
  p.d_depth = d_depth;
  p.d_opacity = d_opacity;
  p.d_colors = d_colors;
  p.d_feats = d_feats;
  p.pair_off = pair_off;
  p.pair_T = pair_T;
  const unsigned tiles = (unsigned)(cam.tiles_x * cam.tiles_y);
  const dim3 grid(tiles, N > 0 ? (N + 31) / 32 : 1);
  if (pair_T) {
    GS_TRACE("k_render_bwd_stored", st);
    if (coupled) k_render_bwd<32, true, 1, true><<<grid, kTilePix, 0, st>>>(p);
    else k_render_bwd<32, false, 1, true><<<grid, kTilePix, 0, st>>>(p);
  } else {
    GS_TRACE("k_render_bwd", st);
    if (coupled) k_render_bwd<32, true, 1><<<grid, kTilePix, 0, st>>>(p);
    else k_render_bwd<32, false, 1><<<grid, kTilePix, 0, st>>>(p);
  }
  return last_launch_status();
}

}  // namespace gsff
