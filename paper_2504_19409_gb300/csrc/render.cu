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

#include "gsff_internal.cuh"

namespace gsff {
namespace {

struct FwdParams {
  CamF cam;
  const int2* ranges;
  const uint32_t* gids;
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
  constexpr int NCs = NC > 0 ? NC : 1;
  __shared__ float2 s_uv[kTilePix];
  __shared__ uint8_t s_wmask[kTilePix];  // bit w: warp w's pixel block passes the skip test
  __shared__ float4 s_co[kTilePix];
  __shared__ float4 s_cd[kTilePix];
  __shared__ float s_f[kTilePix][NCs];
  __shared__ uint32_t s_gid[VIS ? kTilePix : 1];

  const int tile = blockIdx.x;
  const int chunk = blockIdx.y;
  const bool geom = chunk == 0;
  const bool mark = VIS && geom;
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
      const uint32_t g = p.gids[idx];
      const float4 co = p.co[g];
      const float2 u = p.uv[g];
      s_uv[threadIdx.x] = u;
      s_co[threadIdx.x] = co;
      // the skip tests of all 8 warp blocks (2 columns x 4 rows of 8x4 pixels)
      s_wmask[threadIdx.x] = (uint8_t)warp_block_mask<8, 4, false>(u, co, tx, ty);
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
        if (!pair_alpha(s_co[j], uj.x - pxc, uj.y - pyc, pa)) continue;
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
        if (geom) {
          const float4 cd = s_cd[j];
          ac0 = __fmaf_rn(w, cd.x, ac0);
          ac1 = __fmaf_rn(w, cd.y, ac1);
          ac2 = __fmaf_rn(w, cd.z, ac2);
          ad = __fmaf_rn(w, cd.w, ad);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) af[c] = __fmaf_rn(w, s_f[j][c], af[c]);
        T = Tn;
        last = start + j + 1 - rg.x;
        ++cnt;
      }
    }
  }
  if (!inside) return;
  const size_t HW = (size_t)p.cam.W * p.cam.H;
  const size_t pix = (size_t)py * p.cam.W + px;
  if (geom) {
    p.out_rgb[pix] = ac0 + T * p.bg[0];
    p.out_rgb[HW + pix] = ac1 + T * p.bg[1];
    p.out_rgb[2 * HW + pix] = ac2 + T * p.bg[2];
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
}

// ---------------------------------------------------------------------------
struct BwdParams {
  CamF cam;
  const int2* ranges;
  const uint32_t* gids;
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
template <int NC, bool COUPLED, int PPT>
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

  const int tile = blockIdx.x;
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
    if (inside) {
      T[q] = p.T_final[pix];
      last[q] = p.last_idx[pix];
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
  const int maxlast = s_maxlast;

  for (int hi = rg.x + maxlast; hi > rg.x; hi -= BB) {
    const int lo = max(rg.x, hi - BB);
    const int n = hi - lo;
    if ((int)threadIdx.x < n) {
      const uint32_t g = p.gids[lo + threadIdx.x];
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
        T[q] = __fdividef(T[q], om);
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

}  // namespace

gs_status launch_render_fwd(const CamF& cam, const int32_t* ranges, const uint32_t* gids, const float* uv,
                            const float* co, const float* depth, const float* colors, const void* feats, int N,
                            int bf16, int hwc, const float bg[3], float* out_rgb, float* out_depth,
                            float* out_alpha, float* out_feat, float* T_final, int32_t* last_idx,
                            int32_t* n_contrib, uint8_t* visible, cudaStream_t st) {
  FwdParams p;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
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
    if (N <= 0) k_render_fwd<0, true><<<grid, kTilePix, 0, st>>>(p);
    else if (N <= 16) k_render_fwd<16, true><<<grid, kTilePix, 0, st>>>(p);
    else k_render_fwd<32, true><<<grid, kTilePix, 0, st>>>(p);
  } else {
    if (N <= 0) k_render_fwd<0, false><<<grid, kTilePix, 0, st>>>(p);
    else if (N <= 16) k_render_fwd<16, false><<<grid, kTilePix, 0, st>>>(p);
    else k_render_fwd<32, false><<<grid, kTilePix, 0, st>>>(p);
  }
  return last_launch_status();
}

gs_status launch_render_bwd(const CamF& cam, const int32_t* ranges, const uint32_t* gids, const float* uv,
                            const float* co, const float* depth, const float* colors, const void* feats, int N,
                            int bf16, int hwc, const float bg[3], const float* T_final, const int32_t* last_idx,
                            const float* g_rgb, const float* g_depth, const float* g_alpha, const float* g_feat,
                            int coupled, float* d_uv, float* d_conic, float* d_depth, float* d_opacity,
                            float* d_colors, float* d_feats, cudaStream_t st) {
  BwdParams p;
  p.cam = cam;
  p.ranges = reinterpret_cast<const int2*>(ranges);
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
  GS_TRACE("k_render_bwd", st);
  if (N <= 0) {
    k_render_bwd<0, false, 2><<<dim3(tiles, 1), kTilePix / 2, 0, st>>>(p);
  } else if (N <= 16) {
    if (coupled) k_render_bwd<16, true, 1><<<dim3(tiles, 1), kTilePix, 0, st>>>(p);
    else k_render_bwd<16, false, 2><<<dim3(tiles, 1), kTilePix / 2, 0, st>>>(p);
  } else {
    const dim3 grid(tiles, (N + 31) / 32);
    if (coupled) k_render_bwd<32, true, 1><<<grid, kTilePix, 0, st>>>(p);
    else k_render_bwd<32, false, 1><<<grid, kTilePix, 0, st>>>(p);
  }
  return last_launch_status();
}

}  // namespace gsff
