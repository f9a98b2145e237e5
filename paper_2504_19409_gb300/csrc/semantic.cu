// Semantic supervision and read-out of the rendered feature field (Sec. 3.3).
//
//   Eq. 9:  L_s = -(1/HW) sum_p sum_c L_p(c) log F_p(c), with L_p one-hot
//           labels; F is read as per-pixel logits over the N channels
//           normalised by a softmax (the rendered features are unbounded),
//           so L_s = (1/HW) sum_p [logsumexp(F_p) - F_p(l_p)] and
//           dL/dF_p = (softmax(F_p) - onehot(l_p)) / HW. Pixels with a
//           negative label are ignored (no loss, zero gradient).
//   Eq. 10:  predicted labels argmax_c F_p(c) (ties: the lowest channel).
//   Eq. 12: p(l | x) = exp(f(x) . q(l)) / sum_l' exp(f(x) . q(l')), per
//           pixel feature f(x) (M channels) and L query vectors q(l).

#include "gsff_internal.cuh"

namespace gsff {
namespace {

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

// Channel c of pixel p: CHW -> F[c * HW + p], HWC -> F[p * N + c].
__device__ __forceinline__ size_t fidx(int hwc, size_t HW, int N, size_t p, int c) {
  return hwc ? p * (size_t)N + c : (size_t)c * HW + p;
}

__global__ void __launch_bounds__(256) k_semantic_ce(long long HW, int N, int hwc, const float* __restrict__ F,
                                                     const int32_t* __restrict__ labels, float inv_hw,
                                                     float* __restrict__ grad, float* __restrict__ loss) {
  float acc = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (long long)gridDim.x * blockDim.x) {
    const int lab = labels[p];
    if (lab < 0 || lab >= N) {
      if (grad)
        for (int c = 0; c < N; ++c) grad[fidx(hwc, HW, N, p, c)] = 0.f;
      continue;
    }
    float mx = -INFINITY;
    for (int c = 0; c < N; ++c) mx = fmaxf(mx, F[fidx(hwc, HW, N, p, c)]);
    float sum = 0.f;
    for (int c = 0; c < N; ++c) sum += expf(F[fidx(hwc, HW, N, p, c)] - mx);
    const float lse = mx + logf(sum);
    acc += (lse - F[fidx(hwc, HW, N, p, lab)]) * inv_hw;
    if (grad) {
      const float is = 1.f / sum;
      for (int c = 0; c < N; ++c) {
        const size_t i = fidx(hwc, HW, N, p, c);
        const float pr = expf(F[i] - mx) * is;
        grad[i] = (pr - (c == lab ? 1.f : 0.f)) * inv_hw;
      }
    }
  }
  if (loss) {
    __shared__ float s_part[8];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_part[w];
      if (b != 0.f) atomicAdd(loss, b);
    }
  }
}

__global__ void __launch_bounds__(256) k_argmax(long long HW, int N, int hwc, const float* __restrict__ F,
                                                int32_t* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (long long)gridDim.x * blockDim.x) {
    float best = F[fidx(hwc, HW, N, p, 0)];
    int arg = 0;
    for (int c = 1; c < N; ++c) {
      const float v = F[fidx(hwc, HW, N, p, c)];
      if (v > best) {  // strict: ties keep the lowest channel
        best = v;
        arg = c;
      }
    }
    out[p] = arg;
  }
}

// One thread per pixel; the L x M query matrix sits in shared memory (row l =
// q(l)), each step reads 4 of the pixel's channels as a float4 and the 4
// matching entries of every query with one broadcast 16-byte load. LMAX is a
// bound on L (8, 16, 32 or 64).
constexpr int kMaxLabels = 64;

template <int LMAX>
__global__ void __launch_bounds__(512) k_label_probs(long long npix, int M, int L, const float* __restrict__ f,
                                                     const float* __restrict__ q, float* __restrict__ probs,
                                                     int32_t* __restrict__ labels) {
  extern __shared__ __align__(16) float s_q[];  // [L][M]
  for (int i = threadIdx.x; i < M * L; i += blockDim.x) s_q[i] = q[i];
  __syncthreads();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    float z[LMAX];
#pragma unroll
    for (int l = 0; l < LMAX; ++l) z[l] = 0.f;
    const float4* row = reinterpret_cast<const float4*>(f + p * (size_t)M);
#pragma unroll 2
    for (int c4 = 0; c4 < M / 4; ++c4) {
      const float4 v = row[c4];
#pragma unroll
      for (int l = 0; l < LMAX; ++l) {
        if (l < L) {
          const float4 w = *reinterpret_cast<const float4*>(s_q + (size_t)l * M + 4 * c4);
          z[l] = fmaf(v.x, w.x, z[l]);
          z[l] = fmaf(v.y, w.y, z[l]);
          z[l] = fmaf(v.z, w.z, z[l]);
          z[l] = fmaf(v.w, w.w, z[l]);
        }
      }
    }
    float mx = -INFINITY;
    int arg = 0;
#pragma unroll
    for (int l = 0; l < LMAX; ++l)
      if (l < L && z[l] > mx) {  // strict: ties keep the lowest label
        mx = z[l];
        arg = l;
      }
    if (labels) labels[p] = arg;
    if (probs) {
      float sum = 0.f;
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l < L) {
          z[l] = expf(z[l] - mx);
          sum += z[l];
        }
      const float is = 1.f / sum;
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l < L) probs[p * (size_t)L + l] = z[l] * is;
    }
  }
}

int grid_for(long long n, int threads, int per_sm) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * per_sm) b = 152LL * per_sm;
  return (int)(b > 0 ? b : 1);
}

}  // namespace
}  // namespace gsff

using namespace gsff;

extern "C" {

gs_status gs_semantic_ce_grad(int32_t width, int32_t height, int32_t N, int32_t layout, const float* feat,
                              const int32_t* labels, float* grad, float* loss_sum, void* stream) {
  if (width <= 0 || height <= 0 || N <= 0 || N > 4096 || !feat || !labels) return GS_ERR_INVALID_ARG;
  if (layout != GS_LAYOUT_CHW && layout != GS_LAYOUT_HWC) return GS_ERR_INVALID_ARG;
  const long long HW = (long long)width * height;
  GS_TRACE("k_semantic_ce", S(stream));
  k_semantic_ce<<<grid_for(HW, 256, 8), 256, 0, S(stream)>>>(HW, N, layout == GS_LAYOUT_HWC, feat, labels,
                                                             (float)(1.0 / (double)HW), grad, loss_sum);
  return last_launch_status();
}

gs_status gs_argmax_labels(int32_t width, int32_t height, int32_t N, int32_t layout, const float* feat,
                           int32_t* labels, void* stream) {
  if (width <= 0 || height <= 0 || N <= 0 || N > 4096 || !feat || !labels) return GS_ERR_INVALID_ARG;
  if (layout != GS_LAYOUT_CHW && layout != GS_LAYOUT_HWC) return GS_ERR_INVALID_ARG;
  const long long HW = (long long)width * height;
  GS_TRACE("k_argmax", S(stream));
  k_argmax<<<grid_for(HW, 256, 8), 256, 0, S(stream)>>>(HW, N, layout == GS_LAYOUT_HWC, feat, labels);
  return last_launch_status();
}

gs_status gs_label_probs(int64_t npix, int32_t M, int32_t L, const float* feat, const float* queries, float* probs,
                         int32_t* labels, void* stream) {
  if (npix < 0 || M <= 0 || M % 4 != 0 || L <= 0 || L > kMaxLabels || !queries || (npix > 0 && !feat))
    return GS_ERR_INVALID_ARG;
  if (!probs && !labels) return GS_ERR_INVALID_ARG;
  if (!aligned(feat, 16)) return GS_ERR_INVALID_ARG;
  const size_t smem = (size_t)M * L * sizeof(float);
  if (smem > 200 * 1024) return GS_ERR_UNSUPPORTED;
  if (npix == 0) return GS_OK;
  auto launch = [&](auto kernel) -> gs_status {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GS_ERR_CUDA;
    GS_TRACE("k_label_probs", S(stream));
    kernel<<<grid_for(npix, 512, 2), 512, smem, S(stream)>>>(npix, M, L, feat, queries, probs, labels);
    return last_launch_status();
  };
  if (L <= 8) return launch(k_label_probs<8>);
  if (L <= 16) return launch(k_label_probs<16>);
  if (L <= 32) return launch(k_label_probs<32>);
  return launch(k_label_probs<64>);
}

}  // extern "C"
