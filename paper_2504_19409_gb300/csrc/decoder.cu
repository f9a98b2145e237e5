// Per-pixel feature decoder o(.) (Eq. 11, read as a 1x1 lift of the latent
// feature map): y = W2^T gelu(W1^T z + b1) + b2, exact-erf GELU, trained on
// sampled pixels with an MSE loss against the full-width render, and Adam.
//
// The training step is a chain of small kernels: a tiled fp32 SIMT GEMM
// (64x64 tiles, 16-deep K slabs in shared memory, 4x4 outputs per thread,
// arbitrary operand strides so transposes are free, optional split-K with
// atomic accumulation, fused bias / bias+GELU epilogue) plus gather, loss,
// GELU-backward, column-sum, scatter and Adam kernels. The weights enter
// every product as bf16-exact values (the caller keeps fp32 masters and Adam
// writes the bf16-rounded copy), so each product is exact in fp32 and sums
// accumulate in fp32.

#include <math.h>

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;
enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2 };

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_erf_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// C[m, n] = (sum_k A(m, k) B(k, n)) [+ bias[n]] [-> gelu], or += with atomics
// when `atomic_acc` (split-K over gridDim.z chunks of k_chunk).
template <int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, long long lam,
                                              long long lak, const float* __restrict__ B, long long lbk, long long lbn,
                                              float* __restrict__ C, long long ldc, const float* __restrict__ bias,
                                              float* __restrict__ Cpre, int k_chunk, int atomic_acc) {
  __shared__ float sA[kBK][kBM + 4];
  __shared__ float sB[kBK][kBN + 4];
  const int tid = threadIdx.x;
  const int tm = (tid / 16) * 4, tn = (tid % 16) * 4;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int k_begin = blockIdx.z * k_chunk;
  const int k_end = min(K, k_begin + k_chunk);
  float acc[4][4] = {};
  for (int k0 = k_begin; k0 < k_end; k0 += kBK) {
    for (int e = tid; e < kBK * kBM; e += 256) {
      const int kk = e / kBM, mm = e % kBM;
      const int m = m0 + mm, k = k0 + kk;
      sA[kk][mm] = (m < M && k < k_end) ? A[(long long)m * lam + (long long)k * lak] : 0.f;
    }
    for (int e = tid; e < kBK * kBN; e += 256) {
      const int kk = e / kBN, nn = e % kBN;
      const int n = n0 + nn, k = k0 + kk;
      sB[kk][nn] = (n < N && k < k_end) ? B[(long long)k * lbk + (long long)n * lbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][tm + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tn + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn + j;
      if (n >= N) continue;
      float v = acc[i][j];
      float* dst = C + (long long)m * ldc + n;
      if (atomic_acc) {
        atomicAdd(dst, v);
        continue;
      }
      if (EPI != EPI_NONE) v += bias[n];
      if (EPI == EPI_BIAS_GELU) {
        if (Cpre) Cpre[(long long)m * ldc + n] = v;
        v = gelu_erf(v);
      }
      *dst = v;
    }
  }
}

// Pixel sample s of a step (decoder_sample_pixel: the ABI's sampling rule).
__global__ void k_sample(long long S, long long npix, unsigned long long seed, int* __restrict__ idx) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x)
    idx[s] = (int)decoder_sample_pixel(seed, s, npix);
}

__global__ void k_gather(long long S, int d, const int* __restrict__ idx, const float* __restrict__ src,
                         float* __restrict__ dst) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < S * d; e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / d;
    dst[e] = src[(long long)idx[s] * d + (e - s * d)];
  }
}

__global__ void k_scatter_add(long long S, int d, const int* __restrict__ idx, const float* __restrict__ src,
                              float* __restrict__ dst) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < S * d; e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / d;
    atomicAdd(dst + (long long)idx[s] * d + (e - s * d), src[e]);
  }
}

// dY = 2 scale (Y - T) in place of Y; loss += scale sum (Y - T)^2.
__global__ void k_mse_grad(long long n, float* __restrict__ Y, const float* __restrict__ T, float scale,
                           float* __restrict__ loss) {
  float acc = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    Y[e] = 2.f * scale * d;
    acc = fmaf(d, d, acc);
  }
  if (loss) {
    __shared__ float s_part[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_part[w];
      if (b != 0.f) atomicAdd(loss, b * scale);
    }
  }
}

__global__ void k_gelu_bwd(long long n, float* __restrict__ dH, const float* __restrict__ pre) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dH[e] *= gelu_erf_grad(pre[e]);
}

// out[c] += sum_s X[s, c] (block partial sums, one atomic per column and block).
__global__ void __launch_bounds__(256) k_colsum(long long S, int d, const float* __restrict__ X, float* __restrict__ out) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r0 = threadIdx.x >> 5;
  float acc = 0.f;
  if (c < d)
    for (long long s = (long long)blockIdx.y * 8 + r0; s < S; s += (long long)gridDim.y * 8) acc += X[s * d + c];
  __shared__ float s_part[8][32];
  s_part[r0][threadIdx.x & 31] = acc;
  __syncthreads();
  if (threadIdx.x < 32 && c < d) {
    float b = 0.f;
    for (int r = 0; r < 8; ++r) b += s_part[r][threadIdx.x];
    if (b != 0.f) atomicAdd(out + c, b);
  }
}

// Adam (Kingma & Ba 2015) with bias correction; optionally writes the
// bf16-rounded weights (as fp32 values) used by the products.
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       float* __restrict__ p_bf16) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float upd = lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    const float np = p[e] - upd;
    p[e] = np;
    if (p_bf16) p_bf16[e] = __bfloat162float(__float2bfloat16_rn(np));
  }
}

unsigned grid1d(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

template <int EPI>
void gemm(int M, int N, int K, const float* A, long long lam, long long lak, const float* B, long long lbk,
          long long lbn, float* C, long long ldc, const float* bias, float* Cpre, bool atomic_acc, cudaStream_t st) {
  int chunk = K;
  int splits = 1;
  if (atomic_acc) {
    // enough K-splits to fill the GPU (~4 blocks per SM)
    const long long tiles = (long long)((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
    long long want = (152 * 4 + tiles - 1) / tiles;
    chunk = (int)((K + want - 1) / want);
    chunk = ((chunk + kBK - 1) / kBK) * kBK;
    if (chunk < kBK) chunk = kBK;
    splits = (K + chunk - 1) / chunk;
  }
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splits);
  GS_TRACE("k_gemm", st);
  k_gemm<EPI><<<grid, 256, 0, st>>>(M, N, K, A, lam, lak, B, lbk, lbn, C, ldc, bias, Cpre, chunk, atomic_acc ? 1 : 0);
}

struct DecLayout {
  size_t idx, Z, T, PRE, H, Y, DH, DZ, total;
};

DecLayout dec_layout(long long S, int din, int dh, int dout) {
  DecLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.idx = take((size_t)S * 4);
  L.Z = take((size_t)S * din * 4);
  L.T = take((size_t)S * dout * 4);
  L.PRE = take((size_t)S * dh * 4);
  L.H = take((size_t)S * dh * 4);
  L.Y = take((size_t)S * dout * 4);
  L.DH = take((size_t)S * dh * 4);
  L.DZ = take((size_t)S * din * 4);
  L.total = o;
  return L;
}

bool dec_ok(const gs_decoder* d) {
  return d && d->din > 0 && d->din <= 64 && d->dh > 0 && d->dh <= 1024 && d->dout > 0 && d->dout <= 4096 && d->W1 &&
         d->b1 && d->W2 && d->b2;
}

}  // namespace
}  // namespace gsff

using namespace gsff;

extern "C" {

size_t gs_decoder_workspace_bytes(const gs_decoder* dec, int64_t n, int32_t training) {
  if (!dec_ok(dec) || n < 0) return 0;
  if (!training) return align_up((size_t)n * dec->dh * 4, 256);  // hidden activations only
  return dec_layout(n, dec->din, dec->dh, dec->dout).total;
}

gs_status gs_decoder_fwd(const gs_decoder* dec, int64_t npix, const float* z, float* y, void* workspace,
                         size_t workspace_bytes, void* stream) {
  if (!dec_ok(dec) || npix < 0 || (npix > 0 && (!z || !y || !workspace))) return GS_ERR_INVALID_ARG;
  if (npix == 0) return GS_OK;
  if (npix >= (1ll << 31) || workspace_bytes < gs_decoder_workspace_bytes(dec, npix, 0)) return GS_ERR_INVALID_ARG;
  float* H = static_cast<float*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int M = (int)npix;
  gemm<EPI_BIAS_GELU>(M, dec->dh, dec->din, z, dec->din, 1, dec->W1, dec->dh, 1, H, dec->dh, dec->b1, nullptr, false,
                      st);
  gemm<EPI_BIAS>(M, dec->dout, dec->dh, H, dec->dh, 1, dec->W2, dec->dout, 1, y, dec->dout, dec->b2, nullptr, false,
                 st);
  return last_launch_status();
}

gs_status gs_decoder_train(const gs_decoder* dec, int64_t nsample, int64_t npix, uint64_t seed, const float* z_map,
                           const float* target, float loss_scale, void* workspace, size_t workspace_bytes, float* dW1,
                           float* db1, float* dW2, float* db2, float* dz_map, float* loss_sum, void* stream) {
  if (!dec_ok(dec) || nsample <= 0 || npix <= 0 || nsample > (1ll << 31) / 8 || npix >= (1ll << 31)) return GS_ERR_INVALID_ARG;
  if (!z_map || !target || !workspace || !dW1 || !db1 || !dW2 || !db2) return GS_ERR_INVALID_ARG;
  const DecLayout L = dec_layout(nsample, dec->din, dec->dh, dec->dout);
  if (workspace_bytes < L.total) return GS_ERR_INVALID_ARG;
  char* ws = static_cast<char*>(workspace);
  int* idx = reinterpret_cast<int*>(ws + L.idx);
  float* Z = reinterpret_cast<float*>(ws + L.Z);
  float* T = reinterpret_cast<float*>(ws + L.T);
  float* PRE = reinterpret_cast<float*>(ws + L.PRE);
  float* H = reinterpret_cast<float*>(ws + L.H);
  float* Y = reinterpret_cast<float*>(ws + L.Y);
  float* DH = reinterpret_cast<float*>(ws + L.DH);
  float* DZ = reinterpret_cast<float*>(ws + L.DZ);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int S = (int)nsample, din = dec->din, dh = dec->dh, dout = dec->dout;
  {
    GS_TRACE("k_sample", st);
    k_sample<<<grid1d(S), 256, 0, st>>>(S, npix, seed, idx);
  }
  {
    GS_TRACE("k_gather", st);
    k_gather<<<grid1d((long long)S * din), 256, 0, st>>>(S, din, idx, z_map, Z);
    k_gather<<<grid1d((long long)S * dout), 256, 0, st>>>(S, dout, idx, target, T);
  }
  // forward
  gemm<EPI_BIAS_GELU>(S, dh, din, Z, din, 1, dec->W1, dh, 1, H, dh, dec->b1, PRE, false, st);
  gemm<EPI_BIAS>(S, dout, dh, H, dh, 1, dec->W2, dout, 1, Y, dout, dec->b2, nullptr, false, st);
  // loss and dL/dY (in place of Y)
  {
    GS_TRACE("k_mse_grad", st);
    k_mse_grad<<<grid1d((long long)S * dout), 256, 0, st>>>((long long)S * dout, Y, T, loss_scale, loss_sum);
  }
  // dW2 += H^T dY ; db2 += colsum dY ; dH = dY W2^T
  gemm<EPI_NONE>(dh, dout, S, H, 1, dh, Y, dout, 1, dW2, dout, nullptr, nullptr, true, st);
  {
    GS_TRACE("k_colsum", st);
    k_colsum<<<dim3((dout + 31) / 32, 64), 256, 0, st>>>(S, dout, Y, db2);
  }
  gemm<EPI_NONE>(S, dh, dout, Y, dout, 1, dec->W2, 1, dout, DH, dh, nullptr, nullptr, false, st);
  {
    GS_TRACE("k_gelu_bwd", st);
    k_gelu_bwd<<<grid1d((long long)S * dh), 256, 0, st>>>((long long)S * dh, DH, PRE);
  }
  // dW1 += Z^T dPRE ; db1 += colsum dPRE ; dZ = dPRE W1^T, scattered to the pixels
  gemm<EPI_NONE>(din, dh, S, Z, 1, din, DH, dh, 1, dW1, dh, nullptr, nullptr, true, st);
  {
    GS_TRACE("k_colsum", st);
    k_colsum<<<dim3((dh + 31) / 32, 64), 256, 0, st>>>(S, dh, DH, db1);
  }
  if (dz_map) {
    gemm<EPI_NONE>(S, din, dh, DH, dh, 1, dec->W1, 1, dh, DZ, din, nullptr, nullptr, false, st);
    GS_TRACE("k_scatter_add", st);
    k_scatter_add<<<grid1d((long long)S * din), 256, 0, st>>>(S, din, idx, DZ, dz_map);
  }
  return last_launch_status();
}

gs_status gs_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr, float beta1,
                       float beta2, float eps, int32_t step, float* param_bf16, void* stream) {
  if (n < 0 || (n > 0 && (!param || !grad || !m || !v)) || step < 1) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GS_TRACE("k_adam", st);
  k_adam<<<grid1d(n), 256, 0, st>>>(n, param, grad, m, v, lr, beta1, beta2, eps, c1, c2, param_bf16);
  return last_launch_status();
}

}  // extern "C"
