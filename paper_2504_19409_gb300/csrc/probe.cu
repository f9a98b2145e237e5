// Throughput probes: the measured denominators of the compositing kernels'
// arithmetic rooflines. Each kernel runs independent dependency chains long
// enough to saturate one pipe, and leaves its values in a sink so that no
// work is dropped; gs_peak_probe reports how many operations a launch does,
// and the caller times the launch (CUDA events on its stream).
//   kind 0: fp32 fused multiply-add, scalar        (2 flop per FMA)
//   kind 1: fp32 fused multiply-add, packed pairs  (4 flop per instruction)
//   kind 2: ex2.approx (the compositing kernels' exponential; 1 op each)
//   kind 3: mma.sync m16n8k16 bf16 x bf16 -> fp32  (4096 flop per warp op)

#include "gsff_internal.cuh"

namespace gsff {
namespace {

constexpr int kChains = 8;

__global__ void k_probe_ffma(int iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.f + 1e-3f * (threadIdx.x + c);
  const float b = 0.9999f, d = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], b, d);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.f) sink[blockIdx.x] = s;
}

__global__ void k_probe_ffma2(int iters, float* sink) {
  float2 a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = make_float2(1.f + 1e-3f * (threadIdx.x + c), 1.f - 1e-3f * c);
  const float2 b = make_float2(0.9999f, 0.9998f), d = make_float2(1e-4f, 2e-4f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], b, d);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
  if (s == 12345.f) sink[blockIdx.x] = s;
}

__global__ void k_probe_ex2(int iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 0.5f + 1e-3f * (threadIdx.x % 64 + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = ex2_approx(-a[c]);  // stays in [0.5, 1]
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.f) sink[blockIdx.x] = s;
}

__global__ void k_probe_mma(int iters, float* sink) {
  // A 16x16 and B 16x8 bf16 fragments (4 + 2 registers per lane), kChains
  // independent 16x8 fp32 accumulators (4 registers each)
  const uint32_t a0 = 0x3F803F80u + threadIdx.x, a1 = 0x3F003F00u, a2 = 0x3E803E80u, a3 = 0x3F403F40u;
  const uint32_t b0 = 0x3F803F80u, b1 = 0x3F003F00u + (threadIdx.x & 7);
  float acc[kChains][4];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
  if (s == 12345.f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace gsff

using namespace gsff;

extern "C" gs_status gs_peak_probe(int32_t kind, int32_t blocks, int32_t threads, int32_t iters, float* sink,
                                   double* ops, void* stream) {
  if (kind < 0 || kind > 3 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1 ||
      !sink || !ops)
    return GS_ERR_INVALID_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double lanes = (double)blocks * threads * iters * kChains;
  switch (kind) {
    case 0:
      k_probe_ffma<<<blocks, threads, 0, st>>>(iters, sink);
      *ops = 2.0 * lanes;
      break;
    case 1:
      k_probe_ffma2<<<blocks, threads, 0, st>>>(iters, sink);
      *ops = 4.0 * lanes;
      break;
    case 2:
      k_probe_ex2<<<blocks, threads, 0, st>>>(iters, sink);
      *ops = lanes;
      break;
    default:
      k_probe_mma<<<blocks, threads, 0, st>>>(iters, sink);
      *ops = 2.0 * 16 * 8 * 16 * (lanes / 32.0);
      break;
  }
  return last_launch_status();
}
