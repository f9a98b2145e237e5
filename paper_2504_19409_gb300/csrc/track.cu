// Camera tracking (Sec. 3.2): the tracking loss of Eq. 6 and the pose update.
//
//   L = lambda_t m_v m_e L_c + (1 - lambda_t) m_v L_d,
//
// L_c, L_d the L1 colour and depth terms (means over the pixels), m_v the
// 2D visibility mask recorded from the frame's first render, m_e the mask of
// pixels with a significant gradient in the observed image. The pose is
// optimised on its tangent at the current estimate (the left perturbation of
// Eq. 4) and updated as T <- Exp(delta) T; tracking stops when the update's
// translation and rotation fall under tolerances (the convergence of the
// changes of mu_c and W).
//
// Readings where the paper is silent:
//   - m_e: Sobel gradient (1/8-normalised) of the luminance (r + g + b) / 3
//     with replicated borders; an edge pixel has |grad|^2 > tau^2. The
//     decision is taken in binary32 with one fixed order of operations.
//   - m_v: accumulated opacity of the first render above a threshold.
//   - the depth term also requires observed depth > 0 (holes carry no
//     information).
//   - the optimiser is Adam on the 6-vector tangent (separate step sizes for
//     the translation and rotation parts), reset per frame.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

__device__ __forceinline__ float lum(const float* rgb, size_t HW, int W, int x, int y) {
  const size_t p = (size_t)y * W + x;
  return __fmul_rn(__fadd_rn(__fadd_rn(rgb[p], rgb[HW + p]), rgb[2 * HW + p]), 1.f / 3.f);
}

__global__ void __launch_bounds__(256) k_edge_mask(int W, int H, const float* __restrict__ rgb, float tau,
                                                   uint8_t* __restrict__ m_e) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= W || y >= H) return;
  const size_t HW = (size_t)W * H;
  const int xm = max(x - 1, 0), xp = min(x + 1, W - 1), ym = max(y - 1, 0), yp = min(y + 1, H - 1);
  const float a = __fadd_rn(__fadd_rn(lum(rgb, HW, W, xp, ym), __fmul_rn(2.f, lum(rgb, HW, W, xp, y))),
                            lum(rgb, HW, W, xp, yp));
  const float b = __fadd_rn(__fadd_rn(lum(rgb, HW, W, xm, ym), __fmul_rn(2.f, lum(rgb, HW, W, xm, y))),
                            lum(rgb, HW, W, xm, yp));
  const float c = __fadd_rn(__fadd_rn(lum(rgb, HW, W, xm, yp), __fmul_rn(2.f, lum(rgb, HW, W, x, yp))),
                            lum(rgb, HW, W, xp, yp));
  const float d = __fadd_rn(__fadd_rn(lum(rgb, HW, W, xm, ym), __fmul_rn(2.f, lum(rgb, HW, W, x, ym))),
                            lum(rgb, HW, W, xp, ym));
  const float gx = __fmul_rn(__fsub_rn(a, b), 0.125f), gy = __fmul_rn(__fsub_rn(c, d), 0.125f);
  const float mag2 = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
  m_e[(size_t)y * W + x] = mag2 > __fmul_rn(tau, tau) ? 1 : 0;
}

__device__ __forceinline__ float sgn(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(256) k_tracking_grad(int HW, const float* __restrict__ rgb,
                                                       const float* __restrict__ depth,
                                                       const float* __restrict__ gt_rgb,
                                                       const float* __restrict__ gt_depth,
                                                       const float* __restrict__ alpha_ref, float alpha_min,
                                                       const uint8_t* __restrict__ m_e, float sc, float sd,
                                                       float* __restrict__ g_rgb, float* __restrict__ g_depth,
                                                       float* __restrict__ loss) {
  float acc = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const bool mv = alpha_ref[p] > alpha_min;
    const bool col = mv && m_e[p] != 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = (size_t)c * HW + p;
      const float d = rgb[i] - gt_rgb[i];
      g_rgb[i] = col ? sc * sgn(d) : 0.f;
      if (col) acc += sc * fabsf(d);
    }
    const float dg = gt_depth[p];
    const bool dep = mv && dg > 0.f;
    const float d = depth[p] - dg;
    g_depth[p] = dep ? sd * sgn(d) : 0.f;
    if (dep) acc += sd * fabsf(d);
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

// The same terms as k_tracking_grad, kept as sign words (bits 16..18 colour,
// 19 depth; see L1Fwd) for the L1 adjoint: a cotangent is nonzero where its
// mask holds and the difference is not 0, negative where the difference is.
__global__ void __launch_bounds__(256) k_tracking_signs(int HW, const float* __restrict__ rgb,
                                                        const float* __restrict__ depth,
                                                        const float* __restrict__ gt_rgb,
                                                        const float* __restrict__ gt_depth,
                                                        const float* __restrict__ alpha_ref, float alpha_min,
                                                        const uint8_t* __restrict__ m_e, float sc, float sd,
                                                        uint2* __restrict__ signs, float* __restrict__ loss) {
  float acc = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const bool mv = alpha_ref[p] > alpha_min;
    const bool col = mv && m_e[p] != 0;
    uint32_t nz = 0, ng = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = (size_t)c * HW + p;
      const float d = rgb[i] - gt_rgb[i];
      if (col) {
        nz |= (d != 0.f ? 1u : 0u) << (kL1BitRgb + c);
        ng |= (d < 0.f ? 1u : 0u) << (kL1BitRgb + c);
        acc += sc * fabsf(d);
      }
    }
    const float dg = gt_depth[p];
    const bool dep = mv && dg > 0.f;
    const float d = depth[p] - dg;
    if (dep) {
      nz |= (d != 0.f ? 1u : 0u) << kL1BitDepth;
      ng |= (d < 0.f ? 1u : 0u) << kL1BitDepth;
      acc += sd * fabsf(d);
    }
    signs[p] = make_uint2(nz, ng);
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

struct PoseUpdate {
  float lr_trans, lr_rot, beta1, beta2, eps, tol_trans, tol_rot;
  int step;
};

// One thread: Adam on the tangent, then T <- Exp(delta) T with the SE(3)
// exponential (Rodrigues' rotation and the V matrix that maps rho to the
// translation), series forms below 1e-4 rad.
__global__ void k_pose_update(float* __restrict__ pose, const float* __restrict__ d_pose, float* __restrict__ m,
                              float* __restrict__ v, PoseUpdate u, int32_t* __restrict__ converged) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float bc1 = 1.f - powf(u.beta1, (float)u.step), bc2 = 1.f - powf(u.beta2, (float)u.step);
  float dl[6];
  for (int i = 0; i < 6; ++i) {
    const float g = d_pose[i];
    m[i] = u.beta1 * m[i] + (1.f - u.beta1) * g;
    v[i] = u.beta2 * v[i] + (1.f - u.beta2) * g * g;
    const float lr = i < 3 ? u.lr_trans : u.lr_rot;
    dl[i] = -lr * (m[i] / bc1) / (sqrtf(v[i] / bc2) + u.eps);
  }
  const float w0 = dl[3], w1 = dl[4], w2 = dl[5];
  const float phi2 = w0 * w0 + w1 * w1 + w2 * w2, phi = sqrtf(phi2);
  float A, B, C;
  if (phi < 1e-4f) {
    A = 1.f - phi2 / 6.f;
    B = 0.5f - phi2 / 24.f;
    C = 1.f / 6.f - phi2 / 120.f;
  } else {
    const float s = sinf(phi), c = cosf(phi);
    A = s / phi;
    B = (1.f - c) / phi2;
    C = (phi - s) / (phi2 * phi);
  }
  // K = [w]x, K2 = K K
  const float K[9] = {0.f, -w2, w1, w2, 0.f, -w0, -w1, w0, 0.f};
  float K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
  float Rd[9], V[9];
  for (int i = 0; i < 9; ++i) {
    const float I = (i % 4 == 0) ? 1.f : 0.f;
    Rd[i] = I + A * K[i] + B * K2[i];
    V[i] = I + B * K[i] + C * K2[i];
  }
  float td[3];
  for (int i = 0; i < 3; ++i) td[i] = V[3 * i] * dl[0] + V[3 * i + 1] * dl[1] + V[3 * i + 2] * dl[2];
  float R[9], t[3];
  for (int i = 0; i < 9; ++i) R[i] = pose[i];
  for (int i = 0; i < 3; ++i) t[i] = pose[9 + i];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      pose[3 * i + j] = Rd[3 * i] * R[j] + Rd[3 * i + 1] * R[3 + j] + Rd[3 * i + 2] * R[6 + j];
    pose[9 + i] = Rd[3 * i] * t[0] + Rd[3 * i + 1] * t[1] + Rd[3 * i + 2] * t[2] + td[i];
  }
  if (converged) {
    const float tn = sqrtf(td[0] * td[0] + td[1] * td[1] + td[2] * td[2]);
    *converged = (tn < u.tol_trans && phi < u.tol_rot) ? 1 : 0;
  }
}

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace gsff

using namespace gsff;

extern "C" {

gs_status gs_edge_mask(int32_t width, int32_t height, const float* rgb, float tau, uint8_t* m_e, void* stream) {
  if (width <= 0 || height <= 0 || width > (1 << 15) || height > (1 << 15) || !rgb || !m_e || !(tau >= 0.f))
    return GS_ERR_INVALID_ARG;
  const dim3 grid((width + 31) / 32, (height + 7) / 8);
  GS_TRACE("k_edge_mask", S(stream));
  k_edge_mask<<<grid, 256, 0, S(stream)>>>(width, height, rgb, tau, m_e);
  return last_launch_status();
}

gs_status gs_tracking_loss_grad(int32_t width, int32_t height, const float* rgb, const float* depth,
                                const float* gt_rgb, const float* gt_depth, const float* alpha_ref, float alpha_min,
                                const uint8_t* m_e, float lambda_t, float* g_rgb, float* g_depth, float* loss_sum,
                                void* stream) {
  if (width <= 0 || height <= 0 || width > (1 << 15) || height > (1 << 15)) return GS_ERR_INVALID_ARG;
  if (!rgb || !depth || !gt_rgb || !gt_depth || !alpha_ref || !m_e || !g_rgb || !g_depth) return GS_ERR_INVALID_ARG;
  if (!(lambda_t >= 0.f && lambda_t <= 1.f)) return GS_ERR_INVALID_ARG;
  const int HW = width * height;
  const float sc = (float)((double)lambda_t / (3.0 * HW)), sd = (float)((1.0 - (double)lambda_t) / HW);
  int blocks = (HW + 1023) / 1024;
  if (blocks > 152 * 8) blocks = 152 * 8;
  GS_TRACE("k_tracking_grad", S(stream));
  k_tracking_grad<<<blocks, 256, 0, S(stream)>>>(HW, rgb, depth, gt_rgb, gt_depth, alpha_ref, alpha_min, m_e, sc, sd,
                                                 g_rgb, g_depth, loss_sum);
  return last_launch_status();
}

gs_status gs_tracking_loss_signs(int32_t width, int32_t height, const float* rgb, const float* depth,
                                 const float* gt_rgb, const float* gt_depth, const float* alpha_ref, float alpha_min,
                                 const uint8_t* m_e, float lambda_t, uint32_t* l1_signs, float* weights,
                                 float* loss_sum, void* stream) {
  if (width <= 0 || height <= 0 || width > (1 << 15) || height > (1 << 15)) return GS_ERR_INVALID_ARG;
  if (!rgb || !depth || !gt_rgb || !gt_depth || !alpha_ref || !m_e || !l1_signs || !weights) return GS_ERR_INVALID_ARG;
  if (!(lambda_t >= 0.f && lambda_t <= 1.f) || (reinterpret_cast<uintptr_t>(l1_signs) & 7u)) return GS_ERR_INVALID_ARG;
  const int HW = width * height;
  const float sc = (float)((double)lambda_t / (3.0 * HW)), sd = (float)((1.0 - (double)lambda_t) / HW);
  weights[0] = sc;
  weights[1] = sd;
  int blocks = (HW + 1023) / 1024;
  if (blocks > 152 * 8) blocks = 152 * 8;
  GS_TRACE("k_tracking_signs", S(stream));
  k_tracking_signs<<<blocks, 256, 0, S(stream)>>>(HW, rgb, depth, gt_rgb, gt_depth, alpha_ref, alpha_min, m_e, sc, sd,
                                                  reinterpret_cast<uint2*>(l1_signs), loss_sum);
  return last_launch_status();
}

gs_status gs_pose_update(float* pose_dev, const float* d_pose, float* adam_m, float* adam_v, int32_t step,
                         float lr_trans, float lr_rot, float beta1, float beta2, float eps, float tol_trans,
                         float tol_rot, int32_t* converged, void* stream) {
  if (!pose_dev || !d_pose || !adam_m || !adam_v || step < 1) return GS_ERR_INVALID_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f)) return GS_ERR_INVALID_ARG;
  PoseUpdate u;
  u.lr_trans = lr_trans;
  u.lr_rot = lr_rot;
  u.beta1 = beta1;
  u.beta2 = beta2;
  u.eps = eps;
  u.tol_trans = tol_trans;
  u.tol_rot = tol_rot;
  u.step = step;
  GS_TRACE("k_pose_update", S(stream));
  k_pose_update<<<1, 32, 0, S(stream)>>>(pose_dev, d_pose, adam_m, adam_v, u, converged);
  return last_launch_status();
}

}  // extern "C"
