// View-dependent colour from spherical-harmonic coefficients (Sec. 3.1: the
// colour attribute of a Gaussian is given by third-order SH coefficients).
//
// Per Gaussian g and channel c, with d the unit direction from the camera
// centre C = -R^T t to the mean mu:
//     colour_c = max(0, sum_k sh[g][k][c] Y_k(d) + 0.5),
// k = l^2 + l + m over degrees l <= deg (deg <= 3, K = (deg + 1)^2 terms).
// Y_k is the real SH basis with the Condon-Shortley phase, written as
// polynomials in (x, y, z) = d with normalisations from sqrt(pi); the +0.5
// offset and the clamp at zero follow the 3D Gaussian splatting convention
// the paper builds on (the clamp's gradient is zero).
//
// Adjoint: dL/dsh[g][k][c] = Y_k(d) dL/dcolour_c (unclamped channels);
// the direction receives sum_{k,c} sh[g][k][c] dL/dcolour_c grad Y_k(d), and
// d = v / |v| with v = mu - C gives dv = (I - d d^T) dd / |v|, so
// dL/dmu += dv and dL/dC -= dv. Under the left perturbation of the pose
// (Eq. 4) the camera centre moves with the translation part only at first
// order, dC/drho = -R^T, so drho += R sum_g dv_g and dtheta gets nothing.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

struct ShConst {
  float c0, c1, a, b, cc, e, f, g, h, k;
};

__device__ __forceinline__ ShConst sh_const() {
  const float pi = 3.14159265358979323846f;
  ShConst s;
  s.c0 = 0.5f / sqrtf(pi);
  s.c1 = sqrtf(3.f / (4.f * pi));
  s.a = 0.5f * sqrtf(15.f / pi);
  s.b = 0.25f * sqrtf(5.f / pi);
  s.cc = 0.25f * sqrtf(15.f / pi);
  s.e = 0.25f * sqrtf(35.f / (2.f * pi));
  s.f = 0.5f * sqrtf(105.f / pi);
  s.g = 0.25f * sqrtf(21.f / (2.f * pi));
  s.h = 0.25f * sqrtf(7.f / pi);
  s.k = 0.25f * sqrtf(105.f / pi);
  return s;
}

// Y[0..K) at the unit vector (x, y, z).
__device__ __forceinline__ void sh_basis(const ShConst& s, float x, float y, float z, int K, float (&Y)[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = s.c0;
  if (K > 1) {
    Y[1] = -s.c1 * y;
    Y[2] = s.c1 * z;
    Y[3] = -s.c1 * x;
  }
  if (K > 4) {
    Y[4] = s.a * x * y;
    Y[5] = -s.a * y * z;
    Y[6] = s.b * (2.f * zz - xx - yy);
    Y[7] = -s.a * x * z;
    Y[8] = s.cc * (xx - yy);
  }
  if (K > 9) {
    Y[9] = -s.e * y * (3.f * xx - yy);
    Y[10] = s.f * x * y * z;
    Y[11] = -s.g * y * (4.f * zz - xx - yy);
    Y[12] = s.h * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -s.g * x * (4.f * zz - xx - yy);
    Y[14] = s.k * z * (xx - yy);
    Y[15] = -s.e * x * (xx - 3.f * yy);
  }
}

// w . grad Y for weights w[0..K) (the partial derivatives of the polynomials
// above in x, y and z, as functions on R^3).
__device__ __forceinline__ float3 sh_weighted_grad(const ShConst& s, float x, float y, float z, int K,
                                                   const float (&w)[16]) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (K > 1) {
    gy += -s.c1 * w[1];
    gz += s.c1 * w[2];
    gx += -s.c1 * w[3];
  }
  if (K > 4) {
    gx += s.a * y * w[4];
    gy += s.a * x * w[4];
    gy += -s.a * z * w[5];
    gz += -s.a * y * w[5];
    gx += -2.f * s.b * x * w[6];
    gy += -2.f * s.b * y * w[6];
    gz += 4.f * s.b * z * w[6];
    gx += -s.a * z * w[7];
    gz += -s.a * x * w[7];
    gx += 2.f * s.cc * x * w[8];
    gy += -2.f * s.cc * y * w[8];
  }
  if (K > 9) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += -6.f * s.e * x * y * w[9];
    gy += -s.e * (3.f * xx - 3.f * yy) * w[9];
    gx += s.f * y * z * w[10];
    gy += s.f * x * z * w[10];
    gz += s.f * x * y * w[10];
    gx += 2.f * s.g * x * y * w[11];
    gy += -s.g * (4.f * zz - xx - 3.f * yy) * w[11];
    gz += -8.f * s.g * y * z * w[11];
    gx += -6.f * s.h * x * z * w[12];
    gy += -6.f * s.h * y * z * w[12];
    gz += s.h * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    gx += -s.g * (4.f * zz - 3.f * xx - yy) * w[13];
    gy += 2.f * s.g * x * y * w[13];
    gz += -8.f * s.g * x * z * w[13];
    gx += 2.f * s.k * x * z * w[14];
    gy += -2.f * s.k * y * z * w[14];
    gz += s.k * (xx - yy) * w[14];
    gx += -s.e * (3.f * xx - 3.f * yy) * w[15];
    gy += 6.f * s.e * x * y * w[15];
  }
  return make_float3(gx, gy, gz);
}

// Unit direction from the camera centre to mu, and |mu - C|.
__device__ __forceinline__ float3 view_dir(const CamF& cam, const float* mu, float& len, float (&R)[9]) {
  float t[3];
  cam_pose(cam, R, t);
  const float Cx = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
  const float Cy = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
  const float Cz = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
  const float vx = mu[0] - Cx, vy = mu[1] - Cy, vz = mu[2] - Cz;
  len = sqrtf(vx * vx + vy * vy + vz * vz);
  const float il = len > 0.f ? 1.f / len : 0.f;
  return make_float3(vx * il, vy * il, vz * il);
}

__global__ void __launch_bounds__(256) k_sh_colors(const CamF cam, int P, int K, const float* __restrict__ means,
                                                   const float* __restrict__ sh, float* __restrict__ colors) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= P) return;
  const ShConst s = sh_const();
  float len, R[9];
  const float3 d = view_dir(cam, means + 3 * (size_t)gi, len, R);
  float Y[16];
  sh_basis(s, d.x, d.y, d.z, K, Y);
  const float* c = sh + (size_t)gi * K * 3;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float v = 0.5f;
    for (int k = 0; k < K; ++k) v += c[3 * k + ch] * Y[k];
    colors[3 * (size_t)gi + ch] = fmaxf(v, 0.f);
  }
}

__global__ void __launch_bounds__(256) k_sh_colors_bwd(const CamF cam, int P, int K, const float* __restrict__ means,
                                                       const float* __restrict__ sh,
                                                       const float* __restrict__ d_colors, float* __restrict__ d_sh,
                                                       float* __restrict__ d_means, float* __restrict__ d_pose) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  float dv[3] = {0.f, 0.f, 0.f};
  float R[9];
  if (gi < P) {
    const ShConst s = sh_const();
    float len;
    const float3 d = view_dir(cam, means + 3 * (size_t)gi, len, R);
    float Y[16];
    sh_basis(s, d.x, d.y, d.z, K, Y);
    const float* c = sh + (size_t)gi * K * 3;
    float dc[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float v = 0.5f;
      for (int k = 0; k < K; ++k) v += c[3 * k + ch] * Y[k];
      dc[ch] = v < 0.f ? 0.f : d_colors[3 * (size_t)gi + ch];  // clamped channels pass nothing
    }
    float w[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) w[k] = 0.f;
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        if (d_sh) d_sh[((size_t)gi * K + k) * 3 + ch] += Y[k] * dc[ch];
        w[k] += c[3 * k + ch] * dc[ch];
      }
    }
    if (K > 1 && len > 0.f) {
      const float3 gd = sh_weighted_grad(s, d.x, d.y, d.z, K, w);
      const float dot = gd.x * d.x + gd.y * d.y + gd.z * d.z;
      const float il = 1.f / len;
      dv[0] = (gd.x - d.x * dot) * il;
      dv[1] = (gd.y - d.y * dot) * il;
      dv[2] = (gd.z - d.z * dot) * il;
      if (d_means) {
        d_means[3 * (size_t)gi] += dv[0];
        d_means[3 * (size_t)gi + 1] += dv[1];
        d_means[3 * (size_t)gi + 2] += dv[2];
      }
    }
  } else {
    float t[3];
    cam_pose(cam, R, t);
  }
  if (!d_pose) return;
  // drho += R sum_g dv_g: block sum of dv, then three atomics
  __shared__ float s_dv[3][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float x = dv[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) s_dv[i][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float x = 0.f;
    for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) x += s_dv[threadIdx.x][w8];
    s_dv[threadIdx.x][0] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int i = threadIdx.x;
    const float r = R[3 * i] * s_dv[0][0] + R[3 * i + 1] * s_dv[1][0] + R[3 * i + 2] * s_dv[2][0];
    if (r != 0.f) atomicAdd(d_pose + i, r);
  }
}

bool cam_valid(const gs_camera* cam) {
  return cam && cam->width > 0 && cam->height > 0 && cam->fx > 0.f && cam->fy > 0.f;
}

}  // namespace
}  // namespace gsff

using namespace gsff;

extern "C" {

gs_status gs_sh_colors(const gs_camera* cam, int32_t P, int32_t degree, const float* means, const float* sh,
                       float* colors, void* stream) {
  if (!cam_valid(cam) || P < 0 || degree < 0 || degree > 3) return GS_ERR_INVALID_ARG;
  if (P > 0 && (!means || !sh || !colors)) return GS_ERR_INVALID_ARG;
  if (P == 0) return GS_OK;
  const int K = (degree + 1) * (degree + 1);
  GS_TRACE("k_sh_colors", S(stream));
  k_sh_colors<<<(P + 255) / 256, 256, 0, S(stream)>>>(make_cam(*cam), P, K, means, sh, colors);
  return last_launch_status();
}

gs_status gs_sh_colors_bwd(const gs_camera* cam, int32_t P, int32_t degree, const float* means, const float* sh,
                           const float* d_colors, float* d_sh, float* d_means, float* d_pose, void* stream) {
  if (!cam_valid(cam) || P < 0 || degree < 0 || degree > 3) return GS_ERR_INVALID_ARG;
  if (P > 0 && (!means || !sh || !d_colors)) return GS_ERR_INVALID_ARG;
  if (P == 0) return GS_OK;
  const int K = (degree + 1) * (degree + 1);
  GS_TRACE("k_sh_colors_bwd", S(stream));
  k_sh_colors_bwd<<<(P + 255) / 256, 256, 0, S(stream)>>>(make_cam(*cam), P, K, means, sh, d_colors, d_sh, d_means,
                                                          d_pose);
  return last_launch_status();
}

}  // extern "C"
