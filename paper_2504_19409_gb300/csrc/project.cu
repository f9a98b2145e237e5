// EWA projection of 3D Gaussians (Sec. 3.1, Eq. 1) and its adjoint with the
// Lie-algebra pose gradient (Sec. 3.2, Eq. 4).
//
// Forward: one thread per Gaussian, every operation an explicitly rounded
// binary32 operation (__f*_rn, no contraction) in the order documented in
// gsff.h's gs_project, so that tile rectangles and depth keys are
// reproducible bit for bit. HBM-bound: 44 B read, 48 B written per Gaussian.
//
// Backward: one thread per Gaussian recomputes the forward quantities and
// applies the chain rule back to mean, scale and quaternion; the pose
// tangent partials are reduced per block and added atomically.

#include "gsff_internal.cuh"

namespace gsff {
namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }

__global__ void __launch_bounds__(256) k_project(const CamF cam, int P, const float* __restrict__ means,
                                                 const float* __restrict__ scales,
                                                 const float* __restrict__ quats,
                                                 const float* __restrict__ opacity, float2* __restrict__ uv,
                                                 float4* __restrict__ co, float* __restrict__ depth,
                                                 int4* __restrict__ rect, int* __restrict__ touched,
                                                 unsigned long long* __restrict__ n_inst) {
  pdl_wait();
  pdl_trigger();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  int count = 0;
  if (g < P) {
    bool vis = false;
    float u = 0.f, v = 0.f, A = 0.f, B = 0.f, C = 0.f, zc = 0.f, o = 0.f;
    int r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    do {
      const float m0 = means[3 * g], m1 = means[3 * g + 1], m2 = means[3 * g + 2];
      const float s0 = scales[3 * g], s1 = scales[3 * g + 1], s2 = scales[3 * g + 2];
      const float4 q = reinterpret_cast<const float4*>(quats)[g];
      o = opacity[g];
      if (!(isfinite(m0) && isfinite(m1) && isfinite(m2) && isfinite(s0) && isfinite(s1) &&
            isfinite(s2) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w) &&
            isfinite(o)))
        break;
      float R[9], tc[3];
      cam_pose(cam, R, tc);
      const float xc = fa(fa(fa(fm(R[0], m0), fm(R[1], m1)), fm(R[2], m2)), tc[0]);
      const float yc = fa(fa(fa(fm(R[3], m0), fm(R[4], m1)), fm(R[5], m2)), tc[1]);
      zc = fa(fa(fa(fm(R[6], m0), fm(R[7], m1)), fm(R[8], m2)), tc[2]);
      if (!(zc > cam.near_z)) break;
      float qw = q.x, qx = q.y, qy = q.z, qz = q.w;
      const float qq = fa(fa(fa(fm(qw, qw), fm(qx, qx)), fm(qy, qy)), fm(qz, qz));
      if (!(qq > 0.f)) break;
      const float qn = __fsqrt_rn(qq);
      qw = fdv(qw, qn);
      qx = fdv(qx, qn);
      qy = fdv(qy, qn);
      qz = fdv(qz, qn);
      float r[9];
      r[0] = fs(1.f, fm(2.f, fa(fm(qy, qy), fm(qz, qz))));
      r[1] = fm(2.f, fs(fm(qx, qy), fm(qw, qz)));
      r[2] = fm(2.f, fa(fm(qx, qz), fm(qw, qy)));
      r[3] = fm(2.f, fa(fm(qx, qy), fm(qw, qz)));
      r[4] = fs(1.f, fm(2.f, fa(fm(qx, qx), fm(qz, qz))));
      r[5] = fm(2.f, fs(fm(qy, qz), fm(qw, qx)));
      r[6] = fm(2.f, fs(fm(qx, qz), fm(qw, qy)));
      r[7] = fm(2.f, fa(fm(qy, qz), fm(qw, qx)));
      r[8] = fs(1.f, fm(2.f, fa(fm(qx, qx), fm(qy, qy))));
      const float sv[3] = {s0, s1, s2};
      float M[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = fm(r[3 * i + j], sv[j]);
      const float Wf = (float)cam.W, Hf = (float)cam.H;
      const float limx = fm(kGuardBand, fdv(Wf, fm(2.f, cam.fx)));
      const float limy = fm(kGuardBand, fdv(Hf, fm(2.f, cam.fy)));
      const float tx = fdv(xc, zc), ty = fdv(yc, zc);
      const float xcl = fm(fminf(limx, fmaxf(-limx, tx)), zc);
      const float ycl = fm(fminf(limy, fmaxf(-limy, ty)), zc);
      const float zz = fm(zc, zc);
      const float J00 = fdv(cam.fx, zc), J02 = -fdv(fm(cam.fx, xcl), zz);
      const float J11 = fdv(cam.fy, zc), J12 = -fdv(fm(cam.fy, ycl), zz);
      float T[6];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T[j] = fa(fm(J00, R[j]), fm(J02, R[6 + j]));
        T[3 + j] = fa(fm(J11, R[3 + j]), fm(J12, R[6 + j]));
      }
      float V[6];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          V[3 * i + j] = fa(fa(fm(T[3 * i], M[j]), fm(T[3 * i + 1], M[3 + j])), fm(T[3 * i + 2], M[6 + j]));
      const float a = fa(fa(fa(fm(V[0], V[0]), fm(V[1], V[1])), fm(V[2], V[2])), kLowPass);
      const float b = fa(fa(fm(V[0], V[3]), fm(V[1], V[4])), fm(V[2], V[5]));
      const float c = fa(fa(fa(fm(V[3], V[3]), fm(V[4], V[4])), fm(V[5], V[5])), kLowPass);
      const float det = fs(fm(a, c), fm(b, b));
      if (!(det > 0.f) || !isfinite(det)) break;
      A = fdv(c, det);
      B = fdv(-b, det);
      C = fdv(a, det);
      u = fa(fm(cam.fx, tx), cam.cx);
      v = fa(fm(cam.fy, ty), cam.cy);
      if (!isfinite(u) || !isfinite(v)) break;
      const float mid = fm(0.5f, fa(a, c));
      const float lam = fa(mid, __fsqrt_rn(fmaxf(kEigFloor, fs(fm(mid, mid), det))));
      const float rad = ceilf(fm(kSigmas, __fsqrt_rn(lam)));
      if (!isfinite(rad)) break;
      float i0 = ceilf(fs(fs(u, rad), 0.5f)), i1 = floorf(fs(fa(u, rad), 0.5f));
      float j0 = ceilf(fs(fs(v, rad), 0.5f)), j1 = floorf(fs(fa(v, rad), 0.5f));
      i0 = fmaxf(i0, 0.f);
      j0 = fmaxf(j0, 0.f);
      i1 = fminf(i1, Wf - 1.f);
      j1 = fminf(j1, Hf - 1.f);
      if (i0 > i1 || j0 > j1) break;
      r0 = (int)i0 / kTile;
      r1 = (int)j0 / kTile;
      r2 = (int)i1 / kTile + 1;
      r3 = (int)j1 / kTile + 1;
      vis = true;
    } while (false);
    if (vis) {
      uv[g] = make_float2(u, v);
      co[g] = make_float4(A, B, C, o);
      depth[g] = zc;
      rect[g] = make_int4(r0, r1, r2, r3);
      count = (r2 - r0) * (r3 - r1);
    } else {
      uv[g] = make_float2(0.f, 0.f);
      co[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      depth[g] = 0.f;
      rect[g] = make_int4(0, 0, 0, 0);
    }
    touched[g] = count;
  }
  if (n_inst) {
    unsigned long long c = (unsigned long long)count;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_inst, c);
  }
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Adjoint of the projection. The forward quantities are recomputed in plain
// fp32 (the backward needs no bit-exact replay). Chain:
//   conic = inverse(cov)          : dcov = -K G K
//   cov = V V^T + 0.3 I           : dV = 2 dcov V
//   V = T M, T = J W, M = Rq S    : dT = dV M^T, dM = T^T dV, dRq = dM S, ds = diag(Rq^T dM)
//   Rq(q / |q|)                   : quaternion partials, then the projection onto |q|
//   J(z, x', y'), x' = clamp(x/z) z: x' = x when free, +-lim z when clamped
//   u = fx x/z + cx, depth = z, mu_c = W mu + t
//   pose (left perturbation, Eq. 4): drho = dmu_c,
//   dtheta = mu_c x dmu_c + sum_k W_k x dW_k.
// Only the Gaussians that received an image gradient (a small share of a
// frame's) have work: each block first queues those among its kPbPer * 256
// Gaussians in shared memory, then processes the queue densely.
constexpr int kPbPer = 4;
__global__ void __launch_bounds__(256) k_project_bwd(
    const CamF cam, int P, const float* __restrict__ means, const float* __restrict__ scales,
    const float* __restrict__ quats, const float2* __restrict__ d_uv, const float* __restrict__ d_conic,
    const float* __restrict__ d_depth, float* __restrict__ d_means, float* __restrict__ d_scales,
    float* __restrict__ d_quats, float* __restrict__ d_pose) {
  pdl_wait();
  pdl_trigger();
  __shared__ int s_q[kPbPer * 256];
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int base = blockIdx.x * kPbPer * 256;
#pragma unroll
  for (int r = 0; r < kPbPer; ++r) {
    const int g = base + r * 256 + threadIdx.x;
    bool any = false;
    if (g < P) {
      const float2 duv = d_uv[g];
      any = (duv.x != 0.f) | (duv.y != 0.f) | (d_conic[3 * g] != 0.f) | (d_conic[3 * g + 1] != 0.f) |
            (d_conic[3 * g + 2] != 0.f) | (d_depth[g] != 0.f);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, any);
    int at = 0;
    if ((threadIdx.x & 31) == 0 && bal) at = atomicAdd(&s_n, __popc(bal));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (any) s_q[at + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = g;
  }
  __syncthreads();
  const int nq = s_n;
  float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int e = threadIdx.x; e < nq; e += 256) {
    const int g = s_q[e];
    const float2 duv = d_uv[g];
    const float dA = d_conic[3 * g], dB = d_conic[3 * g + 1], dC = d_conic[3 * g + 2];
    const float dd = d_depth[g];
    const float m0 = means[3 * g], m1 = means[3 * g + 1], m2 = means[3 * g + 2];
    float R[9], tc[3];
    cam_pose(cam, R, tc);
    const float x = R[0] * m0 + R[1] * m1 + R[2] * m2 + tc[0];
    const float y = R[3] * m0 + R[4] * m1 + R[5] * m2 + tc[1];
    const float z = R[6] * m0 + R[7] * m1 + R[8] * m2 + tc[2];
    if (z > cam.near_z) {
      const float s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
      const float4 q4 = reinterpret_cast<const float4*>(quats)[g];
      const float qnorm = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
      const float w = q4.x / qnorm, qx = q4.y / qnorm, qy = q4.z / qnorm, qz = q4.w / qnorm;
      float r[9];
      r[0] = 1.f - 2.f * (qy * qy + qz * qz);
      r[1] = 2.f * (qx * qy - w * qz);
      r[2] = 2.f * (qx * qz + w * qy);
      r[3] = 2.f * (qx * qy + w * qz);
      r[4] = 1.f - 2.f * (qx * qx + qz * qz);
      r[5] = 2.f * (qy * qz - w * qx);
      r[6] = 2.f * (qx * qz - w * qy);
      r[7] = 2.f * (qy * qz + w * qx);
      r[8] = 1.f - 2.f * (qx * qx + qy * qy);
      float M[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = r[3 * i + j] * s[j];
      const float limx = kGuardBand * ((float)cam.W / (2.f * cam.fx));
      const float limy = kGuardBand * ((float)cam.H / (2.f * cam.fy));
      const float tx = x / z, ty = y / z;
      const int clx = tx > limx ? 1 : (tx < -limx ? -1 : 0);
      const int cly = ty > limy ? 1 : (ty < -limy ? -1 : 0);
      const float xcl = fminf(limx, fmaxf(-limx, tx)) * z;
      const float ycl = fminf(limy, fmaxf(-limy, ty)) * z;
      const float iz = 1.f / z, iz2 = iz * iz, iz3 = iz2 * iz;
      const float J00 = cam.fx * iz, J02 = -cam.fx * xcl * iz2;
      const float J11 = cam.fy * iz, J12 = -cam.fy * ycl * iz2;
      float T[6];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T[j] = J00 * R[j] + J02 * R[6 + j];
        T[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
      }
      float V[6];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[3 * i + j] = T[3 * i] * M[j] + T[3 * i + 1] * M[3 + j] + T[3 * i + 2] * M[6 + j];
      const float a = V[0] * V[0] + V[1] * V[1] + V[2] * V[2] + kLowPass;
      const float b = V[0] * V[3] + V[1] * V[4] + V[2] * V[5];
      const float c = V[3] * V[3] + V[4] * V[4] + V[5] * V[5] + kLowPass;
      const float idet = 1.f / (a * c - b * b);
      const float K0 = c * idet, K1 = -b * idet, K2 = a * idet;
      // dcov = -K G K with G = [[dA, dB/2], [dB/2, dC]]
      const float G1 = 0.5f * dB;
      const float KG00 = K0 * dA + K1 * G1, KG01 = K0 * G1 + K1 * dC;
      const float KG10 = K1 * dA + K2 * G1, KG11 = K1 * G1 + K2 * dC;
      const float c00 = -(KG00 * K0 + KG01 * K1);
      const float c01 = -(KG00 * K1 + KG01 * K2);
      const float c11 = -(KG10 * K1 + KG11 * K2);
      // dV = 2 dcov V
      float dV[6];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dV[j] = 2.f * (c00 * V[j] + c01 * V[3 + j]);
        dV[3 + j] = 2.f * (c01 * V[j] + c11 * V[3 + j]);
      }
      // dT = dV M^T ; dM = T^T dV
      float dT[6], dM[9];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          dT[3 * i + l] = dV[3 * i] * M[3 * l] + dV[3 * i + 1] * M[3 * l + 1] + dV[3 * i + 2] * M[3 * l + 2];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j) dM[3 * l + j] = T[l] * dV[j] + T[3 + l] * dV[3 + j];
      // M = Rq diag(s)
      float dr[9];
      float ds[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          ds[j] += dM[3 * i + j] * r[3 * i + j];
          dr[3 * i + j] = dM[3 * i + j] * s[j];
        }
      // quaternion partials of each rotation entry
      float dqw = -2.f * qz * dr[1] + 2.f * qy * dr[2] + 2.f * qz * dr[3] - 2.f * qx * dr[5] - 2.f * qy * dr[6] +
                  2.f * qx * dr[7];
      float dqx = 2.f * qy * dr[1] + 2.f * qz * dr[2] + 2.f * qy * dr[3] - 4.f * qx * dr[4] - 2.f * w * dr[5] +
                  2.f * qz * dr[6] + 2.f * w * dr[7] - 4.f * qx * dr[8];
      float dqy = -4.f * qy * dr[0] + 2.f * qx * dr[1] + 2.f * w * dr[2] + 2.f * qx * dr[3] + 2.f * qz * dr[5] -
                  2.f * w * dr[6] + 2.f * qz * dr[7] - 4.f * qy * dr[8];
      float dqz = -4.f * qz * dr[0] - 2.f * w * dr[1] + 2.f * qx * dr[2] + 2.f * w * dr[3] - 4.f * qz * dr[4] +
                  2.f * qy * dr[5] + 2.f * qx * dr[6] + 2.f * qy * dr[7];
      const float dot = w * dqw + qx * dqx + qy * dqy + qz * dqz;
      const float iq = 1.f / qnorm;
      if (d_quats) {
        d_quats[4 * g + 0] += (dqw - w * dot) * iq;
        d_quats[4 * g + 1] += (dqx - qx * dot) * iq;
        d_quats[4 * g + 2] += (dqy - qy * dot) * iq;
        d_quats[4 * g + 3] += (dqz - qz * dot) * iq;
      }
      if (d_scales) {
        d_scales[3 * g + 0] += ds[0];
        d_scales[3 * g + 1] += ds[1];
        d_scales[3 * g + 2] += ds[2];
      }
      // T = J W: dJ = dT W^T (entries 00, 02, 11, 12), dW = J^T dT
      const float dJ00 = dT[0] * R[0] + dT[1] * R[1] + dT[2] * R[2];
      const float dJ02 = dT[0] * R[6] + dT[1] * R[7] + dT[2] * R[8];
      const float dJ11 = dT[3] * R[3] + dT[4] * R[4] + dT[5] * R[5];
      const float dJ12 = dT[3] * R[6] + dT[4] * R[7] + dT[5] * R[8];
      float dW[9];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dW[j] = J00 * dT[j];
        dW[3 + j] = J11 * dT[3 + j];
        dW[6 + j] = J02 * dT[j] + J12 * dT[3 + j];
      }
      float dx = 0.f, dy = 0.f, dz = 0.f;
      dz += -cam.fx * iz2 * dJ00 - cam.fy * iz2 * dJ11 + 2.f * cam.fx * xcl * iz3 * dJ02 +
            2.f * cam.fy * ycl * iz3 * dJ12;
      const float dxcl = -cam.fx * iz2 * dJ02, dycl = -cam.fy * iz2 * dJ12;
      if (clx == 0) dx += dxcl; else dz += (float)clx * limx * dxcl;
      if (cly == 0) dy += dycl; else dz += (float)cly * limy * dycl;
      dx += cam.fx * iz * duv.x;
      dy += cam.fy * iz * duv.y;
      dz += -cam.fx * x * iz2 * duv.x - cam.fy * y * iz2 * duv.y + dd;
      if (d_means) {
        d_means[3 * g + 0] += R[0] * dx + R[3] * dy + R[6] * dz;
        d_means[3 * g + 1] += R[1] * dx + R[4] * dy + R[7] * dz;
        d_means[3 * g + 2] += R[2] * dx + R[5] * dy + R[8] * dz;
      }
      pose[0] += dx;
      pose[1] += dy;
      pose[2] += dz;
      float3 th = cross3(make_float3(x, y, z), make_float3(dx, dy, dz));
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float3 c3 = cross3(make_float3(R[k], R[3 + k], R[6 + k]), make_float3(dW[k], dW[3 + k], dW[6 + k]));
        th.x += c3.x;
        th.y += c3.y;
        th.z += c3.z;
      }
      pose[3] += th.x;
      pose[4] += th.y;
      pose[5] += th.z;
    }
  }
  // block reduction of the pose partials
  __shared__ float red[8][6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float vsum = pose[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = vsum;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float vsum = 0.f;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) vsum += red[wi][threadIdx.x];
    if (vsum != 0.f) atomicAdd(&d_pose[threadIdx.x], vsum);
  }
}

}  // namespace

void launch_project(const CamF& cam, int P, const float* means, const float* scales, const float* quats,
                    const float* opacity, float* uv, float* co, float* depth, int32_t* rect, int32_t* touched,
                    int64_t* n_inst, cudaStream_t st) {
  if (P <= 0) return;
  GS_TRACE("k_project", st);
  launch_pdl(k_project, (P + 255) / 256, 256, 0, st, cam, P, means, scales, quats, opacity, reinterpret_cast<float2*>(uv),
                                             reinterpret_cast<float4*>(co), depth, reinterpret_cast<int4*>(rect),
                                             touched, reinterpret_cast<unsigned long long*>(n_inst));
}

void launch_project_bwd(const CamF& cam, int P, const float* means, const float* scales, const float* quats,
                        const float* d_uv, const float* d_conic, const float* d_depth, float* d_means,
                        float* d_scales, float* d_quats, float* d_pose, cudaStream_t st) {
  if (P <= 0) return;
  GS_TRACE("k_project_bwd", st);
  launch_pdl(k_project_bwd, (P + kPbPer * 256 - 1) / (kPbPer * 256), 256, 0, st, cam, P, means, scales, quats,
                                                 reinterpret_cast<const float2*>(d_uv), d_conic, d_depth, d_means,
                                                 d_scales, d_quats, d_pose);
}

}  // namespace gsff
