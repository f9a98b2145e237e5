// FP64 CPU oracle for the feature-field Gaussian rasterizer.
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load this library. It shares no code with
// the CUDA path: every formula here is written out again from the paper
// (Sec. 3.1, Eq. 1-4) and from the 3D Gaussian splatting rules the paper builds
// on (Kerbl et al. 2023, cited in Sec. 3.1).
//
// Pieces:
//   ora_project_f64      Eq. 1 covariance, EWA projection, culling, radius,
//                        tile rectangle -- all in double.
//   ora_project_b32      binary32 replay of the projection order of
//                        operations that the GPU promises (see the header
//                        comment of that function). Used only so that the
//                        discrete outputs (tile rectangles, depth key bits)
//                        can be compared bit for bit.
//   ora_bin              per-tile lists sorted by (tile, depth, id).
//   ora_render_fwd       Eq. 2-3 front-to-back compositing in double.
//   ora_visibility       per Gaussian, the largest transmittance in front of
//                        it over the pixels where it is blended (Sec. 3.2:
//                        visible when that transmittance exceeds 0.5).
//   ora_edge_mask        tracking edge mask m_e (Sec. 3.2): binary32 replay
//                        of the Sobel test, so the decision matches bit for bit.
//   ora_tracking_grad    cotangents and value of the tracking loss (Eq. 6).
//   ora_pose_update      Adam on the pose tangent and T <- Exp(delta) T.
//   ora_semantic_ce      Eq. 9 cross-entropy of per-pixel logits and its gradient.
//   ora_label_logits_b32 Eq. 12 logits f . q(l) replayed in binary32 with the
//                        GPU's order of fused multiply-adds (for the argmax).
//   ora_label_probs      Eq. 12 probabilities in double.
//   ora_sh_colors        view-dependent colour from SH coefficients (Sec. 3.1),
//                        the basis from Legendre recurrences, its gradient by
//                        forward-mode dual numbers; ora_sh_colors_bwd its adjoint.
//   ora_render_bwd       adjoint of Eq. 2-3 per pixel from the stored list of
//                        blended Gaussians (no division by 1-alpha).
//   ora_project_bwd_f64  adjoint of the projection and the Lie-algebra pose
//                        gradient of Eq. 4.
//
// Camera arrays are 19 doubles: W, H, fx, fy, cx, cy, R[9] (row-major,
// world->camera), t[3], near. mu_c = R mu + t; OpenCV axes (x right, y down,
// z forward); pixel (i, j) has its centre at (i + 0.5, j + 0.5).
//
// Parity pins: closed forms, invariants, brute force and central finite
// differences in the CPU test suite.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <tuple>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// Constants of the 3DGS rules (Sec. 3.1 builds on them; the paper itself is
// silent on their values).
constexpr double kLowPass = 0.3;        // added to the 2D covariance diagonal
constexpr double kGuard = 1.3;          // guard band of the Jacobian clamp
constexpr double kSigmaK = 3.0;         // radius in standard deviations
constexpr double kEigFloor = 0.1;       // floor under the eigenvalue discriminant
constexpr int kTile = 16;               // 16 x 16 pixel tiles
constexpr double kAlphaMax = 0.99;      // alpha clamp
constexpr double kAlphaMin = 1.0 / 255.0;  // skip below this alpha
constexpr double kTStop = 1e-4;         // stop before T drops below this

struct Cam {
  int W, H;
  double fx, fy, cx, cy, R[9], t[3], near_z;
};

Cam load_cam(const double* c) {
  Cam k;
  k.W = (int)c[0];
  k.H = (int)c[1];
  k.fx = c[2];
  k.fy = c[3];
  k.cx = c[4];
  k.cy = c[5];
  for (int i = 0; i < 9; ++i) k.R[i] = c[6 + i];
  for (int i = 0; i < 3; ++i) k.t[i] = c[15 + i];
  k.near_z = c[18];
  return k;
}

// Rotation matrix of a unit quaternion (w, x, y, z), row-major.
void quat_to_rot(const double q[4], double Rq[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  Rq[0] = 1 - 2 * (y * y + z * z);
  Rq[1] = 2 * (x * y - w * z);
  Rq[2] = 2 * (x * z + w * y);
  Rq[3] = 2 * (x * y + w * z);
  Rq[4] = 1 - 2 * (x * x + z * z);
  Rq[5] = 2 * (y * z - w * x);
  Rq[6] = 2 * (x * z - w * y);
  Rq[7] = 2 * (y * z + w * x);
  Rq[8] = 1 - 2 * (x * x + y * y);
}

struct Proj {
  bool vis = false;
  double mc[3];        // camera-space mean
  double qn[4];        // normalised quaternion
  double qnorm;
  double Rq[9];        // rotation of the Gaussian
  double M[9];         // Rq diag(s)
  double Sigma[9];     // Eq. 1: R S S^T R^T
  double xcl, ycl;     // guard-band-clamped x, y
  int clx, cly;        // 0 free, +1 / -1 clamped at +lim / -lim
  double limx, limy;
  double J[6];         // 2x3 Jacobian of the perspective map
  double Tm[6];        // J R (2x3)
  double cov[3];       // 2D covariance a, b, c (with low-pass)
  double conic[3];     // inverse: A, B, C
  double uv[2];
  double depth;
  double radius;
  int rect[4];         // tile rectangle x0, y0, x1, y1 (end exclusive)
};

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Eq. 1 and the EWA projection in double.
void project_one(const Cam& k, const double m[3], const double s[3], const double q[4], double o,
                 Proj& p) {
  p.vis = false;
  if (!finite_all(m, 3) || !finite_all(s, 3) || !finite_all(q, 4) || !std::isfinite(o)) return;
  for (int i = 0; i < 3; ++i)
    p.mc[i] = k.R[3 * i + 0] * m[0] + k.R[3 * i + 1] * m[1] + k.R[3 * i + 2] * m[2] + k.t[i];
  const double x = p.mc[0], y = p.mc[1], z = p.mc[2];
  if (!(z > k.near_z)) return;
  p.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(p.qnorm > 0)) return;
  for (int i = 0; i < 4; ++i) p.qn[i] = q[i] / p.qnorm;
  quat_to_rot(p.qn, p.Rq);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) p.M[3 * i + j] = p.Rq[3 * i + j] * s[j];
  // Sigma = M M^T  (Eq. 1)
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int l = 0; l < 3; ++l) acc += p.M[3 * i + l] * p.M[3 * j + l];
      p.Sigma[3 * i + j] = acc;
    }
  // Jacobian with the guard-band clamp of x/z, y/z.
  p.limx = kGuard * (k.W / (2.0 * k.fx));
  p.limy = kGuard * (k.H / (2.0 * k.fy));
  const double tx = x / z, ty = y / z;
  p.clx = tx > p.limx ? 1 : (tx < -p.limx ? -1 : 0);
  p.cly = ty > p.limy ? 1 : (ty < -p.limy ? -1 : 0);
  p.xcl = std::min(p.limx, std::max(-p.limx, tx)) * z;
  p.ycl = std::min(p.limy, std::max(-p.limy, ty)) * z;
  p.J[0] = k.fx / z;
  p.J[1] = 0;
  p.J[2] = -k.fx * p.xcl / (z * z);
  p.J[3] = 0;
  p.J[4] = k.fy / z;
  p.J[5] = -k.fy * p.ycl / (z * z);
  // Tm = J R
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j)
      p.Tm[3 * i + j] = p.J[3 * i + 0] * k.R[0 + j] + p.J[3 * i + 1] * k.R[3 + j] + p.J[3 * i + 2] * k.R[6 + j];
  // cov2 = Tm Sigma Tm^T + kLowPass I
  double U[6];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int l = 0; l < 3; ++l) acc += p.Tm[3 * i + l] * p.Sigma[3 * l + j];
      U[3 * i + j] = acc;
    }
  double c2[4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double acc = 0;
      for (int l = 0; l < 3; ++l) acc += U[3 * a + l] * p.Tm[3 * b + l];
      c2[2 * a + b] = acc;
    }
  p.cov[0] = c2[0] + kLowPass;
  p.cov[1] = 0.5 * (c2[1] + c2[2]);
  p.cov[2] = c2[3] + kLowPass;
  const double det = p.cov[0] * p.cov[2] - p.cov[1] * p.cov[1];
  if (!(det > 0) || !std::isfinite(det)) return;
  p.conic[0] = p.cov[2] / det;
  p.conic[1] = -p.cov[1] / det;
  p.conic[2] = p.cov[0] / det;
  p.uv[0] = k.fx * x / z + k.cx;
  p.uv[1] = k.fy * y / z + k.cy;
  if (!std::isfinite(p.uv[0]) || !std::isfinite(p.uv[1])) return;
  p.depth = z;
  const double mid = 0.5 * (p.cov[0] + p.cov[2]);
  const double lam = mid + std::sqrt(std::max(kEigFloor, mid * mid - det));
  p.radius = std::ceil(kSigmaK * std::sqrt(lam));
  if (!std::isfinite(p.radius)) return;
  // Pixels whose centre lies within radius of (u, v) along each axis.
  double i0 = std::ceil(p.uv[0] - p.radius - 0.5), i1 = std::floor(p.uv[0] + p.radius - 0.5);
  double j0 = std::ceil(p.uv[1] - p.radius - 0.5), j1 = std::floor(p.uv[1] + p.radius - 0.5);
  i0 = std::max(i0, 0.0);
  j0 = std::max(j0, 0.0);
  i1 = std::min(i1, (double)(k.W - 1));
  j1 = std::min(j1, (double)(k.H - 1));
  if (i0 > i1 || j0 > j1) return;
  p.rect[0] = (int)i0 / kTile;
  p.rect[1] = (int)j0 / kTile;
  p.rect[2] = (int)i1 / kTile + 1;
  p.rect[3] = (int)j1 / kTile + 1;
  p.vis = true;
}

}  // namespace

extern "C" {

int ora_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// FP64 projection. Outputs (all P-long): uv[2], conic[3], depth, cov[3],
// radius, rect[4] (tile x0, y0, x1, y1 with exclusive ends), touched.
// Culled Gaussians get touched = 0 and zeros elsewhere.
void ora_project_f64(const double* cam, int P, const double* means, const double* scales,
                     const double* quats, const double* opac, double* uv, double* conic,
                     double* depth, double* cov, double* radius, int32_t* rect, int32_t* touched) {
  const Cam k = load_cam(cam);
#pragma omp parallel for schedule(static)
  for (int g = 0; g < P; ++g) {
    Proj p;
    project_one(k, means + 3 * g, scales + 3 * g, quats + 4 * g, opac[g], p);
    if (!p.vis) {
      uv[2 * g] = uv[2 * g + 1] = 0;
      conic[3 * g] = conic[3 * g + 1] = conic[3 * g + 2] = 0;
      cov[3 * g] = cov[3 * g + 1] = cov[3 * g + 2] = 0;
      depth[g] = 0;
      radius[g] = 0;
      rect[4 * g] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = 0;
      touched[g] = 0;
      continue;
    }
    uv[2 * g] = p.uv[0];
    uv[2 * g + 1] = p.uv[1];
    for (int i = 0; i < 3; ++i) {
      conic[3 * g + i] = p.conic[i];
      cov[3 * g + i] = p.cov[i];
    }
    depth[g] = p.depth;
    radius[g] = p.radius;
    for (int i = 0; i < 4; ++i) rect[4 * g + i] = p.rect[i];
    touched[g] = (p.rect[2] - p.rect[0]) * (p.rect[3] - p.rect[1]);
  }
}

// binary32 replay of the projection, for bit-exact comparison of the
// discrete outputs. The order of operations below is the one the GPU
// kernel promises; every operation is one IEEE binary32 operation rounded to
// nearest (this file is built with -ffp-contract=off, so no fused
// multiply-add is formed). All sums are evaluated left to right.
//
//   mc_i   = ((R_i0 m0 + R_i1 m1) + R_i2 m2) + t_i
//   qq     = ((w w + x x) + y y) + z z ;  n = sqrt(qq) ; q <- q / n
//   r_ij   = rotation of q, e.g. r00 = 1 - 2 (y y + z z), r01 = 2 (x y - w z)
//   M_ij   = r_ij s_j
//   tx     = x / z ; limx = 1.3 (W / (2 fx)) ; xcl = min(limx, max(-limx, tx)) z
//   J00 = fx / z ; J02 = -((fx xcl) / (z z)) ; J11, J12 alike
//   T0j = J00 R0j + J02 R2j ; T1j = J11 R1j + J12 R2j
//   V_ij   = (T_i0 M_0j + T_i1 M_1j) + T_i2 M_2j
//   a = ((V00 V00 + V01 V01) + V02 V02) + 0.3 ; b = (V00 V10 + V01 V11) + V02 V12 ; c alike
//   det = a c - b b ; A = c / det ; B = -b / det ; C = a / det
//   u = fx tx + cx ; v = fy ty + cy
//   mid = 0.5 (a + c) ; lam = mid + sqrt(max(0.1, mid mid - det)) ; r = ceil(3 sqrt(lam))
//   i0 = max(ceil((u - r) - 0.5), 0) ; i1 = min(floor((u + r) - 0.5), W - 1) ; j alike
// Culling: a non-finite input, z <= near, qq <= 0, det <= 0 or non-finite,
// u, v or r non-finite, or an empty pixel range.
// Sigma' = V V^T equals J R Sigma R^T J^T of Eq. 1 exactly in real
// arithmetic (V = J R M and Sigma = M M^T).
void ora_project_b32(const double* camd, int P, const float* means, const float* scales,
                     const float* quats, const float* opac, float* uv, float* conic, float* depth,
                     int32_t* rect, int32_t* touched) {
  const float fx = (float)camd[2], fy = (float)camd[3], cx = (float)camd[4], cy = (float)camd[5];
  float R[9], t[3];
  for (int i = 0; i < 9; ++i) R[i] = (float)camd[6 + i];
  for (int i = 0; i < 3; ++i) t[i] = (float)camd[15 + i];
  const float near_z = (float)camd[18];
  const int W = (int)camd[0], H = (int)camd[1];
  const float Wf = (float)W, Hf = (float)H;
#pragma omp parallel for schedule(static)
  for (int g = 0; g < P; ++g) {
    auto cull = [&]() {
      uv[2 * g] = uv[2 * g + 1] = 0.f;
      conic[3 * g] = conic[3 * g + 1] = conic[3 * g + 2] = 0.f;
      depth[g] = 0.f;
      rect[4 * g] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = 0;
      touched[g] = 0;
    };
    const float m0 = means[3 * g], m1 = means[3 * g + 1], m2 = means[3 * g + 2];
    const float s0 = scales[3 * g], s1 = scales[3 * g + 1], s2 = scales[3 * g + 2];
    float qw = quats[4 * g], qx = quats[4 * g + 1], qy = quats[4 * g + 2], qz = quats[4 * g + 3];
    const float o = opac[g];
    const float in[11] = {m0, m1, m2, s0, s1, s2, qw, qx, qy, qz, o};
    bool fin = true;
    for (int i = 0; i < 11; ++i) fin = fin && std::isfinite(in[i]);
    if (!fin) { cull(); continue; }
    const float xc = ((R[0] * m0 + R[1] * m1) + R[2] * m2) + t[0];
    const float yc = ((R[3] * m0 + R[4] * m1) + R[5] * m2) + t[1];
    const float zc = ((R[6] * m0 + R[7] * m1) + R[8] * m2) + t[2];
    if (!(zc > near_z)) { cull(); continue; }
    const float qq = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    if (!(qq > 0.f)) { cull(); continue; }
    const float qn = std::sqrt(qq);
    qw = qw / qn; qx = qx / qn; qy = qy / qn; qz = qz / qn;
    float r[9];
    r[0] = 1.f - 2.f * (qy * qy + qz * qz);
    r[1] = 2.f * (qx * qy - qw * qz);
    r[2] = 2.f * (qx * qz + qw * qy);
    r[3] = 2.f * (qx * qy + qw * qz);
    r[4] = 1.f - 2.f * (qx * qx + qz * qz);
    r[5] = 2.f * (qy * qz - qw * qx);
    r[6] = 2.f * (qx * qz - qw * qy);
    r[7] = 2.f * (qy * qz + qw * qx);
    r[8] = 1.f - 2.f * (qx * qx + qy * qy);
    const float sv[3] = {s0, s1, s2};
    float M[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[3 * i + j] = r[3 * i + j] * sv[j];
    const float limx = 1.3f * (Wf / (2.f * fx));
    const float limy = 1.3f * (Hf / (2.f * fy));
    const float tx = xc / zc, ty = yc / zc;
    const float xcl = std::fmin(limx, std::fmax(-limx, tx)) * zc;
    const float ycl = std::fmin(limy, std::fmax(-limy, ty)) * zc;
    const float zz = zc * zc;
    const float J00 = fx / zc, J02 = -((fx * xcl) / zz);
    const float J11 = fy / zc, J12 = -((fy * ycl) / zz);
    float T[6];
    for (int j = 0; j < 3; ++j) {
      T[j] = J00 * R[j] + J02 * R[6 + j];
      T[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    float V[6];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        V[3 * i + j] = (T[3 * i] * M[j] + T[3 * i + 1] * M[3 + j]) + T[3 * i + 2] * M[6 + j];
    const float a = ((V[0] * V[0] + V[1] * V[1]) + V[2] * V[2]) + 0.3f;
    const float b = (V[0] * V[3] + V[1] * V[4]) + V[2] * V[5];
    const float c = ((V[3] * V[3] + V[4] * V[4]) + V[5] * V[5]) + 0.3f;
    const float det = a * c - b * b;
    if (!(det > 0.f) || !std::isfinite(det)) { cull(); continue; }
    const float A = c / det, B = -b / det, C = a / det;
    const float u = fx * tx + cx, v = fy * ty + cy;
    if (!std::isfinite(u) || !std::isfinite(v)) { cull(); continue; }
    const float mid = 0.5f * (a + c);
    const float lam = mid + std::sqrt(std::fmax(0.1f, mid * mid - det));
    const float rad = std::ceil(3.f * std::sqrt(lam));
    if (!std::isfinite(rad)) { cull(); continue; }
    float i0 = std::ceil((u - rad) - 0.5f), i1 = std::floor((u + rad) - 0.5f);
    float j0 = std::ceil((v - rad) - 0.5f), j1 = std::floor((v + rad) - 0.5f);
    i0 = std::fmax(i0, 0.f);
    j0 = std::fmax(j0, 0.f);
    i1 = std::fmin(i1, Wf - 1.f);
    j1 = std::fmin(j1, Hf - 1.f);
    if (i0 > i1 || j0 > j1) { cull(); continue; }
    uv[2 * g] = u;
    uv[2 * g + 1] = v;
    conic[3 * g] = A;
    conic[3 * g + 1] = B;
    conic[3 * g + 2] = C;
    depth[g] = zc;
    const int r0 = (int)i0 / kTile, r1 = (int)j0 / kTile, r2 = (int)i1 / kTile + 1,
              r3 = (int)j1 / kTile + 1;
    rect[4 * g] = r0;
    rect[4 * g + 1] = r1;
    rect[4 * g + 2] = r2;
    rect[4 * g + 3] = r3;
    touched[g] = (r2 - r0) * (r3 - r1);
  }
}

// Per-tile lists: every (tile, gaussian) pair with the tile inside the
// Gaussian's rectangle, ordered by tile, then depth ascending, then id
// ascending (Sec. 3.1: front-to-back by depth). ranges is [num_tiles, 2]
// (start, end). Returns the number of pairs; gids must hold that many (the
// caller sizes it from the sum of touched counts).
int64_t ora_bin(int P, const int32_t* rect, const double* depth, int tiles_x, int tiles_y,
                int32_t* ranges, int32_t* gids) {
  std::vector<std::tuple<int, double, int>> items;
  for (int g = 0; g < P; ++g) {
    const int32_t* r = rect + 4 * g;
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) items.emplace_back(ty * tiles_x + tx, depth[g], g);
  }
  std::sort(items.begin(), items.end());
  const int T = tiles_x * tiles_y;
  for (int t = 0; t < T; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    const int t = std::get<0>(items[i]);
    gids[i] = std::get<2>(items[i]);
    if (i == 0 || std::get<0>(items[i - 1]) != t) ranges[2 * t] = (int32_t)i;
    ranges[2 * t + 1] = (int32_t)i + 1;
  }
  return (int64_t)items.size();
}

}  // extern "C"

namespace {

// One evaluated (pixel, gaussian) pair during the front-to-back walk.
struct Blend {
  int g;          // gaussian id
  double alpha;   // alpha after the clamp
  double G;       // exp(power)
  bool clamped;   // o G > 0.99
  double T;       // transmittance in front of this gaussian
  double dx, dy;  // u - px, v - py
};

// Walk one pixel's tile list front to back (Eq. 2-3 with the 3DGS rules).
// Returns the blended gaussians; sets T_final, last (list position + 1 of the
// last blended) and the smallest decision margin.
void walk_pixel(const int32_t* list, int n, double px, double py, const double* uv,
                const double* conic, const double* opac, std::vector<Blend>& out, double& T_final,
                int& last, double& margin) {
  out.clear();
  double T = 1.0;
  last = 0;
  margin = 1e300;
  for (int k = 0; k < n; ++k) {
    const int g = list[k];
    const double dx = uv[2 * g] - px, dy = uv[2 * g + 1] - py;
    const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
    const double power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
    margin = std::min(margin, std::fabs(power));
    if (power > 0) continue;
    const double G = std::exp(power);
    const double araw = opac[g] * G;
    margin = std::min(margin, std::fabs(araw / kAlphaMax - 1.0));
    const bool clamped = araw > kAlphaMax;
    const double alpha = clamped ? kAlphaMax : araw;
    margin = std::min(margin, std::fabs(alpha / kAlphaMin - 1.0));
    if (alpha < kAlphaMin) continue;
    const double Tn = T * (1.0 - alpha);
    margin = std::min(margin, std::fabs(Tn / kTStop - 1.0));
    if (Tn < kTStop) break;
    out.push_back({g, alpha, G, clamped, T, dx, dy});
    T = Tn;
    last = k + 1;
  }
  T_final = T;
}

}  // namespace

extern "C" {

// Eq. 2-3 in double. Per-Gaussian inputs are double arrays: uv [P,2],
// conic [P,3], opac [P], colors [P,3], depth [P], feats [P,N] (N may be 0).
// Outputs are channel-major images: rgb [3,H,W] (background bg added with
// weight T_final), depth_out [H,W], alpha_out [H,W] = 1 - T_final,
// feat_out [N,H,W]; T_final [H,W]; last_idx [H,W] (list position + 1 of the
// last blended Gaussian); n_contrib [H,W]; margin [H,W] (smallest relative
// distance of any alpha/T decision from its threshold, and |power|).
void ora_render_fwd(const double* cam, int tiles_x, const int32_t* ranges, const int32_t* gids,
                    const double* uv, const double* conic, const double* opac,
                    const double* colors, const double* depth, const double* feats, int N,
                    const double* bg, double* rgb, double* depth_out, double* alpha_out,
                    double* feat_out, double* T_final, int32_t* last_idx, int32_t* n_contrib,
                    double* margin) {
  const int W = (int)cam[0], H = (int)cam[1];
  const int tiles_y = (H + kTile - 1) / kTile;
  const int T = tiles_x * tiles_y;
  const size_t HW = (size_t)H * W;
#pragma omp parallel
  {
    std::vector<Blend> bl;
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
      const int tx = t % tiles_x, ty = t / tiles_x;
      const int s = ranges[2 * t], e = ranges[2 * t + 1];
      for (int j = ty * kTile; j < std::min(H, (ty + 1) * kTile); ++j)
        for (int i = tx * kTile; i < std::min(W, (tx + 1) * kTile); ++i) {
          double Tf, mg;
          int last;
          walk_pixel(gids + s, e - s, i + 0.5, j + 0.5, uv, conic, opac, bl, Tf, last, mg);
          double c[3] = {0, 0, 0}, d = 0;
          const size_t pix = (size_t)j * W + i;
          for (int f = 0; f < N; ++f) feat_out[f * HW + pix] = 0;
          for (const Blend& b : bl) {
            const double w = b.alpha * b.T;
            for (int ch = 0; ch < 3; ++ch) c[ch] += w * colors[3 * b.g + ch];
            d += w * depth[b.g];
            for (int f = 0; f < N; ++f) feat_out[f * HW + pix] += w * feats[(size_t)b.g * N + f];
          }
          for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + pix] = c[ch] + Tf * bg[ch];
          depth_out[pix] = d;
          alpha_out[pix] = 1.0 - Tf;
          T_final[pix] = Tf;
          last_idx[pix] = last;
          n_contrib[pix] = (int32_t)bl.size();
          margin[pix] = mg;
        }
    }
  }
}

// Keyframe visibility (Sec. 3.2): Gaussian g is visible in the frame when it
// is blended at some pixel with transmittance T > 0.5 in front of it. maxT[g]
// receives the largest such T over all pixels (0 if g is blended nowhere), so
// visible = maxT > 0.5 and a caller can see how close each decision is.
void ora_visibility(const double* cam, int tiles_x, const int32_t* ranges, const int32_t* gids,
                    const double* uv, const double* conic, const double* opac, int P, double* maxT) {
  const int W = (int)cam[0], H = (int)cam[1];
  const int tiles_y = (H + kTile - 1) / kTile;
  const int T = tiles_x * tiles_y;
  for (int g = 0; g < P; ++g) maxT[g] = 0.0;
#pragma omp parallel
  {
    std::vector<Blend> bl;
    std::vector<double> mine((size_t)P, 0.0);
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
      const int tx = t % tiles_x, ty = t / tiles_x;
      const int s = ranges[2 * t], e = ranges[2 * t + 1];
      for (int j = ty * kTile; j < std::min(H, (ty + 1) * kTile); ++j)
        for (int i = tx * kTile; i < std::min(W, (tx + 1) * kTile); ++i) {
          double Tf, mg;
          int last;
          walk_pixel(gids + s, e - s, i + 0.5, j + 0.5, uv, conic, opac, bl, Tf, last, mg);
          for (const Blend& b : bl) mine[b.g] = std::max(mine[b.g], b.T);
        }
    }
#pragma omp critical
    for (int g = 0; g < P; ++g) maxT[g] = std::max(maxT[g], mine[g]);
  }
}

// Adjoint of Eq. 2-3. The cotangents g_rgb [3,H,W], g_depth [H,W],
// g_alpha [H,W], g_feat [N,H,W] may be null (zero). coupled = 0 is the
// paper's decoupled feature gradient (Sec. 3.1: the feature cotangent reaches
// only f, not the geometry); coupled = 1 also sends it through alpha, which
// is the true derivative and is used for finite-difference checks.
// Outputs (accumulated, caller zeroes): d_uv [P,2], d_conic [P,3],
// d_opac [P], d_colors [P,3], d_depth [P], d_feats [P,N].
//
// For blended Gaussian i with transmittance T_i in front of it,
// w_i = alpha_i T_i and S_i = prod_{k>i blended} (1 - alpha_k):
//   dL/dc_i = w_i g_C ; dL/dd_i = w_i g_D ; dL/df_i = w_i g_F
//   dL/dalpha_i = T_i [ (c_i - Bc_i).g_C + (d_i - Bd_i) g_D + coupled (f_i - Bf_i).g_F ]
//                 + T_i S_i (g_A - bg.g_C)
// with Bx_i = sum_{j>i} x_j alpha_j prod_{i<k<j} (1 - alpha_k), evaluated by
// Bx_i = alpha_{i+1} x_{i+1} + (1 - alpha_{i+1}) Bx_{i+1}.
// alpha = min(0.99, o exp(power)): dalpha/do = exp(power), dalpha/dpower =
// alpha below the clamp, both 0 at the clamp.
// power = -(A dx^2 + C dy^2)/2 - B dx dy with dx = u - px, dy = v - py.
void ora_render_bwd(const double* cam, int tiles_x, const int32_t* ranges, const int32_t* gids,
                    const double* uv, const double* conic, const double* opac,
                    const double* colors, const double* depth, const double* feats, int N,
                    const double* bg, const double* g_rgb, const double* g_depth,
                    const double* g_alpha, const double* g_feat, int coupled, int P, double* d_uv,
                    double* d_conic, double* d_opac, double* d_colors, double* d_depth,
                    double* d_feats) {
  const int W = (int)cam[0], H = (int)cam[1];
  const int tiles_y = (H + kTile - 1) / kTile;
  const int T = tiles_x * tiles_y;
  const size_t HW = (size_t)H * W;
  const int nthr = ora_num_threads();
  // Per-thread gradient buffers, summed at the end.
  const size_t per = (size_t)P * (2 + 3 + 1 + 3 + 1 + N);
  std::vector<double> buf((size_t)nthr * per, 0.0);
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* my = buf.data() + (size_t)tid * per;
    double* m_uv = my;
    double* m_conic = m_uv + 2 * (size_t)P;
    double* m_op = m_conic + 3 * (size_t)P;
    double* m_col = m_op + (size_t)P;
    double* m_dep = m_col + 3 * (size_t)P;
    double* m_f = m_dep + (size_t)P;
    std::vector<Blend> bl;
    std::vector<double> Bf(N), gF(N);
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
      const int tx = t % tiles_x, ty = t / tiles_x;
      const int s = ranges[2 * t], e = ranges[2 * t + 1];
      for (int j = ty * kTile; j < std::min(H, (ty + 1) * kTile); ++j)
        for (int i = tx * kTile; i < std::min(W, (tx + 1) * kTile); ++i) {
          double Tf, mg;
          int last;
          walk_pixel(gids + s, e - s, i + 0.5, j + 0.5, uv, conic, opac, bl, Tf, last, mg);
          const size_t pix = (size_t)j * W + i;
          double gC[3] = {0, 0, 0}, gD = 0, gA = 0;
          if (g_rgb)
            for (int ch = 0; ch < 3; ++ch) gC[ch] = g_rgb[ch * HW + pix];
          if (g_depth) gD = g_depth[pix];
          if (g_alpha) gA = g_alpha[pix];
          for (int f = 0; f < N; ++f) gF[f] = g_feat ? g_feat[f * HW + pix] : 0.0;
          double Bc[3] = {0, 0, 0}, Bd = 0, S = 1.0;
          std::fill(Bf.begin(), Bf.end(), 0.0);
          const double bgdot = bg[0] * gC[0] + bg[1] * gC[1] + bg[2] * gC[2];
          for (int k = (int)bl.size() - 1; k >= 0; --k) {
            const Blend& b = bl[k];
            const int g = b.g;
            const double w = b.alpha * b.T;
            for (int ch = 0; ch < 3; ++ch) m_col[3 * g + ch] += w * gC[ch];
            m_dep[g] += w * gD;
            for (int f = 0; f < N; ++f) m_f[(size_t)g * N + f] += w * gF[f];
            double da = 0;
            for (int ch = 0; ch < 3; ++ch) da += (colors[3 * g + ch] - Bc[ch]) * gC[ch];
            da += (depth[g] - Bd) * gD;
            if (coupled)
              for (int f = 0; f < N; ++f) da += (feats[(size_t)g * N + f] - Bf[f]) * gF[f];
            da *= b.T;
            da += b.T * S * (gA - bgdot);
            // next (earlier) gaussian sees this one in its suffix
            for (int ch = 0; ch < 3; ++ch) Bc[ch] = b.alpha * colors[3 * g + ch] + (1 - b.alpha) * Bc[ch];
            Bd = b.alpha * depth[g] + (1 - b.alpha) * Bd;
            if (coupled)
              for (int f = 0; f < N; ++f) Bf[f] = b.alpha * feats[(size_t)g * N + f] + (1 - b.alpha) * Bf[f];
            S *= (1 - b.alpha);
            if (b.clamped) continue;
            m_op[g] += da * b.G;
            const double dpow = da * b.alpha;
            const double A = conic[3 * g], Bc_ = conic[3 * g + 1], C = conic[3 * g + 2];
            m_conic[3 * g] += -0.5 * b.dx * b.dx * dpow;
            m_conic[3 * g + 1] += -b.dx * b.dy * dpow;
            m_conic[3 * g + 2] += -0.5 * b.dy * b.dy * dpow;
            m_uv[2 * g] += -(A * b.dx + Bc_ * b.dy) * dpow;
            m_uv[2 * g + 1] += -(Bc_ * b.dx + C * b.dy) * dpow;
          }
        }
    }
  }
  for (int th = 0; th < nthr; ++th) {
    const double* my = buf.data() + (size_t)th * per;
    for (size_t q = 0; q < 2 * (size_t)P; ++q) d_uv[q] += my[q];
    my += 2 * (size_t)P;
    for (size_t q = 0; q < 3 * (size_t)P; ++q) d_conic[q] += my[q];
    my += 3 * (size_t)P;
    for (size_t q = 0; q < (size_t)P; ++q) d_opac[q] += my[q];
    my += (size_t)P;
    for (size_t q = 0; q < 3 * (size_t)P; ++q) d_colors[q] += my[q];
    my += 3 * (size_t)P;
    for (size_t q = 0; q < (size_t)P; ++q) d_depth[q] += my[q];
    my += (size_t)P;
    for (size_t q = 0; q < (size_t)P * N; ++q) d_feats[q] += my[q];
  }
}

// Adjoint of the FP64 projection and the pose gradient of Eq. 4.
// Inputs: cotangents of uv [P,2], conic [P,3] (A, B, C with B the
// off-diagonal entry as stored), depth [P]. Outputs (accumulated):
// d_means [P,3], d_scales [P,3], d_quats [P,4], d_pose [6] = (rho, theta) for
// the left perturbation T <- Exp(tau) T:
//   d mu_c / d tau = [I, -mu_c^x]  ->  drho += dmu_c, dtheta += mu_c x dmu_c
//   d W / d tau    = [0, -W^x] per column W_k  ->  dtheta += W_k x dL/dW_k
// where W is the camera rotation as it enters the Jacobian product J W.
void ora_project_bwd_f64(const double* cam, int P, const double* means, const double* scales,
                         const double* quats, const double* opac, const double* d_uv,
                         const double* d_conic, const double* d_depth, double* d_means,
                         double* d_scales, double* d_quats, double* d_pose) {
  const Cam k = load_cam(cam);
  double pose[6] = {0, 0, 0, 0, 0, 0};
  for (int g = 0; g < P; ++g) {
    Proj p;
    project_one(k, means + 3 * g, scales + 3 * g, quats + 4 * g, opac[g], p);
    if (!p.vis) continue;
    const double* s = scales + 3 * g;
    const double x = p.mc[0], y = p.mc[1], z = p.mc[2];
    double dmc[3] = {0, 0, 0};
    // conic = inverse(cov): dcov = -K G K, G the symmetric cotangent matrix.
    const double K[4] = {p.conic[0], p.conic[1], p.conic[1], p.conic[2]};
    const double Gm[4] = {d_conic[3 * g], 0.5 * d_conic[3 * g + 1], 0.5 * d_conic[3 * g + 1],
                          d_conic[3 * g + 2]};
    double KG[4], dC2[4];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) KG[2 * a + b] = K[2 * a] * Gm[b] + K[2 * a + 1] * Gm[2 + b];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) dC2[2 * a + b] = -(KG[2 * a] * K[b] + KG[2 * a + 1] * K[2 + b]);
    // cov = Tm Sigma Tm^T (+ low-pass): dTm = 2 dC2 Tm Sigma, dSigma = Tm^T dC2 Tm.
    double TS[6];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int l = 0; l < 3; ++l) acc += p.Tm[3 * i + l] * p.Sigma[3 * l + j];
        TS[3 * i + j] = acc;
      }
    double dTm[6];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) dTm[3 * i + j] = 2 * (dC2[2 * i] * TS[j] + dC2[2 * i + 1] * TS[3 + j]);
    double dSig[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) acc += p.Tm[3 * a + i] * dC2[2 * a + b] * p.Tm[3 * b + j];
        dSig[3 * i + j] = acc;
      }
    // Sigma = M M^T: dM = (dSig + dSig^T) M
    double dM[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int l = 0; l < 3; ++l) acc += (dSig[3 * i + l] + dSig[3 * l + i]) * p.M[3 * l + j];
        dM[3 * i + j] = acc;
      }
    // M = Rq diag(s)
    double dRq[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        d_scales[3 * g + j] += dM[3 * i + j] * p.Rq[3 * i + j];
        dRq[3 * i + j] = dM[3 * i + j] * s[j];
      }
    // Rq(qn): partial derivatives of each entry.
    const double w = p.qn[0], qx = p.qn[1], qy = p.qn[2], qz = p.qn[3];
    double dqn[4] = {0, 0, 0, 0};
    // entry: (d/dw, d/dx, d/dy, d/dz)
    const double part[9][4] = {
        {0, 0, -4 * qy, -4 * qz},            // 1 - 2(y^2 + z^2)
        {-2 * qz, 2 * qy, 2 * qx, -2 * w},   // 2(xy - wz)
        {2 * qy, 2 * qz, 2 * w, 2 * qx},     // 2(xz + wy)
        {2 * qz, 2 * qy, 2 * qx, 2 * w},     // 2(xy + wz)
        {0, -4 * qx, 0, -4 * qz},            // 1 - 2(x^2 + z^2)
        {-2 * qx, -2 * w, 2 * qz, 2 * qy},   // 2(yz - wx)
        {-2 * qy, 2 * qz, -2 * w, 2 * qx},   // 2(xz - wy)
        {2 * qx, 2 * w, 2 * qz, 2 * qy},     // 2(yz + wx)
        {0, -4 * qx, -4 * qy, 0},            // 1 - 2(x^2 + y^2)
    };
    for (int e = 0; e < 9; ++e)
      for (int c = 0; c < 4; ++c) dqn[c] += dRq[e] * part[e][c];
    // qn = q / |q|
    double dot = 0;
    for (int c = 0; c < 4; ++c) dot += p.qn[c] * dqn[c];
    for (int c = 0; c < 4; ++c) d_quats[4 * g + c] += (dqn[c] - p.qn[c] * dot) / p.qnorm;
    // Tm = J W: dJ = dTm W^T ; dW = J^T dTm
    double dJ[6], dW[9];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        dJ[3 * i + j] = dTm[3 * i] * k.R[3 * j] + dTm[3 * i + 1] * k.R[3 * j + 1] + dTm[3 * i + 2] * k.R[3 * j + 2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dW[3 * i + j] = p.J[i] * dTm[j] + p.J[3 + i] * dTm[3 + j];
    // J entries: J00 = fx/z, J02 = -fx xcl/z^2, J11 = fy/z, J12 = -fy ycl/z^2
    const double z2 = z * z, z3 = z2 * z;
    dmc[2] += -k.fx / z2 * dJ[0] - k.fy / z2 * dJ[4] + 2 * k.fx * p.xcl / z3 * dJ[2] +
              2 * k.fy * p.ycl / z3 * dJ[5];
    const double dxcl = -k.fx / z2 * dJ[2], dycl = -k.fy / z2 * dJ[5];
    // xcl = clamp(x/z) z: x itself when free, +-lim z when clamped
    if (p.clx == 0) dmc[0] += dxcl; else dmc[2] += p.clx * p.limx * dxcl;
    if (p.cly == 0) dmc[1] += dycl; else dmc[2] += p.cly * p.limy * dycl;
    // u = fx x/z + cx, v = fy y/z + cy, depth = z
    const double du = d_uv[2 * g], dv = d_uv[2 * g + 1];
    dmc[0] += k.fx / z * du;
    dmc[1] += k.fy / z * dv;
    dmc[2] += -k.fx * x / z2 * du - k.fy * y / z2 * dv + d_depth[g];
    // mu_c = R mu + t
    for (int j = 0; j < 3; ++j)
      d_means[3 * g + j] += k.R[j] * dmc[0] + k.R[3 + j] * dmc[1] + k.R[6 + j] * dmc[2];
    // pose (Eq. 4)
    for (int j = 0; j < 3; ++j) pose[j] += dmc[j];
    pose[3] += y * dmc[2] - z * dmc[1];
    pose[4] += z * dmc[0] - x * dmc[2];
    pose[5] += x * dmc[1] - y * dmc[0];
    for (int c = 0; c < 3; ++c) {
      const double Wc[3] = {k.R[c], k.R[3 + c], k.R[6 + c]};
      const double dWc[3] = {dW[c], dW[3 + c], dW[6 + c]};
      pose[3] += Wc[1] * dWc[2] - Wc[2] * dWc[1];
      pose[4] += Wc[2] * dWc[0] - Wc[0] * dWc[2];
      pose[5] += Wc[0] * dWc[1] - Wc[1] * dWc[0];
    }
  }
  for (int j = 0; j < 6; ++j) d_pose[j] += pose[j];
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Per-pixel feature decoder o(.) of Eq. 11, read as a 1x1 lift of the latent
// feature map: y = W2^T gelu(W1^T z + b1) + b2 with the exact (erf) GELU,
// gelu(x) = x (1 + erf(x / sqrt 2)) / 2. Shapes: z [n, din], W1 [din, dh],
// b1 [dh], W2 [dh, dout], b2 [dout], y [n, dout]; all double.
extern "C" {

void ora_decoder_fwd(int n, int din, int dh, int dout, const double* z, const double* W1, const double* b1,
                     const double* W2, const double* b2, double* y) {
#pragma omp parallel for schedule(static)
  for (int p = 0; p < n; ++p) {
    std::vector<double> h(dh);
    for (int j = 0; j < dh; ++j) {
      double a = b1[j];
      for (int i = 0; i < din; ++i) a += z[(size_t)p * din + i] * W1[(size_t)i * dh + j];
      h[j] = 0.5 * a * (1.0 + std::erf(a / std::sqrt(2.0)));
    }
    for (int c = 0; c < dout; ++c) {
      double a = b2[c];
      for (int j = 0; j < dh; ++j) a += h[j] * W2[(size_t)j * dout + c];
      y[(size_t)p * dout + c] = a;
    }
  }
}

// Gradients of L = sum_p sum_c g[p, c] y[p, c] (g given) with respect to
// W1, b1, W2, b2 (accumulated) and z (written). gelu'(x) = Phi(x) + x phi(x).
void ora_decoder_bwd(int n, int din, int dh, int dout, const double* z, const double* W1, const double* b1,
                     const double* W2, const double* g, double* dW1, double* db1, double* dW2, double* db2,
                     double* dz) {
  const double inv_sqrt2 = 1.0 / std::sqrt(2.0), inv_sqrt2pi = 1.0 / std::sqrt(2.0 * M_PI);
  for (int p = 0; p < n; ++p) {
    std::vector<double> a(dh), h(dh), dhv(dh, 0.0);
    for (int j = 0; j < dh; ++j) {
      double s = b1[j];
      for (int i = 0; i < din; ++i) s += z[(size_t)p * din + i] * W1[(size_t)i * dh + j];
      a[j] = s;
      h[j] = 0.5 * s * (1.0 + std::erf(s * inv_sqrt2));
    }
    for (int c = 0; c < dout; ++c) {
      const double gc = g[(size_t)p * dout + c];
      db2[c] += gc;
      for (int j = 0; j < dh; ++j) {
        dW2[(size_t)j * dout + c] += h[j] * gc;
        dhv[j] += W2[(size_t)j * dout + c] * gc;
      }
    }
    for (int i = 0; i < din; ++i) dz[(size_t)p * din + i] = 0.0;
    for (int j = 0; j < dh; ++j) {
      const double d = 0.5 * (1.0 + std::erf(a[j] * inv_sqrt2)) + a[j] * inv_sqrt2pi * std::exp(-0.5 * a[j] * a[j]);
      const double da = dhv[j] * d;
      db1[j] += da;
      for (int i = 0; i < din; ++i) {
        dW1[(size_t)i * dh + j] += z[(size_t)p * din + i] * da;
        dz[(size_t)p * din + i] += W1[(size_t)i * dh + j] * da;
      }
    }
  }
}


// ---- tracking (Sec. 3.2, Eq. 6) ------------------------------------------------

// Edge mask: luminance L = ((r + g) + b) * (1/3), Sobel differences with the
// image border replicated, each divided by 8; edge where gx^2 + gy^2 > tau^2.
// Written with float variables so that every operation rounds to binary32
// in the order the GPU promises (compiled without contraction).
void ora_edge_mask(int W, int H, const float* rgb, float tau, uint8_t* m_e) {
  const size_t HW = (size_t)W * H;
  auto L = [&](int x, int y) {
    const size_t p = (size_t)y * W + x;
    const float s = rgb[p] + rgb[HW + p];
    const float s3 = s + rgb[2 * HW + p];
    return s3 * (1.f / 3.f);
  };
  const float tt = tau * tau;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const int xm = std::max(x - 1, 0), xp = std::min(x + 1, W - 1);
      const int ym = std::max(y - 1, 0), yp = std::min(y + 1, H - 1);
      const float a1 = L(xp, ym) + 2.f * L(xp, y), a = a1 + L(xp, yp);
      const float b1 = L(xm, ym) + 2.f * L(xm, y), b = b1 + L(xm, yp);
      const float c1 = L(xm, yp) + 2.f * L(x, yp), c = c1 + L(xp, yp);
      const float d1 = L(xm, ym) + 2.f * L(x, ym), d = d1 + L(xp, ym);
      const float gx = (a - b) * 0.125f, gy = (c - d) * 0.125f;
      const float gx2 = gx * gx, gy2 = gy * gy;
      const float mag2 = gx2 + gy2;
      m_e[(size_t)y * W + x] = mag2 > tt ? 1 : 0;
    }
}

// Eq. 6: L = lambda/(3HW) sum_{m_v m_e} |C - C_obs| + (1 - lambda)/(HW) sum_{m_v, D_obs > 0} |D - D_obs|,
// m_v = alpha_ref > alpha_min. Returns L; writes dL/dC and dL/dD (sign(0) = 0).
double ora_tracking_grad(int W, int H, const double* rgb, const double* depth, const double* gt_rgb,
                         const double* gt_depth, const double* alpha_ref, double alpha_min, const uint8_t* m_e,
                         double lambda, double* g_rgb, double* g_depth) {
  const size_t HW = (size_t)W * H;
  const double sc = lambda / (3.0 * (double)HW), sd = (1.0 - lambda) / (double)HW;
  auto sign = [](double d) { return d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0); };
  double loss = 0.0;
  for (size_t p = 0; p < HW; ++p) {
    const bool mv = alpha_ref[p] > alpha_min;
    const bool col = mv && m_e[p] != 0;
    for (int c = 0; c < 3; ++c) {
      const double d = rgb[c * HW + p] - gt_rgb[c * HW + p];
      g_rgb[c * HW + p] = col ? sc * sign(d) : 0.0;
      if (col) loss += sc * std::fabs(d);
    }
    const bool dep = mv && gt_depth[p] > 0;
    const double d = depth[p] - gt_depth[p];
    g_depth[p] = dep ? sd * sign(d) : 0.0;
    if (dep) loss += sd * std::fabs(d);
  }
  return loss;
}

// Adam on the 6-vector (rho, theta) and the left update T <- Exp(delta) T,
// Exp(rho, theta) = [R(theta), V(theta) rho] (the closed forms of the SE(3)
// exponential). pose: R row-major then t. converged: |V rho| < tol_t and
// |theta| < tol_r.
int ora_pose_update(double* pose, const double* g, double* m, double* v, int step, double lr_t, double lr_r,
                    double b1, double b2, double eps, double tol_t, double tol_r) {
  double dl[6];
  for (int i = 0; i < 6; ++i) {
    m[i] = b1 * m[i] + (1 - b1) * g[i];
    v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
    const double mh = m[i] / (1 - std::pow(b1, step)), vh = v[i] / (1 - std::pow(b2, step));
    dl[i] = -(i < 3 ? lr_t : lr_r) * mh / (std::sqrt(vh) + eps);
  }
  const double w[3] = {dl[3], dl[4], dl[5]};
  const double phi = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double A, B, C;
  if (phi < 1e-6) {
    A = 1 - phi * phi / 6;
    B = 0.5 - phi * phi / 24;
    C = 1.0 / 6 - phi * phi / 120;
  } else {
    A = std::sin(phi) / phi;
    B = (1 - std::cos(phi)) / (phi * phi);
    C = (phi - std::sin(phi)) / (phi * phi * phi);
  }
  const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9], Rd[9], V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double sum = 0;
      for (int k = 0; k < 3; ++k) sum += K[3 * i + k] * K[3 * k + j];
      K2[3 * i + j] = sum;
    }
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    Rd[i] = I + A * K[i] + B * K2[i];
    V[i] = I + B * K[i] + C * K2[i];
  }
  double td[3], R[9], t[3];
  for (int i = 0; i < 3; ++i) td[i] = V[3 * i] * dl[0] + V[3 * i + 1] * dl[1] + V[3 * i + 2] * dl[2];
  for (int i = 0; i < 9; ++i) R[i] = pose[i];
  for (int i = 0; i < 3; ++i) t[i] = pose[9 + i];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      double sum = 0;
      for (int k = 0; k < 3; ++k) sum += Rd[3 * i + k] * R[3 * k + j];
      pose[3 * i + j] = sum;
    }
    pose[9 + i] = Rd[3 * i] * t[0] + Rd[3 * i + 1] * t[1] + Rd[3 * i + 2] * t[2] + td[i];
  }
  const double tn = std::sqrt(td[0] * td[0] + td[1] * td[1] + td[2] * td[2]);
  return (tn < tol_t && phi < tol_r) ? 1 : 0;
}


// ---- semantics (Sec. 3.3) -------------------------------------------------------

// Eq. 9 with F_p read as logits: loss = (1/HW) sum_p [log sum_c exp F_p(c) - F_p(l_p)],
// grad = (softmax(F_p) - onehot(l_p)) / HW; labels outside [0, N) are ignored.
// Layout: hwc = 0 -> F[c * HW + p], 1 -> F[p * N + c].
double ora_semantic_ce(int W, int H, int N, int hwc, const double* F, const int32_t* labels, double* grad) {
  const size_t HW = (size_t)W * H;
  auto at = [&](size_t p, int c) { return hwc ? p * (size_t)N + c : (size_t)c * HW + p; };
  double loss = 0.0;
  for (size_t p = 0; p < HW; ++p) {
    const int lab = labels[p];
    if (lab < 0 || lab >= N) {
      for (int c = 0; c < N; ++c) grad[at(p, c)] = 0.0;
      continue;
    }
    double mx = -INFINITY;
    for (int c = 0; c < N; ++c) mx = std::max(mx, F[at(p, c)]);
    double sum = 0.0;
    for (int c = 0; c < N; ++c) sum += std::exp(F[at(p, c)] - mx);
    loss += (mx + std::log(sum) - F[at(p, lab)]) / (double)HW;
    for (int c = 0; c < N; ++c)
      grad[at(p, c)] = (std::exp(F[at(p, c)] - mx) / sum - (c == lab ? 1.0 : 0.0)) / (double)HW;
  }
  return loss;
}

// Eq. 12 logits in binary32: z_l = fma(f[M-1], q_l[M-1], ... fma(f[0], q_l[0], 0)),
// one rounding per fused multiply-add in channel order.
void ora_label_logits_b32(long long npix, int M, int L, const float* f, const float* q, float* z) {
  for (long long p = 0; p < npix; ++p)
    for (int l = 0; l < L; ++l) {
      float acc = 0.f;
      for (int c = 0; c < M; ++c) acc = std::fmaf(f[p * M + c], q[(size_t)l * M + c], acc);
      z[p * L + l] = acc;
    }
}

// Eq. 12 probabilities in double.
void ora_label_probs(long long npix, int M, int L, const double* f, const double* q, double* probs) {
  std::vector<double> z((size_t)L);
  for (long long p = 0; p < npix; ++p) {
    double mx = -INFINITY;
    for (int l = 0; l < L; ++l) {
      double acc = 0.0;
      for (int c = 0; c < M; ++c) acc += f[p * M + c] * q[(size_t)l * M + c];
      z[l] = acc;
      mx = std::max(mx, acc);
    }
    double sum = 0.0;
    for (int l = 0; l < L; ++l) sum += std::exp(z[l] - mx);
    for (int l = 0; l < L; ++l) probs[p * L + l] = std::exp(z[l] - mx) / sum;
  }
}


// ---- spherical-harmonic colour (Sec. 3.1) ---------------------------------------

}  // extern "C"

namespace {

// value and the three partial derivatives with respect to the Gaussian's mean
struct Dual {
  double v, d[3];
};
Dual dconst(double c) { return {c, {0, 0, 0}}; }
Dual operator+(Dual a, Dual b) { return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}}; }
Dual operator-(Dual a, Dual b) { return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}}; }
Dual operator*(Dual a, Dual b) {
  return {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1], a.d[2] * b.v + a.v * b.d[2]}};
}
Dual operator*(double c, Dual a) { return {c * a.v, {c * a.d[0], c * a.d[1], c * a.d[2]}}; }
Dual dsqrt(Dual a) {
  const double r = std::sqrt(a.v);
  return {r, {a.d[0] / (2 * r), a.d[1] / (2 * r), a.d[2] / (2 * r)}};
}
Dual ddiv(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, {(a.d[0] - q * b.d[0]) / b.v, (a.d[1] - q * b.d[1]) / b.v, (a.d[2] - q * b.d[2]) / b.v}};
}

double fact(int n) {
  double f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Real SH Y_k, k = l^2 + l + m, l <= lmax, at the unit direction (x, y, z):
// N_l^m Pbar_l^|m|(z) {sqrt2 Re (x + i y)^m | 1 | sqrt2 Im (x + i y)^|m|},
// Pbar_l^m = P_l^m / (1 - z^2)^(m/2) (Condon-Shortley phase included) from
// the three-term recurrence in l, N_l^m = sqrt((2l + 1) (l - m)! / (4 pi (l + m)!)).
void sh_real_basis(int lmax, Dual x, Dual y, Dual z, Dual* Y) {
  const double pi = 3.14159265358979323846;
  Dual re[4], im[4];  // (x + i y)^m
  re[0] = dconst(1);
  im[0] = dconst(0);
  for (int m = 1; m <= lmax; ++m) {
    re[m] = re[m - 1] * x - im[m - 1] * y;
    im[m] = re[m - 1] * y + im[m - 1] * x;
  }
  for (int m = 0; m <= lmax; ++m) {
    Dual P[4];
    double dfact = 1;  // (2m - 1)!!
    for (int i = 1; i <= 2 * m - 1; i += 2) dfact *= i;
    P[m] = dconst(((m % 2) ? -1.0 : 1.0) * dfact);
    if (m + 1 <= lmax) P[m + 1] = (double)(2 * m + 1) * (z * P[m]);
    for (int l = m + 2; l <= lmax; ++l)
      P[l] = (1.0 / (l - m)) * ((double)(2 * l - 1) * (z * P[l - 1]) - (double)(l + m - 1) * P[l - 2]);
    for (int l = m; l <= lmax; ++l) {
      const double N = std::sqrt((2 * l + 1) / (4 * pi) * fact(l - m) / fact(l + m));
      if (m == 0) {
        Y[l * l + l] = N * P[l];
      } else {
        Y[l * l + l + m] = (std::sqrt(2.0) * N) * (P[l] * re[m]);
        Y[l * l + l - m] = (std::sqrt(2.0) * N) * (P[l] * im[m]);
      }
    }
  }
}

// Y_k(d(mu)) with d = (mu - C) / |mu - C| and its gradient in mu.
void sh_at_mean(const double* C, const double* mu, int lmax, Dual* Y) {
  Dual v[3];
  for (int i = 0; i < 3; ++i) v[i] = {mu[i] - C[i], {i == 0 ? 1.0 : 0.0, i == 1 ? 1.0 : 0.0, i == 2 ? 1.0 : 0.0}};
  const Dual len = dsqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  sh_real_basis(lmax, ddiv(v[0], len), ddiv(v[1], len), ddiv(v[2], len), Y);
}

void camera_centre(const double* cam, double* C) {
  const double* R = cam + 6;
  const double* t = cam + 15;
  for (int i = 0; i < 3; ++i) C[i] = -(R[i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2]);
}

}  // namespace

extern "C" {

// The real SH basis Y_k at n unit directions: out [n, (lmax + 1)^2].
void ora_sh_basis(int n, int lmax, const double* dirs, double* out) {
  const int K = (lmax + 1) * (lmax + 1);
  Dual Y[16];
  for (int i = 0; i < n; ++i) {
    sh_real_basis(lmax, dconst(dirs[3 * i]), dconst(dirs[3 * i + 1]), dconst(dirs[3 * i + 2]), Y);
    for (int k = 0; k < K; ++k) out[(size_t)i * K + k] = Y[k].v;
  }
}

// colours [P,3] = max(0, sum_k sh[g][k][c] Y_k(d) + 0.5); sh [P, K, 3], K = (lmax + 1)^2.
void ora_sh_colors(const double* cam, int P, int lmax, const double* means, const double* sh, double* colors) {
  double C[3];
  camera_centre(cam, C);
  const int K = (lmax + 1) * (lmax + 1);
  Dual Y[16];
  for (int g = 0; g < P; ++g) {
    sh_at_mean(C, means + 3 * g, lmax, Y);
    for (int c = 0; c < 3; ++c) {
      double v = 0.5;
      for (int k = 0; k < K; ++k) v += sh[((size_t)g * K + k) * 3 + c] * Y[k].v;
      colors[3 * g + c] = std::max(v, 0.0);
    }
  }
}

// Adjoint: d_sh += Y dcol, d_means += sum_k w_k dY_k/dmu (w_k = sum_c sh dcol),
// d_pose[0..2] += R sum_g (view part of dL/dmu_g) (the centre moves with rho).
void ora_sh_colors_bwd(const double* cam, int P, int lmax, const double* means, const double* sh,
                       const double* d_colors, double* d_sh, double* d_means, double* d_pose) {
  double C[3];
  camera_centre(cam, C);
  const double* R = cam + 6;
  const int K = (lmax + 1) * (lmax + 1);
  Dual Y[16];
  double sum_dmu[3] = {0, 0, 0};
  for (int g = 0; g < P; ++g) {
    sh_at_mean(C, means + 3 * g, lmax, Y);
    double dc[3];
    for (int c = 0; c < 3; ++c) {
      double v = 0.5;
      for (int k = 0; k < K; ++k) v += sh[((size_t)g * K + k) * 3 + c] * Y[k].v;
      dc[c] = v < 0 ? 0.0 : d_colors[3 * g + c];
    }
    double dmu[3] = {0, 0, 0};
    for (int k = 0; k < K; ++k) {
      double w = 0;
      for (int c = 0; c < 3; ++c) {
        d_sh[((size_t)g * K + k) * 3 + c] += Y[k].v * dc[c];
        w += sh[((size_t)g * K + k) * 3 + c] * dc[c];
      }
      for (int i = 0; i < 3; ++i) dmu[i] += w * Y[k].d[i];
    }
    for (int i = 0; i < 3; ++i) {
      d_means[3 * g + i] += dmu[i];
      sum_dmu[i] += dmu[i];
    }
  }
  for (int i = 0; i < 3; ++i) d_pose[i] += R[3 * i] * sum_dmu[0] + R[3 * i + 1] * sum_dmu[1] + R[3 * i + 2] * sum_dmu[2];
}

}  // extern "C"
