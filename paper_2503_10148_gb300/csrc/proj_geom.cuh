// Forward geometry of one (component, camera) pair, shared by the projection
// kernel and its backward so both take the same FP32 decisions
// (near-plane cut, Jacobian limits, singular Sigma2D, colour clamp).
#pragma once

#include "common.cuh"
#include "sh.cuh"

namespace sss {

// Parameters of one component, loaded from the planar scene arrays.
struct CompParams {
  float mu[3], ls[3], q[4], nu_raw, o_raw;
};

__device__ __forceinline__ CompParams load_comp(const sss_params& S, uint32_t i) {
  const size_t n = (size_t)S.n;
  CompParams c;
#pragma unroll
  for (int k = 0; k < 3; ++k) c.mu[k] = __ldg(S.mean + k * n + i);
#pragma unroll
  for (int k = 0; k < 3; ++k) c.ls[k] = __ldg(S.log_scale + k * n + i);
#pragma unroll
  for (int k = 0; k < 4; ++k) c.q[k] = __ldg(S.quat + k * n + i);
  c.nu_raw = __ldg(S.nu + i);
  c.o_raw = __ldg(S.opacity_raw + i);
  return c;
}

// View-independent part: normalised quaternion, rotation, scales and the
// factor M = R S of Sigma = R S S^T R^T = M M^T (Sec. 3.1).
struct CompShape {
  float qn[4], qinv_norm;  // normalised quaternion (w, x, y, z), 1 / |q|
  float R[9];              // row-major rotation
  float s[3];              // exp(log_scale)
  float M[9];              // R diag(s), row-major
};

__device__ __forceinline__ CompShape comp_shape(const CompParams& c) {
  CompShape g;
  float n2 = c.q[0] * c.q[0] + c.q[1] * c.q[1] + c.q[2] * c.q[2] + c.q[3] * c.q[3];
  g.qinv_norm = 1.0f / sqrtf(n2);
#pragma unroll
  for (int k = 0; k < 4; ++k) g.qn[k] = c.q[k] * g.qinv_norm;
  const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
  g.R[0] = 1.0f - 2.0f * (y * y + z * z);
  g.R[1] = 2.0f * (x * y - w * z);
  g.R[2] = 2.0f * (x * z + w * y);
  g.R[3] = 2.0f * (x * y + w * z);
  g.R[4] = 1.0f - 2.0f * (x * x + z * z);
  g.R[5] = 2.0f * (y * z - w * x);
  g.R[6] = 2.0f * (x * z - w * y);
  g.R[7] = 2.0f * (y * z + w * x);
  g.R[8] = 1.0f - 2.0f * (x * x + y * y);
#pragma unroll
  for (int k = 0; k < 3; ++k) g.s[k] = expf(c.ls[k]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) g.M[r * 3 + k] = g.R[r * 3 + k] * g.s[k];
  return g;
}

// View-dependent geometry (Sec. 3.2 Eq. t_2D).
struct ViewGeom {
  bool valid;
  float p[3], inv_z;
  float tx, ty;
  int clx, cly;           // -1 / +1 when x/z (y/z) was limited, else 0
  float limx, limy;
  float j00, j02, j11, j12;
  float T[6];             // J W, rows 0 and 1
  float N[6];             // T M (2x3): Sigma2D = N N^T (+ lowpass I)
  float A, B, C, det;     // Sigma2D (+ lowpass on the diagonal)
  float con[3];           // conic a, b, c
  float m2[2];            // mean2D
  float o, nu;
  bool nu_limited;
};

__device__ __forceinline__ ViewGeom view_geom(const CompParams& c, const CompShape& g, const sss_camera& cam,
                                               const sss_raster_cfg& cfg) {
  ViewGeom v;
  const float* V = cam.viewmat;
  v.p[0] = fmaf(V[2], c.mu[2], fmaf(V[1], c.mu[1], fmaf(V[0], c.mu[0], V[3])));
  v.p[1] = fmaf(V[6], c.mu[2], fmaf(V[5], c.mu[1], fmaf(V[4], c.mu[0], V[7])));
  // depth key: this exact FMA chain (the near-plane cut and the depth order use it)
  v.p[2] = fmaf(V[10], c.mu[2], fmaf(V[9], c.mu[1], fmaf(V[8], c.mu[0], V[11])));
  v.valid = v.p[2] > cfg.znear;
  if (!v.valid) return v;
  v.inv_z = 1.0f / v.p[2];
  v.limx = 1.3f * (0.5f * (float)cam.width / cam.fx);
  v.limy = 1.3f * (0.5f * (float)cam.height / cam.fy);
  const float ux = v.p[0] * v.inv_z, uy = v.p[1] * v.inv_z;
  v.clx = (ux < -v.limx) ? -1 : ((ux > v.limx) ? 1 : 0);
  v.cly = (uy < -v.limy) ? -1 : ((uy > v.limy) ? 1 : 0);
  v.tx = v.clx ? (float)v.clx * v.limx * v.p[2] : v.p[0];
  v.ty = v.cly ? (float)v.cly * v.limy * v.p[2] : v.p[1];
  const float iz2 = v.inv_z * v.inv_z;
  v.j00 = cam.fx * v.inv_z;
  v.j02 = -cam.fx * v.tx * iz2;
  v.j11 = cam.fy * v.inv_z;
  v.j12 = -cam.fy * v.ty * iz2;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v.T[k] = v.j00 * V[0 * 4 + k] + v.j02 * V[2 * 4 + k];
    v.T[3 + k] = v.j11 * V[1 * 4 + k] + v.j12 * V[2 * 4 + k];
  }
  // N = T M; Sigma2D = N N^T.  det(N N^T) = |n0 x n1|^2 (Lagrange identity):
  // a sum of squares, accurate for elongated splats where AC - B^2 cancels.
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      v.N[r * 3 + k] = v.T[r * 3 + 0] * g.M[0 * 3 + k] + v.T[r * 3 + 1] * g.M[1 * 3 + k] + v.T[r * 3 + 2] * g.M[2 * 3 + k];
  const float* n0 = v.N;
  const float* n1 = v.N + 3;
  const float a0 = n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2];
  const float c0 = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
  const float x0 = n0[1] * n1[2] - n0[2] * n1[1], x1 = n0[2] * n1[0] - n0[0] * n1[2], x2 = n0[0] * n1[1] - n0[1] * n1[0];
  v.A = a0 + cfg.lowpass;
  v.B = n0[0] * n1[0] + n0[1] * n1[1] + n0[2] * n1[2];
  v.C = c0 + cfg.lowpass;
  v.det = x0 * x0 + x1 * x1 + x2 * x2 + cfg.lowpass * (a0 + c0 + cfg.lowpass);
  if (!(v.det > 0.0f)) {
    v.valid = false;
    return v;
  }
  const float id = 1.0f / v.det;
  v.con[0] = v.C * id;
  v.con[1] = -v.B * id;
  v.con[2] = v.A * id;
  v.m2[0] = cam.fx * v.p[0] * v.inv_z + cam.cx;
  v.m2[1] = cam.fy * v.p[1] * v.inv_z + cam.cy;
  v.o = tanhf(c.o_raw);
  if (!(fabsf(v.o) >= cfg.tau)) {
    v.valid = false;
    return v;
  }
  v.nu_limited = (c.nu_raw < 1.0f) || (c.nu_raw > 1e4f);
  v.nu = fminf(fmaxf(c.nu_raw, 1.0f), 1e4f);
  return v;
}

// Camera centre -W^T t.
__device__ __forceinline__ void cam_centre(const sss_camera& cam, float* cc) {
  const float* V = cam.viewmat;
#pragma unroll
  for (int k = 0; k < 3; ++k) cc[k] = -(V[0 * 4 + k] * V[3] + V[1 * 4 + k] * V[7] + V[2 * 4 + k] * V[11]);
}

}  // namespace sss
