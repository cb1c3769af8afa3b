// a6: 2D splat gradients -> component parameters (SM "Backward Pass": the
// chain through mu', Sigma' to mu, S, R, c, o, nu).
//
// One thread per (scene, component); the forward geometry is recomputed with
// the same code as the projection (proj_geom.cuh), the gradients of every job
// (view) of the scene are chained back and summed in registers, and each
// parameter gradient is written once (planar, coalesced).
//
// Chain, for one view with upstream g = dL/d(mean2D, conic a b c, o, nu, rgb):
//   conic Q = Sigma2D^-1: dL/dSigma2D = -Q G Q, G = [[ga, gb/2], [gb/2, gc]]
//   Sigma2D = K D K^T with K = T R, T = J W
//   T = J W:  dJ_rc = sum_k dT_rk W_ck (only J00, J02, J11, J12 are non-zero)
//   J(p) = [[fx/z, 0, -fx tx/z^2], [0, fy/z, -fy ty/z^2]], tx = x unless x/z
//     was limited (then tx = +-lim z, and its gradient goes to z)
//   mean2D = (fx x/z + cx, fy y/z + cy);  p = W mu + t
//   Sigma = R D R^T, D = diag(s^2): log-scale and rotation gradients taken in
//     the splat's frame (G' = R^T dL/dSigma R; see the kernel), the rotation
//     as a local rotation omega mapped to the quaternion by q (x) (0, omega/2)
//   rgb = max(SH . Y(d / |d|) + 0.5, 0), d = mu - camera centre:
//     dL/dsh_kc = g_c Y_k (0 where clamped), dL/dd = (I - u u^T)/|d| grad_u
//   o = tanh(raw): dL/draw = go (1 - o^2);  nu: passes where not limited.
#include "proj_geom.cuh"

namespace sss {
namespace {

template <int DEG>
__device__ __forceinline__ void project_bwd_component(const sss_frame_plan& P, int s, uint32_t i, const void* ws,
                                                      const sss_params& G) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const sss_params& S = P.scenes[s];
  const sss_raster_cfg& cfg = P.cfg;
  const CompParams c = load_comp(S, i);
  const CompShape gs = comp_shape(c);
  const float* g2d = ws_ptr<float>(ws, P.ws_off_grad2d);
  const size_t n = (size_t)S.n;

  float d_mu[3] = {0, 0, 0}, d_ls[3] = {0, 0, 0}, bw[3] = {0, 0, 0};
  float d_o = 0.0f, d_nu = 0.0f;
  bool touched = false;
  uint64_t views = 0;  // views (bit q - begin) whose gradient record is non-zero and geometry valid
  const int q0 = P.scene_job_begin[s];

  // geometry: mean (through mean2D and the Jacobian), scale, rotation, o, nu
  for (int q = q0; q < P.scene_job_begin[s + 1]; ++q) {
    const sss_job_desc& J = P.jobs[P.scene_jobs[q]];
    const uint32_t e = J.entry_base + i;
    const float4* gr = reinterpret_cast<const float4*>(g2d + (size_t)e * 12);
    const float4 g0 = gr[0], g1 = gr[1], g2 = gr[2];
    // g0 = (mx, my, ca, cb), g1 = (cc, o, nu, r), g2 = (g, b, -, -)
    if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f && g1.z == 0.f &&
        g1.w == 0.f && g2.x == 0.f && g2.y == 0.f)
      continue;
    const ViewGeom v = view_geom(c, gs, J.cam, cfg);
    if (!v.valid) continue;
    touched = true;
    views |= 1ull << (q - q0);
    const float* V = J.cam.viewmat;
    // Covariance chain, in the splat's own frame.  With Gc the conic gradient
    // as a symmetric matrix [[ga, gb/2], [gb/2, gc]]: dL/dSigma2D = -Q Gc Q
    // (Q = conic), Sigma2D = K D K^T + lowpass I with K = T R (2x3) and
    // D = diag(s^2).  With p_k = Q K_k and u_k = Gc p_k, the gradient w.r.t.
    // Sigma in the local frame is G'_ij = -p_i . u_j, so
    //   dL/dlog_s_k = 2 s_k^2 G'_kk,
    //   dL/domega   = 2 ((d1 - d2) G'_12, (d2 - d0) G'_02, (d0 - d1) G'_01)
    // for a local rotation R (I + [omega]x), and dL/dT = -2 Q U M^T with
    // U_k = s_k u_k.  Only products of well-scaled terms appear: the rotation
    // gradient of a near-isotropic splat comes out as the small difference
    // d_i - d_j times G'_ij instead of a cancellation of large terms.
    const float qa = v.con[0], qb = v.con[1], qc = v.con[2];
    const float ga = g0.z, gbh = 0.5f * g0.w, gc = g1.x;
    float p0[3], p1[3], u0[3], u1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float K0 = v.T[0] * gs.R[0 * 3 + k] + v.T[1] * gs.R[1 * 3 + k] + v.T[2] * gs.R[2 * 3 + k];
      const float K1 = v.T[3] * gs.R[0 * 3 + k] + v.T[4] * gs.R[1 * 3 + k] + v.T[5] * gs.R[2 * 3 + k];
      p0[k] = qa * K0 + qb * K1;
      p1[k] = qb * K0 + qc * K1;
      u0[k] = ga * p0[k] + gbh * p1[k];
      u1[k] = gbh * p0[k] + gc * p1[k];
      d_ls[k] -= 2.0f * gs.s[k] * gs.s[k] * (p0[k] * u0[k] + p1[k] * u1[k]);
    }
    bw[0] += p0[1] * u0[2] + p1[1] * u1[2];
    bw[1] += p0[0] * u0[2] + p1[0] * u1[2];
    bw[2] += p0[0] * u0[1] + p1[0] * u1[1];
    float dj00 = 0.f, dj02 = 0.f, dj11 = 0.f, dj12 = 0.f;
    {
      float qu0[3], qu1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float s2 = gs.s[k] * gs.s[k];
        qu0[k] = s2 * (qa * u0[k] + qb * u1[k]);
        qu1[k] = s2 * (qb * u0[k] + qc * u1[k]);
      }
#pragma unroll
      for (int cidx = 0; cidx < 3; ++cidx) {
        const float dt0 = -2.0f * (qu0[0] * gs.R[cidx * 3 + 0] + qu0[1] * gs.R[cidx * 3 + 1] + qu0[2] * gs.R[cidx * 3 + 2]);
        const float dt1 = -2.0f * (qu1[0] * gs.R[cidx * 3 + 0] + qu1[1] * gs.R[cidx * 3 + 1] + qu1[2] * gs.R[cidx * 3 + 2]);
        dj00 += dt0 * V[0 * 4 + cidx];
        dj02 += dt0 * V[2 * 4 + cidx];
        dj11 += dt1 * V[1 * 4 + cidx];
        dj12 += dt1 * V[2 * 4 + cidx];
      }
    }
    const float iz = v.inv_z, iz2 = iz * iz, iz3 = iz2 * iz;
    const float fx = J.cam.fx, fy = J.cam.fy;
    float dp[3];
    dp[0] = g0.x * fx * iz;
    dp[1] = g0.y * fy * iz;
    dp[2] = -g0.x * fx * v.p[0] * iz2 - g0.y * fy * v.p[1] * iz2;
    dp[2] += -dj00 * fx * iz2 + dj02 * 2.0f * fx * v.tx * iz3 - dj11 * fy * iz2 + dj12 * 2.0f * fy * v.ty * iz3;
    const float dtx = -dj02 * fx * iz2, dty = -dj12 * fy * iz2;
    if (v.clx) dp[2] += dtx * (float)v.clx * v.limx; else dp[0] += dtx;
    if (v.cly) dp[2] += dty * (float)v.cly * v.limy; else dp[1] += dty;
#pragma unroll
    for (int k = 0; k < 3; ++k) d_mu[k] += V[0 * 4 + k] * dp[0] + V[1 * 4 + k] * dp[1] + V[2 * 4 + k] * dp[2];

    d_o += g1.y * (1.0f - v.o * v.o);
    if (!v.nu_limited) d_nu += g1.z;

  }

  // colour, one channel at a time (its K coefficients and their gradients in
  // registers): dL/dsh_kc = sum over views of g_c Y_k (0 where the channel
  // is clamped), and the channel's share of the direction gradient of mu,
  // which is linear in the weights g_c sh_kc
  for (int ch = 0; ch < 3; ++ch) {
    float shc[K], dsh[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      shc[k] = __ldg(S.sh + (size_t)(3 * k + ch) * n + i);
      dsh[k] = 0.0f;
    }
    for (uint64_t m = views; m; m &= m - 1) {
      const int q = q0 + __ffsll((long long)m) - 1;
      const sss_job_desc& J = P.jobs[P.scene_jobs[q]];
      const uint32_t e = J.entry_base + i;
      const float grgb = g2d[(size_t)e * 12 + 7 + ch];
      if (grgb == 0.0f) continue;
      float cc[3];
      cam_centre(J.cam, cc);
      const float dd0 = c.mu[0] - cc[0], dd1 = c.mu[1] - cc[1], dd2 = c.mu[2] - cc[2];
      const float il = 1.0f / sqrtf(dd0 * dd0 + dd1 * dd1 + dd2 * dd2);
      const float ux = dd0 * il, uy = dd1 * il, uz = dd2 * il;
      float Y[K];
      sh_basis<DEG>(ux, uy, uz, Y);
      float raw = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) raw = fmaf(shc[k], Y[k], raw);
      if (raw < 0.0f) continue;  // clamped channel: no gradient
#pragma unroll
      for (int k = 0; k < K; ++k) dsh[k] = fmaf(grgb, Y[k], dsh[k]);
      if (DEG > 0) {
        float wk[K];
#pragma unroll
        for (int k = 0; k < K; ++k) wk[k] = grgb * shc[k];
        float gx, gy, gz;
        sh_grad<DEG>(ux, uy, uz, wk, gx, gy, gz);
        const float dotg = gx * ux + gy * uy + gz * uz;
        d_mu[0] += (gx - ux * dotg) * il;
        d_mu[1] += (gy - uy * dotg) * il;
        d_mu[2] += (gz - uz * dotg) * il;
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) G.sh[(size_t)(3 * k + ch) * n + i] = dsh[k];
  }

  float d_q[4] = {0, 0, 0, 0};
  if (touched) {
    // d_i - d_j = (s_i - s_j)(s_i + s_j); dL/dq = (2 / |q|) Xi(q) dL/domega with
    // Xi(q) v = q (x) (0, v) (right multiplication by a pure quaternion)
    const float* sc = gs.s;
    const float dw0 = -2.0f * (sc[1] - sc[2]) * (sc[1] + sc[2]) * bw[0];
    const float dw1 = -2.0f * (sc[2] - sc[0]) * (sc[2] + sc[0]) * bw[1];
    const float dw2 = -2.0f * (sc[0] - sc[1]) * (sc[0] + sc[1]) * bw[2];
    const float w = gs.qn[0], x = gs.qn[1], y = gs.qn[2], z = gs.qn[3];
    const float f = 2.0f * gs.qinv_norm;
    d_q[0] = f * (-x * dw0 - y * dw1 - z * dw2);
    d_q[1] = f * (w * dw0 - z * dw1 + y * dw2);
    d_q[2] = f * (z * dw0 + w * dw1 - x * dw2);
    d_q[3] = f * (-y * dw0 + x * dw1 + w * dw2);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) G.mean[k * n + i] = d_mu[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) G.log_scale[k * n + i] = d_ls[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) G.quat[k * n + i] = d_q[k];
  G.nu[i] = d_nu;
  G.opacity_raw[i] = d_o;
}

struct GradSet {
  sss_params g[SSS_MAX_SCENES];
};

__global__ void __launch_bounds__(128, 5) k_project_bwd(const sss_frame_plan P, const void* ws, const GradSet G) {
  const uint32_t gidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= P.scene_comp_base[P.n_scenes]) return;
  const int s = scene_of_comp(P, gidx);
  const uint32_t i = gidx - P.scene_comp_base[s];
  switch (P.scenes[s].sh_degree) {
    case 0: project_bwd_component<0>(P, s, i, ws, G.g[s]); break;
    case 1: project_bwd_component<1>(P, s, i, ws, G.g[s]); break;
    case 2: project_bwd_component<2>(P, s, i, ws, G.g[s]); break;
    default: project_bwd_component<3>(P, s, i, ws, G.g[s]); break;
  }
}

}  // namespace
}  // namespace sss

extern "C" int sss_project_bwd(const sss_frame_plan* plan, void* ws, const sss_params* grads, sss_stream_t stream) {
  if (!plan || !ws || !grads) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  sss::GradSet G;
  for (int s = 0; s < P.n_scenes; ++s) {
    const sss_params& g = grads[s];
    if (g.n != P.scenes[s].n || g.sh_degree != P.scenes[s].sh_degree) return SSS_ERR_INVALID_ARG;
    if (g.n > 0 && (!g.mean || !g.log_scale || !g.quat || !g.nu || !g.opacity_raw || !g.sh))
      return SSS_ERR_INVALID_ARG;
    G.g[s] = g;
  }
  const uint32_t total = P.scene_comp_base[P.n_scenes];
  if (total == 0) return SSS_OK;
  sss::k_project_bwd<<<sss::ceil_div(total, 128), 128, 0, (cudaStream_t)stream>>>(P, ws, G);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
