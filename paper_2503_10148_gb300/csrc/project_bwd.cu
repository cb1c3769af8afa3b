// a6: 2D splat gradients -> component parameters (SM "Backward Pass": the
// chain through mu', Sigma' to mu, S, R, c, o, nu).
//
// One thread per (scene, component); the forward geometry is recomputed with
// the same code as the projection (proj_geom.cuh), the gradients of every job
// (view) of the scene are chained back and summed in registers, and each
// parameter gradient is written once (planar, coalesced).
//
// Chain, for one view with upstream g = dL/d(mean2D, conic a b c, o, nu, rgb):
//   conic = Sigma2D^-1, Sigma2D = [[A, B], [B, C]], D = AC - B^2:
//     dA = (-ga C^2 + gb B C - gc B^2) / D^2
//     dB = (2 ga B C - gb (A C + B^2) + 2 gc A B) / D^2
//     dC = (-ga B^2 + gb A B - gc A^2) / D^2
//   Sigma2D = T Sigma T^T (T = J W, rows t0, t1):
//     dL/dSigma (symmetric part) = dA t0 t0^T + dB/2 (t0 t1^T + t1 t0^T) + dC t1 t1^T
//     dL/dt0 = 2 dA Sigma t0 + dB Sigma t1,  dL/dt1 = 2 dC Sigma t1 + dB Sigma t0
//   T = J W:  dJ_rc = sum_k dT_rk W_ck (only J00, J02, J11, J12 are non-zero)
//   J(p) = [[fx/z, 0, -fx tx/z^2], [0, fy/z, -fy ty/z^2]], tx = x unless x/z
//     was limited (then tx = +-lim z, and its gradient goes to z)
//   mean2D = (fx x/z + cx, fy y/z + cy);  p = W mu + t
//   Sigma = M M^T, M = R diag(s): dL/dM = 2 dL/dSigma M,
//     dL/ds_k = sum_r dM_rk R_rk, dL/dlog_s = s dL/ds, dL/dR_rk = dM_rk s_k
//   R(q / |q|): derivative of the quaternion rotation formula, then the
//     projection (I - q q^T) / |q| of the normalisation
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

  float d_mu[3] = {0, 0, 0}, d_Sig[6] = {0, 0, 0, 0, 0, 0}, d_o = 0.0f, d_nu = 0.0f;
  float d_sh[3 * K];
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) d_sh[k] = 0.0f;
  bool touched = false;

  for (int q = P.scene_job_begin[s]; q < P.scene_job_begin[s + 1]; ++q) {
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
    const float* V = J.cam.viewmat;
    const float A = v.A, B = v.B, C = v.C;
    const float id2 = 1.0f / (v.det * v.det);
    const float ga = g0.z, gb = g0.w, gc = g1.x;
    const float dA = (-ga * C * C + gb * B * C - gc * B * B) * id2;
    const float dB = (2.0f * ga * B * C - gb * (A * C + B * B) + 2.0f * gc * A * B) * id2;
    const float dC = (-ga * B * B + gb * A * B - gc * A * A) * id2;
    const float* t0 = v.T;
    const float* t1 = v.T + 3;
    // dL/dSigma (symmetric part), packed xx, xy, xz, yy, yz, zz
    {
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int a = ia[k], b = ib[k];
        d_Sig[k] += dA * t0[a] * t0[b] + 0.5f * dB * (t0[a] * t1[b] + t1[a] * t0[b]) + dC * t1[a] * t1[b];
      }
    }
    // Sigma t0, Sigma t1
    const float* Sg = gs.Sig;
    float st0[3], st1[3];
    st0[0] = Sg[0] * t0[0] + Sg[1] * t0[1] + Sg[2] * t0[2];
    st0[1] = Sg[1] * t0[0] + Sg[3] * t0[1] + Sg[4] * t0[2];
    st0[2] = Sg[2] * t0[0] + Sg[4] * t0[1] + Sg[5] * t0[2];
    st1[0] = Sg[0] * t1[0] + Sg[1] * t1[1] + Sg[2] * t1[2];
    st1[1] = Sg[1] * t1[0] + Sg[3] * t1[1] + Sg[4] * t1[2];
    st1[2] = Sg[2] * t1[0] + Sg[4] * t1[1] + Sg[5] * t1[2];
    float dj00 = 0.f, dj02 = 0.f, dj11 = 0.f, dj12 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float dt0 = 2.0f * dA * st0[k] + dB * st1[k];
      const float dt1 = 2.0f * dC * st1[k] + dB * st0[k];
      dj00 += dt0 * V[0 * 4 + k];
      dj02 += dt0 * V[2 * 4 + k];
      dj11 += dt1 * V[1 * 4 + k];
      dj12 += dt1 * V[2 * 4 + k];
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

    // colour
    float cc[3];
    cam_centre(J.cam, cc);
    float dd[3] = {c.mu[0] - cc[0], c.mu[1] - cc[1], c.mu[2] - cc[2]};
    const float il = 1.0f / sqrtf(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    const float ux = dd[0] * il, uy = dd[1] * il, uz = dd[2] * il;
    float Y[K];
    sh_basis<DEG>(ux, uy, uz, Y);
    float grgb[3] = {g1.w, g2.x, g2.y};
    float wk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) wk[k] = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float raw = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) raw = fmaf(__ldg(S.sh + (size_t)(3 * k + ch) * n + i), Y[k], raw);
      if (raw < 0.0f) continue;  // clamped channel: no gradient
#pragma unroll
      for (int k = 0; k < K; ++k) {
        d_sh[3 * k + ch] += grgb[ch] * Y[k];
        wk[k] += grgb[ch] * __ldg(S.sh + (size_t)(3 * k + ch) * n + i);
      }
    }
    if (DEG > 0) {
      float gx, gy, gz;
      sh_grad<DEG>(ux, uy, uz, wk, gx, gy, gz);
      const float dotg = gx * ux + gy * uy + gz * uz;
      d_mu[0] += (gx - ux * dotg) * il;
      d_mu[1] += (gy - uy * dotg) * il;
      d_mu[2] += (gz - uz * dotg) * il;
    }
  }

  float d_ls[3] = {0, 0, 0}, d_q[4] = {0, 0, 0, 0};
  if (touched) {
    // dL/dM = 2 dSigma_sym M, M = R diag(s)
    const float* R = gs.R;
    float Gs[9] = {d_Sig[0], d_Sig[1], d_Sig[2], d_Sig[1], d_Sig[3], d_Sig[4], d_Sig[2], d_Sig[4], d_Sig[5]};
    float dR[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float dM = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) dM += Gs[r * 3 + a] * R[a * 3 + k] * gs.s[k];
        dM *= 2.0f;
        d_ls[k] += dM * R[r * 3 + k] * gs.s[k];
        dR[r * 3 + k] = dM * gs.s[k];
      }
    const float w = gs.qn[0], x = gs.qn[1], y = gs.qn[2], z = gs.qn[3];
    float dqn[4];
    dqn[0] = 2.0f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2.0f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                     2.0f * x * dR[8]);
    dqn[2] = 2.0f * (-2.0f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                     2.0f * y * dR[8]);
    dqn[3] = 2.0f * (-2.0f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0f * z * dR[4] + y * dR[5] +
                     x * dR[6] + y * dR[7]);
    const float proj = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
#pragma unroll
    for (int k = 0; k < 4; ++k) d_q[k] = (dqn[k] - gs.qn[k] * proj) * gs.qinv_norm;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) G.mean[k * n + i] = d_mu[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) G.log_scale[k * n + i] = d_ls[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) G.quat[k * n + i] = d_q[k];
  G.nu[i] = d_nu;
  G.opacity_raw[i] = d_o;
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) G.sh[k * n + i] = d_sh[k];
}

struct GradSet {
  sss_params g[SSS_MAX_SCENES];
};

__global__ void __launch_bounds__(256) k_project_bwd(const sss_frame_plan P, const void* ws, const GradSet G) {
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
  sss::k_project_bwd<<<sss::ceil_div(total, 256), 256, 0, (cudaStream_t)stream>>>(P, ws, G);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
