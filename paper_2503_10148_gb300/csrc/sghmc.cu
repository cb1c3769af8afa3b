// a7: SGHMC on the means, Adam on every other group (Sec. 3.4 Eq.
// sigmoidUpdate, SM Eq. SGHMC), one thread per component.  Pure streaming:
// per component at SH degree 3 it reads parameters, gradients and moments and
// writes parameters and moments back (about 1.6 KB), so it runs at HBM speed.
//
// Noise: Philox4x32-10 (Salmon et al., SC'11) -- ten rounds of two 32x32->64
// multiplications by the published multipliers on counter words 0 and 2,
// xor of the high halves with words 1, 3 and the round key, a word
// permutation, and a Weyl-sequence key schedule -- on counter
// (component, 0, step_lo, step_hi) under key (seed_lo, seed_hi); the four
// words give three normals by Box-Muller.
#include "common.cuh"

namespace sss {
namespace {

struct StepArgs {
  sss_params p, g;
  float* r;
  float* m;
  float* v;
  float* xi_out;
  float eps, C, k, t0;
  int burn_in;
  uint32_t seed_lo, seed_hi;
  uint64_t step;
  const uint64_t* step_counter;
  float lr[5];
  float beta1, beta2, adam_eps;
  float reg_o, reg_s;  // regulariser weights of the loss
  float* mu_m;         // optional Adam moments of dL/dmu (Adam gradient in SGHMC)
  float* mu_v;
};

// Per-thread view of the step: index and bias corrections 1 / (1 - beta^t).
struct StepNow {
  uint32_t lo, hi;
  float inv_bc1, inv_bc2;
};

__device__ __forceinline__ StepNow step_now(const StepArgs& a) {
  const uint64_t s = a.step_counter ? *a.step_counter : a.step;
  StepNow t;
  t.lo = (uint32_t)s;
  t.hi = (uint32_t)(s >> 32);
  const double tt = (double)s + 1.0;
  t.inv_bc1 = (float)(1.0 / (1.0 - pow((double)a.beta1, tt)));
  t.inv_bc2 = (float)(1.0 / (1.0 - pow((double)a.beta2, tt)));
  return t;
}

// Adam on R rows (stride n) of one component: every load of the group is
// issued before the first update, so each thread keeps 4R loads in flight.
// REG adds a regulariser's gradient, a closed form of the parameter p:
// 1: reg exp(p) (scale term, p = log_scale), 2: reg sign(tanh p)(1 - tanh^2 p)
// (opacity term, p = opacity_raw).
template <int R, int REG = 0>
__device__ __forceinline__ void adam_rows(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                          float* __restrict__ v, size_t n, float lr, const StepArgs& a,
                                          const StepNow& t, float reg = 0.0f) {
  float pp[R], gg[R], mo[R], vo[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    gg[r] = __ldg(g + r * n);
    pp[r] = p[r * n];
    mo[r] = m[r * n];
    vo[r] = v[r * n];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (REG == 1) gg[r] = fmaf(reg, expf(pp[r]), gg[r]);
    if (REG == 2) {
      const float o = tanhf(pp[r]);
      const float sg = o > 0.0f ? 1.0f : (o < 0.0f ? -1.0f : 0.0f);
      gg[r] = fmaf(reg * sg, fmaf(-o, o, 1.0f), gg[r]);
    }
    const float mm = fmaf(a.beta1, mo[r], (1.0f - a.beta1) * gg[r]);
    const float vv = fmaf(a.beta2, vo[r], (1.0f - a.beta2) * gg[r] * gg[r]);
    m[r * n] = mm;
    v[r * n] = vv;
    p[r * n] = pp[r] - lr * (mm * t.inv_bc1) / (sqrtf(vv * t.inv_bc2) + a.adam_eps);
  }
}

template <int DEG>
__device__ __forceinline__ void step_component(const StepArgs& a, uint32_t i, const StepNow& t) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const size_t n = (size_t)a.p.n;
  const float o = tanhf(a.p.opacity_raw[i]);
  const float gate = 1.0f / (1.0f + expf(a.k * (fabsf(o) - a.t0)));
  // three standard normals
  const uint4 w = philox4x32_10(make_uint4(i, 0u, t.lo, t.hi), a.seed_lo, a.seed_hi);
  const float s24 = 1.0f / 16777216.0f;
  const float u1 = (float)((w.x >> 8) + 1u) * s24, u2 = (float)(w.y >> 8) * s24;
  const float u3 = (float)((w.z >> 8) + 1u) * s24, u4 = (float)(w.w >> 8) * s24;
  const float r1 = sqrtf(-2.0f * logf(u1)), r2 = sqrtf(-2.0f * logf(u3));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  float xi[3] = {r1 * cs, r1 * sn, r2 * cospif(2.0f * u4)};
  if (a.xi_out)
#pragma unroll
    for (int c = 0; c < 3; ++c) a.xi_out[c * n + i] = xi[c];
  float noise[3] = {xi[0], xi[1], xi[2]};
  if (a.burn_in) {  // Sigma xi, Sigma = R S S^T R^T of the pre-step parameters
    float q[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = a.p.quat[c * n + i];
    const float inv = 1.0f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float qw = q[0] * inv, qx = q[1] * inv, qy = q[2] * inv, qz = q[3] * inv;
    const float R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                        2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                        2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
    float s2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) s2[c] = expf(2.0f * a.p.log_scale[c * n + i]);
    // Sigma xi = R (s^2 * (R^T xi))
    float t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = s2[k] * (R[0 * 3 + k] * xi[0] + R[1 * 3 + k] * xi[1] + R[2 * 3 + k] * xi[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) noise[r] = R[r * 3 + 0] * t[0] + R[r * 3 + 1] * t[1] + R[r * 3 + 2] * t[2];
  }
  const float sq = sqrtf(2.0f * a.eps * a.C);
  const float fr = 1.0f - a.eps * a.C;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const size_t j = c * n + i;
    float G = a.g.mean[j];
    if (a.mu_m) {  // the Adam gradient in SGHMC: m^ / (sqrt(v^) + eps) of dL/dmu
      const float mm = fmaf(a.beta1, a.mu_m[j], (1.0f - a.beta1) * G);
      const float vv = fmaf(a.beta2, a.mu_v[j], (1.0f - a.beta2) * G * G);
      a.mu_m[j] = mm;
      a.mu_v[j] = vv;
      G = (mm * t.inv_bc1) / (sqrtf(vv * t.inv_bc2) + a.adam_eps);
    }
    const float rr = a.r[j];
    a.r[j] = fr * rr - a.eps * G + sq * xi[c];
    float mu = a.p.mean[j] - a.eps * a.eps * G;
    if (a.burn_in) mu += gate * a.eps * sq * noise[c];
    else mu += gate * a.eps * fr * rr + gate * a.eps * sq * xi[c];
    a.p.mean[j] = mu;
  }
  // Adam: log_scale (rows 0-2 of m, v), quat (3-6), nu (7), opacity (8), sh (9..)
  if (a.reg_s != 0.0f)
    adam_rows<3, 1>(a.p.log_scale + i, a.g.log_scale + i, a.m + i, a.v + i, n, a.lr[0], a, t, a.reg_s);
  else
    adam_rows<3>(a.p.log_scale + i, a.g.log_scale + i, a.m + i, a.v + i, n, a.lr[0], a, t);
  adam_rows<4>(a.p.quat + i, a.g.quat + i, a.m + 3 * n + i, a.v + 3 * n + i, n, a.lr[1], a, t);
  adam_rows<1>(a.p.nu + i, a.g.nu + i, a.m + 7 * n + i, a.v + 7 * n + i, n, a.lr[2], a, t);
  a.p.nu[i] = fminf(fmaxf(a.p.nu[i], 1.0f), 1e4f);
  if (a.reg_o != 0.0f)
    adam_rows<1, 2>(a.p.opacity_raw + i, a.g.opacity_raw + i, a.m + 8 * n + i, a.v + 8 * n + i, n, a.lr[3], a, t,
                    a.reg_o);
  else
    adam_rows<1>(a.p.opacity_raw + i, a.g.opacity_raw + i, a.m + 8 * n + i, a.v + 8 * n + i, n, a.lr[3], a, t);
  constexpr int SH_ROWS = 3 * K;
  constexpr int CH = SH_ROWS % 8 == 0 ? 8 : (SH_ROWS % 4 == 0 ? 4 : 3);
#pragma unroll 1
  for (int c = 0; c < SH_ROWS; c += CH)
    adam_rows<CH>(a.p.sh + c * n + i, a.g.sh + c * n + i, a.m + (9 + c) * n + i, a.v + (9 + c) * n + i, n, a.lr[4],
                  a, t);
}

__global__ void k_step_advance(uint64_t* counter) { *counter += 1; }

__global__ void __launch_bounds__(256) k_sghmc(const StepArgs a) {
  // the step index and its FP64 bias corrections, once per CTA
  __shared__ StepNow s_t;
  if (threadIdx.x == 0) s_t = step_now(a);
  __syncthreads();
  const StepNow t = s_t;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint32_t)a.p.n) return;
  switch (a.p.sh_degree) {
    case 0: step_component<0>(a, i, t); break;
    case 1: step_component<1>(a, i, t); break;
    case 2: step_component<2>(a, i, t); break;
    default: step_component<3>(a, i, t); break;
  }
}

}  // namespace
}  // namespace sss

extern "C" int sss_sghmc_step(const sss_params* params, const sss_params* grads, float* momentum, float* adam_m,
                              float* adam_v, const sss_step_params* sp, float* xi_out, sss_stream_t stream) {
  if (!params || !grads || !momentum || !adam_m || !adam_v || !sp) return SSS_ERR_INVALID_ARG;
  if (params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3 || grads->n != params->n ||
      grads->sh_degree != params->sh_degree)
    return SSS_ERR_INVALID_ARG;
  if (params->n == 0) return SSS_OK;
  if (!(sp->beta1 >= 0.0f && sp->beta1 < 1.0f && sp->beta2 >= 0.0f && sp->beta2 < 1.0f && sp->eps >= 0.0f &&
        sp->C >= 0.0f && sp->reg_opacity >= 0.0f && sp->reg_scale >= 0.0f))
    return SSS_ERR_INVALID_ARG;
  sss::StepArgs a;
  a.p = *params;
  a.g = *grads;
  a.r = momentum;
  a.m = adam_m;
  a.v = adam_v;
  a.xi_out = xi_out;
  a.eps = sp->eps;
  a.C = sp->C;
  a.k = sp->k;
  a.t0 = sp->t0;
  a.burn_in = sp->burn_in;
  a.seed_lo = (uint32_t)sp->seed;
  a.seed_hi = (uint32_t)(sp->seed >> 32);
  a.step = sp->step;
  a.step_counter = sp->step_counter;
  for (int k = 0; k < 5; ++k) a.lr[k] = sp->lr[k];
  a.beta1 = sp->beta1;
  a.beta2 = sp->beta2;
  a.adam_eps = sp->adam_eps;
  a.reg_o = sp->reg_opacity;
  a.reg_s = sp->reg_scale;
  if ((sp->mu_adam_m == nullptr) != (sp->mu_adam_v == nullptr)) return SSS_ERR_INVALID_ARG;
  a.mu_m = sp->mu_adam_m;
  a.mu_v = sp->mu_adam_v;
  sss::k_sghmc<<<sss::ceil_div((size_t)params->n, 256), 256, 0, (cudaStream_t)stream>>>(a);
  SSS_LAUNCH_CHECK();
  if (sp->step_counter) {
    sss::k_step_advance<<<1, 1, 0, (cudaStream_t)stream>>>(sp->step_counter);
    SSS_LAUNCH_CHECK();
  }
  return SSS_OK;
}
