// a7: SGHMC on the means, Adam on every other group (Sec. 3.4 Eq.
// sigmoidUpdate, SM Eq. SGHMC).  Two launches: k_sghmc updates the means
// (one thread per component: the noise, the gate and the momentum), k_adam
// every other parameter row (a 2D grid of (row, block of 1024 components),
// four components per thread with their loads in flight, as 16-byte
// accesses where the layout allows).  Pure streaming:
// per component at SH degree 3 they read parameters, gradients and moments
// and write parameters and moments back (about 1.6 KB), so they run at HBM
// speed.  The updated parameters go to a second set of arrays, which may be
// the input arrays themselves (an update in place).
//
// Noise: Philox4x32-10 (Salmon et al., SC'11) -- ten rounds of two 32x32->64
// multiplications by the published multipliers on counter words 0 and 2,
// xor of the high halves with words 1, 3 and the round key, a word
// permutation, and a Weyl-sequence key schedule -- on counter
// (component, 0, step_lo, step_hi) under key (seed_lo, seed_hi); the four
// words give three normals by Box-Muller.
#include <cmath>
#include <cstdint>
#include <initializer_list>

#include "common.cuh"

namespace sss {
namespace {

struct StepArgs {
  sss_params p, g;  // parameters before the step, gradients
  sss_params q;     // parameters after the step (q's arrays may be p's)
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
  uint32_t* philox_out;  // optional [4][n]: the raw Philox words of the noise
  float ln_beta1, ln_beta2;
};

// Per-thread view of the step: index and bias corrections 1 / (1 - beta^t).
struct StepNow {
  uint32_t lo, hi;
  float inv_bc1, inv_bc2;
};

// Bias corrections 1 / (1 - beta^t) with 1 - beta^t = -expm1(t ln beta) (no
// cancellation for beta near 1); ln beta comes from the host in FP64.
__device__ __forceinline__ StepNow step_now(const StepArgs& a) {
  const uint64_t s = a.step_counter ? *a.step_counter : a.step;
  StepNow t;
  t.lo = (uint32_t)s;
  t.hi = (uint32_t)(s >> 32);
  const float tt = (float)s + 1.0f;
  t.inv_bc1 = -1.0f / expm1f(tt * a.ln_beta1);
  t.inv_bc2 = -1.0f / expm1f(tt * a.ln_beta2);
  return t;
}

// Adam (bias-corrected) on every row of the other groups, one CTA row
// (blockIdx.y) per parameter row: rows 0-2 log_scale (lr[0], + reg_s exp(p)),
// 3-6 quaternion (lr[1]), 7 nu (lr[2], then limited to [1, 1e4]), 8
// opacity_raw (lr[3], + reg_o sign(tanh p)(1 - tanh^2 p)), 9.. SH (lr[4]).
// Each thread updates kPer components with all their loads in flight.
constexpr int kPer = 4;

// Row `row` (numbered as above) of a parameter set of n components.
__device__ __forceinline__ float* param_row(const sss_params& s, int row, size_t n) {
  if (row < 3) return s.log_scale + row * n;
  if (row < 7) return s.quat + (row - 3) * n;
  if (row == 7) return s.nu;
  if (row == 8) return s.opacity_raw;
  return s.sh + (row - 9) * n;
}

// One Adam update (bias-corrected) of parameter pk of row `row`: the
// regulariser's gradient joins gk first; mk and vk are updated in place and
// the new parameter is returned.
__device__ __forceinline__ float adam_update(const StepArgs& a, const StepNow& t, int row, int reg, float lr, float pk,
                                             float gk, float& mk, float& vk) {
  if (reg == 1) gk = fmaf(a.reg_s, expf(pk), gk);
  if (reg == 2) {
    const float o = tanhf(pk);
    const float sg = o > 0.0f ? 1.0f : (o < 0.0f ? -1.0f : 0.0f);
    gk = fmaf(a.reg_o * sg, fmaf(-o, o, 1.0f), gk);
  }
  mk = fmaf(a.beta1, mk, (1.0f - a.beta1) * gk);
  vk = fmaf(a.beta2, vk, (1.0f - a.beta2) * gk * gk);
  float np = pk - lr * (mk * t.inv_bc1) / (sqrtf(vk * t.inv_bc2) + a.adam_eps);
  if (row == 7) np = fminf(fmaxf(np, 1.0f), 1e4f);
  return np;
}

// VEC: n is a multiple of 4 and every array is 16-byte aligned, so a
// thread's kPer = 4 components are adjacent and move as one 16-byte load or
// store per array; otherwise they are strided by the CTA width.
template <bool VEC>
__global__ void __launch_bounds__(256) k_adam(const StepArgs a) {
  __shared__ StepNow s_t;
  if (threadIdx.x == 0) s_t = step_now(a);
  __syncthreads();
  const StepNow t = s_t;
  const int row = blockIdx.y;
  const size_t n = (size_t)a.p.n;
  const float* p = param_row(a.p, row, n);
  float* p_out = param_row(a.q, row, n);
  const float* g = param_row(a.g, row, n);
  const int grp = row < 3 ? 0 : (row < 7 ? 1 : (row == 7 ? 2 : (row == 8 ? 3 : 4)));
  const float lr = a.lr[grp];
  const int reg = (row < 3 && a.reg_s != 0.0f) ? 1 : ((row == 8 && a.reg_o != 0.0f) ? 2 : 0);
  float* m = a.m + row * n;
  float* v = a.v + row * n;
  if (VEC) {
    static_assert(kPer == 4, "one float4 per thread and array");
    const size_t i = ((size_t)blockIdx.x * 256 + threadIdx.x) * 4;
    if (i >= n) return;
    const float4 gg = __ldg(reinterpret_cast<const float4*>(g + i));
    const float4 pp = *reinterpret_cast<const float4*>(p + i);
    float4 mo = *reinterpret_cast<const float4*>(m + i);
    float4 vo = *reinterpret_cast<const float4*>(v + i);
    float4 np;
    np.x = adam_update(a, t, row, reg, lr, pp.x, gg.x, mo.x, vo.x);
    np.y = adam_update(a, t, row, reg, lr, pp.y, gg.y, mo.y, vo.y);
    np.z = adam_update(a, t, row, reg, lr, pp.z, gg.z, mo.z, vo.z);
    np.w = adam_update(a, t, row, reg, lr, pp.w, gg.w, mo.w, vo.w);
    *reinterpret_cast<float4*>(m + i) = mo;
    *reinterpret_cast<float4*>(v + i) = vo;
    *reinterpret_cast<float4*>(p_out + i) = np;
    return;
  }
  const size_t base = (size_t)blockIdx.x * (256 * kPer) + threadIdx.x;
  float pp[kPer], gg[kPer], mo[kPer], vo[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const size_t i = base + 256 * k;
    if (i < n) {
      gg[k] = __ldg(g + i);
      pp[k] = p[i];
      mo[k] = m[i];
      vo[k] = v[i];
    }
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const size_t i = base + 256 * k;
    if (i >= n) continue;
    const float np = adam_update(a, t, row, reg, lr, pp[k], gg[k], mo[k], vo[k]);
    m[i] = mo[k];
    v[i] = vo[k];
    p_out[i] = np;
  }
}

template <int DEG>
__device__ __forceinline__ void step_component(const StepArgs& a, uint32_t i, const StepNow& t) {
  const size_t n = (size_t)a.p.n;
  const float o = tanhf(a.p.opacity_raw[i]);
  const float gate = 1.0f / (1.0f + expf(a.k * (fabsf(o) - a.t0)));
  // three standard normals
  const uint4 w = philox4x32_10(make_uint4(i, 0u, t.lo, t.hi), a.seed_lo, a.seed_hi);
  if (a.philox_out) {
    a.philox_out[i] = w.x;
    a.philox_out[n + i] = w.y;
    a.philox_out[2 * n + i] = w.z;
    a.philox_out[3 * n + i] = w.w;
  }
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
    a.q.mean[j] = mu;
  }
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

extern "C" int sss_sghmc_step_to(const sss_params* params, const sss_params* params_out, const sss_params* grads,
                                 float* momentum, float* adam_m, float* adam_v, const sss_step_params* sp,
                                 float* xi_out, sss_stream_t stream) {
  if (!params || !params_out || !grads || !momentum || !adam_m || !adam_v || !sp) return SSS_ERR_INVALID_ARG;
  if (params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3 || grads->n != params->n ||
      grads->sh_degree != params->sh_degree || params_out->n != params->n ||
      params_out->sh_degree != params->sh_degree)
    return SSS_ERR_INVALID_ARG;
  if (params->n == 0) return SSS_OK;
  if (!(sp->beta1 >= 0.0f && sp->beta1 < 1.0f && sp->beta2 >= 0.0f && sp->beta2 < 1.0f && sp->eps >= 0.0f &&
        sp->C >= 0.0f && sp->reg_opacity >= 0.0f && sp->reg_scale >= 0.0f))
    return SSS_ERR_INVALID_ARG;
  sss::StepArgs a;
  a.p = *params;
  a.q = *params_out;
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
  a.philox_out = sp->philox_out;
  a.ln_beta1 = (float)std::log((double)sp->beta1);
  a.ln_beta2 = (float)std::log((double)sp->beta2);
  // the means first: the gate and the burn-in covariance read the pre-step
  // opacity, quaternion and scale, which the Adam rows then update
  sss::k_sghmc<<<sss::ceil_div((size_t)params->n, 256), 256, 0, (cudaStream_t)stream>>>(a);
  const int rows = 9 + 3 * (params->sh_degree + 1) * (params->sh_degree + 1);
  // 16-byte rows: n a multiple of 4 (each row then starts 16-byte aligned
  // within its array) and every array 16-byte aligned
  bool vec = params->n % 4 == 0 && (reinterpret_cast<uintptr_t>(adam_m) | reinterpret_cast<uintptr_t>(adam_v)) % 16 == 0;
  for (const sss_params* s : {params, params_out, grads})
    for (const float* f : {s->log_scale, s->quat, s->nu, s->opacity_raw, s->sh})
      vec = vec && reinterpret_cast<uintptr_t>(f) % 16 == 0;
  const dim3 grid(sss::ceil_div((size_t)params->n, 256 * sss::kPer), rows);
  if (vec)
    sss::k_adam<true><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  else
    sss::k_adam<false><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  SSS_LAUNCH_CHECK();
  if (sp->step_counter) {
    sss::k_step_advance<<<1, 1, 0, (cudaStream_t)stream>>>(sp->step_counter);
    SSS_LAUNCH_CHECK();
  }
  return SSS_OK;
}

extern "C" int sss_sghmc_step(const sss_params* params, const sss_params* grads, float* momentum, float* adam_m,
                              float* adam_v, const sss_step_params* sp, float* xi_out, sss_stream_t stream) {
  return sss_sghmc_step_to(params, params, grads, momentum, adam_m, adam_v, sp, xi_out, stream);
}
