// Component recycling (Sec. 3.4 "Adding and Recycling Components", Eq.
// relocation; SM "Component Recycling"): near-transparent components are
// moved onto live ones so that the rendered result is unchanged to first
// order.
//
//  1. dead: |o| < dead_opacity; the first floor(max_fraction n) dead
//     components in index order move (o from FP64 tanh of the raw opacity).
//  2. targets: a multinomial over live components with weight |o|,
//     quantised to w = floor(|o| 2^12); with W the weight total and x the
//     first word of Philox4x32-10 on counter (dead rank, 1, step_lo,
//     step_hi), v = (x W) >> 32 and the target is the first index whose
//     inclusive weight prefix exceeds v (exact integer arithmetic).
//  3. the draws are sorted by target (stable, so in dead-rank order); a
//     target keeps at most n_max - 1 copies, N = 1 + copies.
//  4. per target, in FP64: o_new = 1 - (1 - |o|)^(1/N) with o's sign,
//     Sigma_new = F Sigma_old, F = o^2 (B(1/2, (nu+2)/2) / K)^2,
//     K = sum_{i=1..N} sum_{k<i} C(i-1,k) (-1)^k o_new^(k+1)
//         B(1/2, ((k+1)(nu+3)-1)/2)   (nu_new = nu_old; B through ln Gamma),
//     so every log-scale grows by ln(F)/2.
//  5. copies take the target's mean, quaternion, nu, SH, the new opacity and
//     scale, and restart their momentum and Adam moments at zero.
#include <cmath>

#include "common.cuh"

namespace sss {
namespace {

constexpr int RT = 256;
constexpr int kWeightBits = 12;
constexpr uint32_t kStreamWord = 1;  // Philox counter word 1 (the sampler's noise uses 0)

struct RelocLayout {
  size_t dead, w, prefix, bdead, bw, ctrl, dead_idx, keys, vals, hist, tmp_raw, tmp_ls, rank, total;
  uint32_t n, cap, nb, sort_blocks;
};

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

RelocLayout layout(int32_t n, float max_fraction) {
  RelocLayout L{};
  L.n = (uint32_t)n;
  const double c = std::floor((double)max_fraction * (double)n);
  L.cap = (uint32_t)(c < 0.0 ? 0.0 : (c > (double)n ? (double)n : c));
  L.nb = (uint32_t)((n + RT - 1) / RT);
  L.sort_blocks = 3 * device_sm_count();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = up256(off + bytes);
    return o;
  };
  L.dead = take(4 * (size_t)n);
  L.w = take(4 * (size_t)n);
  L.prefix = take(8 * (size_t)n);
  L.bdead = take(4 * (size_t)L.nb + 4);
  L.bw = take(8 * (size_t)L.nb + 8);
  L.ctrl = take(64);  // [0] W total (u64), [2] dead total (u32), [3] moving draws n_sel (u32)
  L.dead_idx = take(4 * (size_t)L.cap + 4);
  L.keys = take(8 * (size_t)L.cap + 8);
  L.vals = take(8 * (size_t)L.cap + 8);
  L.hist = take(4 * ((size_t)256 * L.sort_blocks + 256));
  L.tmp_raw = take(4 * (size_t)n);
  L.tmp_ls = take(12 * (size_t)n);
  L.rank = take(4 * (size_t)L.cap + 4);
  L.total = off;
  return L;
}

struct RelocArgs {
  sss_params p;
  float* momentum;
  float* adam_m;
  float* adam_v;
  int adam_rows;
  double dead_opacity;
  int n_max;
  uint32_t seed_lo, seed_hi, step_lo, step_hi;
  uint32_t* moved_out;
  RelocLayout L;
  char* ws;
};

template <typename T>
__host__ __device__ __forceinline__ T* at(const RelocArgs& A, size_t off) {
  return reinterpret_cast<T*>(A.ws + off);
}

// Block sum of one value per thread (RT threads).
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* s_w) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = 0;
#pragma unroll
  for (int w = 0; w < RT / 32; ++w) t += s_w[w];
  __syncthreads();
  return t;
}

// Inclusive block scan of one value per thread (RT threads).
template <typename T>
__device__ __forceinline__ T block_scan(T v, T* s_w, T& total) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  T before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < RT / 32; ++w) {
    before += (unsigned)w < warp ? s_w[w] : (T)0;
    tot += s_w[w];
  }
  __syncthreads();
  total = tot;
  return before + x;
}

__global__ void __launch_bounds__(RT) k_reloc_flags(const RelocArgs A) {
  __shared__ uint32_t s_d[RT / 32];
  __shared__ unsigned long long s_w[RT / 32];
  const uint32_t i = blockIdx.x * RT + threadIdx.x;
  uint32_t dead = 0, w = 0;
  if (i < A.L.n) {
    const double o = fabs(tanh((double)A.p.opacity_raw[i]));
    dead = o < A.dead_opacity ? 1u : 0u;
    w = dead ? 0u : (uint32_t)floor(o * (double)(1 << kWeightBits));
    at<uint32_t>(A, A.L.dead)[i] = dead;
    at<uint32_t>(A, A.L.w)[i] = w;
  }
  const uint32_t sd = block_sum<uint32_t>(dead, s_d);
  const unsigned long long sw = block_sum<unsigned long long>(w, s_w);
  if (threadIdx.x == 0) {
    at<uint32_t>(A, A.L.bdead)[blockIdx.x] = sd;
    at<unsigned long long>(A, A.L.bw)[blockIdx.x] = sw;
  }
}

// Exclusive scan of the block sums (one CTA); totals into ctrl.
__global__ void __launch_bounds__(RT) k_reloc_scan_blocks(const RelocArgs A) {
  __shared__ uint32_t s_d[RT / 32];
  __shared__ unsigned long long s_w[RT / 32];
  uint32_t* bd = at<uint32_t>(A, A.L.bdead);
  unsigned long long* bw = at<unsigned long long>(A, A.L.bw);
  uint32_t cd = 0;
  unsigned long long cw = 0;
  for (uint32_t base = 0; base < A.L.nb; base += RT) {
    const uint32_t b = base + threadIdx.x;
    const uint32_t vd = b < A.L.nb ? bd[b] : 0u;
    const unsigned long long vw = b < A.L.nb ? bw[b] : 0ull;
    uint32_t td;
    unsigned long long tw;
    const uint32_t id = block_scan<uint32_t>(vd, s_d, td);
    const unsigned long long iw = block_scan<unsigned long long>(vw, s_w, tw);
    if (b < A.L.nb) {
      bd[b] = cd + id - vd;
      bw[b] = cw + iw - vw;
    }
    cd += td;
    cw += tw;
  }
  if (threadIdx.x == 0) {
    unsigned long long* c64 = at<unsigned long long>(A, A.L.ctrl);
    uint32_t* c32 = at<uint32_t>(A, A.L.ctrl);
    c64[0] = cw;
    c32[2] = cd;
    c32[3] = (cw == 0ull) ? 0u : (cd < A.L.cap ? cd : A.L.cap);
  }
}

// Inclusive weight prefix; dead index of every dead rank below the cap.
__global__ void __launch_bounds__(RT) k_reloc_prefix(const RelocArgs A) {
  __shared__ uint32_t s_d[RT / 32];
  __shared__ unsigned long long s_w[RT / 32];
  const uint32_t i = blockIdx.x * RT + threadIdx.x;
  const bool in = i < A.L.n;
  const uint32_t dead = in ? at<uint32_t>(A, A.L.dead)[i] : 0u;
  const unsigned long long w = in ? at<uint32_t>(A, A.L.w)[i] : 0u;
  uint32_t td;
  unsigned long long tw;
  const uint32_t rd = block_scan<uint32_t>(dead, s_d, td) - dead + at<uint32_t>(A, A.L.bdead)[blockIdx.x];
  const unsigned long long pw = block_scan<unsigned long long>(w, s_w, tw) + at<unsigned long long>(A, A.L.bw)[blockIdx.x];
  if (in) {
    at<unsigned long long>(A, A.L.prefix)[i] = pw;
    if (dead && rd < A.L.cap) at<uint32_t>(A, A.L.dead_idx)[rd] = i;
  }
}

// Draw r: target key and value r.
__global__ void __launch_bounds__(RT) k_reloc_draw(const RelocArgs A) {
  const uint32_t r = blockIdx.x * RT + threadIdx.x;
  const uint32_t n_sel = at<uint32_t>(A, A.L.ctrl)[3];
  if (r >= n_sel) return;
  const unsigned long long W = at<unsigned long long>(A, A.L.ctrl)[0];
  const uint4 x = philox4x32_10(make_uint4(r, kStreamWord, A.step_lo, A.step_hi), A.seed_lo, A.seed_hi);
  // v = (x W) >> 32 exactly (W may exceed 2^32): x W_hi + (x W_lo) >> 32 < W
  const unsigned long long xl = x.x;
  const unsigned long long v = xl * (W >> 32) + ((xl * (W & 0xffffffffull)) >> 32);
  const unsigned long long* P = at<unsigned long long>(A, A.L.prefix);
  uint32_t lo = 0, hi = A.L.n - 1;  // first t with P[t] > v exists: P[n-1] = W > v
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P[mid] > v) hi = mid; else lo = mid + 1;
  }
  at<uint32_t>(A, A.L.keys)[r] = lo;
  at<uint32_t>(A, A.L.vals)[r] = r;
}

__device__ __forceinline__ double beta_fn(double x, double y) { return exp(lgamma(x) + lgamma(y) - lgamma(x + y)); }

// Per sorted draw: rank among the draws of its target (up to n_max - 1);
// the first draw of each target computes the target's new opacity and
// log-scales into the temporaries.
__global__ void __launch_bounds__(RT) k_reloc_groups(const RelocArgs A, const uint32_t* __restrict__ skeys) {
  const uint32_t p = blockIdx.x * RT + threadIdx.x;
  const uint32_t n_sel = at<uint32_t>(A, A.L.ctrl)[3];
  if (p >= n_sel) return;
  const uint32_t t = skeys[p];
  uint32_t k = 0;
  while (k < (uint32_t)A.n_max && p >= k + 1 && skeys[p - k - 1] == t) ++k;
  at<uint32_t>(A, A.L.rank)[p] = k;
  if (k < (uint32_t)(A.n_max - 1)) atomicAdd(A.moved_out, 1u);
  if (k != 0) return;
  uint32_t c = 1;
  while (c < (uint32_t)(A.n_max - 1) && p + c < n_sel && skeys[p + c] == t) ++c;
  const int N = (int)c + 1;
  const double o_old = tanh((double)A.p.opacity_raw[t]);
  const double a = fabs(o_old);
  const double o_new = 1.0 - pow(1.0 - a, 1.0 / (double)N);
  const double nu = (double)A.p.nu[t];
  double K = 0.0;
  for (int i = 1; i <= N; ++i) {
    double binom = 1.0, opow = o_new, sgn = 1.0;  // C(i-1, k), o_new^(k+1), (-1)^k
    for (int kk = 0; kk < i; ++kk) {
      K += binom * sgn * opow * beta_fn(0.5, ((double)(kk + 1) * (nu + 3.0) - 1.0) / 2.0);
      binom = binom * (double)(i - 1 - kk) / (double)(kk + 1);
      opow *= o_new;
      sgn = -sgn;
    }
  }
  const double ratio = beta_fn(0.5, (nu + 2.0) / 2.0) / K;
  const double F = a * a * ratio * ratio;
  at<float>(A, A.L.tmp_raw)[t] = (float)atanh(copysign(o_new, o_old));
  const double dls = 0.5 * log(F);
  const size_t n = A.L.n;
#pragma unroll
  for (int j = 0; j < 3; ++j) at<float>(A, A.L.tmp_ls)[j * n + t] = (float)((double)A.p.log_scale[j * n + t] + dls);
}

// Every moving draw: copy the target into the dead component.
__global__ void __launch_bounds__(RT) k_reloc_copy(const RelocArgs A, const uint32_t* __restrict__ skeys,
                                                   const uint32_t* __restrict__ svals) {
  const uint32_t p = blockIdx.x * RT + threadIdx.x;
  const uint32_t n_sel = at<uint32_t>(A, A.L.ctrl)[3];
  if (p >= n_sel || at<uint32_t>(A, A.L.rank)[p] >= (uint32_t)(A.n_max - 1)) return;
  const uint32_t t = skeys[p];
  const uint32_t d = at<uint32_t>(A, A.L.dead_idx)[svals[p]];
  const size_t n = A.L.n;
  const int K3 = 3 * (A.p.sh_degree + 1) * (A.p.sh_degree + 1);
  float* mean = const_cast<float*>(A.p.mean);
  float* quat = const_cast<float*>(A.p.quat);
  float* nu = const_cast<float*>(A.p.nu);
  float* sh = const_cast<float*>(A.p.sh);
  float* raw = const_cast<float*>(A.p.opacity_raw);
  float* ls = const_cast<float*>(A.p.log_scale);
  for (int j = 0; j < 3; ++j) mean[j * n + d] = mean[j * n + t];
  for (int j = 0; j < 4; ++j) quat[j * n + d] = quat[j * n + t];
  nu[d] = nu[t];
  for (int j = 0; j < K3; ++j) sh[j * n + d] = sh[j * n + t];
  raw[d] = at<float>(A, A.L.tmp_raw)[t];
  for (int j = 0; j < 3; ++j) ls[j * n + d] = at<float>(A, A.L.tmp_ls)[j * n + t];
  for (int j = 0; j < 3; ++j) A.momentum[j * n + d] = 0.0f;
  for (int j = 0; j < A.adam_rows; ++j) {
    A.adam_m[j * n + d] = 0.0f;
    A.adam_v[j * n + d] = 0.0f;
  }
}

// Every target: its own new opacity and log-scales.
__global__ void __launch_bounds__(RT) k_reloc_targets(const RelocArgs A, const uint32_t* __restrict__ skeys) {
  const uint32_t p = blockIdx.x * RT + threadIdx.x;
  const uint32_t n_sel = at<uint32_t>(A, A.L.ctrl)[3];
  if (p >= n_sel || at<uint32_t>(A, A.L.rank)[p] != 0u) return;
  const uint32_t t = skeys[p];
  const size_t n = A.L.n;
  const_cast<float*>(A.p.opacity_raw)[t] = at<float>(A, A.L.tmp_raw)[t];
  for (int j = 0; j < 3; ++j) const_cast<float*>(A.p.log_scale)[j * n + t] = at<float>(A, A.L.tmp_ls)[j * n + t];
}

int key_bits(uint32_t n) {
  int b = 1;
  while (b < 32 && (1ull << b) < (unsigned long long)n) ++b;
  return b;
}

}  // namespace
}  // namespace sss

using namespace sss;

extern "C" size_t sss_relocate_scratch_bytes(int32_t n, float max_fraction) {
  if (n < 0 || !(max_fraction >= 0.0f && max_fraction <= 1.0f)) return 0;
  return layout(n, max_fraction).total;
}

extern "C" int sss_relocate(const sss_params* params, float* momentum, float* adam_m, float* adam_v,
                            const sss_relocate_params* rp, uint32_t* moved_out, void* scratch, sss_stream_t stream) {
  if (!params || !momentum || !adam_m || !adam_v || !rp || !moved_out || !scratch) return SSS_ERR_INVALID_ARG;
  if (params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3) return SSS_ERR_INVALID_ARG;
  if (!(rp->max_fraction >= 0.0f && rp->max_fraction <= 1.0f) || !(rp->dead_opacity >= 0.0f) || rp->n_max < 2 ||
      rp->n_max > 64)
    return SSS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) % 256 != 0) return SSS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(moved_out, 0, sizeof(uint32_t), st) != cudaSuccess) return SSS_ERR_CUDA;
  if (params->n == 0) return SSS_OK;
  RelocArgs A{};
  A.p = *params;
  A.momentum = momentum;
  A.adam_m = adam_m;
  A.adam_v = adam_v;
  A.adam_rows = 9 + 3 * (params->sh_degree + 1) * (params->sh_degree + 1);
  A.dead_opacity = (double)rp->dead_opacity;
  A.n_max = rp->n_max;
  A.seed_lo = (uint32_t)rp->seed;
  A.seed_hi = (uint32_t)(rp->seed >> 32);
  A.step_lo = (uint32_t)rp->step;
  A.step_hi = (uint32_t)(rp->step >> 32);
  A.moved_out = moved_out;
  A.L = layout(params->n, rp->max_fraction);
  A.ws = static_cast<char*>(scratch);
  const RelocLayout& L = A.L;
  k_reloc_flags<<<L.nb, RT, 0, st>>>(A);
  k_reloc_scan_blocks<<<1, RT, 0, st>>>(A);
  k_reloc_prefix<<<L.nb, RT, 0, st>>>(A);
  SSS_LAUNCH_CHECK();
  if (L.cap == 0) return SSS_OK;
  const unsigned gcap = ceil_div(L.cap, RT);
  k_reloc_draw<<<gcap, RT, 0, st>>>(A);
  SSS_LAUNCH_CHECK();
  uint32_t* keys = at<uint32_t>(A, L.keys);
  uint32_t* vals = at<uint32_t>(A, L.vals);
  const uint32_t* n_sel_dev = at<uint32_t>(A, L.ctrl) + 3;
  const int bits = key_bits(L.n);
  int rc = radix_sort_pairs(keys, keys + L.cap, vals, vals + L.cap, vals, keys, n_sel_dev, L.cap, bits,
                            (int)L.sort_blocks, at<uint32_t>(A, L.hist), st);
  if (rc != SSS_OK) return rc;
  const int slot = ((bits + 7) / 8) & 1;
  const uint32_t* skeys = keys + (size_t)slot * L.cap;
  const uint32_t* svals = vals + (size_t)slot * L.cap;
  k_reloc_groups<<<gcap, RT, 0, st>>>(A, skeys);
  k_reloc_copy<<<gcap, RT, 0, st>>>(A, skeys, svals);
  k_reloc_targets<<<gcap, RT, 0, st>>>(A, skeys);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
