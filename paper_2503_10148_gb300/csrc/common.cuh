// Internal helpers shared by the libsss kernels (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "sss.h"

namespace sss {

constexpr int kNumSMs = 152;          // GB300: 2 dies x 76 SMs; the SM count
                                      // when no device can be queried
constexpr float kFastNuMax = 64.0f;   // above this nu the log/exp pair runs on
                                      // the accurate path (eval_pair_slow)

// SM count of the current device (cudaDevAttrMultiProcessorCount), or kNumSMs
// when no device is visible (host-only planning).  Sizes the persistent grids
// of the sorts and scans and the grid-stride launches.  A host-side attribute
// query: it enqueues nothing and is allowed while a stream is being captured.
inline int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    (void)cudaGetLastError();
    return kNumSMs;
  }
  return sms;
}

// ------------------------------------------------------------ workspace
template <typename T>
__host__ __device__ inline T* ws_ptr(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}
template <typename T>
__host__ __device__ inline const T* ws_ptr(const void* ws, size_t off) {
  return reinterpret_cast<const T*>(static_cast<const char*>(ws) + off);
}

enum CtrlWord : int { kCtrlPairsNeeded = 0, kCtrlPairsSorted = 1, kCtrlStatus = 2, kCtrlEntries = 3, kCtrlQueue = 8 };

// End of a persistent render launch for the calling warp: counts the warp as
// finished (queue[1]); the last of the grid's warps resets the item counter
// and the finished count, so the next launch starts from item 0.  Every warp
// has taken its last item before it counts itself (the fence orders its last
// take before its count), so nothing touches the counter after the reset.
__device__ __forceinline__ void queue_retire(uint32_t* queue, unsigned lane) {
  if (lane == 0) {
    __threadfence();
    const uint32_t total = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(queue + 1, 1u) == total - 1) {
      queue[0] = 0u;
      queue[1] = 0u;
    }
  }
}

// CTAs of a persistent launch: as many as are resident at once on the
// device (occupancy of `kernel` at `threads` threads per CTA), at most
// `max_ctas`.
template <class K>
inline unsigned persistent_grid(K kernel, int threads, uint32_t max_ctas) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  const uint32_t g = (uint32_t)per_sm * (uint32_t)device_sm_count();
  return g < max_ctas ? g : (max_ctas ? max_ctas : 1u);
}

// ------------------------------------------------------------ job lookup
// Largest j in [0, n) with base(j) <= x; bases are non-decreasing.
__device__ inline int job_of_entry(const sss_frame_plan& P, uint32_t e) {
  int lo = 0, hi = P.n_jobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (P.jobs[mid].entry_base <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ inline int job_of_tile(const sss_frame_plan& P, uint32_t t) {
  int lo = 0, hi = P.n_jobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (P.jobs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ inline int scene_of_comp(const sss_frame_plan& P, uint32_t g) {
  int s = 0;
  while (s + 1 < P.n_scenes && P.scene_comp_base[s + 1] <= g) ++s;
  return s;
}

// ------------------------------------------------------------ launches
#define SSS_LAUNCH_CHECK()                                  \
  do {                                                      \
    if (cudaPeekAtLastError() != cudaSuccess) {             \
      (void)cudaGetLastError();                             \
      return SSS_ERR_CUDA;                                  \
    }                                                       \
  } while (0)

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ splat record
// Render record of one entry, three float4 (48 bytes):
//   a = {mean2D x - ox, mean2D y - oy, conic a, conic b}
//   b = {conic c, o, h_max, nu}
//   c = {r, g, b, origin}   origin = bits of (ox | oy << 16)
// (ox, oy) is the integer pixel nearest to the mean (limited to [0, 16384]):
// (x - ox) is an exact small integer for every pixel x, and the stored
// mean - origin keeps FP32's fine spacing near 0 (within u/2 px of the mean)
// instead of its ~1e-4 px spacing at 1000 px.
// h = a dx^2 + 2 b dx dy + c dy^2 with (dx, dy) = pixel centre - mean2D.
struct SplatRec {
  float4 a, b, c;
};

// MUFU base-2 logarithm and exponential (PTX lg2.approx / ex2.approx; the
// PTX ISA documents their accuracy: about 2^-22 absolute for lg2 and 2^-22
// relative for ex2).  The argument of lg2 here is >= 1, and an ex2 result that
// would be subnormal flushes to 0, which the alpha threshold rejects anyway.
__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------------ packed FP32
// Blackwell issues two FP32 additions, subtractions, multiplications or FMAs
// as one instruction (add/sub/mul/fma.rn.f32x2), each element rounded
// exactly as the scalar operation.  The per-pixel code of the render kernels
// is written once over a value type V -- float (one pixel) or F2 (two pixels
// of a lane) -- with masks MaskT<V> = bool or B2.  The scalar operations use
// the _rn intrinsics, which the compiler does not contract into FMAs, so a
// pixel gets bit-identical values whether it is evaluated alone or in a
// pair, in the forward and in the backward.
// F2 holds its two floats in one 64-bit register (lo = element 0), the
// operand form of the packed instructions; elements are unpacked only for
// element-wise work.
struct F2 {
  unsigned long long v;
};
struct B2 {
  bool x, y;
};
__device__ __forceinline__ F2 f2(float x, float y) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void f2u(F2 a, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
}

#define SSS_PACKED_OP(name, ins)                                                   \
  __device__ __forceinline__ F2 name(F2 a, F2 b) {                                \
    F2 d;                                                                          \
    asm(ins " %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));                      \
    return d;                                                                      \
  }
SSS_PACKED_OP(vadd, "add.rn.f32x2")
SSS_PACKED_OP(vsub, "sub.rn.f32x2")
SSS_PACKED_OP(vmul, "mul.rn.f32x2")
#undef SSS_PACKED_OP

__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <class V>
struct MaskOf;
template <>
struct MaskOf<float> {
  using T = bool;
};
template <>
struct MaskOf<F2> {
  using T = B2;
};
template <class V>
using MaskT = typename MaskOf<V>::T;

template <class V>
__device__ __forceinline__ V vsplat(float v);
template <>
__device__ __forceinline__ float vsplat<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ F2 vsplat<F2>(float v) {
  return f2(v, v);
}

// element-wise helpers (MUFU, min, comparisons, selection, mask logic)
__device__ __forceinline__ float vlg2(float a) { return mufu_lg2(a); }
__device__ __forceinline__ F2 vlg2(F2 a) {
  float x, y;
  f2u(a, x, y);
  return f2(mufu_lg2(x), mufu_lg2(y));
}
__device__ __forceinline__ float vex2(float a) { return mufu_ex2(a); }
__device__ __forceinline__ F2 vex2(F2 a) {
  float x, y;
  f2u(a, x, y);
  return f2(mufu_ex2(x), mufu_ex2(y));
}
// MUFU reciprocal (PTX rcp.approx.ftz: about 1 ulp); one instruction, no
// range handling of a general approximate division
__device__ __forceinline__ float mufu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float vrcp(float a) { return mufu_rcp(a); }
__device__ __forceinline__ F2 vrcp(F2 a) {
  float x, y;
  f2u(a, x, y);
  return f2(mufu_rcp(x), mufu_rcp(y));
}
__device__ __forceinline__ float vlog1p(float a) { return log1pf(a); }
__device__ __forceinline__ F2 vlog1p(F2 a) {
  float x, y;
  f2u(a, x, y);
  return f2(log1pf(x), log1pf(y));
}
__device__ __forceinline__ float vexp(float a) { return expf(a); }
__device__ __forceinline__ F2 vexp(F2 a) {
  float x, y;
  f2u(a, x, y);
  return f2(expf(x), expf(y));
}
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ F2 vmin(F2 a, float b) {
  float x, y;
  f2u(a, x, y);
  return f2(fminf(x, b), fminf(y, b));
}
__device__ __forceinline__ bool vge(float a, float b) { return a >= b; }
__device__ __forceinline__ B2 vge(F2 a, float b) {
  float x, y;
  f2u(a, x, y);
  return B2{x >= b, y >= b};
}
__device__ __forceinline__ B2 vge(F2 a, F2 b) {
  float ax, ay, bx, by;
  f2u(a, ax, ay);
  f2u(b, bx, by);
  return B2{ax >= bx, ay >= by};
}
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ F2 vabs(F2 a) {
  float x, y;
  f2u(a, x, y);
  return f2(fabsf(x), fabsf(y));
}
__device__ __forceinline__ bool vgt(float a, float b) { return a > b; }
__device__ __forceinline__ B2 vgt(F2 a, float b) {
  float x, y;
  f2u(a, x, y);
  return B2{x > b, y > b};
}
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ B2 vlt(F2 a, float b) {
  float x, y;
  f2u(a, x, y);
  return B2{x < b, y < b};
}
__device__ __forceinline__ float vsel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ F2 vsel(B2 m, F2 a, F2 b) {
  float ax, ay, bx, by;
  f2u(a, ax, ay);
  f2u(b, bx, by);
  return f2(m.x ? ax : bx, m.y ? ay : by);
}
__device__ __forceinline__ bool mand(bool a, bool b) { return a && b; }
__device__ __forceinline__ B2 mand(B2 a, B2 b) { return B2{a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ bool mandn(bool a, bool b) { return a && !b; }  // a and not b
__device__ __forceinline__ B2 mandn(B2 a, B2 b) { return B2{a.x && !b.x, a.y && !b.y}; }
__device__ __forceinline__ bool mor(bool a, bool b) { return a || b; }
__device__ __forceinline__ B2 mor(B2 a, B2 b) { return B2{a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ bool many(bool a) { return a; }
__device__ __forceinline__ bool many(B2 a) { return a.x || a.y; }
__device__ __forceinline__ bool mall(bool a) { return a; }
__device__ __forceinline__ bool mall(B2 a) { return a.x && a.y; }
__device__ __forceinline__ float vsum(float a) { return a; }
__device__ __forceinline__ float vsum(F2 a) {
  float x, y;
  f2u(a, x, y);
  return x + y;
}
// element k (0 or 1) of a value or mask
__device__ __forceinline__ float vget(float a, int) { return a; }
__device__ __forceinline__ float vget(F2 a, int k) {
  float x, y;
  f2u(a, x, y);
  return k ? y : x;
}
__device__ __forceinline__ bool mget(bool a, int) { return a; }
__device__ __forceinline__ bool mget(B2 a, int k) { return k ? a.y : a.x; }

// One (splat, pixel) evaluation shared by the forward and backward kernels so
// that both take identical FP32 decisions.  Returns whether the pair
// contributes (|alpha| = |o| T2D >= tau; the tile lists hold only pairs the
// screen extent h <= h_max may reach, and beyond h_max |alpha| < tau, so no
// separate h test is needed); the fields of r are computed either way
// (finite for any finite offsets, alpha already clamped to
// [-alpha_max, alpha_max]), so callers can evaluate all their pixels in
// straight-line code and mask.  The opacity comes split per splat as |o| and
// sign(o): |o| T2D is |o T2D| exactly, and the clamp is one min.  Fast path:
// two MUFU ops (lg2, ex2).  For nu > kFastNuMax the exponent -(nu+2)/2 is
// large enough that the absolute error of lg2.approx would show, so
// eval_pair_slow uses log1pf/expf; callers pick the path per splat (uniform
// over a warp).
template <class V>
struct PairEval {
  V h, t2d, alpha, log_base;  // log_base = ln(1 + h/nu)
  MaskT<V> clamped;
};

// h = dx (a dx + 2 b dy) + c dy^2
template <class V>
__device__ __forceinline__ V conic_h(V dx, V dy, float ca, float cb2, float cc) {
  const V t = vfma(vsplat<V>(ca), dx, vmul(vsplat<V>(cb2), dy));
  return vfma(dx, t, vmul(vmul(vsplat<V>(cc), dy), dy));
}

// CLAMP = false when |o| T2D cannot reach alpha_max (the caller checks |o|
// against alpha_max with a margin for T2D's rounding above 1 near h = 0):
// then the clamp is the identity and is taken out per splat.
template <class V, bool CLAMP = true>
__device__ __forceinline__ MaskT<V> finish_pair(V h, V t2d, V lb, float oabs, float osgn, float tau, float amax,
                                                PairEval<V>& r) {
  const V aabs = vmul(vsplat<V>(oabs), t2d);
  r.h = h;
  r.t2d = t2d;
  if constexpr (CLAMP) {
    r.alpha = vmul(vsplat<V>(osgn), vmin(aabs, amax));
    r.clamped = vgt(aabs, amax);
  } else {
    r.alpha = vmul(vsplat<V>(osgn), aabs);
    if constexpr (std::is_same<V, F2>::value) r.clamped = B2{false, false};
    else r.clamped = false;
  }
  r.log_base = lb;
  return vge(aabs, tau);
}

template <class V, bool CLAMP = true>
__device__ __forceinline__ MaskT<V> eval_pair_fast(V dx, V dy, float ca, float cb2, float cc, float oabs, float osgn,
                                                   float nu, float inv_nu, float tau, float amax, PairEval<V>& r) {
  const V h = conic_h(dx, dy, ca, cb2, cc);
  const float e = fmaf(nu, -0.5f, -1.0f);  // -(nu + 2) / 2
  const V l2 = vlg2(vfma(h, vsplat<V>(inv_nu), vsplat<V>(1.0f)));
  return finish_pair<V, CLAMP>(h, vex2(vmul(vsplat<V>(e), l2)), vmul(l2, vsplat<V>(0.69314718055994531f)), oabs,
                               osgn, tau, amax, r);
}

template <class V>
__device__ __forceinline__ MaskT<V> eval_pair_slow(V dx, V dy, float ca, float cb2, float cc, float oabs, float osgn,
                                                   float nu, float inv_nu, float tau, float amax, PairEval<V>& r) {
  const V h = conic_h(dx, dy, ca, cb2, cc);
  const float e = fmaf(nu, -0.5f, -1.0f);
  const V lb = vlog1p(vmul(h, vsplat<V>(inv_nu)));
  return finish_pair(h, vexp(vmul(vsplat<V>(e), lb)), lb, oabs, osgn, tau, amax, r);
}

// Gaussian kernel (the nu -> infinity limit; records carry nu = +inf):
// T2D = exp(-h/2) = 2^(-h log2(e) / 2), one MUFU op.
template <class V>
__device__ __forceinline__ MaskT<V> eval_pair_gauss(V dx, V dy, float ca, float cb2, float cc, float oabs,
                                                    float osgn, float tau, float amax, PairEval<V>& r) {
  const V h = conic_h(dx, dy, ca, cb2, cc);
  return finish_pair(h, vex2(vmul(h, vsplat<V>(-0.72134752044448170f))), vsplat<V>(0.0f), oabs, osgn, tau, amax,
                     r);
}

// Pixels per value of a lane: pairs when the lane's pixel count is even.
template <int NPIX>
struct LaneVec {
  static constexpr int L = (NPIX % 2 == 0) ? 2 : 1;
  static constexpr int NV = NPIX / L;
};

// Offset of a pixel centre from the splat mean along one axis: fb is the
// lane's first pixel minus the record origin (an exact small integer as a
// float), d the pixel's index inside the lane's block.  fb + (d + 0.5) is
// exact, so the result is rounded once, as (x + 0.5) - mean is.
__device__ __forceinline__ float pixel_offset(float fb, int d, float mean_rel) {
  return (fb + ((float)d + 0.5f)) - mean_rel;
}

// Conservative test: can the ellipse h <= hmax_test reach the axis-aligned box
// [x0, x1] x [y0, y1] of pixel centres?  The minimum of the convex quadratic
// over the box is 0 if the centre is inside, else it lies on an edge facing
// the centre, where it is a clamped 1D minimum.
__device__ __forceinline__ bool ellipse_hits_box(float mx, float my, float ca, float cb, float cc,
                                                 float hmax_test, float x0, float x1, float y0, float y1) {
  bool inx = (mx >= x0) && (mx <= x1);
  bool iny = (my >= y0) && (my <= y1);
  if (inx && iny) return true;
  float hmin = 3.0e38f;
  if (!inx) {
    float dx = (mx < x0 ? x0 : x1) - mx;
    float dy = fminf(fmaxf(-cb * dx / cc, y0 - my), y1 - my);
    float h = ca * dx * dx + 2.0f * cb * dx * dy + cc * dy * dy;
    hmin = fminf(hmin, h);
  }
  if (!iny) {
    float dy = (my < y0 ? y0 : y1) - my;
    float dx = fminf(fmaxf(-cb * dy / ca, x0 - mx), x1 - mx);
    float h = ca * dx * dx + 2.0f * cb * dx * dy + cc * dy * dy;
    hmin = fminf(hmin, h);
  }
  return hmin <= hmax_test;
}

// Relative margin over h_max of the per-warp cull, which skips a splat when
// its ellipse h <= h_max (1 + 2 kHPad) + 1e-3 misses the warp's block of
// pixel centres.  Pixels beyond it have |alpha| below tau by far more than
// the FP32 error of alpha (near |o| = tau, where h_max -> 0, the absolute
// 1e-3 covers it), so the cull never drops a pair the |alpha| >= tau test
// would keep.
constexpr float kHPad = 1e-3f;

__device__ __forceinline__ void rec_origin(float w, int& ox, int& oy) {
  const uint32_t o = __float_as_uint(w);
  ox = (int)(o & 0xffffu);
  oy = (int)(o >> 16);
}

// ------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplications by the published multipliers on counter words 0 and 2,
// xor of the high halves with words 1, 3 and the round key, a word
// permutation, and a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// ------------------------------------------------------------ radix sort
// Stable LSD sort of `count` (key, value) pairs of 32-bit words over key bits
// [0, bits), in the library's workspace conventions (sort.cu): the result
// lands in slot (ceil(bits / 8) & 1) of the two key / value copies; `hist`
// holds 256 * nb + 256 words; count_dev (device) overrides count_max when
// not NULL.  Host function: enqueues kernels on `st`.
int radix_sort_pairs(uint32_t* keys0, uint32_t* keys1, uint32_t* vals0, uint32_t* vals1, const uint32_t* first_vals,
                     const uint32_t* first_keys, const uint32_t* count_dev, uint32_t count_max, int bits, int nb,
                     uint32_t* hist, cudaStream_t st);

// ------------------------------------------------------------ warp staging
// 16-byte asynchronous global -> shared copy (no registers held in flight).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Per-warp staging of splat records, 32 R per batch (slot r*32 + lane is
// staged by lane `lane`), double buffered: a warp gathers batch i+1 with
// cp.async while it evaluates batch i, and no other warp touches its buffers
// (no CTA barrier).  R (1 or 2) is the staging depth the autotuner picks.
template <int R>
struct WarpBuf {
  float4 a[2][32 * R], b[2][32 * R], c[2][32 * R];
  uint32_t e[2][32 * R];
};

// Lane `lane` fills slots r*32 + lane (r < R) of buffer k with records e[r],
// or with an empty slot (h_max < 0, never hit) where !valid[r]; one commit
// group per call.
template <int R>
__device__ __forceinline__ void warp_stage(WarpBuf<R>& S, int k, const SplatRec* __restrict__ rec,
                                           const uint32_t (&e)[R], const bool (&valid)[R], int lane) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int slot = r * 32 + lane;
    if (valid[r]) {
      const float4* src = reinterpret_cast<const float4*>(rec + e[r]);
      cp_async16(&S.a[k][slot], src);
      cp_async16(&S.b[k][slot], src + 1);
      cp_async16(&S.c[k][slot], src + 2);
    } else {
      S.a[k][slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      S.b[k][slot] = make_float4(1.0f, 0.0f, -1.0f, 1.0f);
      S.c[k][slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    S.e[k][slot] = valid[r] ? e[r] : 0u;
  }
  cp_async_commit();
}

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

}  // namespace sss
