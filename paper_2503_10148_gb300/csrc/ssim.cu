// Image loss of Sec. 3.4: (1 - eps) L1 + eps D-SSIM over every image of a
// frame, value and gradient.  SSIM as in 3DGS (the loss the paper cites):
// 11 x 11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2,
// D-SSIM = 1 - mean SSIM over all pixels and channels.
//
// Value pass: one CTA per (32 x 32 tile, channel) of an image.  The tile
// plus a 5-pixel halo of prediction x and target y is staged in shared
// memory (asynchronous copies, zero-filled outside the image); a horizontal 11-tap pass over the 42 rows gives the windowed sums
// of x, y, x^2, y^2, xy, a vertical pass the five window statistics at each
// pixel (both passes register-blocked: a thread makes 4 adjacent outputs
// from 14 loaded values; x and y staged interleaved so that the (x, y) and
// (x^2, y^2) sums run as packed FP32 pairs), then SSIM and its partials
//   a = dS/dmx - 2 mx dS/dsx2 - my dS/dsxy,  b = dS/dsx2,  c = dS/dsxy
// (written to the scratch maps) and the sums of S and |x - y| (one FP64
// atomic per CTA).  Gradient pass: the same tiling over the maps gives
// dS_total/dx = (w * a) + 2 x (w * b) + y (w * c) (the window is symmetric,
// so the adjoint of the windowed sum is the windowed sum).
#include "common.cuh"

namespace sss {
namespace {

constexpr int TX = 32, TY = 32, R = 5, HX = TX + 2 * R, HY = TY + 2 * R, NT = 256;
constexpr int WB = 4;  // outputs per thread along a pass
constexpr int NTAP = 2 * R + 1;
// Row pitches of the shared arrays, odd in words and in 8-byte pairs: the
// horizontal pass gives consecutive lanes consecutive rows (same columns),
// so with an odd pitch every 4-byte access of a warp falls in distinct
// banks and every 8-byte access takes the minimal two wavefronts.
constexpr int HXP = HX + 1, TXP = TX + 1;

struct SsimArgs {
  const float* pred;
  const float* target;
  float* maps;    // [3 maps][3 n_pixels], the frame's image layout each
  double* acc;    // [0] sum |x - y|, [1] sum S
  float w[2 * R + 1];
  float eps, inv_count;
  uint32_t n_pixels;
  uint32_t tile_base[SSS_MAX_JOBS + 1];  // tiles per job, prefix
  const float* dl_dloss;
  float* grad;
  float* loss_out;
};

__device__ __forceinline__ int job_of_ssim_tile(const sss_frame_plan& P, const SsimArgs& A, uint32_t t) {
  int lo = 0, hi = P.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.tile_base[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Stage rows [y0 - R, y0 + TY + R) x cols [x0 - R, x0 + TX + R) of one
// channel plane into s with asynchronous 4-byte copies (all in flight at
// once; pixels outside the image are zero-filled by the copy): warp w takes
// rows w, w + 8, ..., its lanes the columns.  The caller waits
// (stage_wait) and synchronises the CTA.
__device__ __forceinline__ void stage(float (*s)[HXP], const float* plane, int W, int H, int x0, int y0) {
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < HY; r += NT / 32) {
    const int gy = y0 - R + r;
    const bool row_in = gy >= 0 && gy < H;
    const float* row = plane + (size_t)(row_in ? gy : 0) * W;
#pragma unroll
    for (int q = lane; q < HX; q += 32) {
      const int gx = x0 - R + q;
      const bool in = row_in && gx >= 0 && gx < W;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(&s[r][q]);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(in ? row + gx : plane),
                   "r"(in ? 4 : 0)
                   : "memory");
    }
  }
}
// Two planes interleaved: s[r][q] = (plane a, plane b) at the same pixel, so
// that a pixel's pair loads as one 64-bit word (the operand of the packed
// FP32 instructions).
__device__ __forceinline__ void stage2(float2 (*s)[HXP], const float* pa, const float* pb, int W, int H, int x0,
                                       int y0) {
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < HY; r += NT / 32) {
    const int gy = y0 - R + r;
    const bool row_in = gy >= 0 && gy < H;
    const size_t row = (size_t)(row_in ? gy : 0) * W;
#pragma unroll
    for (int q = lane; q < HX; q += 32) {
      const int gx = x0 - R + q;
      const bool in = row_in && gx >= 0 && gx < W;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(&s[r][q].x);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(in ? pa + row + gx : pa),
                   "r"(in ? 4 : 0)
                   : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa + 4u), "l"(in ? pb + row + gx : pb),
                   "r"(in ? 4 : 0)
                   : "memory");
    }
  }
}
__device__ __forceinline__ F2 ld2(const float2& v) {
  F2 r;
  r.v = *reinterpret_cast<const unsigned long long*>(&v);
  return r;
}
__device__ __forceinline__ void st2(float2& d, F2 v) { *reinterpret_cast<unsigned long long*>(&d) = v.v; }

__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(NT) k_ssim_value(const sss_frame_plan P, const SsimArgs A) {
  __shared__ float2 s_xy[HY][HXP];              // (x, y) per pixel
  __shared__ float2 h01[HY][TXP], h23[HY][TXP];  // horizontal sums (x, y), (x^2, y^2)
  __shared__ float h4[HY][TXP];                  // horizontal sum of x y
  __shared__ double red[2][NT / 32];
  const uint32_t t = blockIdx.x;
  const int ch = blockIdx.y;
  const int j = job_of_ssim_tile(P, A, t);
  const sss_job_desc& J = P.jobs[j];
  const int W = J.cam.width, H = J.cam.height;
  const int tiles_x = (W + TX - 1) / TX;
  const int lt = (int)(t - A.tile_base[j]);
  const int x0 = (lt % tiles_x) * TX, y0 = (lt / tiles_x) * TY;
  const size_t plane_off = 3 * (size_t)J.pix_base + (size_t)ch * W * H;
  // Window statistics of x - cx, y - cy with cx, cy the tile's first pixel:
  // the variances E[(x-c)^2] - E[x-c]^2 then carry no cancellation in flat
  // regions (out-of-image pixels stage as 0 and enter as -c, i.e. zero
  // padding is kept; the window weights sum to 1, so the statistics are
  // shift-invariant).  The shift is applied as the staged values are read.
  stage2(s_xy, A.pred + plane_off, A.target + plane_off, W, H, x0, y0);
  stage_wait();
  __syncthreads();
  const float cx = s_xy[R][R].x, cy = s_xy[R][R].y;  // the tile's first pixel (inside the image)
  const F2 cxy = f2(cx, cy);
  // the x and y sums run as packed pairs: (x, y) and (x^2, y^2) per tap,
  // x y alone; each element is rounded as the scalar fmaf would round it
  F2 w2[NTAP];
#pragma unroll
  for (int k = 0; k < NTAP; ++k) w2[k] = vsplat<F2>(A.w[k]);
  // horizontal: item = (row, group of WB columns), rows fastest; windowed
  // sums of x, y, x^2, y^2, xy for WB adjacent columns from WB + 10 staged
  // values
  for (int it = threadIdx.x; it < HY * (TX / WB); it += NT) {
    const int r = it % HY, q0 = (it / HY) * WB;
    F2 v[WB + 2 * R], v2[WB + 2 * R];
    float vxy[WB + 2 * R];
#pragma unroll
    for (int k = 0; k < WB + 2 * R; ++k) {
      v[k] = vsub(ld2(s_xy[r][q0 + k]), cxy);  // (x - cx, y - cy)
      v2[k] = vmul(v[k], v[k]);
      float a, b;
      f2u(v[k], a, b);
      vxy[k] = a * b;
    }
#pragma unroll
    for (int o = 0; o < WB; ++o) {
      F2 s01 = vsplat<F2>(0.f), s23 = vsplat<F2>(0.f);
      float s4 = 0.f;
#pragma unroll
      for (int k = 0; k < NTAP; ++k) {
        s01 = vfma(w2[k], v[o + k], s01);
        s23 = vfma(w2[k], v2[o + k], s23);
        s4 = fmaf(A.w[k], vxy[o + k], s4);
      }
      st2(h01[r][q0 + o], s01);
      st2(h23[r][q0 + o], s23);
      h4[r][q0 + o] = s4;
    }
  }
  __syncthreads();
  // per-thread partials in FP32 (a thread makes TX TY / NT = 4 outputs), then
  // FP64 over the CTA and the frame (FP64 runs at a small fraction of the
  // FP32 rate on this part)
  float l1f = 0.0f, ssf = 0.0f;
  constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
  // vertical: item = (column, group of WB rows)
  for (int it = threadIdx.x; it < TX * (TY / WB); it += NT) {
    const int q = it % TX, r0 = (it / TX) * WB;
    F2 m01[WB], m23[WB];
    float m4[WB];
#pragma unroll
    for (int o = 0; o < WB; ++o) {
      m01[o] = m23[o] = vsplat<F2>(0.f);
      m4[o] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < WB + 2 * R; ++k) {
      const F2 a01 = ld2(h01[r0 + k][q]), a23 = ld2(h23[r0 + k][q]);
      const float a4 = h4[r0 + k][q];
#pragma unroll
      for (int o = 0; o < WB; ++o) {
        const int tap = k - o;
        if (tap < 0 || tap >= NTAP) continue;
        m01[o] = vfma(w2[tap], a01, m01[o]);
        m23[o] = vfma(w2[tap], a23, m23[o]);
        m4[o] = fmaf(A.w[tap], a4, m4[o]);
      }
    }
#pragma unroll
    for (int ob = 0; ob < WB; ++ob) {
    const int r = r0 + ob;
    const int gx = x0 + q, gy = y0 + r;
    float m[5];
    f2u(m01[ob], m[0], m[1]);
    f2u(m23[ob], m[2], m[3]);
    m[4] = m4[ob];
    if (gx >= W || gy >= H) continue;
    const float sx2 = m[2] - m[0] * m[0], sy2 = m[3] - m[1] * m[1], sxy = m[4] - m[0] * m[1];
    const float mx = m[0] + cx, my = m[1] + cy;
    const float A1 = fmaf(2.0f * mx, my, C1), A2 = fmaf(2.0f, sxy, C2);
    const float B1 = fmaf(mx, mx, fmaf(my, my, C1)), B2 = sx2 + sy2 + C2;
    const float D = 1.0f / (B1 * B2);
    const float S = A1 * A2 * D;
    // product forms: no division by A1 or A2 (either can vanish); 1/B1 and
    // 1/B2 as B2 D and B1 D (one reciprocal per pixel)
    const float dS_dmx = 2.0f * my * A2 * D - 2.0f * mx * S * (B2 * D);
    const float dS_dsx2 = -S * (B1 * D);
    const float dS_dsxy = 2.0f * A1 * D;
    const size_t o = plane_off + (size_t)gy * W + gx;
    A.maps[o] = dS_dmx - 2.0f * mx * dS_dsx2 - my * dS_dsxy;
    A.maps[3 * (size_t)A.n_pixels + o] = dS_dsx2;
    A.maps[6 * (size_t)A.n_pixels + o] = dS_dsxy;
    ssf += S;
    l1f += fabsf(s_xy[r + R][q + R].x - s_xy[r + R][q + R].y);
    }
  }
  // CTA sums -> one FP64 atomic each
  double l1 = (double)l1f, ssum = (double)ssf;
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = l1;
    red[1][threadIdx.x >> 5] = ssum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    atomicAdd(A.acc, a);
    atomicAdd(A.acc + 1, b);
  }
}

__global__ void k_ssim_finish(const SsimArgs A) {
  const double l1 = A.acc[0] * (double)A.inv_count;
  const double dssim = 1.0 - A.acc[1] * (double)A.inv_count;
  A.loss_out[1] = (float)l1;
  A.loss_out[2] = (float)dssim;
  A.loss_out[0] = (float)((1.0 - (double)A.eps) * l1 + (double)A.eps * dssim);
}

__global__ void __launch_bounds__(NT) k_ssim_grad(const sss_frame_plan P, const SsimArgs A) {
  __shared__ float2 s_ab[HY][HXP];  // maps a and b per pixel
  __shared__ float s_c[HY][HXP];
  __shared__ float2 h_ab[HY][TXP];
  __shared__ float h_c[HY][TXP];
  const uint32_t t = blockIdx.x;
  const int ch = blockIdx.y;
  const int j = job_of_ssim_tile(P, A, t);
  const sss_job_desc& J = P.jobs[j];
  const int W = J.cam.width, H = J.cam.height;
  const int tiles_x = (W + TX - 1) / TX;
  const int lt = (int)(t - A.tile_base[j]);
  const int x0 = (lt % tiles_x) * TX, y0 = (lt / tiles_x) * TY;
  const size_t plane_off = 3 * (size_t)J.pix_base + (size_t)ch * W * H;
  stage2(s_ab, A.maps + plane_off, A.maps + 3 * (size_t)A.n_pixels + plane_off, W, H, x0, y0);
  stage(s_c, A.maps + 6 * (size_t)A.n_pixels + plane_off, W, H, x0, y0);
  stage_wait();
  __syncthreads();
  // windowed sums of a and b as packed pairs, c alone
  F2 w2[NTAP];
#pragma unroll
  for (int k = 0; k < NTAP; ++k) w2[k] = vsplat<F2>(A.w[k]);
  for (int it = threadIdx.x; it < HY * (TX / WB); it += NT) {
    const int r = it % HY, q0 = (it / HY) * WB;  // rows fastest, as in the value pass
    F2 vab[WB + 2 * R];
    float vc[WB + 2 * R];
#pragma unroll
    for (int k = 0; k < WB + 2 * R; ++k) {
      vab[k] = ld2(s_ab[r][q0 + k]);
      vc[k] = s_c[r][q0 + k];
    }
#pragma unroll
    for (int o = 0; o < WB; ++o) {
      F2 acc = vsplat<F2>(0.f);
      float accc = 0.f;
#pragma unroll
      for (int k = 0; k < NTAP; ++k) {
        acc = vfma(w2[k], vab[o + k], acc);
        accc = fmaf(A.w[k], vc[o + k], accc);
      }
      st2(h_ab[r][q0 + o], acc);
      h_c[r][q0 + o] = accc;
    }
  }
  __syncthreads();
  const float scale = A.dl_dloss ? *A.dl_dloss * A.inv_count : A.inv_count;
  const float w1 = (1.0f - A.eps) * scale, ws = A.eps * scale;
  for (int it = threadIdx.x; it < TX * (TY / WB); it += NT) {
    const int q = it % TX, r0 = (it / TX) * WB;
    // this item's prediction and target values, requested before the
    // windowed sums so that their latency overlaps them
    float xs[WB], ys[WB];
#pragma unroll
    for (int ob = 0; ob < WB; ++ob) {
      const int gx = x0 + q, gy = y0 + r0 + ob;
      const bool in = gx < W && gy < H;
      const size_t o = plane_off + (size_t)(in ? gy : y0) * W + (in ? gx : x0);
      xs[ob] = A.pred[o];
      ys[ob] = A.target[o];
    }
    F2 cab[WB];
    float cc[WB];
#pragma unroll
    for (int o = 0; o < WB; ++o) {
      cab[o] = vsplat<F2>(0.f);
      cc[o] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < WB + 2 * R; ++k) {
      const F2 hab = ld2(h_ab[r0 + k][q]);
      const float hc = h_c[r0 + k][q];
#pragma unroll
      for (int o = 0; o < WB; ++o) {
        const int tap = k - o;
        if (tap < 0 || tap >= NTAP) continue;
        cab[o] = vfma(w2[tap], hab, cab[o]);
        cc[o] = fmaf(A.w[tap], hc, cc[o]);
      }
    }
    float cv[WB][3];
#pragma unroll
    for (int o = 0; o < WB; ++o) {
      f2u(cab[o], cv[o][0], cv[o][1]);
      cv[o][2] = cc[o];
    }
#pragma unroll
    for (int ob = 0; ob < WB; ++ob) {
      const int gx = x0 + q, gy = y0 + r0 + ob;
      if (gx >= W || gy >= H) continue;
      const size_t o = plane_off + (size_t)gy * W + gx;
      const float x = xs[ob], y = ys[ob];
      const float dS = fmaf(2.0f * x, cv[ob][1], fmaf(y, cv[ob][2], cv[ob][0]));
      const float d = x - y;
      const float sg = d > 0.0f ? w1 : (d < 0.0f ? -w1 : 0.0f);
      A.grad[o] = fmaf(-ws, dS, sg);
    }
  }
}

// Byte offset of the two FP64 sums in the scratch (after the nine maps).
size_t acc_offset(uint32_t n_pixels) { return (9 * (size_t)n_pixels * sizeof(float) + 15) & ~(size_t)15; }

// Arguments shared by both passes; false when the plan has no pixels.
bool make_args(const sss_frame_plan& P, float eps, void* scratch, SsimArgs& A) {
  A.maps = static_cast<float*>(scratch);
  A.acc = reinterpret_cast<double*>(static_cast<char*>(scratch) + acc_offset(P.n_pixels));
  // the window: normalised Gaussian, sigma 1.5, evaluated in FP64
  double g[2 * R + 1], tot = 0.0;
  for (int k = 0; k <= 2 * R; ++k) {
    const double d = (double)(k - R);
    g[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
    tot += g[k];
  }
  for (int k = 0; k <= 2 * R; ++k) A.w[k] = (float)(g[k] / tot);
  A.eps = eps;
  A.n_pixels = P.n_pixels;
  A.inv_count = P.n_pixels ? (float)(1.0 / (3.0 * (double)P.n_pixels)) : 0.0f;
  uint32_t t = 0;
  for (int j = 0; j < P.n_jobs; ++j) {
    A.tile_base[j] = t;
    const int W = P.jobs[j].cam.width, H = P.jobs[j].cam.height;
    t += (uint32_t)(((W + TX - 1) / TX) * ((H + TY - 1) / TY));
  }
  A.tile_base[P.n_jobs] = t;
  return t > 0;
}

}  // namespace
}  // namespace sss

using namespace sss;

extern "C" size_t sss_loss_image_scratch_bytes(const sss_frame_plan* plan) {
  if (!plan) return 0;
  return acc_offset(plan->n_pixels) + 2 * sizeof(double);
}

extern "C" int sss_loss_image(const sss_frame_plan* plan, const float* pred, const float* target, float eps_dssim,
                              float* loss_out, void* scratch, sss_stream_t stream) {
  if (!plan || !pred || !target || !loss_out || !scratch) return SSS_ERR_INVALID_ARG;
  if (!(eps_dssim >= 0.0f && eps_dssim <= 1.0f)) return SSS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) % 16 != 0) return SSS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SsimArgs A{};
  A.pred = pred;
  A.target = target;
  A.loss_out = loss_out;
  const bool any = make_args(*plan, eps_dssim, scratch, A);
  if (cudaMemsetAsync(A.acc, 0, 2 * sizeof(double), st) != cudaSuccess) return SSS_ERR_CUDA;
  if (any) {
    k_ssim_value<<<dim3(A.tile_base[plan->n_jobs], 3), NT, 0, st>>>(*plan, A);
    SSS_LAUNCH_CHECK();
  }
  k_ssim_finish<<<1, 1, 0, st>>>(A);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

extern "C" int sss_loss_image_grad(const sss_frame_plan* plan, const float* pred, const float* target,
                                   float eps_dssim, const float* dL_dloss, const void* scratch, float* dL_dpred,
                                   sss_stream_t stream) {
  if (!plan || !pred || !target || !scratch || !dL_dpred) return SSS_ERR_INVALID_ARG;
  if (!(eps_dssim >= 0.0f && eps_dssim <= 1.0f)) return SSS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) % 16 != 0) return SSS_ERR_INVALID_ARG;
  SsimArgs A{};
  A.pred = pred;
  A.target = target;
  A.dl_dloss = dL_dloss;
  A.grad = dL_dpred;
  if (!make_args(*plan, eps_dssim, const_cast<void*>(scratch), A)) return SSS_OK;
  k_ssim_grad<<<dim3(A.tile_base[plan->n_jobs], 3), NT, 0, (cudaStream_t)stream>>>(*plan, A);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
