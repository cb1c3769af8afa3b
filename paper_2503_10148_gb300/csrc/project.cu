// a1: projection of 3D t-components to 2D t-splats (Sec. 3.2 Eq. t_2D).
//
// One thread per (scene, component): the component's parameters (60 floats
// at SH degree 3) are read once, coalesced from the planar arrays, and every
// job (view) of that scene is projected from registers.  Per (job, component)
// entry the kernel writes the 48-byte render record, the FP32 depth key, the
// tile count and the tile rectangle.  HBM traffic per component: 240 B read
// (degree 3) + 64 B written per view.  The screen-space mean is evaluated to
// about 46 bits with error-free FP32 transformations and stored relative to
// the splat's first tile (see SplatRec).
#include "proj_geom.cuh"

namespace sss {

// Unevaluated sum hi + lo of two floats (double-float arithmetic).  Error-free
// transformations: two_sum (Knuth), two_prod with an FMA (the rounding error
// of a*b is fma(a, b, -a*b) exactly).  On this part FP64 runs at a small
// fraction of the FP32 rate, so the extended-precision mean is done in FP32.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

// r0 m0 + r1 m1 + r2 m2 + t, compensated (Ogita, Rump and Oishi's Dot2: as
// accurate as the sum evaluated in twice the precision, then kept as a pair).
__device__ __forceinline__ DF dot3_plus(const float* r, const float* m, float t) {
  DF p = two_prod(r[0], m[0]);
  float s = p.hi, err = p.lo;
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    const DF q = two_prod(r[k], m[k]);
    const DF u = two_sum(s, q.hi);
    s = u.hi;
    err += u.lo + q.lo;
  }
  const DF u = two_sum(s, t);
  return fast_two_sum(u.hi, err + u.lo);
}

// f x / z + c for double-float x, z: a correctly rounded quotient of the
// high parts, refined once with the exact residual.
__device__ __forceinline__ DF screen_coord(float f, DF x, DF z, float c) {
  const float q1 = __fdiv_rn(x.hi, z.hi);
  const float r = fmaf(-q1, z.hi, x.hi) + (x.lo - q1 * z.lo);
  const DF q = fast_two_sum(q1, __fdiv_rn(r, z.hi));
  const DF a = two_prod(f, q.hi);
  const DF s = two_sum(a.hi, c);
  return fast_two_sum(s.hi, fmaf(f, q.lo, a.lo) + s.lo);
}

template <int DEG>
__device__ __forceinline__ void project_component(const sss_frame_plan& P, int s, uint32_t i, void* ws) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const sss_params& S = P.scenes[s];
  const sss_raster_cfg& cfg = P.cfg;
  const CompParams c = load_comp(S, i);
  const CompShape g = comp_shape(c);
  float sh[3 * K];
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) sh[k] = __ldg(S.sh + (size_t)k * S.n + i);

  SplatRec* rec = ws_ptr<SplatRec>(ws, P.ws_off_rec);
  uint32_t* dkey = ws_ptr<uint32_t>(ws, P.ws_off_dkey);
  uint32_t* ntiles = ws_ptr<uint32_t>(ws, P.ws_off_ntiles);
  uint2* rect = ws_ptr<uint2>(ws, P.ws_off_rect);

  for (int q = P.scene_job_begin[s]; q < P.scene_job_begin[s + 1]; ++q) {
    const sss_job_desc& J = P.jobs[P.scene_jobs[q]];
    const uint32_t e = J.entry_base + i;
    const ViewGeom v = view_geom(c, g, J.cam, cfg);
    if (!v.valid) {
      dkey[e] = 0xffffffffu;
      ntiles[e] = 0u;
      rect[e] = make_uint2(0u, 0u);
      continue;
    }
    // mean2D to ~46 bits: in FP32, fx x/z + cx at ~1000 px carries ~1e-4 px
    // of rounding, a large relative error on (pixel - mean) near the centre
    const float* V = J.cam.viewmat;
    const DF pxd = dot3_plus(V + 0, c.mu, V[3]);
    const DF pyd = dot3_plus(V + 4, c.mu, V[7]);
    const DF pzd = dot3_plus(V + 8, c.mu, V[11]);
    const DF mxd = screen_coord(J.cam.fx, pxd, pzd, J.cam.cx);
    const DF myd = screen_coord(J.cam.fy, pyd, pzd, J.cam.cy);
    // extent: |o| T2D(h) >= tau  <=>  h <= h_max (reading of the SM's truncation)
    // Gaussian kernel (nu -> infinity): |o| exp(-h/2) >= tau <=> h <= 2 ln(|o|/tau)
    const bool gauss = cfg.kernel == 1;
    const float hmax = gauss ? 2.0f * logf(fabsf(v.o) / cfg.tau)
                             : v.nu * expm1f(2.0f / (v.nu + 2.0f) * logf(fabsf(v.o) / cfg.tau));
    const float ex = sqrtf(v.A * hmax), ey = sqrtf(v.C * hmax);
    const float fx0 = fmaxf(ceilf(mxd.hi - ex - 0.5f), 0.0f);
    const float fx1 = fminf(floorf(mxd.hi + ex - 0.5f), (float)(J.cam.width - 1));
    const float fy0 = fmaxf(ceilf(myd.hi - ey - 0.5f), 0.0f);
    const float fy1 = fminf(floorf(myd.hi + ey - 0.5f), (float)(J.cam.height - 1));
    uint32_t nt = 0, ox = 0, oy = 0;
    uint2 rc = make_uint2(0u, 0u);
    if (fx0 <= fx1 && fy0 <= fy1) {
      const uint32_t tx0 = (uint32_t)fx0 / (uint32_t)cfg.tile_w, tx1 = (uint32_t)fx1 / (uint32_t)cfg.tile_w;
      const uint32_t ty0 = (uint32_t)fy0 / (uint32_t)cfg.tile_h, ty1 = (uint32_t)fy1 / (uint32_t)cfg.tile_h;
      nt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
      rc = make_uint2(tx0 | (tx1 << 16), ty0 | (ty1 << 16));
      ox = tx0 * (uint32_t)cfg.tile_w;
      oy = ty0 * (uint32_t)cfg.tile_h;
    }
    // view-dependent colour: max(SH . Y(dir) + 0.5, 0)
    float cc[3];
    cam_centre(J.cam, cc);
    float d0 = c.mu[0] - cc[0], d1 = c.mu[1] - cc[1], d2 = c.mu[2] - cc[2];
    const float il = 1.0f / sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float Y[K];
    sh_basis<DEG>(d0 * il, d1 * il, d2 * il, Y);
    float rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float acc = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) acc = fmaf(sh[3 * k + ch], Y[k], acc);
      rgb[ch] = fmaxf(acc, 0.0f);
    }
    SplatRec r;
    // (hi - origin) is exact for |hi - origin| < 1024 px (both on hi's grid)
    r.a = make_float4((mxd.hi - (float)ox) + mxd.lo, (myd.hi - (float)oy) + myd.lo, v.con[0], v.con[1]);
    r.b = make_float4(v.con[2], v.o, hmax, gauss ? __int_as_float(0x7f800000) : v.nu);  // +inf: Gaussian
    r.c = make_float4(rgb[0], rgb[1], rgb[2], __uint_as_float(ox | (oy << 16)));
    rec[e] = r;
    dkey[e] = __float_as_uint(v.p[2]);
    ntiles[e] = nt;
    rect[e] = rc;
  }
}

__global__ void __launch_bounds__(128, 5) k_project(const sss_frame_plan P, void* ws) {
  const uint32_t gidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= P.scene_comp_base[P.n_scenes]) return;
  const int s = scene_of_comp(P, gidx);
  const uint32_t i = gidx - P.scene_comp_base[s];
  switch (P.scenes[s].sh_degree) {
    case 0: project_component<0>(P, s, i, ws); break;
    case 1: project_component<1>(P, s, i, ws); break;
    case 2: project_component<2>(P, s, i, ws); break;
    default: project_component<3>(P, s, i, ws); break;
  }
}

}  // namespace sss

extern "C" int sss_project(const sss_frame_plan* plan, void* ws, sss_stream_t stream) {
  if (!plan || !ws) return SSS_ERR_INVALID_ARG;
  const uint32_t total = plan->scene_comp_base[plan->n_scenes];
  if (total == 0) return SSS_OK;
  sss::k_project<<<sss::ceil_div(total, 128), 128, 0, (cudaStream_t)stream>>>(*plan, ws);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
