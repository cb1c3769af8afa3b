// a1: projection of 3D t-components to 2D t-splats (Sec. 3.2 Eq. t_2D).
//
// One thread per (scene, component): the component's parameters (60 floats
// at SH degree 3) are read once, coalesced from the planar arrays, and every
// job (view) of that scene is projected from registers.  Per (job, component)
// entry the kernel writes the 48-byte render record, the FP32 depth key, the
// tile count and the tile rectangle.  HBM traffic per component: 240 B read
// (degree 3) + 64 B written per view.  The screen-space mean is evaluated to
// about 46 bits with error-free FP32 transformations and stored relative to
// the integer pixel nearest to it (see SplatRec).  The conic is evaluated in
// double-float arithmetic and rounded once to FP32 (conic_df below): in plain
// FP32, a splat elongated along the viewing ray loses most of its 2D
// covariance to cancellation, and its conic to the error of that cancellation.
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

// x / z for double-float x, z: a correctly rounded quotient of the high
// parts, refined once with the exact residual.
__device__ __forceinline__ DF df_div(DF x, DF z) {
  const float q1 = __fdiv_rn(x.hi, z.hi);
  const float r = fmaf(-q1, z.hi, x.hi) + (x.lo - q1 * z.lo);
  return fast_two_sum(q1, __fdiv_rn(r, z.hi));
}

// f x / z + c for double-float x, z.
__device__ __forceinline__ DF screen_coord(float f, DF x, DF z, float c) {
  const DF q = df_div(x, z);
  const DF a = two_prod(f, q.hi);
  const DF s = two_sum(a.hi, c);
  return fast_two_sum(s.hi, fmaf(f, q.lo, a.lo) + s.lo);
}

// ---- double-float products and sums (relative error a few u^2, u = 2^-24;
// a sum's error is relative to the magnitudes of its operands)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = a.hi * b;
  return fast_two_sum(p, fmaf(a.lo, b, fmaf(a.hi, b, -p)));
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ DF df_twice(DF a) { return DF{2.0f * a.hi, 2.0f * a.lo}; }
__device__ __forceinline__ DF df_rcp(DF a) {
  const float r = __frcp_rn(a.hi);
  const float e = fmaf(-r, a.hi, 1.0f) - r * a.lo;  // 1 - r a, the first part exact
  return fast_two_sum(r, r * e);
}
__device__ __forceinline__ bool df_less(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ DF df_dot3(const DF* a, const DF* b) {
  return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}

// M = R diag(s), Sigma = M M^T (Sec. 3.1), in double-float.  With the raw
// quaternion (w, x, y, z) and n2 = |q|^2, the rotation of the normalised
// quaternion is Rn / n2, Rn quadratic in (w, x, y, z): its entries are sums of
// exact products (two_prod), and 1 / n2 is folded into the scales.  The
// scales s = exp(log_scale) are the FP32 values of comp_shape (a relative
// error of s is a relative error of each axis' share of Sigma).
struct ShapeDF {
  DF M[9];  // row-major
};

__device__ __forceinline__ ShapeDF shape_df(const CompParams& c, const CompShape& g) {
  const float w = c.q[0], x = c.q[1], y = c.q[2], z = c.q[3];
  const DF ww = two_prod(w, w), xx = two_prod(x, x), yy = two_prod(y, y), zz = two_prod(z, z);
  const DF xy = two_prod(x, y), wz = two_prod(w, z), xz = two_prod(x, z), wy = two_prod(w, y);
  const DF yz = two_prod(y, z), wx = two_prod(w, x);
  DF Rn[9];
  Rn[0] = df_sub(df_add(ww, xx), df_add(yy, zz));
  Rn[1] = df_twice(df_sub(xy, wz));
  Rn[2] = df_twice(df_add(xz, wy));
  Rn[3] = df_twice(df_add(xy, wz));
  Rn[4] = df_sub(df_add(ww, yy), df_add(xx, zz));
  Rn[5] = df_twice(df_sub(yz, wx));
  Rn[6] = df_twice(df_sub(xz, wy));
  Rn[7] = df_twice(df_add(yz, wx));
  Rn[8] = df_sub(df_add(ww, zz), df_add(xx, yy));
  const DF inv_n2 = df_rcp(df_add(df_add(ww, xx), df_add(yy, zz)));
  ShapeDF m;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const DF sk = df_mul_f(inv_n2, g.s[k]);
#pragma unroll
    for (int r = 0; r < 3; ++r) m.M[r * 3 + k] = df_mul(Rn[r * 3 + k], sk);
  }
  return m;
}

// Reciprocal of a double-float with a normal, non-zero high part: MUFU
// reciprocal (about 1 ulp) and one Newton step on the exact residual.
__device__ __forceinline__ DF df_rcp_normal(DF a) {
  const float r = mufu_rcp(a.hi);
  const float e = fmaf(-r, a.hi, 1.0f) - r * a.lo;
  return fast_two_sum(r, r * e);
}

// ---- packed double-float: two independent double-floats, one per element
// of the f32x2 registers, through the packed FP32 instructions (each element
// rounded as the scalar operation, so every error-free transformation above
// holds element-wise)
struct DF2 {
  F2 hi, lo;
};
__device__ __forceinline__ F2 vneg(F2 a) {
  F2 r;
  asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(r.v) : "l"(a.v));
  return r;
}
__device__ __forceinline__ DF2 df2(DF x, DF y) { return DF2{f2(x.hi, y.hi), f2(x.lo, y.lo)}; }
__device__ __forceinline__ DF2 df2_splat(DF x) { return df2(x, x); }
__device__ __forceinline__ void df2_split(DF2 a, DF& x, DF& y) {
  f2u(a.hi, x.hi, y.hi);
  f2u(a.lo, x.lo, y.lo);
}
__device__ __forceinline__ DF2 fast_two_sum2(F2 a, F2 b) {
  const F2 s = vadd(a, b);
  return DF2{s, vsub(b, vsub(s, a))};
}
__device__ __forceinline__ DF2 df2_mul(DF2 a, DF2 b) {
  const F2 p = vmul(a.hi, b.hi);
  return fast_two_sum2(p, vfma(a.hi, b.lo, vfma(a.lo, b.hi, vfma(a.hi, b.hi, vneg(p)))));
}
__device__ __forceinline__ DF2 df2_mul_f(DF2 a, F2 b) {
  const F2 p = vmul(a.hi, b);
  return fast_two_sum2(p, vfma(a.lo, b, vfma(a.hi, b, vneg(p))));
}
__device__ __forceinline__ DF2 df2_add(DF2 a, DF2 b) {
  const F2 s = vadd(a.hi, b.hi), bb = vsub(s, a.hi);
  const F2 e = vadd(vsub(a.hi, vsub(s, bb)), vsub(b.hi, bb));  // two_sum's error
  return fast_two_sum2(s, vadd(e, vadd(a.lo, b.lo)));
}
__device__ __forceinline__ DF2 df2_sub(DF2 a, DF2 b) { return df2_add(a, DF2{vneg(b.hi), vneg(b.lo)}); }

// The Jacobian's limit 1.3 w / (2 f), with 1.3 as a double-float pair (hi =
// the FP32 nearest, lo = the FP32 nearest to the remainder).
__device__ __forceinline__ DF lim_df(int extent, float f) {
  return df_mul(DF{1.3f, 4.7683717e-08f}, df_mul_f(df_rcp_normal(DF{2.0f * f, 0.0f}), (float)extent));
}

// Conic Sigma2D^-1 and the diagonal of Sigma2D (Sec. 3.2 Eq. t_2D), from the
// double-float camera-space mean p: Sigma2D = N N^T (+ low-pass I) with
// N = J W M and J = diag(fx/z, fy/z) [[1, 0, -ux], [0, 1, -uy]], (ux, uy) the
// limited (x/z, y/z).  The two rows of N are evaluated together, one per
// element of the packed registers.  det Sigma2D = |n0 x n1|^2 (+ low-pass
// terms), a sum of squares.  Each result is rounded once to FP32.
struct ConicDF {
  float con[3], A, C;
};

__device__ __forceinline__ ConicDF conic_df(const ShapeDF& m, DF px, DF py, DF pz, const sss_camera& cam,
                                            const sss_raster_cfg& cfg) {
  const float* V = cam.viewmat;
  const DF iz = df_rcp_normal(pz);  // z > znear > 0
  DF u[2] = {df_mul(px, iz), df_mul(py, iz)};
  const DF lim[2] = {lim_df(cam.width, cam.fx), lim_df(cam.height, cam.fy)};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const DF nl = DF{-lim[r].hi, -lim[r].lo};
    if (df_less(u[r], nl)) u[r] = nl;
    else if (df_less(lim[r], u[r])) u[r] = lim[r];
  }
  const DF2 uu = df2(u[0], u[1]);
  const DF2 rowf = df2_mul_f(df2_splat(iz), f2(cam.fx, cam.fy));
  DF2 U[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    U[k] = df2_sub(DF2{f2(V[0 * 4 + k], V[1 * 4 + k]), f2(0.0f, 0.0f)}, df2_mul_f(uu, f2(V[2 * 4 + k], V[2 * 4 + k])));
  DF2 n[3];
  DF n0[3], n1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    DF2 t = df2_mul(U[0], df2_splat(m.M[0 * 3 + k]));
    t = df2_add(t, df2_mul(U[1], df2_splat(m.M[1 * 3 + k])));
    t = df2_add(t, df2_mul(U[2], df2_splat(m.M[2 * 3 + k])));
    n[k] = df2_mul(rowf, t);
    df2_split(n[k], n0[k], n1[k]);
  }
  DF a, c;
  df2_split(df2_add(df2_add(df2_mul(n[0], n[0]), df2_mul(n[1], n[1])), df2_mul(n[2], n[2])), a, c);
  const DF b = df_dot3(n0, n1);
  // (x0, x1) packed, x2 alone: x = n0 x n1
  const DF2 x01 = df2_sub(df2_mul(df2(n0[1], n0[2]), df2(n1[2], n1[0])), df2_mul(df2(n0[2], n0[0]), df2(n1[1], n1[2])));
  const DF x2 = df_sub(df_mul(n0[0], n1[1]), df_mul(n0[1], n1[0]));
  DF q0, q1;
  df2_split(df2_mul(x01, x01), q0, q1);
  const float lp = cfg.lowpass;
  const DF A = df_add(a, DF{lp, 0.0f}), C = df_add(c, DF{lp, 0.0f});
  const DF det = df_add(df_add(df_add(q0, q1), df_mul(x2, x2)), df_mul_f(df_add(df_add(a, c), DF{lp, 0.0f}), lp));
  const DF id = df_rcp(det);
  ConicDF o;
  o.con[0] = df_mul(C, id).hi;
  o.con[1] = -df_mul(b, id).hi;
  o.con[2] = df_mul(A, id).hi;
  o.A = A.hi;
  o.C = C.hi;
  return o;
}

template <int DEG>
__device__ __forceinline__ void project_component(const sss_frame_plan& P, int s, uint32_t i, void* ws) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const sss_params& S = P.scenes[s];
  const sss_raster_cfg& cfg = P.cfg;
  const CompParams c = load_comp(S, i);
  const CompShape g = comp_shape(c);
  const ShapeDF gd = shape_df(c, g);
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
    const ConicDF cd = conic_df(gd, pxd, pyd, pzd, J.cam, cfg);
    // extent: |o| T2D(h) >= tau  <=>  h <= h_max (reading of the SM's truncation)
    // Gaussian kernel (nu -> infinity): |o| exp(-h/2) >= tau <=> h <= 2 ln(|o|/tau)
    const bool gauss = cfg.kernel == 1;
    const float hmax = gauss ? 2.0f * logf(fabsf(v.o) / cfg.tau)
                             : v.nu * expm1f(2.0f / (v.nu + 2.0f) * logf(fabsf(v.o) / cfg.tau));
    const float ex = sqrtf(cd.A * hmax), ey = sqrtf(cd.C * hmax);
    const float fx0 = fmaxf(ceilf(mxd.hi - ex - 0.5f), 0.0f);
    const float fx1 = fminf(floorf(mxd.hi + ex - 0.5f), (float)(J.cam.width - 1));
    const float fy0 = fmaxf(ceilf(myd.hi - ey - 0.5f), 0.0f);
    const float fy1 = fminf(floorf(myd.hi + ey - 0.5f), (float)(J.cam.height - 1));
    uint32_t nt = 0;
    uint2 rc = make_uint2(0u, 0u);
    if (fx0 <= fx1 && fy0 <= fy1) {
      const uint32_t tx0 = (uint32_t)fx0 / (uint32_t)cfg.tile_w, tx1 = (uint32_t)fx1 / (uint32_t)cfg.tile_w;
      const uint32_t ty0 = (uint32_t)fy0 / (uint32_t)cfg.tile_h, ty1 = (uint32_t)fy1 / (uint32_t)cfg.tile_h;
      nt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
      rc = make_uint2(tx0 | (tx1 << 16), ty0 | (ty1 << 16));
    }
    // origin: the integer pixel nearest to the mean, limited to [0, 16384]
    // (the largest image extent; the packed bits are then an ordinary float)
    const uint32_t ox = (uint32_t)fminf(fmaxf(rintf(mxd.hi), 0.0f), 16384.0f);
    const uint32_t oy = (uint32_t)fminf(fmaxf(rintf(myd.hi), 0.0f), 16384.0f);
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
    // (hi - origin) is exact where the origin is hi rounded (Sterbenz), so the
    // stored mean is rounded once, with an error of at most u/2 px there
    r.a = make_float4((mxd.hi - (float)ox) + mxd.lo, (myd.hi - (float)oy) + myd.lo, cd.con[0], cd.con[1]);
    r.b = make_float4(cd.con[2], v.o, hmax, gauss ? __int_as_float(0x7f800000) : v.nu);  // +inf: Gaussian
    r.c = make_float4(rgb[0], rgb[1], rgb[2], __uint_as_float(ox | (oy << 16)));
    rec[e] = r;
    dkey[e] = __float_as_uint(v.p[2]);
    ntiles[e] = nt;
    rect[e] = rc;
  }
}

__global__ void __launch_bounds__(128, 4) k_project(const sss_frame_plan P, void* ws) {
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
