// a5: closed-form backward of the compositing (SM "Backward Pass").
//
// The forward's CTA/warp/lane layout, or (cfg.bwd_box_h = 16) warp boxes twice
// as high: 2 x 4 pixels a lane, 32 x 64 sub-tiles.  Each pixel walks its tile's list
// from its last contributor back to the front, recomputing the transmittance
// before every contributor as T_k = T_{k+1} / (1 - alpha_k) (no per-pixel
// lists are stored).  With S_k the colour composited behind contributor k
// (plus T_final bg), dC/dalpha_k = T_k rgb_k - S_k / (1 - alpha_k).  Writing
// B_k = S_k / T_{k+1} -- the colour seen behind k, normalised -- this is
// T_k (rgb_k - B_k), and B follows the blend B_{k-1} = alpha_k rgb_k +
// (1 - alpha_k) B_k from B = bg at the back: no division, and the rounding of
// the recovered T_k scales the (often small) difference instead of its two
// large operands.  The kernel carries -alpha (the records are evaluated with
// the opacity's sign flipped) and -g . B, which saves a subtraction per
// pixel.  For a contributor k:
//   dL/drgb   = alpha T_k g                               (g = dL/dC)
//   dL/dalpha = T_k g . (rgb - B)
//   dL/do     = dL/dalpha T2D,  dL/dT2D = dL/dalpha o   (unless alpha was clamped)
//   dL/dh     = dL/dT2D dT2D/dh,  dT2D/dh = -(nu+2)/(2 nu) T2D / (1 + h/nu)
//   dL/dnu    = dL/dT2D T2D [-1/2 ln(1 + h/nu) + (nu+2) h / (2 nu^2 (1 + h/nu))]
//               (mode 1 drops the logarithm, as printed in the SM)
//   dh/dmean2D = -2 conic d,  dh/d(a, b, c) = (dx^2, 2 dx dy, dy^2).
// The factor of dT2D/dnu, f = -1/2 ln(1 + x) + (nu+2) x / (2 nu (1 + x)) with
// x = h/nu, is O(x^2) while its two terms are O(x): evaluated as written it
// cancels.  With u = x / (1 + x) it equals u/nu - g/2, g = ln(1 + x) - u.
// With s = u / (2 - u) = x / (2 + x), ln(1 + x) = 2 atanh(s) and 2 s - u =
// u s, so g = u s + 2 (s^3/3 + s^5/5 + ...), a sum of positive terms; for
// u < 1/4 (s < 1/7) the series to s^9 is used (truncation below 3e-9 of g),
// above that the direct difference (cancellation at most 8x).
// Each warp walks its own contributors back to front, 32 records per round
// staged as in the forward, and evaluates a lane's pixels two at a time
// with packed FP32 instructions where it has an even number of them.  Per splat a lane first sums its pixels (the
// factors common to the splat, o and dT2D/dh's (nu+2)/(2 nu), are applied to
// the sums once); the warp then reduces the 10 sums with a reduce-scatter
// (12 shuffles instead of 10 x 5) and 10 lanes add the totals to the
// splat's record with one RED each.
#include <type_traits>

#include "common.cuh"

namespace sss {
namespace {

// Sums v[0..9] over the warp with 12 shuffles: five halving rounds over lane
// bits 4..0 in which each lane keeps a shrinking set of slots (5, then 3 or
// 2, then 2 or 1, then 1) and sends the rest to its partner.  Returns the
// total of one slot, *slot = its index, or -1 on lanes whose total duplicates
// another lane's (exactly one lane per slot gets a slot index).
__device__ __forceinline__ float warp_reduce_scatter10(const float (&v)[10], unsigned lane, int* slot) {
  constexpr unsigned F = 0xffffffffu;
  const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u, b1 = lane & 2u;
  float w[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) w[i] = (b4 ? v[5 + i] : v[i]) + __shfl_xor_sync(F, b4 ? v[i] : v[5 + i], 16);
  const float y0 = (b3 ? w[3] : w[0]) + __shfl_xor_sync(F, b3 ? w[0] : w[3], 8);
  const float y1 = (b3 ? w[4] : w[1]) + __shfl_xor_sync(F, b3 ? w[1] : w[4], 8);
  const float y2 = w[2] + __shfl_xor_sync(F, w[2], 8);  // used where b3 == 0
  const float send0 = b3 ? (b2 ? y0 : y1) : (b2 ? y0 : y2);
  const float keep0 = b3 ? (b2 ? y1 : y0) : (b2 ? y2 : y0);
  const float z0 = keep0 + __shfl_xor_sync(F, send0, 4);
  const float z1 = y1 + __shfl_xor_sync(F, y1, 4);  // used where b3 == b2 == 0
  const bool two = !b3 && !b2;
  const float send = two ? (b1 ? z0 : z1) : z0;
  const float keep = two ? (b1 ? z1 : z0) : z0;
  float f = keep + __shfl_xor_sync(F, send, 2);
  f += __shfl_xor_sync(F, f, 1);
  const int local = two ? (b1 ? 1 : 0) : (!b3 ? 2 : (!b2 ? 3 : 4));
  *slot = ((lane & 1u) == 0u && (two || !b1)) ? 5 * (b4 ? 1 : 0) + local : -1;
  return f;
}

__device__ __forceinline__ float log1p_minus_u(float u, float log_base) {
  if (u < 0.25f) {
    const float sv = u * mufu_rcp(2.0f - u), s2 = sv * sv;
    float p = fmaf(s2, 2.0f / 9.0f, 2.0f / 7.0f);
    p = fmaf(s2, p, 2.0f / 5.0f);
    p = fmaf(s2, p, 2.0f / 3.0f);
    return fmaf(s2 * sv, p, u * sv);
  }
  return log_base - u;
}
// two pixels: the series in packed form for both, then a per-element choice
__device__ __forceinline__ F2 log1p_minus_u(F2 u, F2 log_base) {
  const F2 sv = vmul(u, vrcp(vsub(vsplat<F2>(2.0f), u))), s2 = vmul(sv, sv);
  F2 p = vfma(s2, vsplat<F2>(2.0f / 9.0f), vsplat<F2>(2.0f / 7.0f));
  p = vfma(s2, p, vsplat<F2>(2.0f / 5.0f));
  p = vfma(s2, p, vsplat<F2>(2.0f / 3.0f));
  const F2 series = vfma(vmul(s2, sv), p, vmul(u, sv));
  return vsel(vlt(u, 0.25f), series, vsub(log_base, u));
}

// One work item: warp (item & 1) of CTA (item >> 1) of the grid form, i.e.
// one warp box of one sub-tile.  S is the calling warp's staging buffer.
template <int PW, int PH, int R, bool PAPER_NU>
__device__ __forceinline__ void bwd_item(const sss_frame_plan& P, void* ws, const float* __restrict__ dl_drgb,
                                         uint32_t item, WarpBuf<R>& S) {
  constexpr int NPIX = PW * PH;
  constexpr uint32_t B = 32 * R;  // records per warp and round
  constexpr int TW = 16 * PW, TH = 16 * PH;
  constexpr int L = LaneVec<NPIX>::L, NV = LaneVec<NPIX>::NV;
  using V = typename std::conditional<L == 2, F2, float>::type;
  using M = MaskT<V>;
  // sub-tiles of the list tile as in the forward; warp w of a sub-tile's
  // 2 x 4 layout
  const sss_raster_cfg& cfg = P.cfg;
  const uint32_t SX = (uint32_t)cfg.tile_w / TW, SY = (uint32_t)cfg.tile_h / TH;
  const uint32_t blk = item >> 1;
  const uint32_t cta = blk >> 2, tile = cta / (SX * SY), sub = cta - tile * (SX * SY);
  const int j = job_of_tile(P, tile);
  const sss_job_desc& J = P.jobs[j];
  const uint32_t lt = tile - J.tile_base;
  const int tx = (int)(lt % (uint32_t)J.tiles_x), ty = (int)(lt / (uint32_t)J.tiles_x);
  const int warp = (int)((blk & 3u) << 1) | (int)(item & 1u);
  const unsigned lane = threadIdx.x & 31;
  const int bx = tx * cfg.tile_w + (int)(sub % SX) * TW + (warp & 1) * 8 * PW;
  const int by = ty * cfg.tile_h + (int)(sub / SX) * TH + (warp >> 1) * 4 * PH;
  const int lx = bx + (lane & 7) * PW, ly = by + (lane >> 3) * PH;
  const int W = J.cam.width, H = J.cam.height;
  const size_t hw = (size_t)W * H;

  const float* Tf = ws_ptr<float>(ws, P.ws_off_T);
  const uint32_t* Lf = ws_ptr<uint32_t>(ws, P.ws_off_last);
  const float* gimg = dl_drgb + 3 * (size_t)J.pix_base;
  // pixel p = L v + k of the lane is value v, element k
  V T[NV], Sg[NV], g[NV][3];  // Sg = -dL/dC . (colour behind)
  uint32_t last[NPIX];
  uint32_t lane_max = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float t[2], gg[2][3];
#pragma unroll
    for (int kk = 0; kk < L; ++kk) {
      const int p = L * v + kk;
      const int x = lx + p % PW, y = ly + p / PW;
      if (x < W && y < H) {
        const size_t o = (size_t)y * W + x;
        t[kk] = Tf[J.pix_base + o];
        last[p] = Lf[J.pix_base + o];
        gg[kk][0] = gimg[o];
        gg[kk][1] = gimg[hw + o];
        gg[kk][2] = gimg[2 * hw + o];
      } else {
        t[kk] = 1.0f;
        last[p] = 0u;
        gg[kk][0] = gg[kk][1] = gg[kk][2] = 0.0f;
      }
      lane_max = max(lane_max, last[p]);
    }
    float sg[2];
#pragma unroll
    for (int kk = 0; kk < L; ++kk)
      sg[kk] = -fmaf(gg[kk][0], cfg.bg[0], fmaf(gg[kk][1], cfg.bg[1], gg[kk][2] * cfg.bg[2]));
    if constexpr (L == 2) {
      T[v] = f2(t[0], t[1]);
      Sg[v] = f2(sg[0], sg[1]);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) g[v][ch] = f2(gg[0][ch], gg[1][ch]);
    } else {
      T[v] = t[0];
      Sg[v] = sg[0];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) g[v][ch] = gg[0][ch];
    }
  }
  const uint32_t warp_max = __reduce_max_sync(0xffffffffu, lane_max);

  const uint2 range = ws_ptr<uint2>(ws, P.ws_off_ranges)[tile];
  const uint32_t* vals = ws_ptr<uint32_t>(ws, P.ws_off_pval) + (size_t)P.pair_slot * P.pair_capacity + range.x;
  const SplatRec* rec = ws_ptr<SplatRec>(ws, P.ws_off_rec);
  float* g2d = ws_ptr<float>(ws, P.ws_off_grad2d);
  const float tau = cfg.tau, amax = cfg.alpha_max;

  // list positions are relative to range.x; pixel p has contributors in
  // [0, last[p]).  The warp walks its own contributors back to front in
  // batches of B: batch i covers [lo_i, hi_i), hi_0 = warp_max (the
  // deepest contributor of the warp's pixels), lo_i = max(hi_i - B, 0);
  // batch i + 1 is gathered and the entry ids of batch i + 2 are loaded
  // while batch i is evaluated.
  const uint32_t n_batches = (warp_max + B - 1) / B;
  auto lo_of = [&](uint32_t i) { return warp_max > (i + 1) * B ? warp_max - (i + 1) * B : 0u; };
  if (n_batches > 0) {
    uint32_t lo = lo_of(0);
    uint32_t e_next[R];
    bool v_next[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t q = lo + r * 32 + lane;
      v_next[r] = q < warp_max;
      e_next[r] = v_next[r] ? __ldg(vals + q) : 0u;
    }
    warp_stage<R>(S, 0, rec, e_next, v_next, lane);
    if (n_batches > 1) {
      const uint32_t lo1 = lo_of(1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t q = lo1 + r * 32 + lane;
        e_next[r] = q < lo ? __ldg(vals + q) : 0u;
      }
    }
    for (uint32_t i = 0; i < n_batches; ++i) {
      lo = lo_of(i);
      const int k = (int)(i & 1);
      if (i + 1 < n_batches) {
        const uint32_t lo1 = lo_of(i + 1);
#pragma unroll
        for (int r = 0; r < R; ++r) v_next[r] = lo1 + r * 32 + lane < lo;
        warp_stage<R>(S, k ^ 1, rec, e_next, v_next, lane);
        const uint32_t lo2 = i + 2 < n_batches ? lo_of(i + 2) : 0u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t q = lo2 + r * 32 + lane;
          e_next[r] = (i + 2 < n_batches && q < lo1) ? __ldg(vals + q) : 0u;
        }
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      unsigned mm[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int sl = rr * 32 + lane;
        const float4 a = S.a[k][sl], b = S.b[k][sl];
        int ox, oy;
        rec_origin(S.c[k][sl].w, ox, oy);
        const bool hit = b.z >= 0.0f &&
                         ellipse_hits_box(a.x, a.y, a.z, a.w, b.x, fmaf(b.z, 2.0f * kHPad, b.z) + 1e-3f,
                                          (float)(bx - ox) + 0.5f, (float)(bx - ox + 8 * PW) - 0.5f,
                                          (float)(by - oy) + 0.5f, (float)(by - oy + 4 * PH) - 0.5f);
        mm[rr] = __ballot_sync(0xffffffffu, hit);
      }
#pragma unroll
      for (int rr = R - 1; rr >= 0; --rr) {
      unsigned m = mm[rr];
      while (m) {
        const int sb = 31 - __clz(m);
        m &= ~(1u << sb);
        const int si = rr * 32 + sb;
        const uint32_t pos = lo + si;
        const float4 a = S.a[k][si], b = S.b[k][si], c = S.c[k][si];
        const float cb2 = 2.0f * a.w;
        const float nu = b.w, inv_nu = mufu_rcp(nu), o = b.y;
        const float oabs = fabsf(o), osgn = copysignf(1.0f, o);
        int ox, oy;
        rec_origin(c.w, ox, oy);
        const float fbx = (float)(lx - ox), fby = (float)(ly - oy);
        float dxs[PW], dys[PH];
#pragma unroll
        for (int ii = 0; ii < PW; ++ii) dxs[ii] = pixel_offset(fbx, ii, a.x);
#pragma unroll
        for (int jj = 0; jj < PH; ++jj) dys[jj] = pixel_offset(fby, jj, a.y);
        V dx[NV], dy[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (L == 2) {
            dx[v] = f2(dxs[(L * v) % PW], dxs[(L * v + 1) % PW]);
            dy[v] = f2(dys[(L * v) / PW], dys[(L * v + 1) / PW]);
          } else {
            dx[v] = dxs[v % PW];
            dy[v] = dys[v / PW];
          }
        }
        // per-lane sums: rgb (v7..9), st = dL/dalpha T2D (v5 = dL/do), st
        // times the nu factor (v6 / o) and, per pixel, q = st / (1 + h/nu),
        // with dL/dh = o (dT2D/dh / T2D) (1 + h/nu) q; dL/dmean and dL/dconic
        // follow from q-weighted moments of the pixel offsets (h is quadratic
        // in the offsets, so its gradients are linear in these moments).
        // Each value is accumulated right after its evaluation, so only one
        // value's evaluation is live at a time.
        const V one = vsplat<V>(1.0f), zero = vsplat<V>(0.0f), ivn = vsplat<V>(inv_nu);
        const V cr = vsplat<V>(c.x), cg = vsplat<V>(c.y), cbl = vsplat<V>(c.z);
        V s5 = zero, s6 = zero, r7 = zero, r8 = zero, r9 = zero, q[NV];
        bool any = false;
        auto accumulate = [&](int v, const PairEval<V>& rv, M okv) {
          M before;  // the splat is in front of the pixel's last contributor
          if constexpr (L == 2) before = B2{pos < last[L * v], pos < last[L * v + 1]};
          else before = pos < last[v];
          const M live = mand(okv, before);
          any = any || many(live);
          const V al = vsel(live, rv.alpha, zero);  // -alpha (the record's sign flipped)
          // T_k = T_{k+1} / (1 - alpha); with al = 0 off the live pixels the
          // MUFU reciprocal of 1 is exactly 1, so T is kept bit for bit
          const V Tk = vmul(T[v], vrcp(vadd(one, al)));
          T[v] = Tk;
          const V w = vmul(al, Tk);  // 0 unless live
          r7 = vfma(w, g[v][0], r7);
          r8 = vfma(w, g[v][1], r8);
          r9 = vfma(w, g[v][2], r9);
          // dL/dalpha = T_k dL/dC . (rgb - B) with B the colour behind; only
          // its projection on dL/dC is needed: Sg = dL/dC . B, and
          // B <- alpha rgb + (1 - alpha) B gives Sg <- Sg + alpha (g.rgb - Sg)
          const V gdiff = vfma(g[v][0], cr, vfma(g[v][1], cg, vfma(g[v][2], cbl, Sg[v])));
          Sg[v] = vfma(al, gdiff, Sg[v]);
          const V dl_da = vsel(mandn(live, rv.clamped), vmul(gdiff, Tk), zero);
          const V st = vmul(dl_da, rv.t2d);
          s5 = vadd(s5, st);
          const V inv_base = vrcp(vfma(rv.h, ivn, one));
          q[v] = vmul(st, inv_base);
          const V u = vmul(vmul(rv.h, ivn), inv_base);  // x / (1 + x)
          // paper form: (nu+2) x / (2 nu (1+x)) = u/2 + u/nu; exact: u/nu - g/2
          const V dnu = PAPER_NU ? vfma(vsplat<V>(0.5f), u, vmul(u, ivn))
                                 : vfma(vsplat<V>(-0.5f), log1p_minus_u(u, rv.log_base), vmul(u, ivn));
          s6 = vfma(st, dnu, s6);
        };
        // all pixels of the lane in straight-line code, masked; nu branch
        // uniform over the warp.  The alpha clamp is the identity when
        // |o| T2D cannot reach alpha_max (the forward makes the same choice,
        // so both take identical decisions).
        if (nu <= kFastNuMax && oabs * 1.0001f <= amax) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            PairEval<V> rv;
            const M okv = eval_pair_fast<V, false>(dx[v], dy[v], a.z, cb2, b.x, oabs, -osgn, nu, inv_nu, tau, amax, rv);
            accumulate(v, rv, okv);
          }
        } else if (nu <= kFastNuMax) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            PairEval<V> rv;
            const M okv = eval_pair_fast(dx[v], dy[v], a.z, cb2, b.x, oabs, -osgn, nu, inv_nu, tau, amax, rv);
            accumulate(v, rv, okv);
          }
        } else if (isinf(nu)) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            PairEval<V> rv;
            const M okv = eval_pair_gauss(dx[v], dy[v], a.z, cb2, b.x, oabs, -osgn, tau, amax, rv);
            accumulate(v, rv, okv);
          }
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            PairEval<V> rv;
            const M okv = eval_pair_slow(dx[v], dy[v], a.z, cb2, b.x, oabs, -osgn, nu, inv_nu, tau, amax, rv);
            accumulate(v, rv, okv);
          }
        }
        // moments of q over the lane's PW x PH pixels from column and row sums
        float m1 = 0.0f, m2 = 0.0f, m3 = 0.0f, m4 = 0.0f, m5 = 0.0f;
        if constexpr (PW == 2 && PH % 2 == 0) {
          // value v is row v: columns packed as (col 0, col 1)
          F2 cq = q[0], cqy = vmul(q[0], dy[0]);  // per-column sums of q and q dy
#pragma unroll
          for (int v = 1; v < NV; ++v) {
            cq = vadd(cq, q[v]);
            cqy = vfma(q[v], dy[v], cqy);
          }
          const F2 dq = vmul(dx[0], cq);
          m1 = vsum(dq);
          m3 = vsum(vmul(dq, dx[0]));
          m4 = vsum(vmul(dx[0], cqy));
#pragma unroll
          for (int jj = 0; jj < PH; jj += 2) {  // per-row sums, two rows at a time
            const F2 dyr = f2(dys[jj], dys[jj + 1]), rq = f2(vsum(q[jj]), vsum(q[jj + 1]));
            const F2 dr = vmul(dyr, rq);
            m2 += vsum(dr);
            m5 += vsum(vmul(dr, dyr));
          }
        } else {
        float cq[PW], cqy[PW], rq[PH];
#pragma unroll
        for (int ii = 0; ii < PW; ++ii) cq[ii] = cqy[ii] = 0.0f;
#pragma unroll
        for (int jj = 0; jj < PH; ++jj) rq[jj] = 0.0f;
#pragma unroll
        for (int p = 0; p < NPIX; ++p) {
          const float qp = vget(q[p / L], p % L);
          cq[p % PW] += qp;
          cqy[p % PW] = fmaf(qp, dys[p / PW], cqy[p % PW]);
          rq[p / PW] += qp;
        }
#pragma unroll
        for (int ii = 0; ii < PW; ++ii) {
          const float dq = dxs[ii] * cq[ii];
          m1 += dq;
          m3 = fmaf(dq, dxs[ii], m3);
          m4 = fmaf(dxs[ii], cqy[ii], m4);
        }
#pragma unroll
        for (int jj = 0; jj < PH; ++jj) {
          const float dq = dys[jj] * rq[jj];
          m2 += dq;
          m5 = fmaf(dq, dys[jj], m5);
        }
        }
        // dT2D/dh / T2D = -(nu+2)/(2 nu) / (1 + h/nu); -1/2 for the Gaussian
        // (nu = inf, inv_nu = 0)
        const float kq = o * (isinf(nu) ? -0.5f : fmaf(nu, -0.5f, -1.0f) * inv_nu);
        m1 *= kq;
        m2 *= kq;
        // dh/dmean = -2 (a dx + b dy, b dx + c dy); dh/dconic = (dx^2, 2 dx dy, dy^2)
        float vv[10];
        vv[0] = -2.0f * fmaf(a.z, m1, a.w * m2);
        vv[1] = -2.0f * fmaf(a.w, m1, b.x * m2);
        vv[2] = kq * m3;
        vv[3] = 2.0f * kq * m4;
        vv[4] = kq * m5;
        vv[5] = vsum(s5);
        vv[6] = o * vsum(s6);
        vv[7] = -vsum(r7);
        vv[8] = -vsum(r8);
        vv[9] = -vsum(r9);
        if (__any_sync(0xffffffffu, any)) {
          int slot;
          const float tot = warp_reduce_scatter10(vv, lane, &slot);
          if (slot >= 0) atomicAdd(g2d + (size_t)S.e[k][si] * 12 + slot, tot);
        }
      }
      }
      __syncwarp();  // every lane is done with buffer k before it is refilled
    }
    cp_async_wait<0>();
  }
}

// Persistent, as the forward: warps take work items from the workspace's
// counter until none is left; the last one resets it.
template <int PW, int PH, int R, bool PAPER_NU>
__global__ void __launch_bounds__(64, PW * PH >= 8 ? 8 : (PW * PH >= 4 ? 12 : 16)) k_render_bwd(const sss_frame_plan P, void* ws,
                                                                           const float* __restrict__ dl_drgb,
                                                                           uint32_t n_items) {
  __shared__ WarpBuf<R> s_wb[2];
  WarpBuf<R>& S = s_wb[threadIdx.x >> 5];
  uint32_t* queue = ws_ptr<uint32_t>(ws, P.ws_off_ctrl) + kCtrlQueue;
  const unsigned lane = threadIdx.x & 31;
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    bwd_item<PW, PH, R, PAPER_NU>(P, ws, dl_drgb, item, S);
  }
  queue_retire(queue, lane);
}

template <int PW, int PH, int R, bool PAPER_NU>
int launch_batch(const sss_frame_plan& P, void* ws, const float* g, cudaStream_t st) {
  const unsigned subs = (unsigned)(P.cfg.tile_w / (16 * PW)) * (unsigned)(P.cfg.tile_h / (16 * PH));
  const uint32_t n_items = 8u * subs * P.n_tiles;  // warps of the grid form
  if (n_items == 0) return SSS_OK;
  const unsigned grid = persistent_grid(k_render_bwd<PW, PH, R, PAPER_NU>, 64, n_items / 2);
  k_render_bwd<PW, PH, R, PAPER_NU><<<grid, 64, 0, st>>>(P, ws, g, n_items);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

template <int PW, int PH, bool PAPER_NU>
int launch_depth(const sss_frame_plan& P, void* ws, const float* g, cudaStream_t st) {
  // records staged per warp and round: cfg.batch = 32 or 64 (checked by the plan)
  return P.cfg.batch == 64 ? launch_batch<PW, PH, 2, PAPER_NU>(P, ws, g, st)
                           : launch_batch<PW, PH, 1, PAPER_NU>(P, ws, g, st);
}

template <int PW, int PH>
int launch_tile(const sss_frame_plan& P, void* ws, const float* g, cudaStream_t st) {
  return P.cfg.nu_grad_mode == 1 ? launch_depth<PW, PH, true>(P, ws, g, st) : launch_depth<PW, PH, false>(P, ws, g, st);
}

}  // namespace
}  // namespace sss

extern "C" int sss_render_bwd(const sss_frame_plan* plan, void* ws, const float* dL_drgb, sss_stream_t stream) {
  if (!plan || !ws || !dL_drgb) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(sss::ws_ptr<float>(ws, P.ws_off_grad2d), 0, 48 * (size_t)P.n_entries, st) != cudaSuccess)
    return SSS_ERR_CUDA;
  // sub-tiles of at most 32 x 32 (lanes of up to 2 x 2 pixels), or 32 x 64
  // (lanes of 2 x 4) with 16-pixel-high warp boxes
  const int pw = (P.cfg.tile_w >= 32 ? 32 : P.cfg.tile_w) / 16;
  const int ph = P.cfg.bwd_box_h == 16 ? 4 : (P.cfg.tile_h >= 32 ? 32 : P.cfg.tile_h) / 16;
  if (pw == 2 && ph == 4) return sss::launch_tile<2, 4>(P, ws, dL_drgb, st);
  if (pw == 1 && ph == 1) return sss::launch_tile<1, 1>(P, ws, dL_drgb, st);
  if (pw == 2 && ph == 1) return sss::launch_tile<2, 1>(P, ws, dL_drgb, st);
  if (pw == 1 && ph == 2) return sss::launch_tile<1, 2>(P, ws, dL_drgb, st);
  if (pw == 2 && ph == 2) return sss::launch_tile<2, 2>(P, ws, dL_drgb, st);
  return SSS_ERR_UNSUPPORTED;
}
