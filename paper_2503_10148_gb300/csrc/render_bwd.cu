// a5: closed-form backward of the compositing (SM "Backward Pass").
//
// Same CTA/warp/lane layout as the forward.  Each pixel walks its tile's list
// from its last contributor back to the front, recomputing the transmittance
// before every contributor as T_k = T_{k+1} / (1 - alpha_k) (no per-pixel
// lists are stored).  With S_k the colour composited behind contributor k
// (plus T_final bg), dC/dalpha_k = T_k rgb_k - S_k / (1 - alpha_k).  Writing
// B_k = S_k / T_{k+1} -- the colour seen behind k, normalised -- this is
// T_k (rgb_k - B_k), and B follows the blend B_{k-1} = alpha_k rgb_k +
// (1 - alpha_k) B_k from B = bg at the back: no division, and the rounding of
// the recovered T_k scales the (often small) difference instead of its two
// large operands.  For a contributor k:
//   dL/drgb   = alpha T_k g                               (g = dL/dC)
//   dL/dalpha = T_k g . (rgb - B)
//   dL/do     = dL/dalpha T2D,  dL/dT2D = dL/dalpha o   (unless alpha was clamped)
//   dL/dh     = dL/dT2D dT2D/dh,  dT2D/dh = -(nu+2)/(2 nu) T2D / (1 + h/nu)
//   dL/dnu    = dL/dT2D T2D [-1/2 ln(1 + h/nu) + (nu+2) h / (2 nu^2 (1 + h/nu))]
//               (mode 1 drops the logarithm, as printed in the SM)
//   dh/dmean2D = -2 conic d,  dh/d(a, b, c) = (dx^2, 2 dx dy, dy^2).
// The factor of dT2D/dnu, f = -1/2 ln(1 + x) + (nu+2) x / (2 nu (1 + x)) with
// x = h/nu, is O(x^2) while its two terms are O(x): evaluated as written it
// cancels.  With u = x / (1 + x) it equals u/nu - g/2, g = ln(1 + x) - u =
// sum_{k>=2} u^k / k (from -ln(1 - u)), a sum of positive terms; for
// u < 1/4 the series to k = 13 is used (truncation < 1e-9 of g), above that the
// direct difference (cancellation at most 8x).
// Records are staged as in the forward (double buffered, next batch loaded
// while this one is processed).  A lane first sums its pixels; the warp then
// reduces the 10 sums with a reduce-scatter (12 shuffles instead of 10 x 5)
// and 10 lanes add the totals to the splat's record with one RED each.
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
    float p = 1.0f / 13.0f;
    p = fmaf(u, p, 1.0f / 12.0f);
    p = fmaf(u, p, 1.0f / 11.0f);
    p = fmaf(u, p, 1.0f / 10.0f);
    p = fmaf(u, p, 1.0f / 9.0f);
    p = fmaf(u, p, 1.0f / 8.0f);
    p = fmaf(u, p, 1.0f / 7.0f);
    p = fmaf(u, p, 1.0f / 6.0f);
    p = fmaf(u, p, 1.0f / 5.0f);
    p = fmaf(u, p, 1.0f / 4.0f);
    p = fmaf(u, p, 1.0f / 3.0f);
    p = fmaf(u, p, 0.5f);
    return u * u * p;
  }
  return log_base - u;
}

template <int PW, int PH, bool PAPER_NU>
__global__ void __launch_bounds__(64, PW * PH >= 4 ? 12 : 16) k_render_bwd(const sss_frame_plan P, void* ws,
                                                       const float* __restrict__ dl_drgb) {
  constexpr int NPIX = PW * PH;
  constexpr int TW = 16 * PW, TH = 16 * PH;
  __shared__ WarpBuf s_wb[2];

  // four CTAs of two warps per tile; warp w of the tile's 2 x 4 layout
  const uint32_t tile = blockIdx.x >> 2;
  WarpBuf& S = s_wb[threadIdx.x >> 5];
  const int j = job_of_tile(P, tile);
  const sss_job_desc& J = P.jobs[j];
  const sss_raster_cfg& cfg = P.cfg;
  const uint32_t lt = tile - J.tile_base;
  const int tx = (int)(lt % (uint32_t)J.tiles_x), ty = (int)(lt / (uint32_t)J.tiles_x);
  const int warp = (int)((blockIdx.x & 3u) << 1) | (int)(threadIdx.x >> 5);
  const unsigned lane = threadIdx.x & 31;
  const int bx = tx * TW + (warp & 1) * 8 * PW, by = ty * TH + (warp >> 1) * 4 * PH;
  const int lx = bx + (lane & 7) * PW, ly = by + (lane >> 3) * PH;
  const int W = J.cam.width, H = J.cam.height;
  const size_t hw = (size_t)W * H;

  const float* Tf = ws_ptr<float>(ws, P.ws_off_T);
  const uint32_t* Lf = ws_ptr<uint32_t>(ws, P.ws_off_last);
  const float* gimg = dl_drgb + 3 * (size_t)J.pix_base;
  float T[NPIX], Sg[NPIX], g[NPIX][3];  // Sg = dL/dC . (colour behind)
  uint32_t last[NPIX];
  uint32_t lane_max = 0;
#pragma unroll
  for (int p = 0; p < NPIX; ++p) {
    const int x = lx + p % PW, y = ly + p / PW;
    if (x < W && y < H) {
      const size_t o = (size_t)y * W + x;
      T[p] = Tf[J.pix_base + o];
      last[p] = Lf[J.pix_base + o];
      g[p][0] = gimg[o];
      g[p][1] = gimg[hw + o];
      g[p][2] = gimg[2 * hw + o];
    } else {
      T[p] = 1.0f;
      last[p] = 0u;
      g[p][0] = g[p][1] = g[p][2] = 0.0f;
    }
    Sg[p] = fmaf(g[p][0], cfg.bg[0], fmaf(g[p][1], cfg.bg[1], g[p][2] * cfg.bg[2]));
    lane_max = max(lane_max, last[p]);
  }
  const uint32_t warp_max = __reduce_max_sync(0xffffffffu, lane_max);

  const uint2 range = ws_ptr<uint2>(ws, P.ws_off_ranges)[tile];
  const uint32_t* vals = ws_ptr<uint32_t>(ws, P.ws_off_pval) + (size_t)P.pair_slot * P.pair_capacity + range.x;
  const SplatRec* rec = ws_ptr<SplatRec>(ws, P.ws_off_rec);
  float* g2d = ws_ptr<float>(ws, P.ws_off_grad2d);
  const float tau = cfg.tau, amax = cfg.alpha_max;

  // list positions are relative to range.x; pixel p has contributors in
  // [0, last[p]).  The warp walks its own contributors back to front in
  // batches of 32: batch i covers [lo_i, hi_i), hi_0 = warp_max (the
  // deepest contributor of the warp's pixels), lo_i = max(hi_i - 32, 0);
  // batch i + 1 is gathered and the entry ids of batch i + 2 are loaded
  // while batch i is evaluated.
  const uint32_t n_batches = (warp_max + 31) / 32;
  auto lo_of = [&](uint32_t i) { return warp_max > (i + 1) * 32 ? warp_max - (i + 1) * 32 : 0u; };
  if (n_batches > 0) {
    uint32_t lo = lo_of(0);
    uint32_t e_next = lo + lane < warp_max ? __ldg(vals + lo + lane) : 0u;
    warp_stage(S, 0, rec, e_next, lo + lane < warp_max, lane);
    if (n_batches > 1) {
      const uint32_t lo1 = lo_of(1);
      e_next = lo1 + lane < lo ? __ldg(vals + lo1 + lane) : 0u;
    }
    for (uint32_t i = 0; i < n_batches; ++i) {
      lo = lo_of(i);
      const int k = (int)(i & 1);
      if (i + 1 < n_batches) {
        const uint32_t lo1 = lo_of(i + 1);
        warp_stage(S, k ^ 1, rec, e_next, lo1 + lane < lo, lane);
        e_next = 0u;
        if (i + 2 < n_batches) {
          const uint32_t lo2 = lo_of(i + 2);
          if (lo2 + lane < lo1) e_next = __ldg(vals + lo2 + lane);
        }
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      unsigned m;
      {
        const float4 a = S.a[k][lane], b = S.b[k][lane];
        int ox, oy;
        rec_origin(S.c[k][lane].w, ox, oy);
        const bool hit = b.z >= 0.0f &&
                         ellipse_hits_box(a.x, a.y, a.z, a.w, b.x, fmaf(b.z, 2.0f * kHPad, b.z) + 1e-3f,
                                          (float)(bx - ox) + 0.5f, (float)(bx - ox + 8 * PW) - 0.5f,
                                          (float)(by - oy) + 0.5f, (float)(by - oy + 4 * PH) - 0.5f);
        m = __ballot_sync(0xffffffffu, hit);
      }
      while (m) {
        const int si = 31 - __clz(m);
        m &= ~(1u << si);
        const uint32_t pos = lo + si;
      const float4 a = S.a[k][si], b = S.b[k][si], c = S.c[k][si];
      const float cb2 = 2.0f * a.w, hpre = fmaf(b.z, kHPad, b.z);
      const float nu = b.w, inv_nu = __fdividef(1.0f, nu), o = b.y;
      int ox, oy;
      rec_origin(c.w, ox, oy);
      const float fbx = (float)(lx - ox), fby = (float)(ly - oy);
      // dT/dh = -(nu+2)/(2 nu) T / (1 + h/nu); -1/2 T for the Gaussian (nu = inf, inv_nu = 0)
      const float e_over_nu = isinf(nu) ? -0.5f : fmaf(nu, -0.5f, -1.0f) * inv_nu;
      // all pixels of the lane in straight-line code, masked; nu branch
      // uniform over the warp
      PairEval r[NPIX];
      bool ok[NPIX];
      float dxs[NPIX], dys[NPIX];
#pragma unroll
      for (int p = 0; p < NPIX; ++p) {
        dxs[p] = pixel_offset(fbx, p % PW, a.x);
        dys[p] = pixel_offset(fby, p / PW, a.y);
      }
      if (nu <= kFastNuMax) {
#pragma unroll
        for (int p = 0; p < NPIX; ++p)
          ok[p] = eval_pair_fast(dxs[p], dys[p], a.z, cb2, b.x, hpre, o, nu, inv_nu, tau, amax, r[p]);
      } else if (isinf(nu)) {
#pragma unroll
        for (int p = 0; p < NPIX; ++p)
          ok[p] = eval_pair_gauss(dxs[p], dys[p], a.z, cb2, b.x, hpre, o, tau, amax, r[p]);
      } else {
#pragma unroll
        for (int p = 0; p < NPIX; ++p)
          ok[p] = eval_pair_slow(dxs[p], dys[p], a.z, cb2, b.x, hpre, o, nu, inv_nu, tau, amax, r[p]);
      }
      // per-lane sums: rgb (v7..9), opacity (v5), nu (v6) and the
      // q-weighted moments of the pixel offsets, q = dL/dh, from which
      // dL/dmean and dL/dconic follow once per splat (h is quadratic in
      // the offsets, so its gradients are linear in these moments)
      float v[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) v[q] = 0.0f;
      float m1 = 0.0f, m2 = 0.0f, m3 = 0.0f, m4 = 0.0f, m5 = 0.0f;
      bool any = false;
#pragma unroll
      for (int p = 0; p < NPIX; ++p) {
        const bool live = ok[p] && pos < last[p];
        any = any || live;
        const float alpha = r[p].alpha;
        const float Tk = live ? T[p] * __fdividef(1.0f, 1.0f - alpha) : T[p];
        T[p] = Tk;
        const float w = live ? alpha * Tk : 0.0f;
        v[7] = fmaf(w, g[p][0], v[7]);
        v[8] = fmaf(w, g[p][1], v[8]);
        v[9] = fmaf(w, g[p][2], v[9]);
        // dL/dalpha = T_k dL/dC . (rgb - B) with B the colour behind; only
        // its projection on dL/dC is needed: Sg = dL/dC . B, and
        // B <- alpha rgb + (1 - alpha) B gives Sg <- Sg + alpha (g.rgb - Sg)
        const float gdiff = fmaf(g[p][0], c.x, fmaf(g[p][1], c.y, g[p][2] * c.z)) - Sg[p];
        Sg[p] = live ? fmaf(alpha, gdiff, Sg[p]) : Sg[p];
        const float dl_da = (live && !r[p].clamped) ? gdiff * Tk : 0.0f;
        v[5] = fmaf(dl_da, r[p].t2d, v[5]);
        const float dl_dt = dl_da * o;
        const float inv_base = __fdividef(1.0f, fmaf(r[p].h, inv_nu, 1.0f));
        const float qh = dl_dt * e_over_nu * r[p].t2d * inv_base;  // dL/dh
        const float u = r[p].h * inv_nu * inv_base;  // x / (1 + x)
        // paper form: (nu+2) x / (2 nu (1+x)) = u/2 + u/nu; exact: u/nu - g/2
        const float dnu = PAPER_NU ? fmaf(0.5f, u, u * inv_nu)
                                   : fmaf(-0.5f, log1p_minus_u(u, r[p].log_base), u * inv_nu);
        v[6] = fmaf(dl_dt * r[p].t2d, dnu, v[6]);
        const float qdx = qh * dxs[p], qdy = qh * dys[p];
        m1 += qdx;
        m2 += qdy;
        m3 = fmaf(qdx, dxs[p], m3);
        m4 = fmaf(qdx, dys[p], m4);
        m5 = fmaf(qdy, dys[p], m5);
      }
      // dh/dmean = -2 (a dx + b dy, b dx + c dy); dh/dconic = (dx^2, 2 dx dy, dy^2)
      v[0] = -2.0f * fmaf(a.z, m1, a.w * m2);
      v[1] = -2.0f * fmaf(a.w, m1, b.x * m2);
      v[2] = m3;
      v[3] = 2.0f * m4;
      v[4] = m5;
      if (__any_sync(0xffffffffu, any)) {
        int slot;
        const float tot = warp_reduce_scatter10(v, lane, &slot);
        if (slot >= 0) atomicAdd(g2d + (size_t)S.e[k][si] * 12 + slot, tot);
      }
      }
      __syncwarp();  // every lane is done with buffer k before it is refilled
    }
    cp_async_wait<0>();
  }
}

template <int PW, int PH, bool PAPER_NU>
int launch_batch(const sss_frame_plan& P, void* ws, const float* g, cudaStream_t st) {
  // 32 records per warp and batch whatever cfg.batch says (checked by the plan)
  k_render_bwd<PW, PH, PAPER_NU><<<4 * P.n_tiles, 64, 0, st>>>(P, ws, g);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

template <int PW, int PH>
int launch_tile(const sss_frame_plan& P, void* ws, const float* g, cudaStream_t st) {
  return P.cfg.nu_grad_mode == 1 ? launch_batch<PW, PH, true>(P, ws, g, st) : launch_batch<PW, PH, false>(P, ws, g, st);
}

}  // namespace
}  // namespace sss

extern "C" int sss_render_bwd(const sss_frame_plan* plan, void* ws, const float* dL_drgb, sss_stream_t stream) {
  if (!plan || !ws || !dL_drgb) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(sss::ws_ptr<float>(ws, P.ws_off_grad2d), 0, 48 * (size_t)P.n_entries, st) != cudaSuccess)
    return SSS_ERR_CUDA;
  const int pw = P.cfg.tile_w / 16, ph = P.cfg.tile_h / 16;
  if (pw == 1 && ph == 1) return sss::launch_tile<1, 1>(P, ws, dL_drgb, st);
  if (pw == 2 && ph == 1) return sss::launch_tile<2, 1>(P, ws, dL_drgb, st);
  if (pw == 1 && ph == 2) return sss::launch_tile<1, 2>(P, ws, dL_drgb, st);
  if (pw == 2 && ph == 2) return sss::launch_tile<2, 2>(P, ws, dL_drgb, st);
  return SSS_ERR_UNSUPPORTED;
}
