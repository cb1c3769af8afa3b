// a4: per-pixel front-to-back compositing with signed alpha
// (Sec. 3.4 Eq. SSS_color; signed opacity Sec. 3.3).
//
// A render sub-tile of (16 PW) x (16 PH) pixels (at most 32 x 32; a list
// tile of the binning may hold several) is covered by eight warp boxes laid
// out 2 x 4; warp box w is (8 PW) x (4 PH) pixels and lane l owns a PW x PH
// block of pixels inside it.  The kernel is persistent: a grid of as many
// two-warp CTAs as fit on the device, whose warps take warp boxes from a
// work counter in index order until none is left.  Warps are
// independent (no CTA barrier): each walks the tile's list in rounds of 32
// or 64 records (cfg.batch; one or two 48-byte records per lane) gathered
// by entry index with cp.async into the warp's own double buffer (the next
// round is in flight while this one is evaluated).  The warp tests the
// staged splats against its box in parallel (exact ellipse/box test) and
// walks only the
// survivors, in list (= depth) order, so pairs whose ellipse misses the
// warp's 32 PW PH pixels cost nothing; it stops when all its pixels are
// done.  A lane's pixels are evaluated two at a time with packed FP32
// instructions where it has an even number of them.
#include <type_traits>

#include "common.cuh"

namespace sss {
namespace {

// One work item: warp (item & 1) of CTA (item >> 1) of the grid form, i.e.
// one warp box of one sub-tile.  S is the calling warp's staging buffer.
template <int PW, int PH, int R, bool COUNT>
__device__ __forceinline__ void fwd_item(const sss_frame_plan& P, void* ws, float* __restrict__ out_rgb, uint32_t item,
                                         WarpBuf<R>& S) {
  constexpr int NPIX = PW * PH;
  constexpr uint32_t B = 32 * R;  // records per warp and round
  constexpr int TW = 16 * PW, TH = 16 * PH;
  constexpr int L = LaneVec<NPIX>::L, NV = LaneVec<NPIX>::NV;
  using V = typename std::conditional<L == 2, F2, float>::type;
  using M = MaskT<V>;
  // a list tile of cfg.tile_w x cfg.tile_h pixels is rendered as SX x SY
  // sub-tiles of TW x TH, each by four CTAs of two warps; warp w of the
  // sub-tile's 2 x 4 layout.  Every sub-tile walks the whole list of its
  // tile (the per-warp cull drops what misses its box).
  const sss_raster_cfg& cfg = P.cfg;
  const uint32_t SX = (uint32_t)cfg.tile_w / TW, SY = (uint32_t)cfg.tile_h / TH;
  const uint32_t blk = item >> 1;
  const uint32_t cta = blk >> 2, tile = cta / (SX * SY), sub = cta - tile * (SX * SY);
  const int warp = (int)((blk & 3u) << 1) | (int)(item & 1u), lane = threadIdx.x & 31;
  const int j = job_of_tile(P, tile);
  const sss_job_desc& J = P.jobs[j];
  const uint32_t lt = tile - J.tile_base;
  const int tx = (int)(lt % (uint32_t)J.tiles_x), ty = (int)(lt / (uint32_t)J.tiles_x);
  const int bx = tx * cfg.tile_w + (int)(sub % SX) * TW + (warp & 1) * 8 * PW;
  const int by = ty * cfg.tile_h + (int)(sub / SX) * TH + (warp >> 1) * 4 * PH;
  const int lx = bx + (lane & 7) * PW, ly = by + (lane >> 3) * PH;
  const int W = J.cam.width, H = J.cam.height;

  // pixel p = L v + k of the lane is value v, element k.  A pixel's
  // threshold is tau while it composites and +inf once it is done (outside
  // the image, or terminated): |alpha| >= +inf never holds, so a done pixel
  // drops out of the compositing update by itself and the common path keeps
  // no done-mask bookkeeping; termination, about once per pixel, is handled
  // in a branch taken when some pixel of the warp terminates.
  const float tau = cfg.tau, amax = cfg.alpha_max, tmin = cfg.t_min;
  V T[NV], C[NV][3], thr[NV];
  uint32_t last[NPIX];
  bool lane_done = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float th[2] = {tau, tau};
#pragma unroll
    for (int k = 0; k < L; ++k) {
      const int p = L * v + k;
      const bool out = !(lx + p % PW < W && ly + p / PW < H);
      th[k] = out ? __int_as_float(0x7f800000) : tau;
      lane_done = lane_done && out;
      last[p] = 0u;
    }
    if constexpr (L == 2) thr[v] = f2(th[0], th[1]);
    else thr[v] = th[0];
    T[v] = vsplat<V>(1.0f);
    C[v][0] = C[v][1] = C[v][2] = vsplat<V>(0.0f);
  }
  bool warp_done = __all_sync(0xffffffffu, lane_done);

  const uint2 range = ws_ptr<uint2>(ws, P.ws_off_ranges)[tile];
  const uint32_t* vals = ws_ptr<uint32_t>(ws, P.ws_off_pval) + (size_t)P.pair_slot * P.pair_capacity + range.x;
  const SplatRec* rec = ws_ptr<SplatRec>(ws, P.ws_off_rec);
  uint32_t n_eval = 0, n_contrib = 0;  // pair counters (COUNT only)

  const uint32_t n_list = range.y - range.x;
  const uint32_t n_batches = (n_list + B - 1) / B;
  if (!warp_done && n_batches > 0) {
    // batch i = list positions [B i, B i + B); batch i + 1 is gathered and
    // the entry ids of batch i + 2 are loaded while batch i is evaluated
    uint32_t e_next[R];
    bool v_next[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t q = r * 32 + lane;
      v_next[r] = q < n_list;
      e_next[r] = v_next[r] ? __ldg(vals + q) : 0u;
    }
    warp_stage<R>(S, 0, rec, e_next, v_next, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t q = B + r * 32 + lane;
      e_next[r] = (n_batches > 1 && q < n_list) ? __ldg(vals + q) : 0u;
    }
    for (uint32_t i = 0; i < n_batches && !warp_done; ++i) {
      const uint32_t p0 = i * B;
      const int k = (int)(i & 1);
      if (i + 1 < n_batches) {
#pragma unroll
        for (int r = 0; r < R; ++r) v_next[r] = p0 + B + r * 32 + lane < n_list;
        warp_stage<R>(S, k ^ 1, rec, e_next, v_next, lane);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t q = p0 + 2 * B + r * 32 + lane;
          e_next[r] = (i + 2 < n_batches && q < n_list) ? __ldg(vals + q) : 0u;
        }
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
      unsigned m;
      {
        const int sl = rr * 32 + lane;
        const float4 a = S.a[k][sl], b = S.b[k][sl];
        int ox, oy;
        rec_origin(S.c[k][sl].w, ox, oy);
        const bool hit = b.z >= 0.0f &&
                         ellipse_hits_box(a.x, a.y, a.z, a.w, b.x, fmaf(b.z, 2.0f * kHPad, b.z) + 1e-3f,
                                          (float)(bx - ox) + 0.5f, (float)(bx - ox + 8 * PW) - 0.5f,
                                          (float)(by - oy) + 0.5f, (float)(by - oy + 4 * PH) - 0.5f);
        m = __ballot_sync(0xffffffffu, hit);
      }
      while (m && !warp_done) {
        const int si = rr * 32 + __ffs(m) - 1;
        m &= m - 1;
        const float4 a = S.a[k][si], b = S.b[k][si], c = S.c[k][si];
        const float cb2 = 2.0f * a.w, inv_nu = mufu_rcp(b.w);
        const float oabs = fabsf(b.y), osgn = copysignf(1.0f, b.y);
        int ox, oy;
        rec_origin(c.w, ox, oy);
        const float fbx = (float)(lx - ox), fby = (float)(ly - oy);
        const uint32_t pos1 = p0 + si + 1;
        V dx[NV], dy[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (L == 2) {
            dx[v] = f2(pixel_offset(fbx, (L * v) % PW, a.x), pixel_offset(fbx, (L * v + 1) % PW, a.x));
            dy[v] = f2(pixel_offset(fby, (L * v) / PW, a.y), pixel_offset(fby, (L * v + 1) / PW, a.y));
          } else {
            dx[v] = pixel_offset(fbx, v % PW, a.x);
            dy[v] = pixel_offset(fby, v / PW, a.y);
          }
        }
        // every pixel of the lane through the same straight-line code (no
        // branches between pixels, so their chains interleave); the nu
        // branch is uniform over the warp
        PairEval<V> r[NV];  // the threshold test is taken below, against each pixel's own threshold
        // the alpha clamp is the identity when |o| T2D cannot reach alpha_max;
        // T2D <= 1 up to the rounding of h near 0 (a few 1e-6 at most for
        // nu <= kFastNuMax), hence the margin
        if (b.w <= kFastNuMax && oabs * 1.0001f <= amax) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
            (void)eval_pair_fast<V, false>(dx[v], dy[v], a.z, cb2, b.x, oabs, osgn, b.w, inv_nu, tau, amax, r[v]);
        } else if (b.w <= kFastNuMax) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
            (void)eval_pair_fast(dx[v], dy[v], a.z, cb2, b.x, oabs, osgn, b.w, inv_nu, tau, amax, r[v]);
        } else if (isinf(b.w)) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
            (void)eval_pair_gauss(dx[v], dy[v], a.z, cb2, b.x, oabs, osgn, tau, amax, r[v]);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v)
            (void)eval_pair_slow(dx[v], dy[v], a.z, cb2, b.x, oabs, osgn, b.w, inv_nu, tau, amax, r[v]);
        }
        const V one = vsplat<V>(1.0f), zero = vsplat<V>(0.0f);
        const V cr = vsplat<V>(c.x), cg = vsplat<V>(c.y), cbl = vsplat<V>(c.z);
        // the splat composites onto pixels whose |alpha| reaches their
        // threshold (tau while live); Tn = T (1 - alpha) there, T elsewhere
        V ae[NV], Tn[NV];
        M add[NV];
        bool lane_term = false;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (COUNT) {
#pragma unroll
            for (int kk = 0; kk < L; ++kk) n_eval += isinf(vget(thr[v], kk)) ? 0u : 1u;
          }
          add[v] = vge(vabs(r[v].alpha), thr[v]);
          ae[v] = vsel(add[v], r[v].alpha, zero);
          Tn[v] = vmul(T[v], vsub(one, ae[v]));
          lane_term = lane_term || many(vlt(Tn[v], tmin));
        }
        if (__any_sync(0xffffffffu, lane_term)) {
          // some pixel of the warp stops before this splat: it keeps its T
          // and colour, and its threshold becomes +inf
          bool ld = true;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            float tx[2], ty[2], ax[2], tt[2];
#pragma unroll
            for (int kk = 0; kk < L; ++kk) {
              tx[kk] = vget(Tn[v], kk);
              ty[kk] = vget(thr[v], kk);
              ax[kk] = vget(ae[v], kk);
              tt[kk] = vget(T[v], kk);
              if (tx[kk] < tmin) {
                ty[kk] = __int_as_float(0x7f800000);
                ax[kk] = 0.0f;
                tx[kk] = tt[kk];
              }
              ld = ld && isinf(ty[kk]);
            }
            if constexpr (L == 2) {
              thr[v] = f2(ty[0], ty[1]);
              ae[v] = f2(ax[0], ax[1]);
              Tn[v] = f2(tx[0], tx[1]);
              add[v] = B2{ax[0] != 0.0f, ax[1] != 0.0f};
            } else {
              thr[v] = ty[0];
              ae[v] = ax[0];
              Tn[v] = tx[0];
              add[v] = ax[0] != 0.0f;
            }
          }
          warp_done = __all_sync(0xffffffffu, ld);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const V w = vmul(ae[v], T[v]);
          C[v][0] = vfma(w, cr, C[v][0]);
          C[v][1] = vfma(w, cg, C[v][1]);
          C[v][2] = vfma(w, cbl, C[v][2]);
          T[v] = Tn[v];
#pragma unroll
          for (int kk = 0; kk < L; ++kk) {
            last[L * v + kk] = mget(add[v], kk) ? pos1 : last[L * v + kk];
            if (COUNT) n_contrib += mget(add[v], kk) ? 1u : 0u;
          }
        }
      }
      }
      __syncwarp();  // every lane is done with buffer k before it is refilled
    }
    cp_async_wait<0>();  // no copy into this warp's buffers outlives the loop
  }

  if (COUNT) {
    const uint32_t ne = __reduce_add_sync(0xffffffffu, n_eval), nc = __reduce_add_sync(0xffffffffu, n_contrib);
    if ((threadIdx.x & 31) == 0 && ne) {
      unsigned long long* ctr = reinterpret_cast<unsigned long long*>(ws_ptr<uint32_t>(ws, P.ws_off_ctrl) + 4);
      atomicAdd(ctr, (unsigned long long)nc);
      atomicAdd(ctr + 1, (unsigned long long)ne);
    }
  }
  float* Tout = ws_ptr<float>(ws, P.ws_off_T);
  uint32_t* Lout = ws_ptr<uint32_t>(ws, P.ws_off_last);
  const size_t hw = (size_t)W * H;
  float* img = out_rgb + 3 * (size_t)J.pix_base;
#pragma unroll
  for (int p = 0; p < NPIX; ++p) {
    const int x = lx + p % PW, y = ly + p / PW;
    if (x < W && y < H) {
      const int v = p / L, kk = p % L;
      const size_t o = (size_t)y * W + x;
      const float Tp = vget(T[v], kk);
      img[o] = fmaf(Tp, cfg.bg[0], vget(C[v][0], kk));
      img[hw + o] = fmaf(Tp, cfg.bg[1], vget(C[v][1], kk));
      img[2 * hw + o] = fmaf(Tp, cfg.bg[2], vget(C[v][2], kk));
      Tout[J.pix_base + o] = Tp;
      Lout[J.pix_base + o] = last[p];
    }
  }
}

// Persistent: a grid of as many CTAs as fit on the device at once, whose
// warps take work items from a counter in the workspace (control word 8) in
// index order -- the order of the grid form, which keeps neighbouring tiles'
// records in L2 together -- until none is left.  No warp waits on another.
// The last warp to finish (control word 9 counts them) resets both words, so
// the next render launch on the workspace starts from item 0.
template <int PW, int PH, int R, bool COUNT>
__global__ void __launch_bounds__(64, 16) k_render_fwd(const sss_frame_plan P, void* ws, float* __restrict__ out_rgb,
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
    fwd_item<PW, PH, R, COUNT>(P, ws, out_rgb, item, S);
  }
  queue_retire(queue, lane);
}

template <int PW, int PH, int R>
int launch_depth(const sss_frame_plan& P, void* ws, float* out, cudaStream_t st) {
  const unsigned subs = (unsigned)(P.cfg.tile_w / (16 * PW)) * (unsigned)(P.cfg.tile_h / (16 * PH));
  const uint32_t n_items = 8u * subs * P.n_tiles;  // warps of the grid form
  if (n_items == 0) return SSS_OK;
  if (P.cfg.count_pairs) {
    const unsigned grid = persistent_grid(k_render_fwd<PW, PH, R, true>, 64, n_items / 2);
    k_render_fwd<PW, PH, R, true><<<grid, 64, 0, st>>>(P, ws, out, n_items);
  } else {
    const unsigned grid = persistent_grid(k_render_fwd<PW, PH, R, false>, 64, n_items / 2);
    k_render_fwd<PW, PH, R, false><<<grid, 64, 0, st>>>(P, ws, out, n_items);
  }
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

template <int PW, int PH>
int launch_batch(const sss_frame_plan& P, void* ws, float* out, cudaStream_t st) {
  // records staged per warp and round: cfg.batch = 32 or 64 (checked by the plan)
  return P.cfg.batch == 64 ? launch_depth<PW, PH, 2>(P, ws, out, st) : launch_depth<PW, PH, 1>(P, ws, out, st);
}

}  // namespace
}  // namespace sss

extern "C" int sss_render_fwd(const sss_frame_plan* plan, void* ws, float* out_rgb, sss_stream_t stream) {
  if (!plan || !ws || !out_rgb) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  cudaStream_t st = (cudaStream_t)stream;
  // render sub-tiles of at most 32 x 32 (lanes of up to 2 x 2 pixels)
  const int pw = (P.cfg.tile_w >= 32 ? 32 : P.cfg.tile_w) / 16, ph = (P.cfg.tile_h >= 32 ? 32 : P.cfg.tile_h) / 16;
  if (pw == 1 && ph == 1) return sss::launch_batch<1, 1>(P, ws, out_rgb, st);
  if (pw == 2 && ph == 1) return sss::launch_batch<2, 1>(P, ws, out_rgb, st);
  if (pw == 1 && ph == 2) return sss::launch_batch<1, 2>(P, ws, out_rgb, st);
  if (pw == 2 && ph == 2) return sss::launch_batch<2, 2>(P, ws, out_rgb, st);
  return SSS_ERR_UNSUPPORTED;
}
