// a4: per-pixel front-to-back compositing with signed alpha
// (Sec. 3.4 Eq. SSS_color; signed opacity Sec. 3.3).
//
// One CTA of 256 threads per image tile of (16 PW) x (16 PH) pixels.  Warps
// are laid out 2 x 4 over the tile; warp w owns an (8 PW) x (4 PH) box and
// lane l a PW x PH block of pixels inside it.  The tile's splat list is
// staged in shared memory B splats at a time (48-byte records gathered by
// entry index, double buffered: the next batch is loaded while this one is
// processed).  Each warp then tests the B staged splats against its own
// box in parallel (one splat per lane, exact ellipse/box test) and walks
// only the survivors, in list (= depth) order, so pairs whose ellipse misses
// the warp's 32 PW PH pixels cost nothing.  A warp stops evaluating when all
// its pixels are done; the CTA stops staging when all warps are done.
#include "common.cuh"

namespace sss {
namespace {

template <int PW, int PH, int B>
__global__ void __launch_bounds__(256) k_render_fwd(const sss_frame_plan P, void* ws, float* __restrict__ out_rgb) {
  constexpr int NPIX = PW * PH;
  constexpr int TW = 16 * PW, TH = 16 * PH;
  constexpr int NW = B / 32;
  __shared__ float4 s_buf[2][3 * B];

  const uint32_t tile = blockIdx.x;
  const int j = job_of_tile(P, tile);
  const sss_job_desc& J = P.jobs[j];
  const sss_raster_cfg& cfg = P.cfg;
  const uint32_t lt = tile - J.tile_base;
  const int tx = (int)(lt % (uint32_t)J.tiles_x), ty = (int)(lt / (uint32_t)J.tiles_x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = tx * TW + (warp & 1) * 8 * PW, by = ty * TH + (warp >> 1) * 4 * PH;
  const int lx = bx + (lane & 7) * PW, ly = by + (lane >> 3) * PH;
  const int W = J.cam.width, H = J.cam.height;

  float T[NPIX], C[NPIX][3];
  uint32_t last[NPIX];
  bool done[NPIX];
#pragma unroll
  for (int p = 0; p < NPIX; ++p) {
    const int x = lx + p % PW, y = ly + p / PW;
    done[p] = !(x < W && y < H);
    T[p] = 1.0f;
    C[p][0] = C[p][1] = C[p][2] = 0.0f;
    last[p] = 0u;
  }
  bool lane_done = true;
#pragma unroll
  for (int p = 0; p < NPIX; ++p) lane_done = lane_done && done[p];
  bool warp_done = __all_sync(0xffffffffu, lane_done);

  const uint2 range = ws_ptr<uint2>(ws, P.ws_off_ranges)[tile];
  const uint32_t* vals = ws_ptr<uint32_t>(ws, P.ws_off_pval) + (size_t)P.pair_slot * P.pair_capacity;
  const SplatRec* rec = ws_ptr<SplatRec>(ws, P.ws_off_rec);
  const float tau = cfg.tau, amax = cfg.alpha_max, tmin = cfg.t_min;
  uint32_t n_eval = 0, n_contrib = 0;  // pair counters for the roofline

  const uint32_t n_list = range.y - range.x;
  const uint32_t n_batches = (n_list + B - 1) / B;
  Stager<B> stg;
  if (n_batches > 0) {
    uint32_t e0[Stager<B>::kL];
    stg.fetch_entries(vals, range.x, min((uint32_t)B, n_list), e0);
    stg.load_records(rec, e0);
    if (n_batches > 1) stg.fetch_entries(vals, range.x + B, min((uint32_t)B, n_list - B), stg.e_next);
    stg.store(s_buf[0], nullptr, e0);
  }
  __syncthreads();
  for (uint32_t i = 0; i < n_batches; ++i) {
    const uint32_t b0 = range.x + i * B;
    // records of batch i+1 and entry ids of batch i+2 go in flight now
    uint32_t e_after[Stager<B>::kL];
    if (i + 1 < n_batches) {
      stg.load_records(rec, stg.e_next);
      if (i + 2 < n_batches) stg.fetch_entries(vals, b0 + 2 * B, min((uint32_t)B, range.y - (b0 + 2 * B)), e_after);
    }
    const float4* s_a = s_buf[i & 1];
    const float4* s_b = s_a + B;
    const float4* s_c = s_a + 2 * B;
    if (!warp_done) {
      unsigned mask[NW];
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        const float4 a = s_a[k * 32 + lane], b = s_b[k * 32 + lane];
        int ox, oy;
        rec_origin(s_c[k * 32 + lane].w, ox, oy);
        const bool hit = b.z >= 0.0f &&
                         ellipse_hits_box(a.x, a.y, a.z, a.w, b.x, fmaf(b.z, 2.0f * kHPad, b.z) + 1e-3f,
                                          (float)(bx - ox) + 0.5f, (float)(bx - ox + 8 * PW) - 0.5f,
                                          (float)(by - oy) + 0.5f, (float)(by - oy + 4 * PH) - 0.5f);
        mask[k] = __ballot_sync(0xffffffffu, hit);
      }
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        unsigned m = mask[k];
        while (m && !warp_done) {
          const int bit = __ffs(m) - 1;
          m &= m - 1;
          const int si = k * 32 + bit;
          const float4 a = s_a[si], b = s_b[si], c = s_c[si];
          const float cb2 = 2.0f * a.w, hpre = fmaf(b.z, kHPad, b.z), inv_nu = __fdividef(1.0f, b.w);
          int ox, oy;
          rec_origin(c.w, ox, oy);
          const float fbx = (float)(lx - ox), fby = (float)(ly - oy);
          const uint32_t pos1 = b0 + si - range.x + 1;
          // every pixel of the lane through the same straight-line code (no
          // branches between pixels, so their chains interleave); the nu
          // branch is uniform over the warp
          PairEval r[NPIX];
          bool ok[NPIX];
          if (b.w <= kFastNuMax) {
#pragma unroll
            for (int p = 0; p < NPIX; ++p)
              ok[p] = eval_pair_fast(pixel_offset(fbx, p % PW, a.x), pixel_offset(fby, p / PW, a.y), a.z, cb2,
                                     b.x, hpre, b.y, b.w, inv_nu, tau, amax, r[p]);
          } else if (isinf(b.w)) {
#pragma unroll
            for (int p = 0; p < NPIX; ++p)
              ok[p] = eval_pair_gauss(pixel_offset(fbx, p % PW, a.x), pixel_offset(fby, p / PW, a.y), a.z, cb2,
                                      b.x, hpre, b.y, tau, amax, r[p]);
          } else {
#pragma unroll
            for (int p = 0; p < NPIX; ++p)
              ok[p] = eval_pair(pixel_offset(fbx, p % PW, a.x), pixel_offset(fby, p / PW, a.y), a.z, cb2, b.x,
                                hpre, b.y, b.w, inv_nu, tau, amax, r[p]);
          }
#pragma unroll
          for (int p = 0; p < NPIX; ++p) {
            n_eval += done[p] ? 0u : 1u;
            const bool live = ok[p] && !done[p];
            const float Tn = T[p] * (1.0f - r[p].alpha);
            const bool term = live && Tn < tmin;  // stops before this splat
            const bool add = live && !term;
            const float w = add ? r[p].alpha * T[p] : 0.0f;
            C[p][0] = fmaf(w, c.x, C[p][0]);
            C[p][1] = fmaf(w, c.y, C[p][1]);
            C[p][2] = fmaf(w, c.z, C[p][2]);
            T[p] = add ? Tn : T[p];
            last[p] = add ? pos1 : last[p];
            done[p] = done[p] || term;
            n_contrib += add ? 1u : 0u;
          }
          bool ld = true;
#pragma unroll
          for (int p = 0; p < NPIX; ++p) ld = ld && done[p];
          warp_done = __all_sync(0xffffffffu, ld);
        }
      }
    }
    if (i + 1 < n_batches) {
      stg.store(s_buf[(i + 1) & 1], nullptr, stg.e_next);
#pragma unroll
      for (int l = 0; l < Stager<B>::kL; ++l) stg.e_next[l] = e_after[l];
    }
    // one barrier per batch: the next buffer is complete and every warp is
    // done with this one; also the CTA-wide early exit
    if (__syncthreads_count(!warp_done) == 0) break;
  }

  {
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
      const size_t o = (size_t)y * W + x;
      img[o] = fmaf(T[p], cfg.bg[0], C[p][0]);
      img[hw + o] = fmaf(T[p], cfg.bg[1], C[p][1]);
      img[2 * hw + o] = fmaf(T[p], cfg.bg[2], C[p][2]);
      Tout[J.pix_base + o] = T[p];
      Lout[J.pix_base + o] = last[p];
    }
  }
}

template <int PW, int PH>
int launch_batch(const sss_frame_plan& P, void* ws, float* out, cudaStream_t st) {
  const unsigned grid = P.n_tiles;
  switch (P.cfg.batch) {
    case 32: k_render_fwd<PW, PH, 32><<<grid, 256, 0, st>>>(P, ws, out); break;
    case 64: k_render_fwd<PW, PH, 64><<<grid, 256, 0, st>>>(P, ws, out); break;
    case 128: k_render_fwd<PW, PH, 128><<<grid, 256, 0, st>>>(P, ws, out); break;
    case 256: k_render_fwd<PW, PH, 256><<<grid, 256, 0, st>>>(P, ws, out); break;
    default: return SSS_ERR_UNSUPPORTED;
  }
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

}  // namespace
}  // namespace sss

extern "C" int sss_render_fwd(const sss_frame_plan* plan, void* ws, float* out_rgb, sss_stream_t stream) {
  if (!plan || !ws || !out_rgb) return SSS_ERR_INVALID_ARG;
  const sss_frame_plan& P = *plan;
  cudaStream_t st = (cudaStream_t)stream;
  const int pw = P.cfg.tile_w / 16, ph = P.cfg.tile_h / 16;
  if (pw == 1 && ph == 1) return sss::launch_batch<1, 1>(P, ws, out_rgb, st);
  if (pw == 2 && ph == 1) return sss::launch_batch<2, 1>(P, ws, out_rgb, st);
  if (pw == 1 && ph == 2) return sss::launch_batch<1, 2>(P, ws, out_rgb, st);
  if (pw == 2 && ph == 2) return sss::launch_batch<2, 2>(P, ws, out_rgb, st);
  return SSS_ERR_UNSUPPORTED;
}
