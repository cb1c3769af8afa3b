// Host side of libsss: frame plans, workspace layout, status queries.
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool side_ok(int s) { return s == 16 || s == 32 || s == 64 || s == 128; }
bool tile_ok(int w, int h) { return side_ok(w) && side_ok(h); }
bool batch_ok(int b) { return b == 32 || b == 64; }

}  // namespace

extern "C" {

int sss_version(void) { return 100; }

void sss_default_cfg(sss_raster_cfg* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->tile_w = 64;  // list tiles of 64 x 64, rendered as 32 x 32 sub-tiles
  cfg->tile_h = 64;
  cfg->batch = 32;
  cfg->nu_grad_mode = 0;
  cfg->tau = 1.0f / 255.0f;
  cfg->t_min = 1e-4f;
  cfg->alpha_max = 0.99f;
  cfg->znear = 0.2f;
  cfg->lowpass = 0.0f;
  cfg->bwd_box_h = 8;
}

const char* sss_status_string(int status) {
  switch (status) {
    case SSS_OK: return "ok";
    case SSS_ERR_INVALID_ARG: return "invalid argument";
    case SSS_ERR_CAPACITY: return "pair capacity exceeded";
    case SSS_ERR_CUDA: return "CUDA error";
    case SSS_ERR_TIMEOUT: return "bounded device wait expired";
    case SSS_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int sss_plan_frame(const sss_params* scenes, int n_scenes, const sss_camera* cams, const int* job_scene,
                   int n_jobs, const sss_raster_cfg* cfg, uint32_t pair_capacity, sss_frame_plan* plan) {
  if (!scenes || !cams || !job_scene || !cfg || !plan) return SSS_ERR_INVALID_ARG;
  if (n_scenes < 1 || n_scenes > SSS_MAX_SCENES || n_jobs < 1 || n_jobs > SSS_MAX_JOBS) return SSS_ERR_INVALID_ARG;
  if (!tile_ok(cfg->tile_w, cfg->tile_h) || !batch_ok(cfg->batch)) return SSS_ERR_UNSUPPORTED;
  if (cfg->nu_grad_mode != 0 && cfg->nu_grad_mode != 1) return SSS_ERR_INVALID_ARG;
  if (cfg->kernel != 0 && cfg->kernel != 1) return SSS_ERR_INVALID_ARG;
  if (cfg->count_pairs != 0 && cfg->count_pairs != 1) return SSS_ERR_INVALID_ARG;
  if (cfg->bwd_box_h != 8 && cfg->bwd_box_h != 16) return SSS_ERR_INVALID_ARG;
  if (cfg->bwd_box_h == 16 && (cfg->tile_w < 32 || cfg->tile_h < 64)) return SSS_ERR_UNSUPPORTED;
  if (!(cfg->tau > 0.0f && cfg->tau < cfg->alpha_max && cfg->alpha_max < 1.0f && cfg->t_min >= 0.0f &&
        cfg->t_min < 1.0f && cfg->lowpass >= 0.0f))
    return SSS_ERR_INVALID_ARG;
  if (pair_capacity == 0 || pair_capacity > 0x7ffffffcu) return SSS_ERR_INVALID_ARG;
  pair_capacity = (pair_capacity + 3u) & ~3u;  // 16-byte aligned pair slots

  std::memset(plan, 0, sizeof(*plan));
  plan->n_jobs = n_jobs;
  plan->n_scenes = n_scenes;
  plan->cfg = *cfg;
  uint64_t comp_total = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const sss_params& p = scenes[s];
    if (p.n < 0 || p.sh_degree < 0 || p.sh_degree > 3) return SSS_ERR_INVALID_ARG;
    if (p.n > 0 && (!p.mean || !p.log_scale || !p.quat || !p.nu || !p.opacity_raw || !p.sh))
      return SSS_ERR_INVALID_ARG;
    plan->scenes[s] = p;
    plan->scene_comp_base[s] = (uint32_t)comp_total;
    comp_total += (uint64_t)p.n;
  }
  if (comp_total > 0x7fffffffull) return SSS_ERR_INVALID_ARG;
  plan->scene_comp_base[n_scenes] = (uint32_t)comp_total;

  uint64_t entries = 0, tiles = 0, pixels = 0;
  for (int j = 0; j < n_jobs; ++j) {
    int s = job_scene[j];
    if (s < 0 || s >= n_scenes) return SSS_ERR_INVALID_ARG;
    const sss_camera& c = cams[j];
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return SSS_ERR_INVALID_ARG;
    if (!(c.fx > 0.0f) || !(c.fy > 0.0f)) return SSS_ERR_INVALID_ARG;
    sss_job_desc& d = plan->jobs[j];
    d.cam = c;
    d.scene = s;
    d.tiles_x = (c.width + cfg->tile_w - 1) / cfg->tile_w;
    d.tiles_y = (c.height + cfg->tile_h - 1) / cfg->tile_h;
    d.entry_base = (uint32_t)entries;
    d.tile_base = (uint32_t)tiles;
    d.pix_base = (uint32_t)pixels;
    entries += (uint64_t)scenes[s].n;
    tiles += (uint64_t)d.tiles_x * d.tiles_y;
    pixels += (uint64_t)c.width * c.height;
  }
  if (entries > 0x7fffffffull || tiles > 0x7fffffffull || 3 * pixels > 0x7fffffffull) return SSS_ERR_INVALID_ARG;
  plan->n_entries = (uint32_t)entries;
  plan->n_tiles = (uint32_t)tiles;
  plan->n_pixels = (uint32_t)pixels;
  plan->pair_capacity = pair_capacity;
  int bits = 1;
  while ((1ull << bits) < tiles) ++bits;
  plan->tile_bits = bits;

  int k = 0;
  for (int s = 0; s < n_scenes; ++s) {
    plan->scene_job_begin[s] = k;
    for (int j = 0; j < n_jobs; ++j)
      if (job_scene[j] == s) plan->scene_jobs[k++] = j;
  }
  plan->scene_job_begin[n_scenes] = k;

  plan->sort_blocks = 3 * sss::device_sm_count();  // resident CTAs of the radix scatter
  int passes = (bits + 7) / 8;
  plan->pair_slot = (uint32_t)(passes & 1);

  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  plan->ws_off_ctrl = take(64);
  plan->ws_off_rec = take(sizeof(sss::SplatRec) * entries);
  plan->ws_off_dkey = take(4 * entries);
  plan->ws_off_ntiles = take(4 * entries);
  plan->ws_off_rect = take(8 * entries);
  // two slots each; slot 1 starts 16-byte aligned (the sort copies chunks
  // with 16-byte transfers when both of its inputs are aligned)
  plan->ws_off_order = take(2 * 4 * ((entries + 3) & ~3ull));
  plan->ws_off_okey = take(2 * 4 * ((entries + 3) & ~3ull));
  plan->ws_off_pkey = take(2 * 4 * (size_t)pair_capacity);
  plan->ws_off_pval = take(2 * 4 * (size_t)pair_capacity);
  plan->ws_off_ranges = take(8 * tiles);
  plan->ws_off_T = take(4 * pixels);
  plan->ws_off_last = take(4 * pixels);
  plan->ws_off_grad2d = take(48 * entries);
  plan->ws_off_hist = take(4 * (size_t)(256 + 4) * (plan->sort_blocks + 1));
  plan->ws_bytes = off;
  return SSS_OK;
}

int sss_read_status(const sss_frame_plan* plan, const void* ws, uint32_t* status_bits, uint32_t* pairs_needed,
                    uint32_t* pairs_sorted, sss_stream_t stream) {
  if (!plan || !ws) return SSS_ERR_INVALID_ARG;
  uint32_t ctrl[16];
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SSS_ERR_CUDA;
  if (cudaMemcpy(ctrl, sss::ws_ptr<uint32_t>(ws, plan->ws_off_ctrl), sizeof(ctrl), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return SSS_ERR_CUDA;
  if (status_bits) *status_bits = ctrl[sss::kCtrlStatus];
  if (pairs_needed) *pairs_needed = ctrl[sss::kCtrlPairsNeeded];
  if (pairs_sorted) *pairs_sorted = ctrl[sss::kCtrlPairsSorted];
  return SSS_OK;
}

}  // extern "C"
