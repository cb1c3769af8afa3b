/*
 * sss.h -- C ABI of libsss, a GB300 (sm_103a) rasterizer for 3D Student
 * Splatting and Scooping (SSS, arXiv 2503.10148).
 *
 * The hot path of the method, one entry point per step:
 *
 *   sss_project      3D t-components -> 2D t-splats         Sec. 3.2 Eq. (t_2D)
 *   sss_bin          depth order + (tile, component) pairs   tile rasterizer of 3DGS
 *   sss_sort         stable radix sort on tile, tile ranges  (SM "Implementation Details")
 *   sss_render_fwd   signed-alpha front-to-back composite    Sec. 3.4 Eq. (SSS_color)
 *   sss_render_bwd   closed-form backward to the 2D splats   SM "Backward Pass"
 *   sss_project_bwd  2D splat gradients -> parameters        SM "Backward Pass" (chain rule)
 *   sss_sghmc_step   SGHMC on mu, Adam on the rest           Sec. 3.4 Eq. (sigmoidUpdate), SM Eq. (SGHMC)
 *   sss_loss_l1      L1 image loss and its gradient          Sec. 3.4 loss (L1 term)
 *   sss_loss_l1_grad its gradient scaled by a device dL/dloss Sec. 3.4 loss (L1 term)
 *   sss_loss_image   L1 + D-SSIM over a frame's images      Sec. 3.4 loss
 *   sss_loss_image_grad  its gradient                       Sec. 3.4 loss
 *   sss_regularizers opacity and scale regularisers         Sec. 3.4 loss
 *   sss_relocate     component recycling                    Sec. 3.4, Eq. relocation
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (SSS_OK = 0 or a negative
 *    SSS_ERR_*); no exception or abort crosses the ABI.  Host-side argument
 *    errors are reported before anything is enqueued.
 *  - Ownership: the caller owns every buffer.  The library allocates no device
 *    or host memory; it reads and writes the buffers it is given plus one
 *    caller-provided workspace whose size sss_plan_frame reports.
 *  - Asynchrony: every device-side call enqueues kernels (and memsets) on the
 *    given stream and returns without synchronising, so a whole frame can be
 *    captured into a CUDA graph.  Data-dependent sizes (the number of
 *    tile/splat pairs) stay on the device; an overflow of the caller's pair
 *    capacity sets a bit in the workspace status word, read with
 *    sss_read_status after the stream has progressed.
 *  - Layout: row-major; per-component fields are planar float32 arrays
 *    [dim][n] (field row d of component i at d*n + i).
 *  - Streams: sss_stream_t is a cudaStream_t (0 = legacy default stream).
 *
 * Readings of points the paper leaves open (truncation rule, alpha clamp,
 * early termination with negative alpha, colour model, projection details,
 * the nu gradient, the SGHMC gate and noise scale) are stated at the fields
 * they govern below.
 */
#ifndef SSS_H
#define SSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sss_stream_t;

/* ---------------------------------------------------------------- status */
#define SSS_OK 0
#define SSS_ERR_INVALID_ARG (-1) /* a size, pointer or option is out of range */
#define SSS_ERR_CAPACITY (-2)    /* pairs needed exceed the pair capacity      */
#define SSS_ERR_CUDA (-3)        /* a CUDA launch or copy failed               */
#define SSS_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up         */
#define SSS_ERR_UNSUPPORTED (-5) /* option not built (e.g. tile size)          */

/* Bits of the device status word (sss_read_status). */
#define SSS_STATUS_PAIR_OVERFLOW 1u

/* ---------------------------------------------------------------- limits */
#define SSS_MAX_JOBS 64   /* (scene, camera) jobs in one frame */
#define SSS_MAX_SCENES 8  /* distinct scenes in one frame       */

/* --------------------------------------------------------------- scene */
/* One mixture of 3D Student's t components (Sec. 3.2 Eq. t-dist).
 * Device pointers, planar float32 [dim][n]:
 *   mean        [3][n]   component centre mu
 *   log_scale   [3][n]   S = diag(exp(log_scale)); Sigma = R S S^T R^T (Sec. 3.1)
 *   quat        [4][n]   rotation (w, x, y, z); normalised before use
 *   nu          [n]      degrees of freedom; limited to [1, 1e4] before use
 *                        (SM "Implementation Details"); gradient is zero
 *                        where the limit binds
 *   opacity_raw [n]      o = tanh(opacity_raw) in (-1, 1); o > 0 splats,
 *                        o < 0 scoops (Sec. 3.3)
 *   sh          [3K][n]  real spherical-harmonic colour, K = (sh_degree+1)^2,
 *                        row 3k + c = coefficient k of channel c; basis with
 *                        the Condon-Shortley phase, index l*l + l + m.
 * The rasterizer only reads these; sss_sghmc_step updates them in place. */
typedef struct sss_params {
  float* mean;
  float* log_scale;
  float* quat;
  float* nu;
  float* opacity_raw;
  float* sh;
  int32_t n;         /* components, >= 0 */
  int32_t sh_degree; /* 0..3 */
} sss_params;

/* ------------------------------------------------------------- camera */
/* Pinhole camera.  viewmat = row-major 3x4 [W | t] world -> camera (the
 * affine map of Eq. t_2D); camera axes x right, y down, z forward.
 * Pixel (i, j) is sampled at (i + 0.5, j + 0.5). */
typedef struct sss_camera {
  float viewmat[12];
  float fx, fy, cx, cy;
  int32_t width, height; /* 1 .. 16384 */
} sss_camera;

/* ------------------------------------------------------ raster options */
typedef struct sss_raster_cfg {
  int32_t tile_w, tile_h; /* 16, 32, 64 (default) or 128 pixels each: the
                             tiles of the pair lists; the render runs
                             sub-tiles of at most 32 x 32 (eight warps,
                             lanes of up to 2 x 2 pixels; 32 x 64 and 2 x 4
                             in the backward with bwd_box_h = 16), each
                             walking its tile's whole list                 */
  int32_t batch;          /* records each warp stages in shared memory per
                             round (double buffered, cp.async): 32 or 64,
                             one or two per lane                          */
  int32_t nu_grad_mode;   /* 0: exact dT/dnu (default); 1: the SM's printed
                             form, which omits -1/2 ln(1 + h/nu) T2D          */
  float tau;              /* alpha threshold, 1/255: a splat contributes to a
                             pixel iff |o T2D| >= tau (our reading of the SM's
                             nu-dependent truncation); the screen extent is
                             the box of the ellipse h <= h_max with
                             h_max = nu ((|o|/tau)^(2/(nu+2)) - 1)            */
  float t_min;            /* early termination, 1e-4: stop before the splat
                             that would bring the transmittance below t_min;
                             0 disables (transmittance can rise when o < 0)   */
  float alpha_max;        /* alpha limited to [-alpha_max, alpha_max], 0.99  */
  float znear;            /* components with camera z <= znear are culled,
                             0.2; decided on the FP32 depth key              */
  float lowpass;          /* added to the diagonal of Sigma2D; 0 in the
                             paper's final model, 0.3 in its ablation         */
  float bg[3];            /* background colour                                */
  int32_t kernel;         /* 0: Student's t (default); 1: Gaussian, the limit
                             nu -> infinity, T2D = exp(-h/2) with extent
                             h <= 2 ln(|o|/tau) and no nu gradient (the
                             paper's "SGHMC + 3DGS" ablation kernel)          */
  int32_t count_pairs;    /* 0 (default): no counting; 1: the forward also
                             counts evaluated and contributing (splat,
                             pixel) pairs into ctrl[4..7] (a diagnostic for
                             work figures; costs a few % of the forward)     */
  int32_t bwd_box_h;      /* height in pixels of a warp's box in the backward
                             render: 8 (default; 16 x 8 boxes, 2 x 2 pixels
                             per lane) or 16 (16 x 16 boxes, 2 x 4 pixels per
                             lane; needs tile_w >= 32 and tile_h >= 64).  A
                             box twice as high halves the per-splat work of
                             large splats at a lower occupancy: a choice per
                             workload, not a change of any result's value   */
} sss_raster_cfg;

/* Fills *cfg with the defaults quoted above. */
void sss_default_cfg(sss_raster_cfg* cfg);

/* ---------------------------------------------------------- frame plan */
/* A frame is a batch of jobs; job j renders scene job_scene[j] through
 * camera cams[j].  Views of one scene share one parameter read in
 * sss_project.  The plan is plain data: it may be copied, kept and reused
 * for any number of frames with the same scenes, cameras and options.
 *
 * Entries: job j owns entries [entry_base[j], entry_base[j] + n of its
 * scene); entry e = entry_base[j] + i is component i seen by job j.
 * Tiles: job j owns global tiles [tile_base[j], tile_base[j] + tiles_x[j] *
 * tiles_y[j]), row-major.  Pixels: job j owns pixels [pix_base[j],
 * pix_base[j] + width*height); image outputs are [3][H][W] per job at
 * 3 * pix_base[j] floats, per-pixel scalars at pix_base[j].
 *
 * Workspace: ws_bytes bytes, 256-byte aligned, owned by the caller; each
 * ws_off_* field is the byte offset of a region documented below. */
typedef struct sss_job_desc {
  sss_camera cam;
  int32_t scene;
  int32_t tiles_x, tiles_y;
  uint32_t entry_base;
  uint32_t tile_base;
  uint32_t pix_base;
} sss_job_desc;

typedef struct sss_frame_plan {
  int32_t n_jobs, n_scenes;
  sss_raster_cfg cfg;
  sss_params scenes[SSS_MAX_SCENES];
  uint32_t scene_comp_base[SSS_MAX_SCENES + 1]; /* prefix of scene sizes */
  sss_job_desc jobs[SSS_MAX_JOBS];               /* in the caller's order */
  int32_t scene_jobs[SSS_MAX_JOBS];              /* job indices grouped by
                                                    scene                   */
  int32_t scene_job_begin[SSS_MAX_SCENES + 1];   /* jobs of scene s are
                                                    scene_jobs[begin[s] ..
                                                    begin[s+1])            */
  uint32_t n_entries, n_tiles, n_pixels;
  uint32_t pair_capacity;
  int32_t tile_bits; /* ceil(log2(n_tiles)) */
  /* workspace regions (byte offsets) */
  size_t ws_bytes;
  size_t ws_off_rec;     /* float4[3][n_entries]: 2D splat records:
                            {mean2D - origin, conic a, conic b},
                            {conic c, o, h_max, nu}, {rgb, origin bits}
                            with origin = the integer pixel nearest to
                            mean2D, limited to [0, 16384]
                            (x | y << 16)                                   */
  size_t ws_off_dkey;    /* uint32[n_entries]: FP32 depth-key bits          */
  size_t ws_off_ntiles;  /* uint32[n_entries]: tiles touched                */
  size_t ws_off_rect;    /* uint2[n_entries]: tile rect (x0|x1<<16, y0|y1<<16) */
  size_t ws_off_order;   /* uint32[2][n4]: depth-sorted entries (slot 0),
                            n4 = n_entries rounded up to a multiple of 4    */
  size_t ws_off_okey;    /* uint32[2][n4]: sort keys (ping-pong)            */
  size_t ws_off_pkey;    /* uint32[2][pair_capacity]: tile key per pair     */
  size_t ws_off_pval;    /* uint32[2][pair_capacity]: entry per pair        */
  size_t ws_off_ranges;  /* uint2[n_tiles]: [start, end) per tile           */
  size_t ws_off_T;       /* float[n_pixels]: final transmittance            */
  size_t ws_off_last;    /* uint32[n_pixels]: 1 + list position of the last
                            contributor in the tile's range (0 = none)      */
  size_t ws_off_grad2d;  /* float[n_entries][12]: dL/d(mean2D x,y, conic
                            a,b,c, o, nu, r,g,b, -, -)                     */
  size_t ws_off_hist;    /* scratch for the radix sort and the scans        */
  size_t ws_off_ctrl;    /* uint32[16]: [0] pairs needed, [1] pairs sorted,
                            [2] status bits, [3] entries, [4..5] uint64
                            contributing (splat, pixel) pairs and [6..7]
                            uint64 evaluated pairs of the forwards run with
                            cfg.count_pairs = 1, [8..9] the work-item
                            counter and finished-warp count of the
                            persistent render kernels (back to 0 after each
                            render launch); reset by sss_bin                 */
  int32_t sort_blocks;   /* persistent CTAs used by the sorts and scans     */
  uint32_t pair_slot;    /* which half of pkey/pval holds the sorted pairs  */
} sss_frame_plan;

/* Host only.  Builds a plan for n_jobs jobs.  scenes[s] holds device
 * pointers (not dereferenced here); job_scene[j] in [0, n_scenes).
 * pair_capacity bounds the (tile, splat) pairs of one frame; the plan
 * rounds it up to a multiple of 4 (plan->pair_capacity), so that both pair
 * slots start 16-byte aligned; at most 2^31 - 4.
 * Errors: SSS_ERR_INVALID_ARG for counts outside the limits, sh_degree not in
 * 0..3, non-positive image sizes, a job referring to a missing scene, totals
 * above 2^31; SSS_ERR_UNSUPPORTED for a tile size or batch not built. */
int sss_plan_frame(const sss_params* scenes, int n_scenes, const sss_camera* cams, const int* job_scene,
                   int n_jobs, const sss_raster_cfg* cfg, uint32_t pair_capacity, sss_frame_plan* plan);

/* ---------------------------------------------------------- hot path */
/* a1. Projects every (job, component) entry: camera-space mean, FP32 depth
 * key, Sigma = R S S^T R^T, EWA Jacobian J at the mean (x/z and y/z limited
 * to 1.3 x the half-FOV tangent), Sigma2D = (J W Sigma W^T J^T)_{1:2,1:2} +
 * lowpass I, conic = Sigma2D^-1, mean2D, o = tanh(raw), nu limited to [1,1e4],
 * h_max, the screen box and tile rectangle, and the view-dependent colour
 * max(SH . Y(dir) + 0.5, 0), dir = normalised (mu - camera centre).  Culled
 * entries (behind znear, singular Sigma2D, |o| < tau) touch no tile.
 * ws: the plan's workspace.  Errors: SSS_ERR_INVALID_ARG (null plan or ws),
 * SSS_ERR_CUDA (launch failure). */
int sss_project(const sss_frame_plan* plan, void* ws, sss_stream_t stream);

/* a2. Orders all entries by (FP32 depth key, entry index) with a stable LSD
 * radix sort, scans their tile counts in that order and emits one
 * (global tile id, entry) pair per touched tile, rectangle rows in order.
 * Pairs beyond pair_capacity are not written; the status word gets
 * SSS_STATUS_PAIR_OVERFLOW and ctrl[0] the number needed. */
int sss_bin(const sss_frame_plan* plan, void* ws, sss_stream_t stream);

/* a3. Stable LSD radix sort of the pairs on the tile id (tile_bits bits).
 * Because pairs were emitted in depth order, the result is the pair list
 * sorted by (tile, depth key, entry), i.e. the (tile | depth) key order with
 * ties broken by component index.  Then the [start, end) range of every
 * tile.  Sorts min(needed, capacity) pairs. */
int sss_sort(const sss_frame_plan* plan, void* ws, sss_stream_t stream);

/* a4. Per pixel, front to back over its tile's range:
 *   alpha = clamp(o T2D(h), -alpha_max, alpha_max), T2D = (1 + h/nu)^-(nu+2)/2,
 *   skipped when |o T2D| < tau; C += rgb alpha T; T *= (1 - alpha); stop
 *   before a splat that would make T < t_min; finally C += T bg.
 * out_rgb: device float[3 * n_pixels], [3][H][W] per job at 3*pix_base[j].
 * Also writes the final T and last-contributor positions into ws.  Runs as
 * a persistent grid (as many CTAs as are resident at once) whose warps take
 * (sub-tile, warp box) items from a counter in the workspace; two render
 * launches on one workspace must therefore not overlap on the GPU. */
int sss_render_fwd(const sss_frame_plan* plan, void* ws, float* out_rgb, sss_stream_t stream);

/* a5. Given dL/dC (device float[3 * n_pixels], same layout as out_rgb),
 * walks every pixel's contributors back to front, recovering T_k =
 * T_{k+1} / (1 - alpha_k), and accumulates into the workspace's grad2d:
 *   dL/drgb = alpha T dL/dC,  dL/dalpha = dL/dC . (T rgb - S / (1 - alpha)),
 *   dalpha/do = T2D, dT2D/dh = -(nu+2)/(2nu) (1 + h/nu)^-(nu+4)/2,
 *   dT2D/dnu = T2D [-1/2 ln(1 + h/nu) + (nu+2) h / (2 nu^2 (1 + h/nu))],
 *   dh/dmean2D, dh/dconic,
 * S being the colour composited behind the splat plus T_final bg.  Needs the
 * workspace state of sss_render_fwd of the same frame. */
int sss_render_bwd(const sss_frame_plan* plan, void* ws, const float* dL_drgb, sss_stream_t stream);

/* a6. Chains the 2D gradients of every job of scene s back to scene s's
 * parameters (through mean2D, J, Sigma, the quaternion, the SH colour and
 * its viewing direction, tanh and the nu limit) and sums over the jobs.
 * grads[s] gives device arrays with the parameter layout (overwritten).
 * grads must hold plan->n_scenes entries with n and sh_degree matching. */
int sss_project_bwd(const sss_frame_plan* plan, void* ws, const sss_params* grads, sss_stream_t stream);

/* a7. One sampler step on one scene, in place (Sec. 3.4, SM "SGHMC").
 *   o = tanh(opacity_raw), gate g = sigmoid(-k (|o| - t0)) (k = 100,
 *   t0 = 0.005: open for components more transparent than 0.005),
 *   xi ~ N(0, I3): Box-Muller on Philox4x32-10 of counter (i, 0, step_lo,
 *   step_hi) and key (seed_lo, seed_hi), u1 = ((w0 >> 8) + 1) 2^-24,
 *   u2 = (w1 >> 8) 2^-24 (and w2, w3 for the third normal),
 *   r'  = (1 - eps C) r - eps G + sqrt(2 eps C) xi,      G = dL/dmu
 *   mu' = mu - eps^2 G + g eps (1 - eps C) r + g eps sqrt(2 eps C) xi,
 *   burn-in: mu' = mu - eps^2 G + g eps sqrt(2 eps C) Sigma xi (no friction).
 * Adam (bias-corrected, t = step + 1) on log_scale, quat, nu, opacity_raw,
 * sh with lr[0..4]; nu limited to [1, 1e4] afterwards.
 * The regularisers of the loss (Sec. 3.4) enter here, their gradients being
 * closed forms of the parameters: Adam sees G + reg_opacity sign(o)(1 - o^2)
 * for opacity_raw (d/draw of reg_opacity |o|) and G + reg_scale exp(s_j) for
 * log_scale_j (d/ds_j of reg_scale sqrt(lambda_j), sqrt(lambda_j) being the
 * scale exp(s_j)); zero weights leave the step unchanged.
 *   momentum   device float[3][n]
 *   adam_m/v   device float[(9 + 3K)][n]: rows log_scale(3), quat(4), nu,
 *              opacity_raw, sh(3K)
 *   xi_out     optional device float[3][n] (NULL to skip) */
typedef struct sss_step_params {
  float eps, C, k, t0;
  int32_t burn_in;
  uint64_t seed, step;
  float lr[5];
  float beta1, beta2, adam_eps;
  uint64_t* step_counter; /* optional device counter: when non-NULL the step
                             index is read from it (instead of `step`) and
                             incremented by one after the update, so a
                             graph-replayed step draws fresh noise and
                             bias-corrects with the right t */
  float reg_opacity;      /* eps_o of the loss, >= 0 */
  float reg_scale;        /* eps_Sigma of the loss, >= 0 */
  float* mu_adam_m;       /* optional device float[3][n] (both or neither):
                             Adam moments of dL/dmu; when given, G in the
                             SGHMC update is Adam's m^ / (sqrt(v^) + adam_eps)
                             of dL/dmu (Implementation Details: the Adam
                             gradient in SGHMC) and the moments are updated */
  float* mu_adam_v;
  uint32_t* philox_out;   /* optional device uint32[4][n] (NULL to skip):
                             the four Philox4x32-10 words each component's
                             normals were drawn from (row w = word w), so a
                             caller can check the generator bit for bit */
} sss_step_params;

int sss_sghmc_step(const sss_params* params, const sss_params* grads, float* momentum, float* adam_m,
                   float* adam_v, const sss_step_params* sp, float* xi_out, sss_stream_t stream);

/* The same step with the updated parameters written to params_out (device
 * arrays of the same layout, n and sh_degree) instead of over params, which
 * it then only reads; momentum, the Adam moments and the step counter are
 * updated in place as above.  params_out's arrays are either params' own
 * (the step in place: sss_sghmc_step is this call with params_out = params)
 * or arrays that overlap none of params'.  Lets a caller keep the pre-step
 * parameters, e.g. to run repeated steps from one configuration without
 * copying it back.  Errors as sss_sghmc_step, and SSS_ERR_INVALID_ARG for a
 * NULL params_out or one whose n or sh_degree differs. */
int sss_sghmc_step_to(const sss_params* params, const sss_params* params_out, const sss_params* grads,
                      float* momentum, float* adam_m, float* adam_v, const sss_step_params* sp, float* xi_out,
                      sss_stream_t stream);

/* L1 term of the loss (Sec. 3.4): loss_out[0] = sum |pred - target| / count
 * (overwritten; the partial sums are added in an unspecified order) and,
 * when dL_dpred is not NULL, dL_dpred = sign(pred - target) / count (0 where
 * equal).  count floats; pred, target, dL_dpred device arrays, loss_out one
 * device float. */
int sss_loss_l1(const float* pred, const float* target, uint32_t count, float* dL_dpred, float* loss_out,
                sss_stream_t stream);

/* Gradient of the L1 term for a caller that holds dL/dloss on the device
 * (an autograd backward): dL_dpred = dL_dloss[0] * sign(pred - target) /
 * count, dL_dloss[0] taken as 1 when dL_dloss is NULL.  Same layout as
 * sss_loss_l1; dL_dpred is overwritten. */
int sss_loss_l1_grad(const float* pred, const float* target, uint32_t count, const float* dL_dloss,
                     float* dL_dpred, sss_stream_t stream);

/* Image loss of Sec. 3.4 over every image of a frame:
 *   L = (1 - eps_dssim) L1 + eps_dssim (1 - SSIM),
 * L1 and SSIM both averaged over all pixels and channels of all jobs.  SSIM
 * as in 3DGS (the loss the paper cites): 11 x 11 Gaussian window with sigma
 * 1.5 (weights normalised to 1), zero padding outside each image,
 * C1 = 0.01^2, C2 = 0.03^2; windows never cross images.
 *   pred, target  device float[3 * n_pixels], the layout of sss_render_fwd's
 *                 out_rgb for this plan
 *   loss_out      device float[3]: L, L1, 1 - SSIM (overwritten)
 *   scratch       device buffer of sss_loss_image_scratch_bytes(plan)
 *                 bytes, 16-byte aligned: receives the per-pixel SSIM
 *                 partials that sss_loss_image_grad needs.
 * Errors: SSS_ERR_INVALID_ARG for NULL pointers, a misaligned scratch or
 * eps_dssim outside [0, 1]. */
size_t sss_loss_image_scratch_bytes(const sss_frame_plan* plan);
int sss_loss_image(const sss_frame_plan* plan, const float* pred, const float* target, float eps_dssim,
                   float* loss_out, void* scratch, sss_stream_t stream);

/* dL/dpred of sss_loss_image, scaled by dL_dloss[0] (device float; 1 when
 * NULL): (1 - eps) sign(x - y) / count - eps (w*a + 2 x (w*b) + y (w*c)) /
 * count, where a, b, c are the SSIM partials the value call left in
 * `scratch` (same plan, pred and target) and w* the windowed sum.  dL_dpred
 * (overwritten) has the layout of pred. */
int sss_loss_image_grad(const sss_frame_plan* plan, const float* pred, const float* target, float eps_dssim,
                        const float* dL_dloss, const void* scratch, float* dL_dpred, sss_stream_t stream);

/* Value of the regularisers of Sec. 3.4 for one scene:
 *   loss_out[0] = reg_opacity sum_i |tanh(opacity_raw_i)|
 *               + reg_scale sum_i sum_j exp(log_scale_ij)
 * (sqrt(lambda_ij) of Sigma_i = R S S^T R^T is the scale exp(log_scale_ij)).
 * loss_out: one device float, overwritten.  Their gradients are added by
 * sss_sghmc_step (reg_opacity, reg_scale of sss_step_params). */
int sss_regularizers(const sss_params* params, float reg_opacity, float reg_scale, float* loss_out,
                     sss_stream_t stream);

/* Component recycling (Sec. 3.4 "Adding and Recycling Components", Eq.
 * relocation, SM "Component Recycling"), in place on one scene:
 *  - dead: |o| = |tanh(opacity_raw)| < dead_opacity (FP64); the first
 *    floor(max_fraction n) dead components in index order move;
 *  - each draws a target from the multinomial over live components with
 *    weight floor(|o| 2^12): x = word 0 of Philox4x32-10 on counter
 *    (dead rank, 1, step_lo, step_hi) and key (seed_lo, seed_hi),
 *    v = (x W) >> 32 (W the weight total), target = the first index whose
 *    inclusive weight prefix exceeds v;
 *  - a target keeps its first n_max - 1 draws in dead-rank order (later ones
 *    stay dead); with N = 1 + copies, in FP64:
 *      o_new = 1 - (1 - |o|)^(1/N) (sign of o),
 *      Sigma_new = F Sigma_old, F = o^2 (B(1/2, (nu+2)/2) / K)^2,
 *      K = sum_{i=1..N} sum_{k<i} C(i-1,k) (-1)^k o_new^(k+1)
 *          B(1/2, ((k+1)(nu+3)-1)/2), nu kept, B from ln Gamma,
 *    i.e. every log-scale of the target grows by ln(F)/2;
 *  - the copies take the target's mean, quaternion, nu, SH, new opacity and
 *    scale; their momentum and Adam moments (layouts of sss_sghmc_step) are
 *    set to zero.
 *   params     device parameters of the scene, modified in place
 *   moved_out  device uint32: number of components moved (overwritten)
 *   scratch    device buffer of sss_relocate_scratch_bytes(n, max_fraction)
 *              bytes, 256-byte aligned.
 * Errors: SSS_ERR_INVALID_ARG for NULL pointers, a misaligned scratch,
 * max_fraction outside [0, 1], dead_opacity < 0 or n_max outside [2, 64]. */
typedef struct sss_relocate_params {
  float dead_opacity; /* 0.005: the sampler's gate opens below it */
  float max_fraction; /* 0.05: at most 5 % of the components per call */
  int32_t n_max;      /* at most n_max - 1 copies per target */
  uint64_t seed, step;
} sss_relocate_params;

size_t sss_relocate_scratch_bytes(int32_t n, float max_fraction);
int sss_relocate(const sss_params* params, float* momentum, float* adam_m, float* adam_v,
                 const sss_relocate_params* rp, uint32_t* moved_out, void* scratch, sss_stream_t stream);

/* -------------------------------------------- no-allocation forward */
/* No counterpart in the paper.  A forward render of one small frame for
 * callers that cannot allocate device memory when they render: a plug-in in
 * a host application that owns all device memory through its own pool or
 * budget, or a real-time render thread that must not take the allocator's
 * locks or wait for the device synchronisation cudaMalloc can imply.  The
 * whole workspace lives in one file-scope __device__ array of
 * SSS_STATIC_ARENA_BYTES in the library, so the caller passes only the scene,
 * the camera, the options and the output image.
 *   scene    device parameters of one scene, n <= SSS_STATIC_MAX_COMPONENTS
 *   cam      width * height <= SSS_STATIC_MAX_PIXELS
 *   out_rgb  device float[3][height][width]
 * Same computation as sss_project + sss_bin + sss_sort + sss_render_fwd on a
 * one-job frame, bit for bit.  Allocates nothing (no cudaMalloc, cudaFree or
 * allocating library call).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and caches
 * it for the life of the process; a cudaDeviceReset of that device
 * invalidates the cached address, so calls after one are not supported.
 * Every call on a device shares the one array and leaves its contents
 * behind (the kernels reset what must start at zero): calls whose work
 * overlaps on the GPU (other streams or host threads) race, so serialise
 * them.  The call enqueues its kernels on `stream` and then synchronises
 * `stream` (a blocking wait) to read the overflow status before it returns.
 * Errors: SSS_ERR_INVALID_ARG (null pointer, size beyond the limits, bad
 * options; nothing enqueued), SSS_ERR_CAPACITY (the frame's workspace does
 * not fit the array, nothing enqueued; or its tile pairs overflowed the rest
 * of the array, in which case out_rgb holds an incomplete image),
 * SSS_ERR_CUDA. */
#define SSS_STATIC_ARENA_BYTES (32u << 20)
#define SSS_STATIC_MAX_COMPONENTS 65536
#define SSS_STATIC_MAX_PIXELS (1024 * 1024)
int sss_render_static(const sss_params* scene, const sss_camera* cam, const sss_raster_cfg* cfg, float* out_rgb,
                      sss_stream_t stream);

/* ----------------------------------------------------------- status */
/* Synchronises the stream, then copies the workspace control words to the
 * host: status bits, pairs needed, pairs sorted.  Any pointer may be NULL. */
int sss_read_status(const sss_frame_plan* plan, const void* ws, uint32_t* status_bits, uint32_t* pairs_needed,
                    uint32_t* pairs_sorted, sss_stream_t stream);

/* Human-readable text for a status code. */
const char* sss_status_string(int status);

/* Library version (major * 10000 + minor * 100 + patch). */
int sss_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SSS_H */
