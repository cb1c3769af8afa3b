/*
 * sss_oracle.c -- FP64 CPU oracle for the Student Splatting and Scooping
 * (SSS) rasterizer hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes, and the passage each part follows:
 *   - orc_project     one 3D t-component -> 2D t-splat: Sec. 3.2 Eq. (t_2D)
 *                     (mu2D, Sigma2D = (J W Sigma W^T J^T)_{1:2,1:2}),
 *                     Sigma = R S S^T R^T (Sec. 3.1), signed opacity via
 *                     tanh (Sec. 3.3), nu limited to [1, 1e4] and no low-pass
 *                     filter (SM "Implementation Details"), SH colour
 *                     (Sec. 3.1: c in R^27 / R^48 as spherical harmonics).
 *   - orc_render      per-pixel front-to-back composite with signed alpha,
 *                     Sec. 3.4 Eq. (SSS_color), brute force over all
 *                     components sorted by (FP32 depth key, index); no tiles.
 *   - orc_backward    SM "Backward Pass": dL/dalpha from the compositing
 *                     recurrence, dT/dh (SM Eq. for the h(x) trick) and the
 *                     exact dT/dnu; the projection part (dh/dmu', dSigma'/d..)
 *                     is the derivative of the plainly written projection
 *                     taken by the complex-step method (Squire & Trapp 1998),
 *                     exact to rounding.
 *   - orc_sghmc_step  Sec. 3.4 Eq. (sigmoidUpdate) and SM Eq. (SGHMC) on mu,
 *                     Adam (Kingma & Ba 2015) on every other group.
 *   - orc_philox4x32_10  counter-based generator of Salmon et al., SC'11.
 *
 * Readings taken where the paper is silent or inconsistent are listed in the
 * repository's design document; each one is also stated at its use below.
 *
 * Parity notes: every function is a literal restatement; no blocking, fusion
 * or reordering beyond the definition.  The only shortcut is in orc_render:
 * a pair is skipped when h exceeds the value at which |o| T2D equals
 * tau * (1 - 1e-2); that is exactly equivalent to the |alpha| >= tau test it
 * precedes (the skipped pairs all have |alpha| < tau) and keeps the near-tau
 * bookkeeping (windows of at most 1e-2) intact.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

#define ORC_PI 3.14159265358979323846

/* --- parameter layout: planar theta[(12 + 3K) n] ------------------------ */
#define TH_MEAN(n) 0
#define TH_LS(n) (3 * (size_t)(n))
#define TH_Q(n) (6 * (size_t)(n))
#define TH_NU(n) (10 * (size_t)(n))
#define TH_O(n) (11 * (size_t)(n))
#define TH_SH(n) (12 * (size_t)(n))

/* --- projection record, doubles ----------------------------------------- */
enum {
  P_VALID, P_MX, P_MY, P_COV_A, P_COV_B, P_COV_C, P_CON_A, P_CON_B, P_CON_C,
  P_DEPTH, P_O, P_NU, P_R, P_G, P_B, P_CLAMP_R, P_CLAMP_G, P_CLAMP_B, P_HMAX,
  P_PX0, P_PX1, P_PY0, P_PY1, P_TX0, P_TX1, P_TY0, P_TY1, P_NTILES, P_ES, P_STRIDE
};

/* --- 2D gradient record, doubles ---------------------------------------- */
enum { G_MX, G_MY, G_CA, G_CB, G_CC, G_O, G_NU, G_R, G_G, G_B, G_STRIDE };

/* render flags */
#define F_NEAR_TAU 1
#define F_NEAR_TMIN 2

typedef struct {
  double V[12]; /* row-major [R|t] */
  double fx, fy, cx, cy;
  int width, height;
} ocam;

typedef struct {
  double tau, t_min, alpha_max, znear, lowpass, bg[3];
  int tile_w, tile_h, nu_grad_mode;
  int kernel; /* 0: Student's t (Eq. t_2D); 1: Gaussian, the nu -> infinity
                 limit exp(-h/2) (Sec. 3.1; the paper's SGHMC + 3DGS ablation) */
} ocfg;

static ocam read_cam(const double* c, const int* wh) {
  ocam k;
  memcpy(k.V, c, 12 * sizeof(double));
  k.fx = c[12]; k.fy = c[13]; k.cx = c[14]; k.cy = c[15];
  k.width = wh[0]; k.height = wh[1];
  return k;
}

static ocfg read_cfg(const double* d, const int* i) {
  ocfg g;
  g.tau = d[0]; g.t_min = d[1]; g.alpha_max = d[2]; g.znear = d[3]; g.lowpass = d[4];
  g.bg[0] = d[5]; g.bg[1] = d[6]; g.bg[2] = d[7];
  g.tile_w = i[0]; g.tile_h = i[1]; g.nu_grad_mode = i[2]; g.kernel = i[3];
  return g;
}

int orc_version(void) { return 1; }

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* Real spherical harmonics                                                  */
/* ======================================================================== */
/* Y_{l,m} for m = -l..l at index l*l + l + m, with the Condon-Shortley phase:
 *   m = 0 : K_l^0 P_l^0(z)
 *   m > 0 : sqrt2 K_l^m P_l^m(cos th) cos(m phi)
 *   m < 0 : sqrt2 K_l^|m| P_l^|m|(cos th) sin(|m| phi)
 * K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  P_l^m = Q_l^m(z) sin^m(th) and
 * sin^m(th) e^{i m phi} = (x + i y)^m on the unit sphere, so everything is a
 * polynomial in (x, y, z); Q_l^m follows the associated Legendre recurrence.
 * Written with cx so the complex-step derivative passes through it. */
static double fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return f;
}

static void sh_basis_cx(int deg, cx x, cx y, cx z, cx* out) {
  cx cm = 1.0, sm = 0.0; /* Re, Im of (x + i y)^m */
  for (int m = 0; m <= deg; ++m) {
    if (m > 0) {
      cx c2 = x * cm - y * sm;
      cx s2 = x * sm + y * cm;
      cm = c2;
      sm = s2;
    }
    double qmm = 1.0;
    for (int k = 1; k <= m; ++k) qmm *= -(2.0 * k - 1.0);
    cx q_prev = 0.0, q_cur = qmm; /* Q_{l-1}^m, Q_l^m starting at l = m */
    for (int l = m; l <= deg; ++l) {
      if (l == m + 1) {
        q_prev = q_cur;
        q_cur = (2.0 * m + 1.0) * z * q_prev;
      } else if (l > m + 1) {
        cx q_next = ((2.0 * l - 1.0) * z * q_cur - (double)(l + m - 1) * q_prev) / (double)(l - m);
        q_prev = q_cur;
        q_cur = q_next;
      }
      double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * fact(l - m) / fact(l + m));
      if (m == 0) {
        out[l * l + l] = K * q_cur;
      } else {
        out[l * l + l + m] = sqrt(2.0) * K * q_cur * cm;
        out[l * l + l - m] = sqrt(2.0) * K * q_cur * sm;
      }
    }
  }
}

void orc_sh_basis(int degree, const double* dir, double* out) {
  cx tmp[100];
  if (degree < 0 || degree > 8) return;
  sh_basis_cx(degree, dir[0], dir[1], dir[2], tmp);
  for (int k = 0; k < (degree + 1) * (degree + 1); ++k) out[k] = creal(tmp[k]);
}

/* ======================================================================== */
/* The 2D Student's t kernel (Sec. 3.2 Eq. t_2D, unnormalised)               */
/* ======================================================================== */
double orc_t2d(double h, double nu) { return pow(1.0 + h / nu, -(nu + 2.0) / 2.0); }

/* ======================================================================== */
/* Projection of one component into one view (Sec. 3.2 Eq. t_2D)            */
/* ======================================================================== */
/* Outputs, in the order of the 2D gradient record: mean2D (2), conic (3),
 * o, nu, rgb (3).  Also depth, Sigma2D and the colour clamp mask.
 * Returns 1 if the component is in front of the near plane and its Sigma2D is
 * positive definite, else 0.
 * Readings: near plane znear on camera-space z; the Jacobian J of the
 * perspective map is evaluated at the camera-space mean with x/z and y/z
 * limited to 1.3 times the half-FOV tangent (the EWA convention of 3DGS, on
 * which the paper builds); quaternion (w,x,y,z) normalised before use;
 * colour = SH . Y(dir) + 0.5 clamped below at 0 with dir = normalised
 * (mu - camera centre). */
static int project_cx(const cx* mu, const cx* ls, const cx* q, cx nu_in, cx o_raw,
                      const cx* sh, int sh_deg, const ocam* cam, const ocfg* cfg,
                      cx out[G_STRIDE], cx* depth, cx cov[3], int clampmask[3]) {
  const double* V = cam->V;
  cx p[3];
  for (int r = 0; r < 3; ++r)
    p[r] = V[r * 4 + 0] * mu[0] + V[r * 4 + 1] * mu[1] + V[r * 4 + 2] * mu[2] + V[r * 4 + 3];
  *depth = p[2];
  if (!(creal(p[2]) > 0.0)) return 0; /* near-plane culling is decided on the FP32 depth key */

  /* Sigma = R S S^T R^T (Sec. 3.1) */
  cx qn = csqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  cx w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
  cx Rq[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
              2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
              2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
  cx s[3] = {cexp(ls[0]), cexp(ls[1]), cexp(ls[2])};
  cx M[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[r * 3 + c] = Rq[r * 3 + c] * s[c];
  cx Sig[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      cx acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += M[r * 3 + k] * M[c * 3 + k];
      Sig[r * 3 + c] = acc;
    }

  /* EWA Jacobian of (x,y,z) -> (fx x/z + cx, fy y/z + cy) at p */
  double limx = 1.3 * (cam->width / (2.0 * cam->fx));
  double limy = 1.3 * (cam->height / (2.0 * cam->fy));
  double ux = creal(p[0]) / creal(p[2]), uy = creal(p[1]) / creal(p[2]);
  cx tx = (ux < -limx) ? -limx * p[2] : ((ux > limx) ? limx * p[2] : p[0]);
  cx ty = (uy < -limy) ? -limy * p[2] : ((uy > limy) ? limy * p[2] : p[1]);
  cx J[6] = {cam->fx / p[2], 0.0, -cam->fx * tx / (p[2] * p[2]),
             0.0, cam->fy / p[2], -cam->fy * ty / (p[2] * p[2])};
  /* A = J W (2x3), W = rotation part of the view matrix */
  cx A[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c)
      A[r * 3 + c] = J[r * 3 + 0] * V[0 * 4 + c] + J[r * 3 + 1] * V[1 * 4 + c] + J[r * 3 + 2] * V[2 * 4 + c];
  /* Sigma2D = (A Sigma A^T) */
  cx AS[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      cx acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += A[r * 3 + k] * Sig[k * 3 + c];
      AS[r * 3 + c] = acc;
    }
  cx S2[4];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      cx acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += AS[r * 3 + k] * A[c * 3 + k];
      S2[r * 2 + c] = acc;
    }
  cov[0] = S2[0] + cfg->lowpass;
  cov[1] = 0.5 * (S2[1] + S2[2]);
  cov[2] = S2[3] + cfg->lowpass;
  cx det = cov[0] * cov[2] - cov[1] * cov[1];
  if (!(creal(det) > 0.0)) return 0;

  out[G_MX] = cam->fx * p[0] / p[2] + cam->cx;
  out[G_MY] = cam->fy * p[1] / p[2] + cam->cy;
  out[G_CA] = cov[2] / det;
  out[G_CB] = -cov[1] / det;
  out[G_CC] = cov[0] / det;
  out[G_O] = ctanh(o_raw);
  double nur = creal(nu_in);
  out[G_NU] = (nur < 1.0) ? (cx)1.0 : ((nur > 1e4) ? (cx)1e4 : nu_in);

  /* colour from spherical harmonics at the viewing direction */
  double campos[3];
  for (int c = 0; c < 3; ++c)
    campos[c] = -(V[0 * 4 + c] * V[3] + V[1 * 4 + c] * V[7] + V[2 * 4 + c] * V[11]);
  cx d[3] = {mu[0] - campos[0], mu[1] - campos[1], mu[2] - campos[2]};
  cx dn = csqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  cx Y[16];
  sh_basis_cx(sh_deg, d[0] / dn, d[1] / dn, d[2] / dn, Y);
  int K = (sh_deg + 1) * (sh_deg + 1);
  for (int c = 0; c < 3; ++c) {
    cx acc = 0.5;
    for (int k = 0; k < K; ++k) acc += sh[k * 3 + c] * Y[k];
    if (creal(acc) < 0.0) {
      clampmask[c] = 1;
      acc = 0.0;
    } else {
      clampmask[c] = 0;
    }
    out[G_R + c] = acc;
  }
  return 1;
}

/* Gather component i's parameters as cx (imaginary parts zero). */
static void gather_cx(int n, int sh_deg, const double* th, size_t i, cx* buf) {
  int K = (sh_deg + 1) * (sh_deg + 1);
  for (int c = 0; c < 3; ++c) buf[c] = th[TH_MEAN(n) + c * (size_t)n + i];
  for (int c = 0; c < 3; ++c) buf[3 + c] = th[TH_LS(n) + c * (size_t)n + i];
  for (int c = 0; c < 4; ++c) buf[6 + c] = th[TH_Q(n) + c * (size_t)n + i];
  buf[10] = th[TH_NU(n) + i];
  buf[11] = th[TH_O(n) + i];
  for (int k = 0; k < 3 * K; ++k) buf[12 + k] = th[TH_SH(n) + k * (size_t)n + i];
}

static int project_buf(const cx* buf, int sh_deg, const ocam* cam, const ocfg* cfg, cx out[G_STRIDE],
                       cx* depth, cx cov[3], int clampmask[3]) {
  return project_cx(buf, buf + 3, buf + 6, buf[10], buf[11], buf + 12, sh_deg, cam, cfg, out, depth, cov,
                    clampmask);
}

/* Depth key: camera-space z of mu in FP32, evaluated as
 *   fma(W20, mu_x, ...) chain: fmaf(W22, mu_z, fmaf(W21, mu_y, fmaf(W20, mu_x, t_z)))
 * on the FP32 values of the camera and the mean.  The per-pixel order
 * (depth key, index) and the near-plane cut are discrete decisions; both sides
 * take them on this FP32 key (the rasterizer's precision), so they agree bit
 * for bit; all geometry stays FP64. */
static float depth_key(const ocam* cam, const double* th, int n, size_t i) {
  float mx = (float)th[TH_MEAN(n) + i], my = (float)th[TH_MEAN(n) + (size_t)n + i];
  float mz = (float)th[TH_MEAN(n) + 2 * (size_t)n + i];
  const double* V = cam->V;
  return fmaf((float)V[10], mz, fmaf((float)V[9], my, fmaf((float)V[8], mx, (float)V[11])));
}

/* Largest h at which |o| T2D(h) >= a (a < |o|):  nu ((|o|/a)^{2/(nu+2)} - 1). */
static double h_limit(double o_abs, double nu, double a) {
  return nu * expm1(2.0 / (nu + 2.0) * log(o_abs / a));
}

/* The splat kernel of the chosen family and its extent: the t profile of
 * Eq. t_2D, or the Gaussian exp(-h/2) (the limit nu -> infinity) for which
 * |o| exp(-h/2) >= a  <=>  h <= 2 ln(|o| / a). */
static double kernel_value(double h, double nu, const ocfg* cfg) {
  return cfg->kernel == 1 ? exp(-0.5 * h) : orc_t2d(h, nu);
}
static double kernel_limit(double o_abs, double nu, double a, const ocfg* cfg) {
  return cfg->kernel == 1 ? 2.0 * log(o_abs / a) : h_limit(o_abs, nu, a);
}

/* Scale of the rounding error of an evaluation of Sigma2D, relative to its
 * smallest eigenvalue: |J W|_F^2 s_max^2 / lambda_min(Sigma2D).  Evaluating
 * Sigma2D = (J W R S)(J W R S)^T with unit roundoff e perturbs it by a few e
 * times |J W|_F^2 s_max^2 (rotation and products rounded on the scale of the
 * largest axis), and a perturbation dS of Sigma2D moves h = d^T Sigma2D^-1 d
 * by at most |dS| h / lambda_min.  Used only for the ambiguity windows. */
static double error_scale(int n, const double* th, size_t i, const ocam* cam, const double* rec) {
  const double* V = cam->V;
  double mu[3], p[3];
  for (int c = 0; c < 3; ++c) mu[c] = th[TH_MEAN(n) + c * (size_t)n + i];
  for (int r = 0; r < 3; ++r) p[r] = V[r * 4 + 0] * mu[0] + V[r * 4 + 1] * mu[1] + V[r * 4 + 2] * mu[2] + V[r * 4 + 3];
  double limx = 1.3 * (cam->width / (2.0 * cam->fx)), limy = 1.3 * (cam->height / (2.0 * cam->fy));
  double tx = fmin(fmax(p[0] / p[2], -limx), limx) * p[2], ty = fmin(fmax(p[1] / p[2], -limy), limy) * p[2];
  double J[6] = {cam->fx / p[2], 0.0, -cam->fx * tx / (p[2] * p[2]), 0.0, cam->fy / p[2], -cam->fy * ty / (p[2] * p[2])};
  double t2 = 0.0;
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) {
      double a = J[r * 3 + 0] * V[0 * 4 + c] + J[r * 3 + 1] * V[1 * 4 + c] + J[r * 3 + 2] * V[2 * 4 + c];
      t2 += a * a;
    }
  double lmax = th[TH_LS(n) + i];
  for (int c = 1; c < 3; ++c) lmax = fmax(lmax, th[TH_LS(n) + c * (size_t)n + i]);
  const double A = rec[P_COV_A], B = rec[P_COV_B], C = rec[P_COV_C];
  const double tr = A + C, det = A * C - B * B;
  const double lmin = 2.0 * det / (tr + sqrt(fmax(tr * tr - 4.0 * det, 0.0)));
  return t2 * exp(2.0 * lmax) / lmin;
}

static void project_record(int n, int sh_deg, const double* th, size_t i, const ocam* cam, const ocfg* cfg,
                           double* rec) {
  cx buf[12 + 48];
  cx out[G_STRIDE], depth, cov[3];
  int cm[3] = {0, 0, 0};
  gather_cx(n, sh_deg, th, i, buf);
  memset(rec, 0, P_STRIDE * sizeof(double));
  float dk = depth_key(cam, th, n, i);
  rec[P_DEPTH] = (double)dk;
  if (!(dk > (float)cfg->znear)) return;
  int ok = project_buf(buf, sh_deg, cam, cfg, out, &depth, cov, cm);
  if (!ok) return;
  double o = creal(out[G_O]);
  /* A component with |o| < tau can never reach |alpha| >= tau. */
  if (!(fabs(o) >= cfg->tau)) return;
  rec[P_VALID] = 1.0;
  rec[P_MX] = creal(out[G_MX]);
  rec[P_MY] = creal(out[G_MY]);
  rec[P_COV_A] = creal(cov[0]);
  rec[P_COV_B] = creal(cov[1]);
  rec[P_COV_C] = creal(cov[2]);
  rec[P_CON_A] = creal(out[G_CA]);
  rec[P_CON_B] = creal(out[G_CB]);
  rec[P_CON_C] = creal(out[G_CC]);
  rec[P_O] = o;
  rec[P_NU] = creal(out[G_NU]);
  for (int c = 0; c < 3; ++c) {
    rec[P_R + c] = creal(out[G_R + c]);
    rec[P_CLAMP_R + c] = cm[c];
  }
  /* Extent (reading of SM "Implementation Details" on truncation): the splat
   * is cut where |alpha| = |o| T2D falls below tau, i.e. h <= h_max.  The
   * pixel centres (i + 0.5, j + 0.5) inside the bounding box of that ellipse
   * give the pixel range; the tiles covering it give the tile rectangle. */
  double hmax = kernel_limit(fabs(o), rec[P_NU], cfg->tau, cfg);
  rec[P_HMAX] = hmax;
  double ex = sqrt(rec[P_COV_A] * hmax), ey = sqrt(rec[P_COV_C] * hmax);
  double px0 = ceil(rec[P_MX] - ex - 0.5), px1 = floor(rec[P_MX] + ex - 0.5);
  double py0 = ceil(rec[P_MY] - ey - 0.5), py1 = floor(rec[P_MY] + ey - 0.5);
  if (px0 < 0) px0 = 0;
  if (py0 < 0) py0 = 0;
  if (px1 > cam->width - 1) px1 = cam->width - 1;
  if (py1 > cam->height - 1) py1 = cam->height - 1;
  rec[P_PX0] = px0; rec[P_PX1] = px1; rec[P_PY0] = py0; rec[P_PY1] = py1;
  if (px0 > px1 || py0 > py1) {
    rec[P_TX0] = 0; rec[P_TX1] = -1; rec[P_TY0] = 0; rec[P_TY1] = -1; rec[P_NTILES] = 0;
    return;
  }
  long tx0 = (long)px0 / cfg->tile_w, tx1 = (long)px1 / cfg->tile_w;
  long ty0 = (long)py0 / cfg->tile_h, ty1 = (long)py1 / cfg->tile_h;
  rec[P_TX0] = tx0; rec[P_TX1] = tx1; rec[P_TY0] = ty0; rec[P_TY1] = ty1;
  rec[P_NTILES] = (double)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
  rec[P_ES] = error_scale(n, th, i, cam, rec);
}

void orc_project(int n, int sh_deg, const double* theta, const double* camd, const int* wh, const double* cfgd,
                 const int* cfgi, double* out) {
  ocam cam = read_cam(camd, wh);
  ocfg cfg = read_cfg(cfgd, cfgi);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) project_record(n, sh_deg, theta, (size_t)i, &cam, &cfg, out + (size_t)i * P_STRIDE);
}

/* ======================================================================== */
/* Per-pixel composite (Sec. 3.4 Eq. SSS_color)                              */
/* ======================================================================== */
typedef struct { double depth; long idx; } dkey;

static int cmp_dkey(const void* a, const void* b) {
  const dkey* x = (const dkey*)a;
  const dkey* y = (const dkey*)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Valid components sorted by (depth, index). */
static long* sorted_valid(int n, const double* proj, long* count) {
  dkey* keys = (dkey*)malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
  long m = 0;
  for (long i = 0; i < n; ++i)
    if (proj[(size_t)i * P_STRIDE + P_VALID] != 0.0) {
      keys[m].depth = proj[(size_t)i * P_STRIDE + P_DEPTH];
      keys[m].idx = i;
      ++m;
    }
  qsort(keys, (size_t)m, sizeof(dkey), cmp_dkey);
  long* order = (long*)malloc(sizeof(long) * (size_t)(m > 0 ? m : 1));
  for (long k = 0; k < m; ++k) order[k] = keys[k].idx;
  free(keys);
  *count = m;
  return order;
}

/* One contributor of a pixel, kept for the backward pass. */
typedef struct { long idx; double alpha, T, t2d, h, dx, dy; int clamped; double errT; } contrib;

typedef struct { contrib* v; long n, cap; } cvec;

static void cvec_push(cvec* c, contrib x) {
  if (c->n == c->cap) {
    c->cap = c->cap ? 2 * c->cap : 256;
    c->v = (contrib*)realloc(c->v, sizeof(contrib) * (size_t)c->cap);
  }
  c->v[c->n++] = x;
}

/* Ambiguity window of one (pixel, splat) decision.  Which splats contribute
 * to a pixel is decided by |alpha| >= tau and by T' >= t_min; where such a
 * decision lies within the rounding error of an FP32 evaluation (the
 * precision of the paper's rasterizer), both outcomes are correct results.
 * The window bounds, to first order, the relative error of alpha evaluated
 * in FP32 from a projection whose conic is evaluated in double-float
 * arithmetic (pairs of FP32, unit roundoff about 4 u^2) and rounded once to
 * FP32, as the sum of:
 *   - the scales exp(log_scale) in FP32 (at most 2 ulp, 4 u, each; squared in
 *     Sigma2D, a relative perturbation of each axis' share): 8 u h;
 *   - the double-float evaluation of the conic: 64 u^2 E h, E the error scale
 *     of the record (error_scale above; the FP32 evaluation of the same
 *     expressions measured at most 10.2 u E h, and 64 u^2 is 16 times the
 *     double-float unit roundoff);
 *   - the conic rounded to FP32: u q, q the sum of the magnitudes of the three
 *     terms of h;
 *   - the screen mean stored relative to the integer pixel nearest to it
 *     (limited to [0, 16384]): 2 u (|m - origin| + 1) per coordinate, times
 *     |dh/dm|;
 *   - evaluating h in FP32 from the offsets: 6 u q;
 * times |dlnT2D/dh| = (nu+2) / (2 nu (1 + h/nu)) (1/2 for the Gaussian); plus,
 * with e = (nu+2)/2 and T2D = 2^(-e log2(1 + h/nu)) evaluated as the kernel
 * does:
 *   - hardware log2 / exp2 of 2^-22 error (absolute for log2, times the
 *     exponent e; relative for exp2);
 *   - the argument 1 + h/nu from a 1-ulp hardware reciprocal of nu and one
 *     FMA: 3 u relative, times e;
 *   - the exponent -e log2(1 + h/nu), e and the product each rounded once:
 *     2 u of |ln T2D| = 2 u e ln(1 + h/nu) (for the Gaussian, the FP32
 *     constant log2(e) / 2 and its product with h: 2 u of h / 2);
 *   - the opacity, FP32 tanh of at most 2 ulp (4 u), and its product with
 *     T2D: 5 u.
 * Capped at 1e-2 (the prefilter evaluates every pair with
 * |alpha| >= tau (1 - 1e-2)). */
#define ORC_U (1.0 / 16777216.0)
#define ORC_MUFU (1.0 / 4194304.0)
static double alpha_window(const double* r, double h, double dx, double dy, const ocfg* cfg) {
  const double u = ORC_U;
  const double ca = r[P_CON_A], cb = r[P_CON_B], cc = r[P_CON_C];
  const double q = fabs(ca) * dx * dx + 2.0 * fabs(cb * dx * dy) + fabs(cc) * dy * dy;
  const double ox = fmin(fmax(rint(r[P_MX]), 0.0), 16384.0), oy = fmin(fmax(rint(r[P_MY]), 0.0), 16384.0);
  const double gm = 2.0 * fabs(ca * dx + cb * dy) * 2.0 * u * (fabs(r[P_MX] - ox) + 1.0) +
                    2.0 * fabs(cb * dx + cc * dy) * 2.0 * u * (fabs(r[P_MY] - oy) + 1.0);
  const double dh = 8.0 * u * h + 64.0 * u * u * r[P_ES] * h + gm + 7.0 * u * q;
  double w;
  if (cfg->kernel == 1) {
    w = 0.5 * dh + ORC_MUFU + u * h;
  } else {
    const double nu = r[P_NU], e = 0.5 * (nu + 2.0);
    w = e / nu / (1.0 + h / nu) * dh + log(2.0) * e * ORC_MUFU + 3.0 * u * e + 2.0 * u * e * log1p(h / nu) +
        ORC_MUFU;
  }
  w += 5.0 * u;
  return w < 1e-2 ? w : 1e-2;
}

/* h = d^T Sigma2D^-1 d of a projection record at the offset d = (dx, dy)
 * from its mean (Sec. 3.2 Eq. t_2D). */
static double record_h(const double* r, double dx, double dy) {
  return r[P_CON_A] * dx * dx + 2.0 * r[P_CON_B] * dx * dy + r[P_CON_C] * dy * dy;
}

/* Composite pixel (px, py) (integer indices; sample point at the centre).
 * Readings: alpha = o T2D, skipped when |alpha| < tau; alpha clamped to
 * [-alpha_max, alpha_max]; front-to-back, stop before the component that
 * would bring T below t_min (t_min = 0 disables); background added with the
 * final transmittance.
 * Ambiguous decisions (alpha_window above; for the termination test, T' within
 * the accumulated relative error of an FP32 T, 2 u + window |alpha| / |1 -
 * alpha| per composited splat) set a flag bit; the j-th ambiguous decision met
 * on the way is taken the other way when bit j of `flip` is set (the other
 * correct result), and their number is returned in *n_amb. */
static void composite_pixel(const double* proj, const long* order, long m, const double* hpre, const ocfg* cfg,
                            long px, long py, uint32_t flip, double rgb[3], double* T_out, int* ncontrib,
                            long* last, int* flags, int* n_amb, cvec* keep) {
  double u = (double)px + 0.5, v = (double)py + 0.5;
  double T = 1.0, C[3] = {0, 0, 0};
  double errT = 0.0; /* relative error bound of an FP32 T along this path */
  int nc = 0, fl = 0, ev = 0;
  long lst = -1;
  for (long k = 0; k < m; ++k) {
    long i = order[k];
    const double* r = proj + (size_t)i * P_STRIDE;
    double dx = u - r[P_MX], dy = v - r[P_MY];
    double h = record_h(r, dx, dy);
    if (h > hpre[i]) continue; /* |alpha| < tau (1 - 1e-2) for sure */
    double t2d = kernel_value(h, r[P_NU], cfg);
    double alpha = r[P_O] * t2d;
    const double W = alpha_window(r, h, dx, dy, cfg);
    int include = fabs(alpha) >= cfg->tau;
    if (fabs(fabs(alpha) - cfg->tau) <= W * cfg->tau) {
      fl |= F_NEAR_TAU;
      if (ev < 32 && ((flip >> ev) & 1u)) include = !include;
      ++ev;
    }
    if (!include) continue;
    int clamped = 0;
    if (alpha > cfg->alpha_max) { alpha = cfg->alpha_max; clamped = 1; }
    if (alpha < -cfg->alpha_max) { alpha = -cfg->alpha_max; clamped = 1; }
    double Tn = T * (1.0 - alpha);
    double errTn = errT + 2.0 * ORC_U + W * fabs(alpha) / fabs(1.0 - alpha);
    if (cfg->t_min > 0.0) {
      int term = Tn < cfg->t_min;
      if (fabs(Tn - cfg->t_min) <= errTn * Tn) {
        fl |= F_NEAR_TMIN;
        if (ev < 32 && ((flip >> ev) & 1u)) term = !term;
        ++ev;
      }
      if (term) break;
    }
    if (keep) {
      contrib c = {i, alpha, T, t2d, h, dx, dy, clamped, errTn};
      cvec_push(keep, c);
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] += r[P_R + ch] * alpha * T;
    T = Tn;
    errT = errTn;
    ++nc;
    lst = i;
  }
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch] + T * cfg->bg[ch];
  *T_out = T;
  *ncontrib = nc;
  *last = lst;
  *flags = fl;
  if (n_amb) *n_amb = ev;
}

/* The ambiguity window (alpha_window above) and the FP64 alpha of npairs
 * (component, pixel) pairs: component idx[k] of the projection records at
 * the pixel centre (px[k], py[k]).  For the tests that check the window
 * against an FP32 evaluation. */
void orc_pair_windows(const double* proj, const double* cfgd, const int* cfgi, long npairs, const long* idx,
                      const double* px, const double* py, double* out_h, double* out_alpha, double* out_w) {
  const ocfg cfg = read_cfg(cfgd, cfgi);
  for (long k = 0; k < npairs; ++k) {
    const double* r = proj + (size_t)idx[k] * P_STRIDE;
    const double dx = px[k] - r[P_MX], dy = py[k] - r[P_MY];
    const double h = record_h(r, dx, dy);
    out_h[k] = h;
    out_alpha[k] = r[P_O] * kernel_value(h, r[P_NU], &cfg);
    out_w[k] = alpha_window(r, h, dx, dy, &cfg);
  }
}

static double* prefilter_bounds(int n, const double* proj, const ocfg* cfg) {
  double* hpre = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (long i = 0; i < n; ++i) {
    const double* r = proj + (size_t)i * P_STRIDE;
    hpre[i] = r[P_VALID] != 0.0 ? kernel_limit(fabs(r[P_O]), r[P_NU], cfg->tau * (1.0 - 1e-2), cfg) : -1.0;
  }
  return hpre;
}

/* Render npix pixels (linear indices pix[k] = y * width + x; pix == NULL means
 * all width*height pixels in order).  out_rgb is [3][npix].  flip (optional,
 * [npix]): per pixel, which ambiguous decisions to take the other way;
 * out_namb (optional): the number of ambiguous decisions met. */
void orc_render(int n, const double* proj, int width, int height, const double* cfgd, const int* cfgi, long npix,
                const int64_t* pix, const uint32_t* flip, double* out_rgb, double* out_T, int32_t* out_n,
                int64_t* out_last, int32_t* out_flags, int32_t* out_namb) {
  ocfg cfg = read_cfg(cfgd, cfgi);
  long m;
  long* order = sorted_valid(n, proj, &m);
  double* hpre = prefilter_bounds(n, proj, &cfg);
  (void)height;
#pragma omp parallel for schedule(dynamic, 64)
  for (long k = 0; k < npix; ++k) {
    long lin = pix ? (long)pix[k] : k;
    long px = lin % width, py = lin / width;
    double rgb[3], T;
    int nc, fl, na;
    long lst;
    composite_pixel(proj, order, m, hpre, &cfg, px, py, flip ? flip[k] : 0u, rgb, &T, &nc, &lst, &fl, &na, NULL);
    for (int c = 0; c < 3; ++c) out_rgb[(size_t)c * npix + k] = rgb[c];
    if (out_T) out_T[k] = T;
    if (out_n) out_n[k] = nc;
    if (out_last) out_last[k] = lst;
    if (out_flags) out_flags[k] = fl;
    if (out_namb) out_namb[k] = na;
  }
  free(order);
  free(hpre);
}

/* The compositing path of npix pixels (linear indices pix[k]): up to max_k
 * contributors each, in order, with their index, (clamped) alpha, the
 * transmittance T in front of them and the bound on the relative error of an
 * FP32 transmittance behind them (the termination window's errT).  For the
 * tests that check that bound against an FP32 compositing. */
void orc_pixel_paths(int n, const double* proj, int width, const double* cfgd, const int* cfgi, long npix,
                     const int64_t* pix, int max_k, int32_t* out_count, int64_t* out_idx, double* out_alpha,
                     double* out_T, double* out_errT) {
  ocfg cfg = read_cfg(cfgd, cfgi);
  long m;
  long* order = sorted_valid(n, proj, &m);
  double* hpre = prefilter_bounds(n, proj, &cfg);
#pragma omp parallel for schedule(dynamic, 16)
  for (long k = 0; k < npix; ++k) {
    const long lin = (long)pix[k];
    double rgb[3], T;
    int nc, fl, na;
    long lst;
    cvec keep = {NULL, 0, 0};
    composite_pixel(proj, order, m, hpre, &cfg, lin % width, lin / width, 0u, rgb, &T, &nc, &lst, &fl, &na, &keep);
    const long c = keep.n < max_k ? keep.n : max_k;
    out_count[k] = (int32_t)c;
    for (long j = 0; j < c; ++j) {
      const size_t o = (size_t)k * max_k + j;
      out_idx[o] = keep.v[j].idx;
      out_alpha[o] = keep.v[j].alpha;
      out_T[o] = keep.v[j].T;
      out_errT[o] = keep.v[j].errT;
    }
    free(keep.v);
  }
  free(order);
  free(hpre);
}

/* ======================================================================== */
/* Backward (SM "Backward Pass")                                             */
/* ======================================================================== */
/* dT2D/dh, SM Eq. for the h(x) trick: -(nu+2)/(2 nu) (1 + h/nu)^{-(nu+4)/2}. */
static double dT_dh(double h, double nu) { return -(nu + 2.0) / (2.0 * nu) * pow(1.0 + h / nu, -(nu + 4.0) / 2.0); }

/* dT2D/dnu.  Mode 0 (exact): the derivative of (1 + h/nu)^{-(nu+2)/2} with
 * both the base and the exponent depending on nu,
 *   T2D [ -1/2 ln(1 + h/nu) + (nu+2) h / (2 nu^2 (1 + h/nu)) ].
 * Mode 1 (paper): the printed SM result (nu+2)/2 h/nu^2 (1 + h/nu)^{-(nu+4)/2},
 * which holds the exponent fixed. */
static double dT_dnu(double h, double nu, int mode) {
  double g = 1.0 + h / nu;
  double second = (nu + 2.0) / 2.0 * h / (nu * nu) * pow(g, -(nu + 4.0) / 2.0);
  if (mode == 1) return second;
  return -0.5 * log1p(h / nu) * pow(g, -(nu + 2.0) / 2.0) + second;
}

/* Accumulate dL/d(2D record) for one pixel from its contributors.
 * With S the colour contributed behind contributor k and T_f the final
 * transmittance, C = sum_k rgb_k alpha_k T_k + T_f bg gives
 *   dC/drgb_k   = alpha_k T_k
 *   dC/dalpha_k = T_k rgb_k - (S_k + T_f bg) / (1 - alpha_k). */
static void pixel_backward(const double* proj, const cvec* cs, double T_final, const double g[3], const ocfg* cfg,
                           double* g2d, double* g2abs, double* g2absn) {
  const double ncon = (double)cs->n; /* contributors of this pixel */
  double S[3] = {0, 0, 0};
  for (long k = cs->n - 1; k >= 0; --k) {
    const contrib* c = &cs->v[k];
    const double* r = proj + (size_t)c->idx * P_STRIDE;
    double* gr = g2d + (size_t)c->idx * G_STRIDE;
    double* ga = g2abs ? g2abs + (size_t)c->idx * G_STRIDE : NULL;
    double* gan = g2absn ? g2absn + (size_t)c->idx * G_STRIDE : NULL;
    double dL_dalpha = 0.0, dL_dalpha_mag = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      double dC_dalpha = c->T * r[P_R + ch] - (S[ch] + T_final * cfg->bg[ch]) / (1.0 - c->alpha);
      dL_dalpha += g[ch] * dC_dalpha;
      dL_dalpha_mag += fabs(g[ch]) * (c->T * fabs(r[P_R + ch]) +
                                      fabs(S[ch] + T_final * cfg->bg[ch]) / (1.0 - c->alpha));
      double d_rgb = g[ch] * c->alpha * c->T;
#pragma omp atomic
      gr[G_R + ch] += d_rgb;
      if (ga) {
#pragma omp atomic
        ga[G_R + ch] += fabs(d_rgb);
#pragma omp atomic
        gan[G_R + ch] += fabs(d_rgb) * ncon;
      }
    }
    for (int ch = 0; ch < 3; ++ch) S[ch] += r[P_R + ch] * c->alpha * c->T;
    if (c->clamped) continue; /* clamp: alpha independent of o and T2D */
    double nu = r[P_NU];
    double d_o = dL_dalpha * c->t2d;
    double dL_dT = dL_dalpha * r[P_O];
    const int gauss = cfg->kernel == 1;
    double dL_dh = dL_dT * (gauss ? -0.5 * exp(-0.5 * c->h) : dT_dh(c->h, nu));
    double d_nu = gauss ? 0.0 : dL_dT * dT_dnu(c->h, nu, cfg->nu_grad_mode);
    /* h = a dx^2 + 2 b dx dy + c dy^2 with (dx, dy) = u - mean2D */
    double d_mx = dL_dh * (-2.0 * (r[P_CON_A] * c->dx + r[P_CON_B] * c->dy));
    double d_my = dL_dh * (-2.0 * (r[P_CON_B] * c->dx + r[P_CON_C] * c->dy));
    double d_ca = dL_dh * c->dx * c->dx;
    double d_cb = dL_dh * 2.0 * c->dx * c->dy;
    double d_cc = dL_dh * c->dy * c->dy;
#pragma omp atomic
    gr[G_MX] += d_mx;
#pragma omp atomic
    gr[G_MY] += d_my;
#pragma omp atomic
    gr[G_CA] += d_ca;
#pragma omp atomic
    gr[G_CB] += d_cb;
#pragma omp atomic
    gr[G_CC] += d_cc;
#pragma omp atomic
    gr[G_O] += d_o;
    /* dL/d(limited nu); the limit's own derivative is applied in the chain */
#pragma omp atomic
    gr[G_NU] += d_nu;
    if (ga) {
      /* Magnitudes of the summands, each taken on the operands of the
       * subtractions inside it (T rgb and S / (1 - alpha) in dC/dalpha; the two
       * terms of dT/dnu): the scale a floating-point evaluation rounds
       * against. */
      double dT_mag = fabs(r[P_O]) * dL_dalpha_mag;
      double dh_mag = dT_mag * (gauss ? 0.5 * exp(-0.5 * c->h) : fabs(dT_dh(c->h, nu)));
      double nu_mag = gauss ? 0.0 : 0.5 * log1p(c->h / nu) + (nu + 2.0) / 2.0 * c->h / (nu * nu) / (1.0 + c->h / nu);
      const double t[7] = {
          dh_mag * 2.0 * (fabs(r[P_CON_A] * c->dx) + fabs(r[P_CON_B] * c->dy)),
          dh_mag * 2.0 * (fabs(r[P_CON_B] * c->dx) + fabs(r[P_CON_C] * c->dy)),
          dh_mag * c->dx * c->dx,
          dh_mag * 2.0 * fabs(c->dx * c->dy),
          dh_mag * c->dy * c->dy,
          dL_dalpha_mag * c->t2d,
          dT_mag * c->t2d * nu_mag};
      for (int o = 0; o < 7; ++o) {
#pragma omp atomic
        ga[o] += t[o];
#pragma omp atomic
        gan[o] += t[o] * ncon;
      }
    }
  }
}

/* Full backward over n_views views.
 *   theta    planar parameters (layout above)
 *   cams     [n_views][16], whs [n_views][2]
 *   npix     [n_views] pixel counts; pix concatenated linear indices or NULL
 *            (then every view uses all its pixels)
 *   dL_dC    concatenated per view [3][npix_v]
 *   grad2d   optional [n_views][n][G_STRIDE] output (dL/d 2D record)
 *   grad     [(12 + 3K) n] output, dL/dtheta summed over views
 *   grad2d_abs, grad_abs  optional: the same sums taken over magnitudes --
 *            per pixel the absolute values of the operands of every
 *            subtraction inside a term (T rgb and S / (1 - alpha) in
 *            dC/dalpha, the two terms of dT/dnu), then |Jacobian| times those
 *            -- i.e. the scale a floating-point evaluation of the same sums
 *            rounds against
 *   grad_absn optional: as grad_abs with every pixel's magnitudes weighted by
 *            its number of contributors (a transmittance recovered through
 *            the whole list carries a rounding proportional to that count)
 * The 2D -> 3D chain uses the complex-step derivative of project_cx. */
void orc_backward(int n, int sh_deg, const double* theta, int n_views, const double* cams, const int* whs,
                  const double* cfgd, const int* cfgi, const int64_t* npix, const int64_t* pix, const uint32_t* flip,
                  const double* dL_dC, double* grad2d, double* grad, double* grad2d_abs, double* grad_abs,
                  double* grad_absn, double* grad2d_absn) {
  ocfg cfg = read_cfg(cfgd, cfgi);
  int K = (sh_deg + 1) * (sh_deg + 1);
  size_t P = (size_t)(12 + 3 * K);
  memset(grad, 0, sizeof(double) * P * (size_t)n);
  if (grad_abs) memset(grad_abs, 0, sizeof(double) * P * (size_t)n);
  if (grad_absn) memset(grad_absn, 0, sizeof(double) * P * (size_t)n);
  double* proj = (double*)malloc(sizeof(double) * P_STRIDE * (size_t)(n > 0 ? n : 1));
  double* g2 = (double*)malloc(sizeof(double) * G_STRIDE * (size_t)(n > 0 ? n : 1));
  double* g2a = (grad2d_abs || grad_abs) ? (double*)malloc(sizeof(double) * G_STRIDE * (size_t)(n > 0 ? n : 1))
                                         : NULL;
  double* g2an = g2a ? (double*)malloc(sizeof(double) * G_STRIDE * (size_t)(n > 0 ? n : 1)) : NULL;
  size_t pix_off = 0, dl_off = 0, flip_off = 0;
  for (int v = 0; v < n_views; ++v) {
    ocam cam = read_cam(cams + 16 * v, whs + 2 * v);
    long np = npix ? (long)npix[v] : (long)cam.width * cam.height;
    const int64_t* pv = pix ? pix + pix_off : NULL;
    const uint32_t* fl_v = flip ? flip + flip_off : NULL;
    orc_project(n, sh_deg, theta, cams + 16 * v, whs + 2 * v, cfgd, cfgi, proj);
    memset(g2, 0, sizeof(double) * G_STRIDE * (size_t)n);
    if (g2a) memset(g2a, 0, sizeof(double) * G_STRIDE * (size_t)n);
    if (g2an) memset(g2an, 0, sizeof(double) * G_STRIDE * (size_t)n);
    long m;
    long* order = sorted_valid(n, proj, &m);
    double* hpre = prefilter_bounds(n, proj, &cfg);
    const double* dl = dL_dC + dl_off;
#pragma omp parallel
    {
      cvec cs = {NULL, 0, 0};
#pragma omp for schedule(dynamic, 32)
      for (long k = 0; k < np; ++k) {
        long lin = pv ? (long)pv[k] : k;
        long px = lin % cam.width, py = lin / cam.width;
        double rgb[3], T;
        int nc, fl;
        long lst;
        cs.n = 0;
        composite_pixel(proj, order, m, hpre, &cfg, px, py, fl_v ? fl_v[k] : 0u, rgb, &T, &nc, &lst, &fl, NULL,
                        &cs);
        double g[3] = {dl[k], dl[(size_t)np + k], dl[2 * (size_t)np + k]};
        pixel_backward(proj, &cs, T, g, &cfg, g2, g2a, g2an);
      }
      free(cs.v);
    }
    free(order);
    free(hpre);
    if (grad2d) memcpy(grad2d + (size_t)v * G_STRIDE * n, g2, sizeof(double) * G_STRIDE * (size_t)n);
    if (grad2d_abs) memcpy(grad2d_abs + (size_t)v * G_STRIDE * n, g2a, sizeof(double) * G_STRIDE * (size_t)n);
    if (grad2d_absn) memcpy(grad2d_absn + (size_t)v * G_STRIDE * n, g2an, sizeof(double) * G_STRIDE * (size_t)n);

    /* chain to the 3D parameters, complex step of step size hc */
    const double hc = 1e-20;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) {
      const double* gi = g2 + (size_t)i * G_STRIDE;
      const double* gai = g2a ? g2a + (size_t)i * G_STRIDE : NULL;
      const double* gani = g2an ? g2an + (size_t)i * G_STRIDE : NULL;
      int any = 0;
      for (int j = 0; j < G_STRIDE; ++j) any |= (gi[j] != 0.0) || (gai && gai[j] != 0.0);
      if (!any) continue;
      cx buf[12 + 48];
      gather_cx(n, sh_deg, theta, (size_t)i, buf);
      for (size_t j = 0; j < P; ++j) {
        cx save = buf[j];
        buf[j] = creal(save) + I * hc;
        cx out[G_STRIDE], depth, cov[3];
        int cm[3];
        int ok = project_buf(buf, sh_deg, &cam, &cfg, out, &depth, cov, cm);
        buf[j] = save;
        if (!ok) continue;
        double acc = 0.0, acc_abs = 0.0, acc_absn = 0.0;
        for (int o = 0; o < G_STRIDE; ++o) {
          acc += gi[o] * (cimag(out[o]) / hc);
          if (gai) {
            acc_abs += gai[o] * fabs(cimag(out[o]) / hc);
            acc_absn += gani[o] * fabs(cimag(out[o]) / hc);
          }
        }
        /* theta index of parameter j of component i */
        size_t row;
        if (j < 3) row = TH_MEAN(n) + j * (size_t)n;
        else if (j < 6) row = TH_LS(n) + (j - 3) * (size_t)n;
        else if (j < 10) row = TH_Q(n) + (j - 6) * (size_t)n;
        else if (j == 10) row = TH_NU(n);
        else if (j == 11) row = TH_O(n);
        else row = TH_SH(n) + (j - 12) * (size_t)n;
        grad[row + (size_t)i] += acc;
        if (grad_abs) grad_abs[row + (size_t)i] += acc_abs;
        if (grad_absn) grad_absn[row + (size_t)i] += acc_absn;
      }
    }
    pix_off += pv ? (size_t)np : 0;
    flip_off += (size_t)np;
    dl_off += 3 * (size_t)np;
  }
  free(proj);
  free(g2);
  free(g2a);
  free(g2an);
}

/* ======================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11)                                                  */
/* ======================================================================== */
/* One round: two 32x32->64 multiplications of counter words 0 and 2 by the
 * published multipliers; the high halves are xored with the other two words
 * and the round key, the words are permuted.  The key is advanced by the
 * Weyl constants (golden ratio and sqrt(3) - 1 in 32-bit fixed point) before
 * every round after the first. */
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for component i at a given step, Box-Muller on the
 * four Philox words of counter (i, 0, step_lo, step_hi) under key
 * (seed_lo, seed_hi).  Uniforms: u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1],
 * u2 = (w1 >> 8) 2^-24 in [0, 1); likewise (w2, w3). */
void orc_normals3(uint64_t seed, uint64_t step, uint32_t i, double* z) {
  uint32_t ctr[4] = {i, 0u, (uint32_t)step, (uint32_t)(step >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  const double s24 = 1.0 / 16777216.0;
  double u1 = ((double)(w[0] >> 8) + 1.0) * s24, u2 = (double)(w[1] >> 8) * s24;
  double u3 = ((double)(w[2] >> 8) + 1.0) * s24, u4 = (double)(w[3] >> 8) * s24;
  double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
  z[0] = r1 * cos(2.0 * ORC_PI * u2);
  z[1] = r1 * sin(2.0 * ORC_PI * u2);
  z[2] = r2 * cos(2.0 * ORC_PI * u4);
}

/* ======================================================================== */
/* SGHMC on mu, Adam on the rest (Sec. 3.4 Eq. sigmoidUpdate, SM Eq. SGHMC)  */
/* ======================================================================== */
/* sp: eps, C, k, t0, lr_logscale, lr_quat, lr_nu, lr_opacity, lr_sh, beta1,
 *     beta2, adam_eps.   burn_in: 0/1.
 * Readings (the printed indices and noise variance disagree with the SM
 * derivation; this follows the derivation, which is self-consistent):
 *   g   = sigmoid(-k (|o| - t0)), o = tanh(opacity_raw)     (gate, t0 = 1 - t)
 *   xi  ~ N(0, I_3) from Philox, G = dL/dmu (raw gradient)
 *   r'  = (1 - eps C) r - eps G + sqrt(2 eps C) xi
 *   mu' = mu - eps^2 G + g eps (1 - eps C) r + g eps sqrt(2 eps C) xi
 *   burn-in: mu' = mu - eps^2 G + g eps sqrt(2 eps C) Sigma xi (no friction
 *   term; Sigma = R S S^T R^T of the pre-step parameters); r' as above.
 * Adam: m' = b1 m + (1-b1) g, v' = b2 v + (1-b2) g^2,
 *       p' = p - lr (m'/(1-b1^t)) / (sqrt(v'/(1-b2^t)) + eps_adam), t = step+1,
 *       nu' limited to [1, 1e4] afterwards.
 * All arrays share theta's planar layout except r [3][n]; m, v have theta's
 * size (their mean slots are unused).  xi_out [3][n] receives the normals. */
void orc_sghmc_step(int n, int sh_deg, double* theta, const double* grad, double* r, double* m, double* v,
                    const double* sp, int burn_in, uint64_t seed, uint64_t step, double* xi_out) {
  int K = (sh_deg + 1) * (sh_deg + 1);
  size_t N = (size_t)n;
  double eps = sp[0], C = sp[1], kk = sp[2], t0 = sp[3];
  double b1 = sp[9], b2 = sp[10], aeps = sp[11];
  double t = (double)step + 1.0;
  double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double o = tanh(theta[TH_O(n) + i]);
    double g = 1.0 / (1.0 + exp(kk * (fabs(o) - t0)));
    double xi[3];
    orc_normals3(seed, step, (uint32_t)i, xi);
    if (xi_out)
      for (int c = 0; c < 3; ++c) xi_out[c * N + i] = xi[c];
    double noise[3] = {xi[0], xi[1], xi[2]};
    if (burn_in) {
      /* Sigma xi with Sigma = R S S^T R^T from the pre-step parameters */
      double q[4], qn = 0.0;
      for (int c = 0; c < 4; ++c) {
        q[c] = theta[TH_Q(n) + c * N + i];
        qn += q[c] * q[c];
      }
      qn = sqrt(qn);
      double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
      double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                     2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                     2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
      double s2[3];
      for (int c = 0; c < 3; ++c) s2[c] = exp(2.0 * theta[TH_LS(n) + c * N + i]);
      for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int b = 0; b < 3; ++b) {
          double sig = 0.0;
          for (int k = 0; k < 3; ++k) sig += R[a * 3 + k] * s2[k] * R[b * 3 + k];
          acc += sig * xi[b];
        }
        noise[a] = acc;
      }
    }
    double sq = sqrt(2.0 * eps * C);
    for (int c = 0; c < 3; ++c) {
      size_t j = TH_MEAN(n) + c * N + i;
      double G = grad[j];
      double rr = r[c * N + i];
      double r_new = (1.0 - eps * C) * rr - eps * G + sq * xi[c];
      double mu = theta[j] - eps * eps * G;
      if (burn_in) mu += g * eps * sq * noise[c];
      else mu += g * eps * (1.0 - eps * C) * rr + g * eps * sq * xi[c];
      theta[j] = mu;
      r[c * N + i] = r_new;
    }
    /* Adam groups: log-scale, quaternion, nu, opacity, SH */
    size_t begin[5] = {TH_LS(n), TH_Q(n), TH_NU(n), TH_O(n), TH_SH(n)};
    int rows[5] = {3, 4, 1, 1, 3 * K};
    for (int grp = 0; grp < 5; ++grp) {
      double lr = sp[4 + grp];
      for (int c = 0; c < rows[grp]; ++c) {
        size_t j = begin[grp] + c * N + i;
        double gg = grad[j];
        double mm = b1 * m[j] + (1.0 - b1) * gg;
        double vv = b2 * v[j] + (1.0 - b2) * gg * gg;
        m[j] = mm;
        v[j] = vv;
        theta[j] -= lr * (mm / bc1) / (sqrt(vv / bc2) + aeps);
      }
    }
    double* nu = &theta[TH_NU(n) + i];
    if (*nu < 1.0) *nu = 1.0;
    if (*nu > 1e4) *nu = 1e4;
  }
}
