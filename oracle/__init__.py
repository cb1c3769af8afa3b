"""FP64 CPU oracle for the Student Splatting and Scooping rasterizer.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product library.  It shares no code
with the CUDA path; the only common module is the seeded input generator,
which holds none of the method's arithmetic.

The arithmetic lives in ``sss_oracle.c`` (plain C, FP64, OpenMP over pixels);
this module only marshals numpy arrays.  Function-by-function citations are in
that file.  ``bin_sort_reference`` (the tile-list reference) is plain numpy
here: a lexicographic sort of (tile, depth bits, index) tuples.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# projection record fields (doubles), same order as sss_oracle.c
P_FIELDS = ("valid mx my cov_a cov_b cov_c con_a con_b con_c depth o nu r g b "
            "clamp_r clamp_g clamp_b hmax px0 px1 py0 py1 tx0 tx1 ty0 ty1 ntiles es").split()
P = {name: i for i, name in enumerate(P_FIELDS)}
P_STRIDE = len(P_FIELDS)
# 2D gradient record fields: dL/d(mean2D x, y, conic a, b, c, o, nu, r, g, b)
G_FIELDS = ("mx", "my", "ca", "cb", "cc", "o", "nu", "r", "g", "b")
G_STRIDE = len(G_FIELDS)

F_NEAR_TAU, F_NEAR_TMIN = 1, 2

DEFAULT_CFG = dict(tau=1.0 / 255.0, t_min=1e-4, alpha_max=0.99, znear=0.2, lowpass=0.0,
                   bg=(0.0, 0.0, 0.0), tile_w=16, tile_h=16, nu_grad_mode=0, kernel=0)

_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def _nullable(base):
    def from_param(cls, obj):
        if obj is None:
            return None
        return base.from_param(obj)
    return type(base.__name__ + "_or_null", (base,), {"from_param": classmethod(from_param)})


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_project.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _ip, _dp, _ip, _dp]
        L.orc_project.restype = None
        L.orc_render.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp, _ip, ctypes.c_long,
                                 _nullable(_lp), _nullable(_up), _dp, _nullable(_dp), _nullable(_ip),
                                 _nullable(_lp), _nullable(_ip), _nullable(_ip)]
        L.orc_render.restype = None
        L.orc_backward.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _ip, _dp, _ip,
                                   _nullable(_lp), _nullable(_lp), _nullable(_up), _dp, _nullable(_dp), _dp,
                                   _nullable(_dp), _nullable(_dp), _nullable(_dp), _nullable(_dp)]
        L.orc_backward.restype = None
        L.orc_sghmc_step.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                                     ctypes.c_uint64, ctypes.c_uint64, _nullable(_dp)]
        L.orc_sghmc_step.restype = None
        L.orc_philox4x32_10.argtypes = [_up, _up, _up]
        L.orc_philox4x32_10.restype = None
        L.orc_normals3.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _dp]
        L.orc_normals3.restype = None
        L.orc_t2d.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_t2d.restype = ctypes.c_double
        L.orc_sh_basis.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_sh_basis.restype = None
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_pair_windows.argtypes = [_dp, _dp, _ip, ctypes.c_long, _lp, _dp, _dp, _dp, _dp, _dp]
        L.orc_pair_windows.restype = None
        L.orc_pixel_paths.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _ip, ctypes.c_long, _lp, ctypes.c_int,
                                      _ip, _lp, _dp, _dp, _dp]
        L.orc_pixel_paths.restype = None
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def n_sh(sh_degree: int) -> int:
    return (sh_degree + 1) ** 2


def theta_from_scene(scene) -> np.ndarray:
    """Planar FP64 parameter vector: mean 3n, log_scale 3n, quat 4n, nu n,
    opacity_raw n, sh 3Kn (same row order as the scene's arrays)."""
    parts = [scene["mean"], scene["log_scale"], scene["quat"], scene["nu"][None],
             scene["opacity_raw"][None], scene["sh"]]
    return np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).reshape(-1, scene["n"])
                                                for p in parts], axis=0).reshape(-1))


def theta_slices(n: int, sh_degree: int) -> dict:
    K = n_sh(sh_degree)
    rows = dict(mean=(0, 3), log_scale=(3, 6), quat=(6, 10), nu=(10, 11), opacity_raw=(11, 12),
                sh=(12, 12 + 3 * K))
    return {k: slice(a * n, b * n) for k, (a, b) in rows.items()}


def split_theta(theta: np.ndarray, n: int, sh_degree: int) -> dict:
    out = {}
    for k, s in theta_slices(n, sh_degree).items():
        a = theta[s]
        out[k] = a.reshape(-1, n) if k not in ("nu", "opacity_raw") else a
    return out


def cam_arrays(cam):
    d = np.zeros(16, np.float64)
    d[:12] = np.asarray(cam.viewmat, np.float64).reshape(-1)
    d[12:] = (cam.fx, cam.fy, cam.cx, cam.cy)
    return d, np.array([cam.width, cam.height], np.int32)


def cfg_arrays(cfg=None):
    c = dict(DEFAULT_CFG)
    if cfg:
        c.update(cfg)
    d = np.array([c["tau"], c["t_min"], c["alpha_max"], c["znear"], c["lowpass"], *c["bg"]], np.float64)
    i = np.array([c["tile_w"], c["tile_h"], c["nu_grad_mode"], c.get("kernel", 0)], np.int32)
    return d, i


# ---------------------------------------------------------------------------
# oracle entry points
# ---------------------------------------------------------------------------

def project(scene_or_theta, cam, cfg=None, *, n=None, sh_degree=None) -> np.ndarray:
    """[n][P_STRIDE] FP64 projection records for one view."""
    if isinstance(scene_or_theta, dict):
        theta = theta_from_scene(scene_or_theta)
        n, sh_degree = scene_or_theta["n"], scene_or_theta["sh_degree"]
    else:
        theta = np.ascontiguousarray(scene_or_theta, np.float64)
    assert 0 <= sh_degree <= 3
    cd, wh = cam_arrays(cam)
    fd, fi = cfg_arrays(cfg)
    out = np.zeros((n, P_STRIDE), np.float64)
    lib().orc_project(n, sh_degree, theta, cd, wh, fd, fi, out)
    return out


def render(proj: np.ndarray, cam, cfg=None, pix=None, flip=None) -> dict:
    """Brute-force composite of the pixels ``pix`` (linear y*W+x; None = all).

    ``flags`` marks pixels with a decision (|alpha| >= tau, T' >= t_min)
    within the rounding error of an FP32 evaluation, ``n_amb`` counts those
    decisions; ``flip`` (one uint32 per pixel) takes the j-th of them the
    other way where bit j is set: the other correct results."""
    fd, fi = cfg_arrays(cfg)
    n = proj.shape[0]
    pix_arr = None if pix is None else np.ascontiguousarray(pix, np.int64)
    npix = cam.width * cam.height if pix is None else len(pix_arr)
    flip_arr = None if flip is None else np.ascontiguousarray(flip, np.uint32)
    assert flip_arr is None or len(flip_arr) == npix
    rgb = np.zeros((3, npix), np.float64)
    T = np.zeros(npix, np.float64)
    nc = np.zeros(npix, np.int32)
    last = np.zeros(npix, np.int64)
    flags = np.zeros(npix, np.int32)
    namb = np.zeros(npix, np.int32)
    lib().orc_render(n, np.ascontiguousarray(proj), cam.width, cam.height, fd, fi, npix, pix_arr, flip_arr, rgb, T,
                     nc, last, flags, namb)
    return dict(rgb=rgb, T=T, n_contrib=nc, last=last, flags=flags, n_amb=namb)


def backward(scene_or_theta, cams, cfg, dl_dc, pix=None, *, n=None, sh_degree=None, want_grad2d=False,
             want_abs=False, flip=None):
    """Analytic FP64 gradient of L = sum(dl_dc * C) w.r.t. theta.

    dl_dc: list (one per view) of [3][npix_v] (or [3][H][W]) arrays.
    pix:   None (all pixels) or a list of linear-index arrays per view.
    flip:  None or a list (one per view) of uint32 per pixel: the forward
           each pixel is differentiated through takes its ambiguous decisions
           as in ``render(..., flip=...)``.
    Returns grad theta (planar) and, if asked, grad2d [views][n][G_STRIDE];
    with want_abs also the sums of |summand| for both (grad_abs, grad2d_abs),
    the scale against which a floating-point evaluation of the same sums
    rounds."""
    if isinstance(scene_or_theta, dict):
        theta = theta_from_scene(scene_or_theta)
        n, sh_degree = scene_or_theta["n"], scene_or_theta["sh_degree"]
    else:
        theta = np.ascontiguousarray(scene_or_theta, np.float64)
    V = len(cams)
    cds = np.concatenate([cam_arrays(c)[0] for c in cams])
    whs = np.concatenate([cam_arrays(c)[1] for c in cams])
    fd, fi = cfg_arrays(cfg)
    if pix is None:
        npix = None
        pix_cat = None
        dl = np.concatenate([np.asarray(d, np.float64).reshape(3, -1).reshape(-1) for d in dl_dc])
    else:
        npix = np.array([len(p) for p in pix], np.int64)
        pix_cat = np.ascontiguousarray(np.concatenate([np.asarray(p, np.int64) for p in pix]))
        dl = np.concatenate([np.asarray(d, np.float64).reshape(3, -1).reshape(-1) for d in dl_dc])
    dl = np.ascontiguousarray(dl)
    flip_cat = None
    if flip is not None:
        flip_cat = np.ascontiguousarray(np.concatenate([np.asarray(f, np.uint32).reshape(-1) for f in flip]))
        assert len(flip_cat) * 3 == len(dl)
    grad = np.zeros_like(theta)
    g2d = np.zeros((V, n, G_STRIDE), np.float64) if want_grad2d else None
    gabs = np.zeros_like(theta) if want_abs else None
    gabsn = np.zeros_like(theta) if want_abs else None
    g2abs = np.zeros((V, n, G_STRIDE), np.float64) if (want_abs and want_grad2d) else None
    g2absn = np.zeros((V, n, G_STRIDE), np.float64) if (want_abs and want_grad2d) else None
    lib().orc_backward(n, sh_degree, theta, V, cds, whs, fd, fi, npix, pix_cat, flip_cat, dl, g2d, grad, g2abs, gabs,
                       gabsn, g2absn)
    out = (grad,)
    if want_grad2d:
        out += (g2d,)
    if want_abs:
        out += (Magnitudes(gabs, gabsn),) + ((Magnitudes(g2abs, g2absn),) if want_grad2d else ())
    return out if len(out) > 1 else grad


class Magnitudes:
    """Per-element magnitude sums of a gradient: ``abs`` = sum of |summand|
    (taken on the operands of every subtraction inside a summand), ``absn`` =
    the same with each pixel's terms weighted by its contributor count."""

    def __init__(self, abs_, absn):
        self.abs = abs_
        self.absn = absn

    def __getitem__(self, sl):
        return Magnitudes(self.abs[sl], self.absn[sl])


SGHMC_DEFAULTS = dict(eps=1e-3, C=0.5, k=100.0, t0=0.005, lr=(5e-3, 1e-3, 1e-2, 5e-2, 2.5e-3),
                      beta1=0.9, beta2=0.999, adam_eps=1e-15)


def sghmc_step(theta, grad, r, m, v, *, n, sh_degree, params=None, burn_in=False, seed=0, step=0):
    """One SGHMC (mu) + Adam (rest) step; returns new (theta, r, m, v, xi)."""
    p = dict(SGHMC_DEFAULTS)
    if params:
        p.update(params)
    sp = np.array([p["eps"], p["C"], p["k"], p["t0"], *p["lr"], p["beta1"], p["beta2"], p["adam_eps"]],
                  np.float64)
    th = np.array(theta, np.float64, copy=True)
    rr = np.array(r, np.float64, copy=True)
    mm = np.array(m, np.float64, copy=True)
    vv = np.array(v, np.float64, copy=True)
    xi = np.zeros(3 * n, np.float64)
    lib().orc_sghmc_step(n, sh_degree, th, np.ascontiguousarray(grad, np.float64), rr, mm, vv, sp,
                         int(bool(burn_in)), int(seed), int(step), xi)
    return th, rr, mm, vv, xi.reshape(3, n)


def adam_preconditioned(g_mu, m, v, *, step: int, beta1: float, beta2: float, adam_eps: float):
    """The Adam gradient used in SGHMC (Implementation Details): updates the
    moments of dL/dmu and returns (m^ / (sqrt(v^) + eps), m', v') with the
    bias corrections of step t = step + 1.  Plain numpy, FP64."""
    g = np.asarray(g_mu, np.float64)
    m2 = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v2 = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    t = step + 1
    mhat = m2 / (1.0 - beta1 ** t)
    vhat = v2 / (1.0 - beta2 ** t)
    return mhat / (np.sqrt(vhat) + adam_eps), m2, v2


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32), out)
    return out


def normals3(seed: int, step: int, i: int) -> np.ndarray:
    z = np.zeros(3, np.float64)
    lib().orc_normals3(int(seed), int(step), int(i), z)
    return z


def pair_windows(proj: np.ndarray, cfg, idx, px, py):
    """(h, alpha, window) of (component, pixel-centre) pairs: the FP64
    values and the ambiguity window of the alpha threshold decision."""
    fd, fi = cfg_arrays(cfg)
    idx = np.ascontiguousarray(idx, np.int64)
    px = np.ascontiguousarray(px, np.float64)
    py = np.ascontiguousarray(py, np.float64)
    h, a, w = (np.zeros(idx.size) for _ in range(3))
    lib().orc_pair_windows(np.ascontiguousarray(proj), fd, fi, idx.size, idx, px, py, h, a, w)
    return h, a, w


def pixel_paths(proj: np.ndarray, cam, cfg, pix, max_k: int = 512):
    """Per pixel (linear indices pix) its contributors in compositing order:
    (count [npix], index, alpha, T in front, errT behind [npix][max_k]), errT
    being the termination window's bound on an FP32 transmittance."""
    fd, fi = cfg_arrays(cfg)
    pix = np.ascontiguousarray(pix, np.int64)
    n = proj.shape[0]
    cnt = np.zeros(pix.size, np.int32)
    idx = np.zeros((pix.size, max_k), np.int64)
    a, T, e = (np.zeros((pix.size, max_k)) for _ in range(3))
    lib().orc_pixel_paths(n, np.ascontiguousarray(proj), int(cam.width), fd, fi, pix.size, pix, int(max_k), cnt, idx,
                          a, T, e)
    return cnt, idx, a, T, e


def t2d(h: float, nu: float) -> float:
    return float(lib().orc_t2d(float(h), float(nu)))


def sh_basis(degree: int, direction) -> np.ndarray:
    out = np.zeros((degree + 1) ** 2, np.float64)
    lib().orc_sh_basis(int(degree), np.ascontiguousarray(direction, np.float64), out)
    return out


# ---------------------------------------------------------------------------
# tile binning and sorting reference (plain numpy)
# ---------------------------------------------------------------------------

def bin_sort_reference(rects, depth_bits, tiles_x, tile_base):
    """Reference tile list: for every entry e (flattened (view, component)
    index) and every tile in its inclusive tile rectangle rects[e] =
    (tx0, tx1, ty0, ty1) emit (global tile id, depth bits, e); sort the tuples
    lexicographically.  tiles_x[e] and tile_base[e] give the tile-grid width
    and first global tile id of the entry's view.  Returns (tile, entry)
    arrays in sorted order."""
    rects = np.asarray(rects, np.int64)
    tiles_x = np.asarray(tiles_x, np.int64)
    tile_base = np.asarray(tile_base, np.int64)
    nx = np.maximum(rects[:, 1] - rects[:, 0] + 1, 0)
    ny = np.maximum(rects[:, 3] - rects[:, 2] + 1, 0)
    cnt = nx * ny
    e = np.repeat(np.arange(len(rects), dtype=np.int64), cnt)
    start = np.cumsum(cnt) - cnt
    k = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(start, cnt)
    nxe = nx[e]
    tx = rects[e, 0] + k % np.maximum(nxe, 1)
    ty = rects[e, 2] + k // np.maximum(nxe, 1)
    tile = tile_base[e] + ty * tiles_x[e] + tx
    db = np.asarray(depth_bits, np.uint32)[e].astype(np.int64)
    order = np.lexsort((e, db, tile))
    return tile[order], e[order]


# ---------------------------------------------------------------------------
# FP64 central finite differences (O4)
# ---------------------------------------------------------------------------

def fd_gradient(theta, n, sh_degree, cams, cfg, dl_dc, which, h=1e-6):
    """Central differences of L = sum_views sum(dl_dc * C) w.r.t. theta[j]
    for j in ``which``.  Only the pixels inside the perturbed component's
    pixel box (union over +h and -h) can change, so L is summed over those.

    Returns (grad, smooth): smooth[k] is False when a pixel's contributor
    count, last contributor or near-threshold flags differ between the two
    sides, i.e. the difference straddles a discrete event."""
    theta = np.ascontiguousarray(theta, np.float64)
    grads = np.zeros(len(which), np.float64)
    smooth = np.ones(len(which), bool)
    for k, j in enumerate(which):
        comp = int(j) % n
        total = 0.0
        for v, cam in enumerate(cams):
            w = np.asarray(dl_dc[v], np.float64).reshape(3, -1)
            sides = []
            for sgn in (+1.0, -1.0):
                th = theta.copy()
                th[j] += sgn * h
                sides.append((th, project(th, cam, cfg, n=n, sh_degree=sh_degree)))
            boxes = [pr[comp] for _, pr in sides if pr[comp, P["valid"]] != 0.0
                     and pr[comp, P["px0"]] <= pr[comp, P["px1"]]
                     and pr[comp, P["py0"]] <= pr[comp, P["py1"]]]
            if not boxes:
                continue
            x0 = int(min(b[P["px0"]] for b in boxes)); x1 = int(max(b[P["px1"]] for b in boxes))
            y0 = int(min(b[P["py0"]] for b in boxes)); y1 = int(max(b[P["py1"]] for b in boxes))
            xs, ys = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1))
            pix = (ys * cam.width + xs).reshape(-1).astype(np.int64)
            outs = [render(pr, cam, cfg, pix) for _, pr in sides]
            Lp = float(np.sum(w[:, pix] * outs[0]["rgb"]))
            Lm = float(np.sum(w[:, pix] * outs[1]["rgb"]))
            total += (Lp - Lm) / (2.0 * h)
            if (np.any(outs[0]["n_contrib"] != outs[1]["n_contrib"])
                    or np.any(outs[0]["last"] != outs[1]["last"])
                    or np.any(outs[0]["flags"] != outs[1]["flags"])):
                smooth[k] = False
        grads[k] = total
    return grads, smooth
