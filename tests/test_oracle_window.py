"""The oracle's ambiguity window (which alpha-threshold decisions an FP32
rasterizer may take either way) against an FP32 evaluation of alpha.

The kernel's chain from a 2D record to |alpha| is emulated on the CPU in
float32 with exact fused multiply-adds (through float64), from a record
rounded as the kernel stores it: the conic rounded once to FP32, the mean
relative to the integer pixel nearest to it, the opacity in FP32.  The
hardware approximations are emulated at their documented worst case: the
MUFU reciprocal of nu at 1 ulp, log2 at 2^-22 absolute, exp2 at 2^-22
relative, and tanh at 2 ulp, each taken both ways.  The window must bound
the largest deviation from the FP64 alpha, relative to it, for every pair.
Pairs are seeded pixel centres inside each component's extent, weighted
towards the alpha = tau boundary where the decisions lie.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_10148_gb300 import inputs

F32, F64 = np.float32, np.float64
FIELDS = ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh")


def _cfg(kernel):
    """The oracle's default options at the FP32 values a rasterizer holds."""
    c = dict(oracle.DEFAULT_CFG, kernel=kernel)
    for k in ("tau", "t_min", "alpha_max", "znear"):
        c[k] = float(F32(c[k]))
    return c


def _f32_camera(cam):
    return inputs.Camera(np.asarray(cam.viewmat, F32).astype(F64), float(F32(cam.fx)), float(F32(cam.fy)),
                         float(F32(cam.cx)), float(F32(cam.cy)), int(cam.width), int(cam.height))


def _fma(a, b, c):
    """float32 fused multiply-add (the float64 product of two float32 is exact)."""
    return (np.asarray(a, F64) * np.asarray(b, F64) + np.asarray(c, F64)).astype(F32)


def _ulp(x):
    return np.spacing(np.abs(np.asarray(x, F32))).astype(F64)


def _worst(x, bound, sign):
    """The float32 farthest from the exact x on the side `sign` that lies
    within `bound` of it: an approximation at its documented maximum error."""
    x = np.asarray(x, F64)
    c = (x + sign * bound).astype(F32)
    over = np.abs(c.astype(F64) - x) > bound
    c = np.where(over, np.nextafter(c, (x - sign * bound).astype(F32)), c)
    return c.astype(F32)


def _pairs(proj, cam, rng, per_comp):
    """Component indices and integer pixel coordinates: per valid component,
    pixels of its extent box, half drawn near the boundary ellipse."""
    P = oracle.P
    ok = (proj[:, P["valid"]] != 0) & (proj[:, P["ntiles"]] > 0)
    idx = np.flatnonzero(ok)
    r = proj[idx]
    A, B, C, hm = r[:, P["cov_a"]], r[:, P["cov_b"]], r[:, P["cov_c"]], r[:, P["hmax"]]
    l11 = np.sqrt(A)
    l21 = B / l11
    l22 = np.sqrt(np.maximum(C - l21 ** 2, 0.0))
    comp = np.repeat(idx, per_comp)
    k = np.repeat(np.arange(idx.size), per_comp)
    th = rng.uniform(0, 2 * np.pi, comp.size)
    rad = np.where(rng.random(comp.size) < 0.5, rng.uniform(0.9, 1.0, comp.size), np.sqrt(rng.random(comp.size)))
    s = np.sqrt(hm[k]) * rad
    x = r[k, P["mx"]] + s * l11[k] * np.cos(th)
    y = r[k, P["my"]] + s * (l21[k] * np.cos(th) + l22[k] * np.sin(th))
    px, py = np.floor(x), np.floor(y)
    keep = (px >= 0) & (px < cam.width) & (py >= 0) & (py < cam.height)
    return comp[keep], px[keep], py[keep]


def _emulated_aabs(proj, comp, px, py, kernel, so, sr, sl, se, con=None):
    """|alpha| of the pairs through the emulated FP32 chain, with tanh, the
    reciprocal of nu, log2 and exp2 each at its worst case on the side of the
    sign given for it (so, sr, sl, se).  con: the pairs' FP32 conic (a, b, c);
    by default the FP64 record's, rounded once."""
    P = oracle.P
    r = proj[comp]
    if con is None:
        ca, cb, cc = (r[:, P[k]].astype(F32) for k in ("con_a", "con_b", "con_c"))
    else:
        ca, cb, cc = con
    mx, my = r[:, P["mx"]], r[:, P["my"]]
    ox, oy = np.clip(np.rint(mx), 0, 16384), np.clip(np.rint(my), 0, 16384)
    mxr, myr = (mx - ox).astype(F32), (my - oy).astype(F32)
    dx = ((px - ox + 0.5).astype(F32) - mxr).astype(F32)  # (pixel - origin + 0.5) exact, one rounding
    dy = ((py - oy + 0.5).astype(F32) - myr).astype(F32)
    t = _fma(ca, dx, ((F32(2) * cb) * dy).astype(F32))
    h = _fma(dx, t, ((cc * dy).astype(F32) * dy).astype(F32))
    o = np.abs(r[:, P["o"]])
    o32 = _worst(o, 2 * _ulp(o), so)  # tanh: 2 ulp
    if kernel == 1:
        p = (h * F32(-0.72134752044448170)).astype(F32)
    else:
        nu = r[:, P["nu"]].astype(F32)
        inv = _worst(1.0 / nu.astype(F64), _ulp(1.0 / nu.astype(F64)), sr)  # reciprocal: 1 ulp
        x1 = _fma(h, inv, F32(1))
        l2 = _worst(np.log2(x1.astype(F64)), 2.0 ** -22, sl)  # log2: 2^-22 absolute
        e = (nu * F32(-0.5) - F32(1)).astype(F32)
        p = (e * l2).astype(F32)
    ex = np.exp2(p.astype(F64))
    t2d = _worst(ex, 2.0 ** -22 * ex, se)  # exp2: 2^-22 relative
    return np.minimum((o32 * t2d).astype(F32), F32(oracle.DEFAULT_CFG["alpha_max"]))


def _emulated_alpha_range(proj, cfgd, comp, px, py, kernel, con=None):
    """Smallest and largest |alpha| the emulated FP32 chain gives over the
    worst cases of the hardware approximations."""
    lo = np.full(comp.size, np.inf)
    hi = np.full(comp.size, -np.inf)
    for so in (-1, 1):
        for sr in (-1, 1):
            for sl in (-1, 1):
                for se in (-1, 1):
                    a = _emulated_aabs(proj, comp, px, py, kernel, so, sr, sl, se, con).astype(F64)
                    lo, hi = np.minimum(lo, a), np.maximum(hi, a)
    return lo, hi


# ---- the projection's double-float conic, emulated (pairs of float32 with
# exact error-free transformations), as a rasterizer computes it from the
# FP32 parameters: exact products of the raw quaternion, the rotation folded
# with the FP32 scales, the two rows of J W M, det = |n0 x n1|^2, each result
# rounded once
def _two_sum(a, b):
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    return s, ((a - (s - bb)) + (b - bb)).astype(F32)


def _fast_two_sum(a, b):
    s = (a + b).astype(F32)
    return s, (b - (s - a)).astype(F32)


def _two_prod(a, b):
    p = (a * b).astype(F32)
    return p, _fma(a, b, -p)


def _dmul(A, B):
    p = (A[0] * B[0]).astype(F32)
    return _fast_two_sum(p, _fma(A[0], B[1], _fma(A[1], B[0], _fma(A[0], B[0], -p))))


def _dmulf(A, b):
    p = (A[0] * b).astype(F32)
    return _fast_two_sum(p, _fma(A[1], b, _fma(A[0], b, -p)))


def _dadd(A, B):
    s, e = _two_sum(A[0], B[0])
    return _fast_two_sum(s, (e + (A[1] + B[1]).astype(F32)).astype(F32))


def _dneg(A):
    return -A[0], -A[1]


def _drcp(A):
    r = (F32(1) / A[0]).astype(F32)
    e = (_fma(-r, A[0], np.ones_like(r)) - (r * A[1]).astype(F32)).astype(F32)
    return _fast_two_sum(r, (r * e).astype(F32))


def _df(x):
    x = np.asarray(x, F32)
    return x, np.zeros_like(x)


def _dot3_plus(r, m, t):
    s, err = _two_prod(r[0], m[0])
    for k in (1, 2):
        q = _two_prod(r[k], m[k])
        s, e = _two_sum(s, q[0])
        err = (err + (e + q[1]).astype(F32)).astype(F32)
    s, e = _two_sum(s, t)
    return _fast_two_sum(s, (err + e).astype(F32))


def _conic_df(mu, ls_scale, q, cam, lp):
    """Conic (a, b, c) of every component for the camera, from FP32 means,
    scales and quaternions."""
    V = np.asarray(cam.viewmat, F32).reshape(3, 4)
    full = lambda v: np.full_like(mu[0], F32(v))
    w, x, y, z = q
    pr = {k: _two_prod(a, b) for k, (a, b) in dict(ww=(w, w), xx=(x, x), yy=(y, y), zz=(z, z), xy=(x, y),
                                                   wz=(w, z), xz=(x, z), wy=(w, y), yz=(y, z), wx=(w, x)).items()}
    two = lambda A: (A[0] * F32(2), A[1] * F32(2))
    Rn = [[_dadd(_dadd(pr["ww"], pr["xx"]), _dneg(_dadd(pr["yy"], pr["zz"]))), two(_dadd(pr["xy"], _dneg(pr["wz"]))),
           two(_dadd(pr["xz"], pr["wy"]))],
          [two(_dadd(pr["xy"], pr["wz"])), _dadd(_dadd(pr["ww"], pr["yy"]), _dneg(_dadd(pr["xx"], pr["zz"]))),
           two(_dadd(pr["yz"], _dneg(pr["wx"])))],
          [two(_dadd(pr["xz"], _dneg(pr["wy"]))), two(_dadd(pr["yz"], pr["wx"])),
           _dadd(_dadd(pr["ww"], pr["zz"]), _dneg(_dadd(pr["xx"], pr["yy"])))]]
    inv = _drcp(_dadd(_dadd(pr["ww"], pr["xx"]), _dadd(pr["yy"], pr["zz"])))
    sig = [_dmulf(inv, ls_scale[k]) for k in range(3)]
    M = [[_dmul(Rn[j][k], sig[k]) for k in range(3)] for j in range(3)]
    p = [_dot3_plus([full(V[r, k]) for k in range(3)], mu, full(V[r, 3])) for r in range(3)]
    iz = _drcp(p[2])
    u = [_dmul(p[0], iz), _dmul(p[1], iz)]
    for r, (ext, f) in enumerate(((cam.width, cam.fx), (cam.height, cam.fy))):
        lim = _dmul((full(1.3), full(4.7683717e-08)), _dmulf(_drcp(_df(full(F32(2) * F32(f)))), F32(ext)))
        lo = (u[r][0] < -lim[0]) | ((u[r][0] == -lim[0]) & (u[r][1] < -lim[1]))
        hi = (u[r][0] > lim[0]) | ((u[r][0] == lim[0]) & (u[r][1] > lim[1]))
        u[r] = (np.where(lo, -lim[0], np.where(hi, lim[0], u[r][0])),
                np.where(lo, -lim[1], np.where(hi, lim[1], u[r][1])))
    rowf = [_dmulf(iz, F32(cam.fx)), _dmulf(iz, F32(cam.fy))]
    U = [[_dadd(_df(full(V[r, k])), _dneg(_dmulf(u[r], V[2, k]))) for k in range(3)] for r in range(2)]
    N = [[_dmul(rowf[r], _dadd(_dadd(_dmul(U[r][0], M[0][k]), _dmul(U[r][1], M[1][k])), _dmul(U[r][2], M[2][k])))
          for k in range(3)] for r in range(2)]
    dot = lambda a, b: _dadd(_dadd(_dmul(a[0], b[0]), _dmul(a[1], b[1])), _dmul(a[2], b[2]))
    a, c, b = dot(N[0], N[0]), dot(N[1], N[1]), dot(N[0], N[1])
    xr = [_dadd(_dmul(N[0][1], N[1][2]), _dneg(_dmul(N[0][2], N[1][1]))),
          _dadd(_dmul(N[0][2], N[1][0]), _dneg(_dmul(N[0][0], N[1][2]))),
          _dadd(_dmul(N[0][0], N[1][1]), _dneg(_dmul(N[0][1], N[1][0])))]
    lpv = full(lp)
    A, C = _dadd(a, _df(lpv)), _dadd(c, _df(lpv))
    det = _dadd(dot(xr, xr), _dmulf(_dadd(_dadd(a, c), _df(lpv)), F32(lp)))
    iv = _drcp(det)
    return _dmul(C, iv)[0], _dneg(_dmul(b, iv))[0], _dmul(A, iv)[0]


@pytest.mark.parametrize("kernel", [0, 1])
def test_window_bounds_an_fp32_evaluation_of_alpha(kernel):
    scene = inputs.subset_scene(inputs.scene_sphere_shell(100_000, seed=1), np.arange(0, 100_000, 5))
    cam = _f32_camera(inputs.sphere_cameras(8, width=800, height=800)[3])
    cfgd = _cfg(kernel)
    s32 = {k: (np.asarray(v, F32) if k in FIELDS else v) for k, v in scene.items()}
    proj = oracle.project(s32, cam, cfgd)
    comp, px, py = _pairs(proj, cam, np.random.default_rng(3), per_comp=12)
    h, alpha, w = oracle.pair_windows(proj, cfgd, comp, px + 0.5, py + 0.5)
    lo, hi = _emulated_alpha_range(proj, cfgd, comp, px, py, kernel)
    a = np.abs(alpha)
    live = a >= 0.5 * cfgd["tau"]  # the pairs whose decision the window governs (and a margin below)
    assert live.sum() > 50_000
    dev = np.maximum(np.abs(hi - a), np.abs(lo - a))[live] / a[live]
    ratio = dev / w[live]
    print(f"kernel {kernel}: {int(live.sum())} pairs, deviation / window: median {np.median(ratio):.3f}, "
          f"max {ratio.max():.3f}")
    assert ratio.max() <= 1.0


@pytest.mark.parametrize("kernel", [0, 1])
def test_window_bounds_the_fp32_projection_and_evaluation(kernel):
    """As the test above, with each record computed as a rasterizer computes
    it: the double-float conic from the FP32 parameters, with the scales
    exp(log_scale) at 2 ulp to either side.  This covers the projection's part
    of the window as well (the scales, the double-float chain, the conic's
    rounding)."""
    scene = inputs.subset_scene(inputs.scene_sphere_shell(100_000, seed=1), np.arange(0, 100_000, 5))
    cam = _f32_camera(inputs.sphere_cameras(8, width=800, height=800)[3])
    cfgd = _cfg(kernel)
    s32 = {k: (np.asarray(v, F32) if k in FIELDS else v) for k, v in scene.items()}
    proj = oracle.project(s32, cam, cfgd)
    comp, px, py = _pairs(proj, cam, np.random.default_rng(4), per_comp=12)
    h, alpha, w = oracle.pair_windows(proj, cfgd, comp, px + 0.5, py + 0.5)
    mu = [s32["mean"][k] for k in range(3)]
    q = [s32["quat"][k] for k in range(4)]
    a = np.abs(alpha)
    lo = np.full(comp.size, np.inf)
    hi = np.full(comp.size, -np.inf)
    for ss in (-1, 1):  # expf: 2 ulp
        sc = [_worst(np.exp(s32["log_scale"][k].astype(F64)), 2 * _ulp(np.exp(s32["log_scale"][k].astype(F64))), ss)
              for k in range(3)]
        ca, cb, cc = _conic_df(mu, sc, q, cam, cfgd["lowpass"])
        l, hh = _emulated_alpha_range(proj, cfgd, comp, px, py, kernel, con=(ca[comp], cb[comp], cc[comp]))
        lo, hi = np.minimum(lo, l), np.maximum(hi, hh)
    live = a >= 0.5 * cfgd["tau"]
    assert live.sum() > 50_000
    ratio = np.maximum(np.abs(hi - a), np.abs(lo - a))[live] / a[live] / w[live]
    print(f"kernel {kernel}: {int(live.sum())} pairs from emulated records, deviation / window: median "
          f"{np.median(ratio):.3f}, max {ratio.max():.3f}")
    assert ratio.max() <= 1.0


@pytest.mark.parametrize("side", [-1, 1])
def test_termination_window_bounds_an_fp32_compositing(side):
    """Along every sampled pixel's path the oracle's bound errT on the
    relative error of an FP32 transmittance (2u per composited splat plus the
    splat's window times |alpha| / |1 - alpha|) must hold for the emulated
    FP32 compositing T <- T (1 - alpha), with the hardware approximations at
    their worst case on one side for every splat."""
    scene = inputs.scene_sphere_shell(100_000, seed=1)
    cam = _f32_camera(inputs.sphere_cameras(8, width=800, height=800)[5])
    cfgd = _cfg(0)
    s32 = {k: (np.asarray(v, F32) if k in FIELDS else v) for k, v in scene.items()}
    proj = oracle.project(s32, cam, cfgd)
    pix = np.random.default_rng(7).choice(cam.width * cam.height, 3000, replace=False)
    cnt, idx, alpha, T64, errT = oracle.pixel_paths(proj, cam, cfgd, pix, max_k=1024)
    assert cnt.max() < 1024 and np.mean(cnt) > 20
    px, py = (pix % cam.width).astype(F64), (pix // cam.width).astype(F64)
    T32 = np.ones(pix.size, F32)
    worst = 0.0
    for j in range(int(cnt.max())):
        live = j < cnt
        if not live.any():
            break
        k = np.flatnonzero(live)
        # every approximation on the side that moves |alpha| by `side` (a larger 1/nu or log2 lowers it)
        aabs = _emulated_aabs(proj, idx[k, j], px[k], py[k], 0, side, -side, -side, side)
        a32 = (np.sign(alpha[k, j]).astype(F32) * aabs).astype(F32)
        T32[k] = (T32[k] * (F32(1) - a32).astype(F32)).astype(F32)
        Tn = T64[k, j] * (1.0 - alpha[k, j])
        ratio = np.abs(T32[k].astype(F64) - Tn) / (errT[k, j] * np.abs(Tn))
        worst = max(worst, float(ratio.max()))
    print(f"side {side}: {pix.size} pixels, {int(cnt.sum())} composited splats, mean path {cnt.mean():.0f}, "
          f"T deviation / bound: max {worst:.3f}")
    assert worst <= 1.0
