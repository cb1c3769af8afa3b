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


def _emulated_aabs(proj, comp, px, py, kernel, so, sr, sl, se):
    """|alpha| of the pairs through the emulated FP32 chain, with tanh, the
    reciprocal of nu, log2 and exp2 each at its worst case on the side of the
    sign given for it (so, sr, sl, se)."""
    P = oracle.P
    r = proj[comp]
    ca, cb, cc = (r[:, P[k]].astype(F32) for k in ("con_a", "con_b", "con_c"))
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


def _emulated_alpha_range(proj, cfgd, comp, px, py, kernel):
    """Smallest and largest |alpha| the emulated FP32 chain gives over the
    worst cases of the hardware approximations."""
    lo = np.full(comp.size, np.inf)
    hi = np.full(comp.size, -np.inf)
    for so in (-1, 1):
        for sr in (-1, 1):
            for sl in (-1, 1):
                for se in (-1, 1):
                    a = _emulated_aabs(proj, comp, px, py, kernel, so, sr, sl, se).astype(F64)
                    lo, hi = np.minimum(lo, a), np.maximum(hi, a)
    return lo, hi


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
