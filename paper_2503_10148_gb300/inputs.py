"""Seeded synthetic scenes and cameras for the Student-splatting rasterizer.

This module is shared by the CUDA path, the tests and the FP64 oracle's
callers.  It only draws random numbers and builds camera poses; it contains
none of the rasterizer's arithmetic (no projection, no compositing, no
gradients, no optimiser step).

Parameter layout (one scene), every field planar ``[dim][N]`` float32:

    mean        [3][N]   component centre mu
    log_scale   [3][N]   S = diag(exp(log_scale))
    quat        [4][N]   rotation quaternion (w, x, y, z), not normalised
    nu          [N]      degrees of freedom, meaningful range [1, 1e4]
    opacity_raw [N]      o = tanh(opacity_raw), o in (-1, 1); o < 0 scoops
    sh          [K*3][N] spherical-harmonic colour, K = (degree+1)^2,
                         row k*3 + c holds coefficient k of channel c

The recipes follow the paper's workloads (Sec. 4 datasets are replaced by
seeded synthetic scenes of the same scale: component counts of the order of
the paper's parameter-efficiency study, Sec. 4.3, and the "down-scaled"
large-scene resolutions of the SM implementation details).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Real spherical harmonic of degree 0: 1 / (2 sqrt(pi)).  Used only to turn a
# drawn RGB value into the DC coefficient that reproduces it.
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclasses.dataclass
class Camera:
    """Pinhole camera. ``viewmat`` is the row-major 3x4 [R|t] world->camera
    map; camera axes are x right, y down, z forward (positive depth)."""

    viewmat: np.ndarray  # (3, 4) float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def position(self) -> np.ndarray:
        R = self.viewmat[:, :3]
        t = self.viewmat[:, 3]
        return -R.T @ t


def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), *, width: int,
            height: int, fov_x_deg: float = 50.0) -> Camera:
    """Camera at ``position`` looking at ``target`` with horizontal FOV."""
    c = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    u = np.asarray(up, dtype=np.float64)
    if abs(float(f @ u)) > 0.99:  # looking along the up axis: pick another
        u = np.array([0.0, 0.0, 1.0])
    right = np.cross(f, u)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ c
    fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return Camera(np.concatenate([R, t[:, None]], axis=1), fx, fx, width / 2.0,
                  height / 2.0, int(width), int(height))


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors spread evenly on the sphere (golden-angle spiral)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    y = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - y * y))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), y, r * np.sin(phi)], axis=1)


def sphere_cameras(n: int, *, radius: float = 3.0, width: int, height: int,
                   fov_x_deg: float = 50.0) -> list[Camera]:
    return [look_at(radius * d, width=width, height=height, fov_x_deg=fov_x_deg)
            for d in fibonacci_directions(n)]


def random_sphere_camera(rng: np.random.Generator, *, radius: float = 3.0, width: int,
                         height: int, fov_x_deg: float = 50.0) -> Camera:
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return look_at(radius * d, width=width, height=height, fov_x_deg=fov_x_deg)


def _unit_quats(rng, n):
    q = rng.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q


def _signed_opacity_raw(rng, n, lo, hi, frac_negative):
    o = rng.uniform(lo, hi, size=n)
    neg = rng.permutation(n)[: int(round(frac_negative * n))]
    o[neg] = -o[neg]
    return np.arctanh(o)


def _log_uniform(rng, n, lo, hi):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))


def _pack(mean, log_scale, quat, nu, opacity_raw, sh, sh_degree):
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)  # noqa: E731
    return {
        "mean": f(mean), "log_scale": f(log_scale), "quat": f(quat), "nu": f(nu),
        "opacity_raw": f(opacity_raw), "sh": f(sh), "sh_degree": int(sh_degree),
        "n": int(mean.shape[1]),
    }


def scene_uniform_cube(n: int, seed: int) -> dict:
    """Tiny-scene recipe: mu ~ U[-1,1]^3, log-scale ~ N(-3, 0.5), uniform unit
    quaternions, nu log-uniform in [1, 8], |o| ~ U(0.05, 0.9) with 20% negated
    (scooping), SH degree 0 with RGB ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-1.0, 1.0, size=(3, n))
    log_scale = rng.normal(-3.0, 0.5, size=(3, n))
    quat = _unit_quats(rng, n)
    nu = _log_uniform(rng, n, 1.0, 8.0)
    o_raw = _signed_opacity_raw(rng, n, 0.05, 0.9, 0.20)
    rgb = rng.uniform(0.0, 1.0, size=(3, n))
    sh = (rgb - 0.5) / _Y00
    return _pack(mean, log_scale, quat, nu, o_raw, sh, 0)


def scene_sphere_shell(n: int, seed: int) -> dict:
    """Shell recipe: mu = (1 + N(0, 0.05)) * uniform direction, log-scale ~
    N(-4, 0.5), nu log-uniform in [1, 16], 25% scooping, SH degree 3 with
    coefficients ~ N(0, 0.1)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    mean = d * (1.0 + rng.normal(0.0, 0.05, size=n))
    log_scale = rng.normal(-4.0, 0.5, size=(3, n))
    quat = _unit_quats(rng, n)
    nu = _log_uniform(rng, n, 1.0, 16.0)
    o_raw = _signed_opacity_raw(rng, n, 0.05, 0.9, 0.25)
    sh = rng.normal(0.0, 0.1, size=(16 * 3, n))
    return _pack(mean, log_scale, quat, nu, o_raw, sh, 3)


def scene_clusters_ground(n: int, seed: int) -> dict:
    """Large-scene recipe: 80% of the components in 6 isotropic Gaussian
    clusters (centres ~ U[-1,1]^3, sigma 0.3), 20% on a ground plane y = -1
    over [-2,2]^2 with N(0, 0.01) thickness; log-scale ~ N(-4, 0.7), SH degree
    3 with coefficients ~ N(0, 0.1), nu log-uniform in [1, 32], 30% scooping."""
    rng = np.random.default_rng(seed)
    n_cl = int(round(0.8 * n))
    n_gp = n - n_cl
    centres = rng.uniform(-1.0, 1.0, size=(6, 3))
    which = rng.integers(0, 6, size=n_cl)
    cl = centres[which].T + rng.normal(0.0, 0.3, size=(3, n_cl))
    gp = np.stack([rng.uniform(-2.0, 2.0, n_gp), -1.0 + rng.normal(0.0, 0.01, n_gp),
                   rng.uniform(-2.0, 2.0, n_gp)])
    mean = np.concatenate([cl, gp], axis=1)
    perm = rng.permutation(n)
    mean = mean[:, perm]
    log_scale = rng.normal(-4.0, 0.7, size=(3, n))
    quat = _unit_quats(rng, n)
    nu = _log_uniform(rng, n, 1.0, 32.0)
    o_raw = _signed_opacity_raw(rng, n, 0.05, 0.9, 0.30)
    sh = rng.normal(0.0, 0.1, size=(16 * 3, n))
    return _pack(mean, log_scale, quat, nu, o_raw, sh, 3)


# ---------------------------------------------------------------------------
# Named workloads (sizes and seeds fixed).
# ---------------------------------------------------------------------------

def tiny_cube_2k():
    """2,000 components, one 128x128 camera at (0,0,3), seed 0."""
    scene = scene_uniform_cube(2000, seed=0)
    cams = [look_at((0.0, 0.0, 3.0), width=128, height=128)]
    return scene, cams


def shell_100k_8views():
    """100k components on a noisy sphere shell, 8 cameras at 800x800, seed 1."""
    scene = scene_sphere_shell(100_000, seed=1)
    cams = sphere_cameras(8, width=800, height=800)
    return scene, cams


def clusters_1p5m_4views():
    """1.5M components (6 clusters + ground plane), 4 views at 1297x840, seed 2."""
    scene = scene_clusters_ground(1_500_000, seed=2)
    cams = sphere_cameras(4, width=1297, height=840)
    return scene, cams


def gradcheck_cube_50k():
    """50k components with the tiny-scene distribution, one 256x256 view, seed 3."""
    scene = scene_uniform_cube(50_000, seed=3)
    cams = [look_at((0.0, 0.0, 3.0), width=256, height=256)]
    return scene, cams


def serving_scenes(sizes=(200_000, 1_000_000, 3_000_000), seed=4):
    """Resident scenes for the render server (large-scene distribution)."""
    return [scene_clusters_ground(n, seed=seed + i) for i, n in enumerate(sizes)]


SERVE_RESOLUTIONS = ((256, 256), (800, 800), (1297, 840), (1920, 1080))


def subset_scene(scene: dict, idx) -> dict:
    """Components ``idx`` of ``scene`` (keeps the planar layout)."""
    idx = np.asarray(idx)
    out = {k: (np.ascontiguousarray(v[..., idx]) if isinstance(v, np.ndarray) else v)
           for k, v in scene.items()}
    out["n"] = int(len(idx))
    return out


def linear_loss_weights(cams, seed: int):
    """Seeded dL/dC images w ~ U(-1, 1), one [3][H][W] float32 array per view
    (the loss L = sum(w * C) has exactly dL/dC = w)."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, size=(3, c.height, c.width)).astype(np.float32)
            for c in cams]


def target_images(cams, seed: int):
    """Seeded target images in [0, 1] for the L1 training loss."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.0, 1.0, size=(3, c.height, c.width)).astype(np.float32)
            for c in cams]
