"""The seeded synthetic inputs follow the recipes they state (no GPU):
distributions of scale, nu, opacity sign and size, rotations, colour
coefficients, the cluster / ground split of the large-scene recipe, the
named workloads' sizes, and determinism under a seed."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2503_10148_gb300 import inputs  # noqa: E402


def _opacity(scene):
    return np.tanh(scene["opacity_raw"].astype(np.float64))


def _check_common(scene, n, ls_mu, ls_sd, nu_hi, frac_neg, sh_deg):
    assert scene["n"] == n and scene["sh_degree"] == sh_deg
    assert scene["mean"].shape == (3, n) and scene["log_scale"].shape == (3, n)
    assert scene["quat"].shape == (4, n) and scene["nu"].shape == (n,) and scene["opacity_raw"].shape == (n,)
    assert scene["sh"].shape == (3 * (sh_deg + 1) ** 2, n)
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        assert scene[f].dtype == np.float32 and scene[f].flags.c_contiguous
    se = 5.0 / math.sqrt(3 * n)  # 5 standard errors
    ls = scene["log_scale"].astype(np.float64)
    assert abs(ls.mean() - ls_mu) < 5 * ls_sd / math.sqrt(3 * n) and abs(ls.std() - ls_sd) < ls_sd * se
    q = scene["quat"].astype(np.float64)
    assert np.allclose(np.linalg.norm(q, axis=0), 1.0, atol=1e-6)
    nu = scene["nu"].astype(np.float64)
    assert nu.min() >= 1.0 - 1e-6 and nu.max() <= nu_hi * (1 + 1e-6)
    # log-uniform: log nu uniform on [0, log hi], mean log(hi) / 2, sd log(hi) / sqrt(12)
    lg = np.log(nu)
    assert abs(lg.mean() - math.log(nu_hi) / 2) < 5 * math.log(nu_hi) / math.sqrt(12 * n)
    o = _opacity(scene)
    a = np.abs(o)
    assert a.min() >= 0.05 - 1e-6 and a.max() <= 0.9 + 1e-6
    assert abs(np.mean(o < 0) - frac_neg) <= 1.0 / n  # the scooping fraction, exactly rounded
    assert abs(a.mean() - 0.475) < 5 * 0.245 / math.sqrt(n)  # |o| ~ U(0.05, 0.9)


def test_tiny_scene_recipe():
    s = inputs.scene_uniform_cube(40_000, seed=5)
    _check_common(s, 40_000, -3.0, 0.5, 8.0, 0.20, 0)
    m = s["mean"]
    assert m.min() >= -1.0 and m.max() <= 1.0 and abs(float(m.mean())) < 0.01
    rgb = s["sh"].astype(np.float64) * 0.28209479177387814 + 0.5  # SH degree 0: rgb = Y00 c + 0.5
    assert rgb.min() >= -1e-6 and rgb.max() <= 1 + 1e-6 and abs(rgb.mean() - 0.5) < 0.01


def test_shell_recipe():
    s = inputs.scene_sphere_shell(40_000, seed=6)
    _check_common(s, 40_000, -4.0, 0.5, 16.0, 0.25, 3)
    r = np.linalg.norm(s["mean"].astype(np.float64), axis=0)
    assert abs(r.mean() - 1.0) < 0.002 and abs(r.std() - 0.05) < 0.002
    sh = s["sh"].astype(np.float64)
    assert abs(sh.mean()) < 0.002 and abs(sh.std() - 0.1) < 0.002


def test_large_scene_recipe_clusters_and_ground():
    n = 100_000
    s = inputs.scene_clusters_ground(n, seed=7)
    _check_common(s, n, -4.0, 0.7, 32.0, 0.30, 3)
    y = s["mean"][1].astype(np.float64)
    x, z = s["mean"][0].astype(np.float64), s["mean"][2].astype(np.float64)
    ground = (np.abs(y + 1.0) < 0.05) & (np.abs(x) <= 2.0) & (np.abs(z) <= 2.0)
    # 20 % on the ground plane (plus the few cluster points that fall in the slab)
    assert 0.20 <= ground.mean() < 0.21
    gy = y[ground]
    assert abs(gy.mean() + 1.0) < 0.001 and abs(gy.std() - 0.01) < 0.002
    sh = s["sh"].astype(np.float64)
    assert abs(sh.std() - 0.1) < 0.002


def test_named_workloads_sizes_and_cameras():
    s, cams = inputs.tiny_cube_2k()
    assert s["n"] == 2000 and [(c.width, c.height) for c in cams] == [(128, 128)]
    s, cams = inputs.gradcheck_cube_50k()
    assert s["n"] == 50_000 and [(c.width, c.height) for c in cams] == [(256, 256)]
    s, cams = inputs.shell_100k_8views()
    assert s["n"] == 100_000 and s["sh_degree"] == 3 and [(c.width, c.height) for c in cams] == [(800, 800)] * 8
    s, cams = inputs.clusters_1p5m_4views()
    assert s["n"] == 1_500_000 and s["sh_degree"] == 3 and [(c.width, c.height) for c in cams] == [(1297, 840)] * 4
    assert inputs.SERVE_RESOLUTIONS == ((256, 256), (800, 800), (1297, 840), (1920, 1080))


@pytest.mark.parametrize("gen", [inputs.scene_uniform_cube, inputs.scene_sphere_shell, inputs.scene_clusters_ground])
def test_generators_are_deterministic_under_a_seed(gen):
    a, b, c = gen(3000, seed=11), gen(3000, seed=11), gen(3000, seed=12)
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        assert np.array_equal(a[f], b[f]), f
    assert not np.array_equal(a["mean"], c["mean"])


def test_cameras_look_at_the_target_with_a_50_degree_horizontal_fov():
    cams = inputs.sphere_cameras(6, width=1297, height=840)
    for c in cams:
        V = np.asarray(c.viewmat, dtype=np.float64).reshape(3, 4)
        R, t = V[:, :3], V[:, 3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) > 0
        centre = -R.T @ t
        assert abs(np.linalg.norm(centre) - 3.0) < 1e-9  # on the radius-3 sphere
        p = R @ np.zeros(3) + t  # the origin, in camera coordinates
        assert p[2] > 0 and abs(p[0]) < 1e-9 and abs(p[1]) < 1e-9  # straight ahead
        assert c.fx == c.fy and abs(2 * math.degrees(math.atan(c.width / (2 * c.fx))) - 50.0) < 1e-9
        assert (c.cx, c.cy) == (c.width / 2, c.height / 2)
    d = inputs.fibonacci_directions(64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0) and np.linalg.norm(d.mean(0)) < 0.05
