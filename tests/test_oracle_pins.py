"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these calls the CUDA path.  Each test checks the oracle against
something other than itself: a library routine (scipy's spherical harmonics,
multivariate t density, quadrature, rotations), a closed form, a published
known-answer vector, an invariant, or brute force.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_10148_gb300 import inputs

TAU = 1.0 / 255.0


def _cfg(**kw):
    c = dict(oracle.DEFAULT_CFG)
    c.update(kw)
    return c


def _one_component(mean, log_scale, quat, nu, o, rgb=None, sh=None, sh_degree=0):
    n = 1
    if sh is None:
        sh = (np.asarray(rgb, np.float64) - 0.5) / (0.5 / math.sqrt(math.pi))
    return {
        "mean": np.asarray(mean, np.float64).reshape(3, 1),
        "log_scale": np.asarray(log_scale, np.float64).reshape(3, 1),
        "quat": np.asarray(quat, np.float64).reshape(4, 1),
        "nu": np.array([nu], np.float64), "opacity_raw": np.array([math.atanh(o)], np.float64),
        "sh": np.asarray(sh, np.float64).reshape(-1, 1), "sh_degree": sh_degree, "n": n,
    }


def _concat_scenes(a, b):
    out = {}
    for k in ("mean", "log_scale", "quat", "sh"):
        out[k] = np.concatenate([np.asarray(a[k], np.float64), np.asarray(b[k], np.float64)], axis=1)
    for k in ("nu", "opacity_raw"):
        out[k] = np.concatenate([np.asarray(a[k], np.float64), np.asarray(b[k], np.float64)])
    out["n"] = a["n"] + b["n"]
    out["sh_degree"] = a["sh_degree"]
    return out


# ---------------------------------------------------------------------------
# P9: Philox4x32-10 published known-answer vectors
# ---------------------------------------------------------------------------

def test_philox_known_answer_vectors(golden_dir):
    rows = 0
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            got = oracle.philox4x32_10(w[0:4], w[4:6])
            assert [int(x) for x in got] == w[6:10]
            rows += 1
    assert rows == 3


def test_philox_normals_moments_and_independence():
    """10^6 Box-Muller normals: mean 0, variance 1, no correlation between the
    three dimensions or between consecutive steps (counter-based streams)."""
    n = 200_000
    z = np.array([oracle.normals3(1234, 7, i) for i in range(n)])
    z2 = np.array([oracle.normals3(1234, 8, i) for i in range(n)])
    assert np.all(np.abs(z.mean(axis=0)) < 0.012)
    assert np.all(np.abs(z.var(axis=0) - 1.0) < 0.015)
    c = np.corrcoef(np.concatenate([z, z2[:, :1]], axis=1).T)
    assert np.max(np.abs(c - np.eye(4))) < 0.012
    # determinism: the same (seed, step, index) gives the same numbers
    assert np.array_equal(oracle.normals3(1234, 7, 5), z[5])
    # kurtosis of a normal is 3
    k = ((z - z.mean(0)) ** 4).mean(0) / z.var(0) ** 2
    assert np.all(np.abs(k - 3.0) < 0.08)


# ---------------------------------------------------------------------------
# Spherical harmonics against scipy's complex Y_l^m
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("degree", [0, 1, 2, 3, 6])
def test_sh_basis_matches_scipy(degree):
    rng = np.random.default_rng(degree)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta = math.acos(d[2])
        phi = math.atan2(d[1], d[0])
        ours = oracle.sh_basis(degree, d)
        for l in range(degree + 1):
            for m in range(-l, l + 1):
                Y = special.sph_harm_y(l, abs(m), theta, phi)
                if m == 0:
                    ref = Y.real
                elif m > 0:
                    ref = math.sqrt(2.0) * Y.real
                else:
                    ref = math.sqrt(2.0) * Y.imag
                assert ours[l * l + l + m] == pytest.approx(ref, abs=1e-13)


def test_sh_basis_is_orthonormal_on_sphere():
    """Monte-Carlo check of orthonormality over the unit sphere."""
    rng = np.random.default_rng(0)
    d = rng.normal(size=(40000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = np.array([oracle.sh_basis(3, x) for x in d])
    G = 4.0 * math.pi * (Y.T @ Y) / len(d)
    assert np.max(np.abs(G - np.eye(16))) < 0.06


# ---------------------------------------------------------------------------
# P1: marginalising the 3D t along a ray gives the 2D t (SM "Integral along a ray")
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_ray_marginal_is_2d_t(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    Sig = A @ A.T + 0.3 * np.eye(3)
    Pm = np.linalg.inv(Sig)
    nu = float(np.exp(rng.uniform(0.0, math.log(32.0))))
    mu = rng.normal(size=3)

    def t3(z, x1, x2):
        d = np.array([x1 - mu[0], x2 - mu[1], z - mu[2]])
        return (1.0 + d @ Pm @ d / nu) ** (-(nu + 3.0) / 2.0)

    centre, _ = integrate.quad(t3, -np.inf, np.inf, args=(mu[0], mu[1]), epsabs=0, epsrel=1e-12, limit=400)
    beta = special.beta(0.5, (nu + 2.0) / 2.0)
    assert centre == pytest.approx(beta * math.sqrt(nu / Pm[2, 2]), rel=1e-9)
    S2inv = np.linalg.inv(Sig[:2, :2])
    for _ in range(5):
        x = mu[:2] + rng.normal(size=2) * 2.0
        val, _ = integrate.quad(t3, -np.inf, np.inf, args=(x[0], x[1]), epsabs=0, epsrel=1e-12, limit=400)
        d = x - mu[:2]
        h = float(d @ S2inv @ d)
        assert val / centre == pytest.approx(oracle.t2d(h, nu), rel=1e-8)


# ---------------------------------------------------------------------------
# The 2D kernel against scipy's multivariate t density; nu = 1 (Cauchy)
# ---------------------------------------------------------------------------

def test_t2d_is_normalised_multivariate_t_ratio():
    rng = np.random.default_rng(1)
    for nu in (1.0, 1.7, 4.0, 31.0, 500.0):
        A = rng.normal(size=(2, 2))
        S = A @ A.T + 0.2 * np.eye(2)
        mt = stats.multivariate_t(loc=np.zeros(2), shape=S, df=nu)
        for _ in range(5):
            u = rng.normal(size=2) * 3
            h = float(u @ np.linalg.solve(S, u))
            assert oracle.t2d(h, nu) == pytest.approx(mt.pdf(u) / mt.pdf(np.zeros(2)), rel=1e-10)


def test_t2d_cauchy_closed_form():
    for h in (0.0, 0.1, 1.0, 7.5, 100.0):
        assert oracle.t2d(h, 1.0) == pytest.approx((1.0 + h) ** -1.5, rel=1e-14)


def test_t2d_gaussian_limit():
    for h in (0.0, 0.5, 2.0, 9.0):
        assert oracle.t2d(h, 1e8) == pytest.approx(math.exp(-h / 2.0), rel=1e-6)


# ---------------------------------------------------------------------------
# P2: projection -- mean2D, the EWA Jacobian, Sigma2D = (J W Sigma W^T J^T)_{1:2,1:2}
# ---------------------------------------------------------------------------

def _persp(p, cam):
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


@pytest.mark.parametrize("seed", range(5))
def test_projection_against_numeric_jacobian_and_scipy_rotation(seed):
    rng = np.random.default_rng(10 + seed)
    cam = inputs.look_at(np.array([0.4, -0.3, 3.2]), width=200, height=150)
    # non-square pixels and an off-centre principal point
    cam.fy = cam.fx * 0.83
    cam.cx, cam.cy = 97.25, 80.5
    mean = rng.uniform(-0.5, 0.5, size=3)
    ls = rng.normal(-2.0, 0.4, size=3)
    q = rng.normal(size=4)
    sc = _one_component(mean, ls, q * 1.7, 3.0, 0.8, rgb=[0.3, 0.4, 0.5])
    rec = oracle.project(sc, cam)[0]
    assert rec[oracle.P["valid"]] == 1.0
    R = cam.viewmat[:, :3]
    t = cam.viewmat[:, 3]
    p = R @ mean + t
    # the depth key is FP32 (it only orders and culls): within FP32 rounding
    assert rec[oracle.P["depth"]] == pytest.approx(p[2], rel=3e-7)
    m2 = _persp(p, cam)
    assert rec[oracle.P["mx"]] == pytest.approx(m2[0], rel=1e-13)
    assert rec[oracle.P["my"]] == pytest.approx(m2[1], rel=1e-13)
    # numeric Jacobian of the perspective map at p (central differences)
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1e-6 * max(1.0, abs(p[k]))
        J[:, k] = (_persp(p + e, cam) - _persp(p - e, cam)) / (2 * e[k])
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
    Sig = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
    S2 = J @ R @ Sig @ R.T @ J.T
    assert rec[oracle.P["cov_a"]] == pytest.approx(S2[0, 0], rel=1e-7)
    assert rec[oracle.P["cov_b"]] == pytest.approx(S2[0, 1], rel=1e-6, abs=1e-9 * abs(S2[0, 0]))
    assert rec[oracle.P["cov_c"]] == pytest.approx(S2[1, 1], rel=1e-7)
    C = np.linalg.inv(S2)
    assert rec[oracle.P["con_a"]] == pytest.approx(C[0, 0], rel=1e-6)
    assert rec[oracle.P["con_c"]] == pytest.approx(C[1, 1], rel=1e-6)


def test_affine_closure_by_sampling():
    """Samples of a 3D t pushed through the linearised camera map have the
    covariance nu/(nu-2) * Sigma2D, Sigma2D being the oracle's projection."""
    cam = inputs.look_at((0.0, 0.0, 3.0), width=256, height=256)
    mean = np.array([0.1, -0.2, 0.3])
    ls = np.array([-1.5, -2.0, -1.8])
    q = np.array([0.9, 0.2, -0.3, 0.1])
    nu = 8.0
    sc = _one_component(mean, ls, q, nu, 0.9, rgb=[0.5, 0.5, 0.5])
    rec = oracle.project(sc, cam)[0]
    R = cam.viewmat[:, :3]
    p = R @ mean + cam.viewmat[:, 3]
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1e-6
        J[:, k] = (_persp(p + e, cam) - _persp(p - e, cam)) / 2e-6
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
    x = stats.multivariate_t(loc=mean, shape=Sig, df=nu).rvs(size=400_000, random_state=3)
    y = (x - mean) @ (J @ R).T
    cov = np.cov(y.T) * (nu - 2.0) / nu
    ref = np.array([[rec[oracle.P["cov_a"]], rec[oracle.P["cov_b"]]],
                    [rec[oracle.P["cov_b"]], rec[oracle.P["cov_c"]]]])
    assert np.max(np.abs(cov - ref)) < 0.03 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# P3: a single component renders as rgb * o * T2D where |alpha| >= tau
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nu,o", [(1.0, 0.9), (3.3, -0.6), (25.0, 0.35), (2.0, -0.999), (6.0, 0.999)])
def test_single_component_closed_form(nu, o):
    cam = inputs.look_at((0.0, 0.0, 3.0), width=96, height=80)
    rng = np.random.default_rng(int(nu * 10))
    sh = rng.normal(0, 0.3, size=(16, 3))
    sh[0] += 1.0
    sc = _one_component([0.05, -0.04, 0.1], [-2.2, -2.6, -2.4], [0.8, 0.1, 0.3, -0.2], nu, o,
                        sh=sh.reshape(-1), sh_degree=3)
    rec = oracle.project(sc, cam)[0]
    # colour from scipy's spherical harmonics at the viewing direction
    d = np.array([0.05, -0.04, 0.1]) - cam.position
    d /= np.linalg.norm(d)
    th, ph = math.acos(d[2]), math.atan2(d[1], d[0])
    Y = []
    for l in range(4):
        for m in range(-l, l + 1):
            c = special.sph_harm_y(l, abs(m), th, ph)
            Y.append(c.real if m == 0 else math.sqrt(2) * (c.real if m > 0 else c.imag))
    rgb = np.maximum(np.asarray(Y) @ sh + 0.5, 0.0)
    assert np.allclose(rec[[oracle.P["r"], oracle.P["g"], oracle.P["b"]]], rgb, rtol=1e-12, atol=1e-14)
    out = oracle.render(oracle.project(sc, cam), cam, _cfg(t_min=0.0))
    S = np.array([[rec[oracle.P["cov_a"]], rec[oracle.P["cov_b"]]],
                  [rec[oracle.P["cov_b"]], rec[oracle.P["cov_c"]]]])
    m2 = np.array([rec[oracle.P["mx"]], rec[oracle.P["my"]]])
    mt = stats.multivariate_t(loc=m2, shape=S, df=nu)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    u = np.stack([xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5], axis=1)
    t2 = mt.pdf(u) / mt.pdf(m2)
    alpha = o * t2
    keep = np.abs(np.abs(alpha) - TAU) > 1e-6
    on = np.abs(alpha) >= TAU
    alpha = np.clip(alpha, -0.99, 0.99)  # reading: alpha limited to [-0.99, 0.99]
    if abs(o) > 0.99:
        assert np.sum(np.abs(alpha) == 0.99) > 0
    expect = np.where(on, alpha, 0.0)[None, :] * rgb[:, None]
    assert on.sum() > 50
    assert np.allclose(out["rgb"][:, keep], expect[:, keep], rtol=1e-9, atol=1e-12)
    assert np.allclose(out["T"][keep], np.where(on, 1.0 - alpha, 1.0)[keep], rtol=1e-12)
    # extent: every lit pixel lies inside the pixel box and tile rectangle
    lit = np.flatnonzero(np.abs(out["rgb"]).sum(axis=0) > 0)
    lx, ly = lit % cam.width, lit // cam.width
    assert lx.min() >= rec[oracle.P["px0"]] and lx.max() <= rec[oracle.P["px1"]]
    assert ly.min() >= rec[oracle.P["py0"]] and ly.max() <= rec[oracle.P["py1"]]
    # at h = h_max the alpha threshold is met exactly
    assert abs(o) * oracle.t2d(rec[oracle.P["hmax"]], nu) == pytest.approx(TAU, rel=1e-12)
    # and the pixel box is the tight one: the pixel centres between the
    # extreme x and y of the ellipse h = h_max, found here by sampling its
    # boundary d = sqrt(h_max) L (cos t, sin t) with L L^T = Sigma2D
    Lc = np.linalg.cholesky(S)
    t = np.linspace(0.0, 2.0 * math.pi, 200_001)
    d = math.sqrt(rec[oracle.P["hmax"]]) * (Lc @ np.stack([np.cos(t), np.sin(t)]))
    ex, ey = d[0].max(), d[1].max()
    assert rec[oracle.P["px0"]] == max(math.ceil(m2[0] - ex - 0.5), 0)
    assert rec[oracle.P["px1"]] == min(math.floor(m2[0] + ex - 0.5), cam.width - 1)
    assert rec[oracle.P["py0"]] == max(math.ceil(m2[1] - ey - 0.5), 0)
    assert rec[oracle.P["py1"]] == min(math.floor(m2[1] + ey - 0.5), cam.height - 1)


def test_projection_limits_nu_to_the_paper_range():
    """SM Implementation Details: nu is kept in [1, 1e4].  The projected nu is
    the limited one, and a component beyond the limit renders exactly as one
    at the limit."""
    cam = inputs.look_at((0.0, 0.0, 3.0), width=64, height=48)
    nus = [0.25, 1.0, 7.5, 9999.0, 1e4, 3e5]
    recs = [oracle.project(_one_component([0.02, 0.01, 0.0], [-1.9, -2.1, -2.0], [0.9, 0.2, -0.1, 0.3], nu, 0.7,
                                          rgb=[0.6, 0.3, 0.2]), cam)[0] for nu in nus]
    assert [r[oracle.P["nu"]] for r in recs] == [1.0, 1.0, 7.5, 9999.0, 1e4, 1e4]
    img = [oracle.render(r[None], cam, _cfg())["rgb"] for r in recs]
    assert np.array_equal(img[0], img[1]) and np.array_equal(img[4], img[5])
    assert not np.array_equal(img[3], img[4])


# ---------------------------------------------------------------------------
# P4: nu -> infinity gives a Gaussian splat compositor
# ---------------------------------------------------------------------------

def _gaussian_composite(proj, cam, tau):
    """Textbook Gaussian front-to-back compositor over the same 2D records."""
    valid = np.flatnonzero(proj[:, oracle.P["valid"]] != 0)
    order = valid[np.lexsort((valid, proj[valid, oracle.P["depth"]]))]
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    ux, uy = xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5
    T = np.ones_like(ux)
    C = np.zeros((3, ux.size))
    for i in order:
        r = proj[i]
        dx, dy = ux - r[oracle.P["mx"]], uy - r[oracle.P["my"]]
        h = r[oracle.P["con_a"]] * dx * dx + 2 * r[oracle.P["con_b"]] * dx * dy + r[oracle.P["con_c"]] * dy * dy
        a = r[oracle.P["o"]] * np.exp(-0.5 * h)
        a = np.where(np.abs(a) >= tau, np.clip(a, -0.99, 0.99), 0.0)
        C += r[[oracle.P["r"], oracle.P["g"], oracle.P["b"]]][:, None] * (a * T)[None]
        T = T * (1 - a)
    return C, T


def test_large_nu_matches_gaussian_compositor():
    sc = inputs.scene_uniform_cube(40, seed=11)
    sc = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["log_scale"] = sc["log_scale"] + 1.0
    sc["nu"] = np.full(40, 1e4)
    cam = inputs.look_at((0.0, 0.0, 3.0), width=64, height=64)
    tau = 1e-9
    cfg = _cfg(t_min=0.0, tau=tau)
    proj = oracle.project(sc, cam, cfg)
    out = oracle.render(proj, cam, cfg)
    Cg, Tg = _gaussian_composite(proj, cam, tau)
    hh = np.linspace(0, 200, 200001)
    delta = np.max(np.abs((1 + hh / 1e4) ** (-(1e4 + 2) / 2) - np.exp(-hh / 2)))
    assert delta < 1e-3
    bound = 4 * 40 * delta * max(1.0, proj[:, oracle.P["r"]:oracle.P["b"] + 1].max())
    assert np.max(np.abs(out["rgb"] - Cg)) < bound
    assert np.max(np.abs(out["T"] - Tg)) < bound
    # and the difference is not zero: the t kernel is not the Gaussian
    assert np.max(np.abs(out["rgb"] - Cg)) > 0


# ---------------------------------------------------------------------------
# P6: scooping only ever lowers accumulated density (Sec. 3.3, Fig. negative)
# ---------------------------------------------------------------------------

def test_scooping_lowers_and_splatting_raises_density():
    base = inputs.scene_uniform_cube(150, seed=5)
    base = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in base.items()}
    cam = inputs.look_at((0.0, 0.0, 3.0), width=64, height=64)
    cfg = _cfg(t_min=0.0)
    ref = oracle.render(oracle.project(base, cam, cfg), cam, cfg)
    for z in (-0.8, 0.0, 0.9):
        for o in (-0.7, 0.7):
            extra = _one_component([0.02, 0.03, z], [-1.6, -1.7, -1.5], [1, 0, 0, 0], 2.0, o, rgb=[0.2, 0.9, 0.4])
            out = oracle.render(oracle.project(_concat_scenes(base, extra), cam, cfg), cam, cfg)
            if o < 0:
                assert np.all(1 - out["T"] <= 1 - ref["T"] + 1e-14)
                assert np.any(1 - out["T"] < 1 - ref["T"] - 1e-3)
            else:
                assert np.all(1 - out["T"] >= 1 - ref["T"] - 1e-14)
    zero = _one_component([0.0, 0.0, 0.0], [-1.6, -1.7, -1.5], [1, 0, 0, 0], 2.0, 0.0, rgb=[1, 1, 1])
    out = oracle.render(oracle.project(_concat_scenes(base, zero), cam, cfg), cam, cfg)
    assert np.array_equal(out["rgb"], ref["rgb"]) and np.array_equal(out["T"], ref["T"])


def test_negative_component_carves_a_hole():
    """Torus idea of Fig. negative: a co-located negative component removes
    density at the centre while leaving the far ring untouched."""
    cam = inputs.look_at((0.0, 0.0, 3.0), width=64, height=64)
    cfg = _cfg(t_min=0.0)
    pos = _one_component([0, 0, 0], [-1.0, -1.0, -1.0], [1, 0, 0, 0], 5.0, 0.8, rgb=[1, 1, 1])
    neg = _one_component([0, 0, 0.001], [-2.2, -2.2, -2.2], [1, 0, 0, 0], 5.0, -0.9, rgb=[1, 1, 1])
    a = oracle.render(oracle.project(pos, cam, cfg), cam, cfg)
    b = oracle.render(oracle.project(_concat_scenes(pos, neg), cam, cfg), cam, cfg)
    centre = 32 * 64 + 32
    # transmittance is a product: the negative component multiplies it by
    # (1 - alpha_neg) = 1 + 0.9 T2D, close to 1.9 at the centre
    assert 1.85 < b["T"][centre] / a["T"][centre] <= 1.9
    assert 1 - b["T"][centre] < 0.8 * (1 - a["T"][centre])
    corner = 2 * 64 + 2
    assert b["T"][corner] == a["T"][corner]


# ---------------------------------------------------------------------------
# termination rule, depth order
# ---------------------------------------------------------------------------

def test_termination_keeps_transmittance_above_t_min():
    sc = inputs.scene_uniform_cube(8000, seed=0)
    cam = inputs.look_at((0.0, 0.0, 3.0), width=64, height=64)
    out = oracle.render(oracle.project(sc, cam), cam)
    assert out["T"].min() >= 1e-4
    off = oracle.render(oracle.project(sc, cam, _cfg(t_min=0.0)), cam, _cfg(t_min=0.0))
    assert off["T"].min() < 1e-4
    assert np.all(off["n_contrib"] >= out["n_contrib"])


def _ambiguity_scene(a_list, px, py, nu=2.0):
    """Components stacked on the optical axis (front to back by a small depth
    step) whose alpha at the centre of pixel (px, py) is a_list[k], seen by a
    48 x 40 camera."""
    cam = inputs.look_at((0.0, 0.0, 3.0), width=48, height=40)

    def build(o_list):
        comps = [_one_component([0.0, 0.0, -0.01 * k], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0], nu, o,
                                rgb=[0.9 - 0.2 * k, 0.3, 0.2 + 0.1 * k]) for k, o in enumerate(o_list)]
        sc = comps[0]
        for c in comps[1:]:
            sc = _concat_scenes(sc, c)
        return sc

    recs = oracle.project(build([0.5] * len(a_list)), cam)
    o_list = []
    for rec, a in zip(recs, a_list):
        dx, dy = px + 0.5 - rec[oracle.P["mx"]], py + 0.5 - rec[oracle.P["my"]]
        h = rec[oracle.P["con_a"]] * dx * dx + 2 * rec[oracle.P["con_b"]] * dx * dy + rec[oracle.P["con_c"]] * dy * dy
        o_list.append(a / oracle.t2d(h, nu))
    return build(o_list), cam


def test_ambiguous_decisions_flip_to_the_nearby_results():
    """A decision within the FP32 window is flagged and counted, and flipping
    it gives the result of a tiny perturbation across the threshold: an
    |alpha| 1e-7 above tau (included; flipped: as if just below, excluded),
    and a T' 1e-7 above t_min (continued; flipped: terminated before that
    splat, i.e. the image without it)."""
    px, py = 23, 19
    pix = np.array([py * 48 + px])
    up, cam = _ambiguity_scene([TAU * (1 + 1e-7)], px, py)
    down, _ = _ambiguity_scene([TAU * (1 - 1e-7)], px, py)
    far, _ = _ambiguity_scene([TAU * (1 - 1e-3)], px, py)
    r_up = oracle.render(oracle.project(up, cam), cam, _cfg(), pix)
    assert r_up["flags"][0] == oracle.F_NEAR_TAU and r_up["n_amb"][0] == 1 and r_up["n_contrib"][0] == 1
    r_flip = oracle.render(oracle.project(up, cam), cam, _cfg(), pix, flip=[1])
    r_down = oracle.render(oracle.project(down, cam), cam, _cfg(), pix)
    r_far = oracle.render(oracle.project(far, cam), cam, _cfg(), pix)
    assert r_down["flags"][0] == oracle.F_NEAR_TAU and r_far["flags"][0] == 0
    assert r_flip["n_contrib"][0] == 0 and np.array_equal(r_flip["rgb"], r_down["rgb"])
    assert np.array_equal(r_flip["rgb"], r_far["rgb"]) and r_flip["T"][0] == 1.0
    # termination: T after three splats 1e-7 above t_min
    t_min = 1e-4
    cfg = _cfg(t_min=t_min)
    T2 = (1.0 - 0.9) * (1.0 - 0.9)
    sc2, _ = _ambiguity_scene([0.9, 0.9, 1.0 - t_min * (1 + 1e-7) / T2, 0.5], px, py)
    r = oracle.render(oracle.project(sc2, cam), cam, cfg, pix)
    assert r["flags"][0] == oracle.F_NEAR_TMIN and r["n_amb"][0] == 1
    assert r["n_contrib"][0] == 3 and r["T"][0] == pytest.approx(t_min * (1 + 1e-7), rel=1e-9)
    rf = oracle.render(oracle.project(sc2, cam), cam, cfg, pix, flip=[1])
    assert rf["n_contrib"][0] == 2 and rf["T"][0] == pytest.approx(T2, rel=1e-12)
    two, _ = _ambiguity_scene([0.9, 0.9], px, py)
    r2 = oracle.render(oracle.project(two, cam), cam, cfg, pix)
    assert np.allclose(rf["rgb"], r2["rgb"], rtol=1e-12, atol=0)
    # the windows are narrow: a decision 1e-3 away is not ambiguous
    sc3, _ = _ambiguity_scene([0.9, 0.9, 1.0 - t_min * (1 + 1e-3) / T2, 0.5], px, py)
    assert oracle.render(oracle.project(sc3, cam), cam, cfg, pix)["flags"][0] == 0


def test_front_component_occludes_back_component():
    cam = inputs.look_at((0.0, 0.0, 3.0), width=32, height=32)
    front = _one_component([0, 0, 0.5], [-1.5] * 3, [1, 0, 0, 0], 2.0, 0.99, rgb=[1, 0, 0])
    back = _one_component([0, 0, -0.5], [-1.5] * 3, [1, 0, 0, 0], 2.0, 0.99, rgb=[0, 0, 1])
    for sc in (_concat_scenes(front, back), _concat_scenes(back, front)):
        out = oracle.render(oracle.project(sc, cam), cam)
        c = 16 * 32 + 16
        assert out["rgb"][0, c] > 0.9 and out["rgb"][2, c] < 0.1 * out["rgb"][0, c]


# ---------------------------------------------------------------------------
# P7: analytic FP64 gradients against FP64 central differences
# ---------------------------------------------------------------------------

def _grad_scene(n=160, seed=21):
    sc = inputs.scene_uniform_cube(n, seed=seed)
    rng = np.random.default_rng(seed)
    sh = rng.normal(0.0, 0.2, size=(48, n))
    sh[0:3] = sc["sh"]
    sc = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["sh"] = sh
    sc["sh_degree"] = 3
    sc["log_scale"] = sc["log_scale"] + 0.6
    return sc


def _pick_params(sc, per_group, seed):
    n, deg = sc["n"], sc["sh_degree"]
    sl = oracle.theta_slices(n, deg)
    rng = np.random.default_rng(seed)
    out = []
    for name in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        s = sl[name]
        out += [(name, int(j)) for j in rng.choice(np.arange(s.start, s.stop), per_group, replace=False)]
    return out


def test_analytic_gradient_matches_central_differences():
    sc = _grad_scene()
    cam = inputs.look_at((0.2, 0.1, 3.0), width=56, height=48)
    w = inputs.linear_loss_weights([cam], seed=9)
    theta = oracle.theta_from_scene(sc)
    g = oracle.backward(sc, [cam], None, w)
    picks = _pick_params(sc, 10, seed=2)
    fd, smooth = oracle.fd_gradient(theta, sc["n"], 3, [cam], None, w, [j for _, j in picks])
    checked = 0
    groups = {}
    for (name, j), f, ok in zip(picks, fd, smooth):
        groups.setdefault(name, []).append((g[j], f, ok))
    for name, vals in groups.items():
        scale = max(abs(f) for _, f, _ in vals)
        for a, f, ok in vals:
            if not ok:
                continue
            assert abs(a - f) <= 1e-6 * max(abs(f), 1e-3 * scale) + 1e-9, (name, a, f)
            checked += 1
        assert any(abs(f) > 0 for _, f, _ in vals), name
    assert checked >= 50


def test_summand_magnitudes_bound_the_gradient():
    """grad_abs sums operand magnitudes of the summands: it bounds |grad|
    (triangle inequality) and equals it for a single contributor on a black
    background (no subtraction inside the term)."""
    sc = _grad_scene(n=60, seed=4)
    cam = inputs.look_at((0.2, 0.1, 3.0), width=40, height=32)
    w = inputs.linear_loss_weights([cam], seed=2)
    g, g2, mag, mag2 = oracle.backward(sc, [cam], None, w, want_grad2d=True, want_abs=True)
    ga, g2a = mag.abs, mag2.abs
    assert np.all(ga >= np.abs(g) * (1 - 1e-12)) and np.all(g2a >= np.abs(g2) * (1 - 1e-12))
    assert np.any(ga > np.abs(g) * 1.5)  # cancellation does occur
    assert np.all(mag.absn >= ga * (1 - 1e-12))  # weights are contributor counts >= 1
    one = _one_component([0.05, -0.04, 0.1], [-2.2, -2.6, -2.4], [0.8, 0.1, 0.3, -0.2], 3.0, 0.7, rgb=[0.2, 0.5, 0.7])
    pix = [np.array([40 * 16 + 20], np.int64)]
    dl = [np.array([[0.3], [0.0], [0.0]])]  # one channel: no cancellation across channels
    g, g2, mag, mag2 = oracle.backward(one, [cam], None, dl, pix, want_grad2d=True, want_abs=True)
    g2a = mag2.abs
    # dL/do and dL/drgb of a lone contributor on black are single products
    keep = [5, 7, 8, 9]
    assert np.allclose(g2a[..., keep], np.abs(g2[..., keep]), rtol=1e-13, atol=0)
    assert np.all(g2a >= np.abs(g2) * (1 - 1e-13))


def test_paper_printed_nu_gradient_disagrees_with_differences():
    """The printed SM dT/dnu holds the exponent fixed; it misses the
    -1/2 ln(1 + h/nu) T2D term, so it fails against finite differences where
    the exact form passes."""
    sc = _grad_scene()
    cam = inputs.look_at((0.2, 0.1, 3.0), width=56, height=48)
    w = inputs.linear_loss_weights([cam], seed=9)
    theta = oracle.theta_from_scene(sc)
    sl = oracle.theta_slices(sc["n"], 3)["nu"]
    g_exact = oracle.backward(sc, [cam], None, w)
    g_paper = oracle.backward(sc, [cam], _cfg(nu_grad_mode=1), w)
    idx = [j for j in range(sl.start, sl.stop) if abs(g_exact[j]) > 1e-3][:12]
    fd, smooth = oracle.fd_gradient(theta, sc["n"], 3, [cam], None, w, idx)
    bad = 0
    for j, f, ok in zip(idx, fd, smooth):
        if not ok:
            continue
        assert abs(g_exact[j] - f) <= 1e-6 * abs(f) + 1e-9
        bad += abs(g_paper[j] - f) > 1e-2 * abs(f)
    assert bad >= len(idx) // 2
    # other groups are unaffected by the nu-gradient mode
    other = np.ones_like(theta, bool)
    other[sl] = False
    # (equal up to the summation order of the OpenMP accumulation)
    assert np.allclose(g_exact[other], g_paper[other], rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------------------
# P8: SGHMC special cases (Sec. 3.4 Eq. sigmoidUpdate, SM Eq. SGHMC)
# ---------------------------------------------------------------------------

def _step_setup(n=500, seed=3):
    sc = inputs.scene_uniform_cube(n, seed=seed)
    theta = oracle.theta_from_scene(sc)
    rng = np.random.default_rng(seed)
    grad = rng.normal(size=theta.shape)
    r = rng.normal(size=3 * n) * 0.1
    m = rng.normal(size=theta.shape) * 0.01
    v = np.abs(rng.normal(size=theta.shape)) * 0.01
    return sc, theta, grad, r, m, v


def test_sghmc_gate_open_is_textbook_sghmc():
    """g = 1: mu' = mu + eps r' (Chen et al. 2014 with M = I)."""
    sc, theta, grad, r, m, v = _step_setup()
    n = sc["n"]
    p = dict(t0=10.0, eps=2e-2, C=0.7)
    th, rr, _, _, xi = oracle.sghmc_step(theta, grad, r, m, v, n=n, sh_degree=0, params=p, seed=5, step=3)
    mu0, mu1 = theta[:3 * n], th[:3 * n]
    assert np.allclose(mu1 - mu0, p["eps"] * rr, rtol=1e-12, atol=1e-15)
    # and r' = (1 - eps C) r - eps G + sqrt(2 eps C) xi, xi the Philox normals
    assert np.allclose(xi[:, 7], oracle.normals3(5, 3, 7), rtol=0, atol=0)


def test_sghmc_heavy_ball_when_no_friction():
    """g = 1, C = 0: no noise, r' = r - eps G and mu' = mu + eps r' (heavy ball)."""
    sc, theta, grad, r, m, v = _step_setup()
    n = sc["n"]
    eps = 0.05
    th, rr, _, _, _ = oracle.sghmc_step(theta, grad, r, m, v, n=n, sh_degree=0,
                                       params=dict(t0=10.0, eps=eps, C=0.0), seed=1, step=0)
    assert np.allclose(rr, r - eps * grad[:3 * n], rtol=1e-13, atol=1e-16)
    assert np.allclose(th[:3 * n], theta[:3 * n] + eps * (r - eps * grad[:3 * n]), rtol=1e-13, atol=1e-16)


def test_sghmc_gate_closed_is_scaled_gradient_step():
    """g = 0: the SM notes mu is then updated by eps^2 G alone."""
    sc, theta, grad, r, m, v = _step_setup()
    n = sc["n"]
    eps = 0.03
    th, _, _, _, _ = oracle.sghmc_step(theta, grad, r, m, v, n=n, sh_degree=0,
                                      params=dict(t0=-10.0, eps=eps, C=0.5), seed=1, step=0)
    assert np.allclose(th[:3 * n], theta[:3 * n] - eps * eps * grad[:3 * n], rtol=1e-14, atol=1e-17)


def test_sghmc_gate_switches_at_opacity_threshold():
    """The gate is half open at |o| = 0.005, mostly open below, closed above
    (Sec. 3.4: active only for opacity lower than 0.005)."""
    n = 4
    sc = inputs.scene_uniform_cube(n, seed=0)
    theta = oracle.theta_from_scene(sc)
    ops = np.array([0.0, 0.005, -0.005, 0.2])
    theta[oracle.theta_slices(n, 0)["opacity_raw"]] = np.arctanh(ops)
    grad = np.zeros_like(theta)
    r = np.ones(3 * n)
    eps, C = 0.1, 0.0
    th, _, _, _, _ = oracle.sghmc_step(theta, grad, r, np.zeros_like(theta), np.zeros_like(theta), n=n,
                                      sh_degree=0, params=dict(eps=eps, C=C), seed=0, step=0)
    g = (th[:n] - theta[:n]) / eps  # first mean row: g * eps * r with r = 1
    assert g[1] == pytest.approx(0.5, abs=1e-12) and g[2] == pytest.approx(0.5, abs=1e-12)
    assert g[0] > 0.6 and g[3] < 1e-8


def test_burn_in_noise_scales_with_covariance():
    """Burn-in with an isotropic Sigma = s^2 I: the noise is s^2 times the
    post-burn-in noise and there is no friction term."""
    sc, theta, grad, r, m, v = _step_setup(n=50)
    n = sc["n"]
    sl = oracle.theta_slices(n, 0)
    theta[sl["log_scale"]] = -1.3
    theta[sl["opacity_raw"]] = 0.0  # g = sigmoid(0.5)
    p = dict(eps=0.02, C=0.4)
    th, _, _, _, xi = oracle.sghmc_step(theta, grad, r, m, v, n=n, sh_degree=0, params=p, burn_in=True,
                                       seed=8, step=2)
    gate = 1.0 / (1.0 + math.exp(-0.5))
    s2 = math.exp(-2.6)
    expect = theta[:3 * n] - p["eps"] ** 2 * grad[:3 * n] + gate * p["eps"] * math.sqrt(2 * p["eps"] * p["C"]) * s2 * xi.reshape(-1)
    assert np.allclose(th[:3 * n], expect, rtol=1e-12, atol=1e-15)


def test_burn_in_noise_is_anisotropic_covariance_times_xi():
    """Burn-in with a rotated, anisotropic Sigma = R diag(e^{2s}) R^T (Sec. 3.4:
    the noise is multiplied by Sigma during burn-in).  Sigma is built here from
    scipy's rotation of each quaternion (scalar-last order) and distinct
    log-scales per axis, so a transposed rotation (R^T D R) or a swapped axis
    in the oracle fails.  The momentum update keeps its friction term."""
    n = 40
    sc, theta, grad, r, m, v = _step_setup(n=n, seed=11)
    sl = oracle.theta_slices(n, 0)
    rng = np.random.default_rng(17)
    q = rng.normal(size=(4, n))
    q[0] += 0.3  # away from the identity, both signs of w present
    theta[sl["quat"]] = q.reshape(-1)
    ls = np.stack([np.full(n, -0.4), np.full(n, -1.1), np.full(n, -2.0)]) + rng.uniform(-0.2, 0.2, (3, n))
    theta[sl["log_scale"]] = ls.reshape(-1)
    o = rng.uniform(-0.02, 0.02, n)
    theta[sl["opacity_raw"]] = np.arctanh(o)
    p = dict(eps=0.03, C=0.6, k=100.0, t0=0.005)
    th, rr, _, _, xi = oracle.sghmc_step(theta, grad, r, m, v, n=n, sh_degree=0, params=p, burn_in=True,
                                        seed=21, step=6)
    rot = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], axis=1)).as_matrix()  # [n][3][3]
    D = np.exp(2.0 * ls).T  # [n][3]
    Sigma = np.einsum("nij,nj,nkj->nik", rot, D, rot)
    noise = np.einsum("nij,jn->in", Sigma, xi)  # [3][n]
    gate = 1.0 / (1.0 + np.exp(p["k"] * (np.abs(o) - p["t0"])))
    sq = math.sqrt(2.0 * p["eps"] * p["C"])
    G = grad[:3 * n].reshape(3, n)
    mu0 = theta[:3 * n].reshape(3, n)
    expect_mu = mu0 - p["eps"] ** 2 * G + gate * p["eps"] * sq * noise
    assert np.allclose(th[:3 * n].reshape(3, n), expect_mu, rtol=1e-12, atol=1e-15)
    expect_r = (1.0 - p["eps"] * p["C"]) * r.reshape(3, n) - p["eps"] * G + sq * xi
    assert np.allclose(rr.reshape(3, n), expect_r, rtol=1e-12, atol=1e-15)
    # the rotation matters: with R^T D R the displacement would differ
    wrong = np.einsum("nji,nj,njk->nik", rot, D, rot)
    assert np.max(np.abs(np.einsum("nij,jn->in", wrong, xi) - noise)) > 1e-3


def test_adam_two_steps_from_nonzero_moments_follow_the_recurrence():
    """Two consecutive steps from non-zero first and second moments (Adam,
    Kingma & Ba 2015, on every group but the means): the recurrence written
    out here, with the bias corrections of steps t = s + 1 and s + 2.  The
    moments differ from each other and from zero, so an update that mixes m
    and v, drops a bias correction or uses the wrong step fails."""
    n = 60
    sc, theta, grad, r, _, _ = _step_setup(n=n, seed=13)
    rng = np.random.default_rng(29)
    m0 = rng.normal(size=theta.shape) * 0.3
    v0 = rng.uniform(0.05, 2.0, size=theta.shape)
    grad2 = rng.normal(size=theta.shape)
    lr = (1e-2, 2e-3, 5e-2, 3e-2, 4e-3)
    b1, b2, eps_a = 0.85, 0.995, 1e-6
    p = dict(lr=lr, beta1=b1, beta2=b2, adam_eps=eps_a)
    s = 4
    th1, r1, m1, v1, _ = oracle.sghmc_step(theta, grad, r, m0, v0, n=n, sh_degree=0, params=p, seed=2, step=s)
    th2, _, m2, v2, _ = oracle.sghmc_step(th1, grad2, r1, m1, v1, n=n, sh_degree=0, params=p, seed=2, step=s + 1)
    sl = oracle.theta_slices(n, 0)
    for name, l in zip(("log_scale", "quat", "nu", "opacity_raw", "sh"), lr):
        j = sl[name]
        pp, mm, vv = theta[j].copy(), m0[j].copy(), v0[j].copy()
        for t, g in ((s + 1, grad[j]), (s + 2, grad2[j])):
            mm = b1 * mm + (1.0 - b1) * g
            vv = b2 * vv + (1.0 - b2) * g * g
            pp = pp - l * (mm / (1.0 - b1 ** t)) / (np.sqrt(vv / (1.0 - b2 ** t)) + eps_a)
            if name == "nu":
                pp = np.clip(pp, 1.0, 1e4)
        assert np.allclose(m2[j], mm, rtol=1e-13, atol=0)
        assert np.allclose(v2[j], vv, rtol=1e-13, atol=0)
        assert np.allclose(th2[j], pp, rtol=1e-12, atol=1e-15)


def test_adam_first_step_moves_by_learning_rate():
    """First Adam step with zero moments: |delta p| = lr |g| / (|g| + eps)."""
    sc, theta, grad, r, _, _ = _step_setup(n=200)
    n = sc["n"]
    lr = (1e-2, 2e-3, 5e-2, 3e-2, 4e-3)
    th, _, m1, v1, _ = oracle.sghmc_step(theta, grad, r, np.zeros_like(theta), np.zeros_like(theta), n=n,
                                        sh_degree=0, params=dict(lr=lr), seed=0, step=0)
    sl = oracle.theta_slices(n, 0)
    for name, l in zip(("log_scale", "quat", "opacity_raw", "sh"), (lr[0], lr[1], lr[3], lr[4])):
        d = th[sl[name]] - theta[sl[name]]
        assert np.allclose(np.abs(d), l, rtol=1e-9)
        assert np.all(np.sign(d) == -np.sign(grad[sl[name]]))
    nu_new = th[sl["nu"]]
    assert np.all(nu_new >= 1.0) and np.all(nu_new <= 1e4)


def test_nu_is_limited_after_update():
    sc, theta, grad, r, m, v = _step_setup(n=20)
    n = sc["n"]
    sl = oracle.theta_slices(n, 0)["nu"]
    theta[sl] = 1.0
    grad[sl] = 1.0  # pushes nu down
    th, *_ = oracle.sghmc_step(theta, grad, r, np.zeros_like(theta), np.zeros_like(theta), n=n, sh_degree=0,
                               params=dict(lr=(0, 0, 0.5, 0, 0)), seed=0, step=0)
    assert np.all(th[sl] == 1.0)


# ---------------------------------------------------------------------------
# P10: tile-list reference against brute force
# ---------------------------------------------------------------------------

def test_bin_sort_reference_matches_brute_force():
    rng = np.random.default_rng(4)
    E = 300
    tiles_x = np.array([7] * 150 + [5] * 150)
    tile_base = np.array([0] * 150 + [7 * 6] * 150)
    rects = []
    for e in range(E):
        tx0 = rng.integers(0, tiles_x[e]); tx1 = rng.integers(tx0 - 1, tiles_x[e])
        ty0 = rng.integers(0, 6); ty1 = rng.integers(ty0, 6)
        rects.append((tx0, tx1, ty0, ty1))
    depth_bits = rng.integers(0, 50, size=E).astype(np.uint32)  # many ties
    tiles, ents = oracle.bin_sort_reference(rects, depth_bits, tiles_x, tile_base)
    brute = []
    for e, (tx0, tx1, ty0, ty1) in enumerate(rects):
        for ty in range(ty0, ty1 + 1):
            for tx in range(tx0, tx1 + 1):
                brute.append((int(tile_base[e] + ty * tiles_x[e] + tx), int(depth_bits[e]), e))
    brute.sort()
    assert list(tiles) == [b[0] for b in brute]
    assert list(ents) == [b[2] for b in brute]
