"""Pins of the oracle's variants (the Adam gradient in SGHMC) against closed
forms."""
import numpy as np
import pytest

import oracle


def test_adam_gradient_with_a_constant_gradient_is_g_over_abs_g():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step, so the normalised gradient is g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    g = rng.normal(size=20) * 10.0 ** rng.uniform(-6, 1, size=20)
    m = np.zeros(20)
    v = np.zeros(20)
    for step in range(5):
        G, m, v = oracle.adam_preconditioned(g, m, v, step=step, beta1=0.9, beta2=0.999, adam_eps=1e-8)
        assert np.allclose(G, g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_adam_gradient_first_step_and_moment_updates():
    g = np.array([2.0, -0.5, 0.0])
    m0 = np.array([0.1, 0.2, 0.3])
    v0 = np.array([0.01, 0.02, 0.03])
    G, m, v = oracle.adam_preconditioned(g, m0, v0, step=3, beta1=0.8, beta2=0.99, adam_eps=1e-6)
    assert np.allclose(m, 0.8 * m0 + 0.2 * g) and np.allclose(v, 0.99 * v0 + 0.01 * g * g)
    want = (m / (1 - 0.8 ** 4)) / (np.sqrt(v / (1 - 0.99 ** 4)) + 1e-6)
    assert np.allclose(G, want, rtol=1e-14)


# --------------------------------------------------------------------- Gaussian kernel (nu -> infinity)

def test_gaussian_kernel_mode_is_the_textbook_gaussian_compositor():
    """kernel = 1 renders exp(-h/2) splats: equal, to rounding, to a textbook
    Gaussian front-to-back compositor over the same 2D records, with the
    extent h <= 2 ln(|o|/tau)."""
    from test_oracle_pins import _cfg, _gaussian_composite
    from paper_2503_10148_gb300 import inputs
    sc = inputs.scene_uniform_cube(60, seed=12)
    sc = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["log_scale"] = sc["log_scale"] + 1.0
    cam = inputs.look_at((0.0, 0.0, 3.0), width=48, height=40)
    tau = 1e-9
    cfg = dict(_cfg(t_min=0.0, tau=tau), kernel=1)
    proj = oracle.project(sc, cam, cfg)
    o = np.abs(proj[:, oracle.P["o"]])
    valid = proj[:, oracle.P["valid"]] != 0
    assert np.allclose(proj[valid, oracle.P["hmax"]], 2.0 * np.log(o[valid] / tau), rtol=1e-12)
    out = oracle.render(proj, cam, cfg)
    Cg, Tg = _gaussian_composite(proj, cam, tau)
    assert np.max(np.abs(out["rgb"] - Cg)) < 1e-12 and np.max(np.abs(out["T"] - Tg)) < 1e-12


def test_gaussian_kernel_gradient_against_differences():
    """Analytic gradient of the Gaussian mode against central differences of
    its own forward (nu gets no gradient)."""
    from test_oracle_pins import _cfg
    from paper_2503_10148_gb300 import inputs
    sc = inputs.scene_uniform_cube(30, seed=13)
    sc = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    cam = inputs.look_at((0.0, 0.3, 3.0), width=40, height=32)
    cfg = dict(_cfg(t_min=0.0), kernel=1)
    ws = inputs.linear_loss_weights([cam], 4)
    g = oracle.backward(sc, [cam], cfg, ws)
    n = sc["n"]
    sl = oracle.theta_slices(n, 0)
    theta = oracle.theta_from_scene(sc)
    assert np.all(g[sl["nu"]] == 0.0)
    rng = np.random.default_rng(1)
    picks = []
    for name in ("mean", "log_scale", "quat", "opacity_raw", "sh"):
        cand = np.arange(sl[name].start, sl[name].stop)
        cand = cand[np.abs(g[cand]) > 1e-3 * np.abs(g[sl[name]]).max()]
        picks += list(rng.choice(cand, 4, replace=False))
    fd, smooth = oracle.fd_gradient(theta, n, 0, [cam], cfg, ws, picks)
    for j, f, ok in zip(picks, fd, smooth):
        if ok:
            assert g[j] == pytest.approx(f, rel=1e-5, abs=1e-9)
