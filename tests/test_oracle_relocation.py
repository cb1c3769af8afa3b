"""Pins of the recycling oracle (oracle/relocation.py; Eq. relocation and the
SM's "Component Recycling") against closed forms, numerical integration and
counting -- independent of the oracle's own formulas."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import relocation as RL
from paper_2503_10148_gb300 import inputs


@pytest.mark.parametrize("o,nu", [(0.3, 1.0), (0.95, 4.0), (-0.6, 30.0)])
def test_one_copy_changes_nothing(o, nu):
    assert RL.relocated_opacity(o, 1) == pytest.approx(o, rel=1e-15)
    assert RL.scale_factor(o, nu, 1) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("o,N", [(0.3, 2), (0.99, 7), (-0.5, 3), (0.01, 32)])
def test_opacity_conservation(o, N):
    o_new = RL.relocated_opacity(o, N)
    assert math.copysign(1.0, o_new) == math.copysign(1.0, o)
    assert (1.0 - abs(o_new)) ** N == pytest.approx(1.0 - abs(o), rel=1e-13)


@pytest.mark.parametrize("alpha", [2.0, 3.5, 17.0])
def test_beta_equals_the_profile_integral(alpha):
    val, _ = integrate.quad(lambda u: (1.0 + u * u) ** (-alpha), -np.inf, np.inf, epsabs=0, epsrel=1e-13)
    assert RL.beta(0.5, alpha - 0.5) == pytest.approx(val, rel=1e-11)


@pytest.mark.parametrize("o,nu,N", [(0.5, 1.0, 2), (0.9, 3.0, 4), (0.99, 8.0, 7), (0.2, 25.0, 3), (-0.7, 2.0, 5)])
def test_integrated_colour_is_preserved(o, nu, N):
    """The recycled stack of N identical components (geometric sum of the
    compositing recurrence: 1 - (1 - o_new f)^N) carries the same integral
    along a ray as the old component (the condition Eq. relocation solves)."""
    sigma_old = 0.37
    F = RL.scale_factor(o, nu, N)
    o_new = abs(RL.relocated_opacity(o, N))
    e = -(nu + 3.0) / 2.0
    old, _ = integrate.quad(lambda x: abs(o) * (1 + x * x / (nu * sigma_old)) ** e, -np.inf, np.inf, epsrel=1e-12)
    new, _ = integrate.quad(lambda x: 1.0 - (1.0 - o_new * (1 + x * x / (nu * F * sigma_old)) ** e) ** N, -np.inf,
                            np.inf, epsrel=1e-12)
    assert new == pytest.approx(old, rel=1e-8)


def test_draws_follow_the_weights_and_hit_the_boundaries():
    w = np.array([0, 3, 0, 1, 4, 0, 2], np.int64)
    t = RL.draw_targets(w, 20000, seed=5, step=2)
    assert np.all(w[t] > 0)
    freq = np.bincount(t, minlength=len(w)) / len(t)
    assert np.allclose(freq, w / w.sum(), atol=0.012)
    # the draw maps x = 0 to the first live index and x = 2^32 - 1 to the last
    prefix = np.cumsum(w)
    W = int(prefix[-1])
    assert int(np.searchsorted(prefix, (0 * W) >> 32, side="right")) == 1
    assert int(np.searchsorted(prefix, ((2 ** 32 - 1) * W) >> 32, side="right")) == 6


def _scene(n, dead_frac, seed):
    sc = inputs.scene_uniform_cube(n, seed=seed)
    rng = np.random.default_rng(seed)
    dead = rng.random(n) < dead_frac
    sc["opacity_raw"] = np.where(dead, rng.uniform(-0.004, 0.004, n), sc["opacity_raw"])
    return sc, dead


def test_relocate_caps_copies_and_state():
    n = 4000
    sc, dead = _scene(n, 0.1, 3)
    mom = np.ones((3, n))
    m = np.ones((12, n))
    v = np.ones((12, n))
    out, r_, m_, v_, moved, tg = RL.relocate(sc, mom, m, v, n_max=3, seed=9, step=4)
    assert len(moved) <= int(0.05 * n) and len(moved) > 0
    assert np.all(dead[moved]) and not np.any(dead[tg])
    counts = np.bincount(tg, minlength=n)
    assert counts.max() <= 2  # n_max - 1
    o_old = np.tanh(sc["opacity_raw"])
    o_new = np.tanh(out["opacity_raw"])
    for t in np.unique(tg):
        N = counts[t] + 1
        assert (1 - abs(o_new[t])) ** N == pytest.approx(1 - abs(o_old[t]), rel=1e-12)
        assert np.sign(o_new[t]) == np.sign(o_old[t])
    for d, t in zip(moved, tg):
        for f in ("mean", "quat", "sh", "log_scale"):
            assert np.array_equal(out[f][:, d], out[f][:, t]), f
        assert out["nu"][d] == out["nu"][t] and out["opacity_raw"][d] == out["opacity_raw"][t]
        assert np.all(r_[:, d] == 0) and np.all(m_[:, d] == 0) and np.all(v_[:, d] == 0)
    untouched = np.setdiff1d(np.arange(n), np.concatenate([moved, tg]))
    assert np.array_equal(out["mean"][:, untouched], sc["mean"][:, untouched])
    assert np.all(r_[:, untouched] == 1)


def test_relocate_degenerate_cases():
    n = 500
    sc, _ = _scene(n, 0.0, 4)
    z = np.zeros((3, n))
    out, *_, moved, _ = RL.relocate(sc, z, np.zeros((12, n)), np.zeros((12, n)))
    assert len(moved) == 0 and np.array_equal(out["opacity_raw"], sc["opacity_raw"])
    sc["opacity_raw"] = np.zeros(n)  # everything dead: nothing to copy from
    out, *_, moved, _ = RL.relocate(sc, z, np.zeros((12, n)), np.zeros((12, n)))
    assert len(moved) == 0


def test_relocate_binding_cap_and_preserved_integral():
    """Few live components, many dead: the copy cap binds.  The number moved
    per target follows from the raw draws; every target's new scale, read
    back from its log-scale, preserves the integrated colour of Eq.
    relocation for the N that the target ended with."""
    n = 400
    sc = inputs.scene_uniform_cube(n, seed=6)
    rng = np.random.default_rng(6)
    live = rng.choice(n, 12, replace=False)
    raw = rng.uniform(-0.004, 0.004, n)
    raw[live] = sc["opacity_raw"][live]
    sc["opacity_raw"] = raw
    z = np.zeros((3, n))
    n_max = 3
    out, *_, moved, tg = RL.relocate(sc, z, np.zeros((12, n)), np.zeros((12, n)), n_max=n_max, max_fraction=0.25,
                                     seed=11, step=1)
    dead, w = RL.weights(raw, 0.005)
    draws = RL.draw_targets(w, int(0.25 * n), 11, 1)
    per = np.bincount(draws, minlength=n)
    assert len(moved) == int(np.minimum(per, n_max - 1).sum())
    counts = np.bincount(tg, minlength=n)
    assert counts.max() == n_max - 1
    o_old = np.tanh(raw)
    for t in np.unique(tg):
        N = counts[t] + 1
        F = np.exp(2.0 * (out["log_scale"][:, t] - sc["log_scale"][:, t]))
        assert np.allclose(F, F[0], rtol=1e-12)
        nu = float(sc["nu"][t])
        o_new = abs(np.tanh(out["opacity_raw"][t]))
        e = -(nu + 3.0) / 2.0
        old, _ = integrate.quad(lambda x: abs(o_old[t]) * (1 + x * x / nu) ** e, -np.inf, np.inf, epsrel=1e-12)
        new, _ = integrate.quad(lambda x: 1.0 - (1.0 - o_new * (1 + x * x / (nu * F[0])) ** e) ** N, -np.inf, np.inf,
                                epsrel=1e-12)
        assert new == pytest.approx(old, rel=1e-8), (t, N)
