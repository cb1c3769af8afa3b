"""Component recycling on the GPU (sss_relocate) against the FP64 oracle.

Index work (which components move, where to) is compared exactly: the
parameters a copy takes from its target are bit-identical, and the set of
moved components follows from them.  The recomputed opacity and log-scales
are FP64 on both sides, rounded to FP32 once: 2 ulp."""
import numpy as np
import pytest
import torch

from oracle import relocation as RL
from paper_2503_10148_gb300 import frame, inputs

from gpu_util import DEV, f32_scene, require_gpu

pytestmark = pytest.mark.gpu

DEAD = float(np.float32(0.005))
FRAC = float(np.float32(0.05))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _scene(n, dead_frac, seed, sh_degree=0, live=None):
    sc = inputs.scene_uniform_cube(n, seed=seed)
    if sh_degree:
        rng = np.random.default_rng(seed + 100)
        K = (sh_degree + 1) ** 2
        sc["sh"] = rng.normal(0, 0.1, size=(3 * K, n))
        sc["sh_degree"] = sh_degree
    rng = np.random.default_rng(seed)
    dead = rng.random(n) < dead_frac
    sc["opacity_raw"] = np.where(dead, rng.uniform(-0.004, 0.004, n), sc["opacity_raw"])
    if live is not None:
        keep = rng.choice(n, live, replace=False)
        raw = rng.uniform(-0.004, 0.004, n)
        raw[keep] = sc["opacity_raw"][keep]
        sc["opacity_raw"] = raw
    return f32_scene(sc)


def _run(sc_np, **kw):
    sc = frame.Scene.from_numpy(sc_np, DEV)
    st = frame.SamplerState(sc)
    for t in (st.r, st.m, st.v):
        t.fill_(1.0)
    moved = frame.relocate(sc, st, dead_opacity=DEAD, **kw)
    torch.cuda.synchronize()
    return sc.to_numpy(), st, int(moved.cpu()[0])


def _ulps(a, b):
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    return np.abs(a.view(np.int32).astype(np.int64) - b.view(np.int32).astype(np.int64))


def _compare(sc_np, n_max, max_fraction=FRAC, seed=3, step=5):
    got, st, n_moved = _run(sc_np, max_fraction=max_fraction, n_max=n_max, seed=seed, step=step)
    n = sc_np["n"]
    K = (sc_np["sh_degree"] + 1) ** 2
    ones = np.ones
    want, r_, m_, v_, moved, tg = RL.relocate(sc_np, ones((3, n)), ones((9 + 3 * K, n)), ones((9 + 3 * K, n)),
                                              dead_opacity=DEAD, max_fraction=max_fraction, n_max=n_max, seed=seed,
                                              step=step)
    assert n_moved == len(moved)
    for f in ("mean", "quat", "sh"):
        assert np.array_equal(got[f], want[f].astype(np.float32)), f
    assert np.array_equal(got["nu"], want["nu"].astype(np.float32))
    assert _ulps(got["opacity_raw"], want["opacity_raw"]).max() <= 2
    assert _ulps(got["log_scale"], want["log_scale"]).max() <= 2
    assert np.array_equal(st.r.cpu().numpy(), r_.astype(np.float32))
    assert np.array_equal(st.m.cpu().numpy(), m_.astype(np.float32))
    assert np.array_equal(st.v.cpu().numpy(), v_.astype(np.float32))
    return n_moved, moved, tg


def test_relocate_matches_oracle_small():
    n_moved, moved, tg = _compare(_scene(4000, 0.1, 3), n_max=32)
    assert n_moved == int(FRAC * 4000)


def test_relocate_matches_oracle_binding_cap_sh3():
    sc = _scene(3000, 0.0, 4, sh_degree=3, live=15)
    n_moved, moved, tg = _compare(sc, n_max=3, max_fraction=float(np.float32(0.3)))
    assert np.bincount(tg).max() == 2 and n_moved < int(np.float32(0.3) * 3000)


def test_relocate_matches_oracle_200k():
    n_moved, _, _ = _compare(_scene(200_000, 0.08, 5), n_max=32, seed=12, step=77)
    assert n_moved == int(FRAC * 200_000)


def test_relocate_degenerate_inputs():
    sc = _scene(2000, 0.0, 6)
    got, st, n_moved = _run(sc)
    assert n_moved == 0 and np.array_equal(got["opacity_raw"], sc["opacity_raw"].astype(np.float32))
    sc["opacity_raw"] = np.zeros(2000, np.float32)  # nothing alive to copy from
    got, st, n_moved = _run(sc)
    assert n_moved == 0 and np.all(st.r.cpu().numpy() == 1.0)
