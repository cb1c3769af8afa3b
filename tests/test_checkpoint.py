"""Checkpoint and resume (no GPU): exact round trip of everything the
sampler step reads, in-place loads that keep the tensors' memory, refusal
of mismatched or damaged files, atomic replacement, and a resumed step that
matches the uninterrupted one (the oracle's step stands in for the kernel:
both are functions of the same saved state)."""
import os
import sys

import numpy as np
import pytest
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2503_10148_gb300 import checkpoint, frame, inputs  # noqa: E402

STEP = (1 << 32) + 7  # beyond 32 bits: both words of the Philox counter matter
SEED = (1 << 40) + 99


def _run_state(n=500, deg=3, seed=0):
    rng = np.random.default_rng(seed)
    sc = frame.Scene.from_numpy(inputs.scene_sphere_shell(n, seed=seed + 1), "cpu") if deg == 3 else \
        frame.Scene.from_numpy(inputs.scene_uniform_cube(n, seed=seed + 1), "cpu")
    st = frame.SamplerState(sc)
    for x in (st.r, st.m, st.v):
        x.copy_(torch.as_tensor(rng.normal(size=tuple(x.shape)).astype(np.float32)))
    st.v.abs_()
    return sc, st


def test_round_trip_is_exact(tmp_path):
    sc, st = _run_state()
    mu = (torch.randn(3, sc.n), torch.rand(3, sc.n))
    path = str(tmp_path / "run.ckpt")
    checkpoint.save(path, sc, st, torch.tensor([STEP], dtype=torch.int64), seed=SEED, mu_adam=mu)
    got = checkpoint.load(path, device="cpu")
    assert got["step"] == STEP and got["seed"] == SEED
    for f in frame.FIELDS:
        assert torch.equal(got["scene"].t[f], sc.t[f]), f
    for a, b in ((got["state"].r, st.r), (got["state"].m, st.m), (got["state"].v, st.v)):
        assert torch.equal(a, b)
    assert torch.equal(got["mu_adam"][0], mu[0]) and torch.equal(got["mu_adam"][1], mu[1])
    assert got["scene"].n == sc.n and got["scene"].sh_degree == sc.sh_degree


def test_load_into_keeps_the_tensors_memory_and_sets_the_step_counter(tmp_path):
    sc, st = _run_state(seed=3)
    path = str(tmp_path / "run.ckpt")
    checkpoint.save(path, sc, st, STEP, seed=SEED)
    dst_sc, dst_st = sc.zeros_like(), frame.SamplerState(sc)
    ptrs = [dst_sc.t[f].data_ptr() for f in frame.FIELDS] + [dst_st.r.data_ptr(), dst_st.m.data_ptr()]
    counter = torch.zeros(1, dtype=torch.int64)
    meta = checkpoint.load_into(path, dst_sc, dst_st, step_counter=counter)
    assert meta == {"step": STEP, "seed": SEED} and int(counter) == STEP
    assert ptrs == [dst_sc.t[f].data_ptr() for f in frame.FIELDS] + [dst_st.r.data_ptr(), dst_st.m.data_ptr()]
    for f in frame.FIELDS:
        assert torch.equal(dst_sc.t[f], sc.t[f]), f
    assert torch.equal(dst_st.v, st.v)


def test_mismatches_and_damaged_files_are_refused(tmp_path):
    sc, st = _run_state()
    path = str(tmp_path / "run.ckpt")
    checkpoint.save(path, sc, st, 5)
    other, other_st = _run_state(n=499)
    with pytest.raises(ValueError, match="n=500"):
        checkpoint.load_into(path, other, other_st)
    small, small_st = _run_state(n=500, deg=0)
    with pytest.raises(ValueError):
        checkpoint.load_into(path, small, small_st)
    with pytest.raises(ValueError, match="dL/dmu"):
        checkpoint.load_into(path, sc, st, mu_adam=(torch.zeros(3, 500), torch.zeros(3, 500)))
    bad = str(tmp_path / "bad.npz")
    with open(path, "rb") as f, open(bad, "wb") as g:
        z = dict(np.load(f))
        z["sampler_m"] = z["sampler_m"][:-1]  # one row short
        np.savez(g, **z)
    with pytest.raises(ValueError, match="sampler_m"):
        checkpoint.load(bad, device="cpu")
    with pytest.raises(ValueError):
        checkpoint.save(str(tmp_path / "x"), sc, st, -1)


def test_a_failed_save_leaves_the_previous_checkpoint(tmp_path, monkeypatch):
    sc, st = _run_state()
    path = str(tmp_path / "run.ckpt")
    checkpoint.save(path, sc, st, 1)
    before = open(path, "rb").read()

    def boom(*a, **k):
        raise OSError("disk full")

    monkeypatch.setattr(checkpoint.np, "savez", boom)
    with pytest.raises(OSError):
        checkpoint.save(path, sc, st, 2)
    assert open(path, "rb").read() == before
    assert sorted(os.listdir(tmp_path)) == ["run.ckpt"]  # no temporary left behind


def _oracle_args(sc, st):
    """The scene and state in the oracle's layout (moments with unused mean rows)."""
    n = sc.n
    theta = oracle.theta_from_scene(sc.to_numpy())
    pad = np.zeros(3 * n)
    m = np.concatenate([pad, st.m.numpy().astype(np.float64).reshape(-1)])
    v = np.concatenate([pad, st.v.numpy().astype(np.float64).reshape(-1)])
    return theta, st.r.numpy().astype(np.float64).reshape(-1), m, v


def _store(sc, st, theta, r, m, v):
    """Write an oracle state back as the FP32 arrays a run keeps."""
    n = sc.n
    sl = oracle.theta_slices(n, sc.sh_degree)
    for f in frame.FIELDS:
        sc.t[f].copy_(torch.as_tensor(theta[sl[f]].astype(np.float32).reshape(sc.t[f].shape)))
    st.r.copy_(torch.as_tensor(r.astype(np.float32).reshape(3, n)))
    st.m.copy_(torch.as_tensor(m[3 * n:].astype(np.float32).reshape(st.m.shape)))
    st.v.copy_(torch.as_tensor(v[3 * n:].astype(np.float32).reshape(st.v.shape)))


def test_a_resumed_step_matches_the_uninterrupted_run(tmp_path):
    sc, st = _run_state(n=300, seed=7)
    n, deg = sc.n, sc.sh_degree
    rng = np.random.default_rng(8)
    g1, g2 = (rng.normal(size=oracle.theta_slices(n, deg)["sh"].stop) for _ in range(2))
    kw = dict(n=n, sh_degree=deg, seed=SEED)
    # step 1, then the FP32 state a run keeps
    theta, r, m, v = _oracle_args(sc, st)
    th, r, m, v, _ = oracle.sghmc_step(theta, g1, r, m, v, step=STEP, **kw)
    _store(sc, st, th, r, m, v)
    # uninterrupted: step 2 straight away
    theta, r, m, v = _oracle_args(sc, st)
    th_a, r_a, m_a, v_a, xi_a = oracle.sghmc_step(theta, g2, r, m, v, step=STEP + 1, **kw)
    # interrupted: save, load into a fresh run, step 2 from what was loaded
    path = str(tmp_path / "run.ckpt")
    checkpoint.save(path, sc, st, STEP + 1, seed=SEED)
    got = checkpoint.load(path, device="cpu")
    theta, r, m, v = _oracle_args(got["scene"], got["state"])
    th_b, r_b, m_b, v_b, xi_b = oracle.sghmc_step(theta, g2, r, m, v, step=got["step"], n=n, sh_degree=deg,
                                                  seed=got["seed"])
    for a, b in ((th_a, th_b), (r_a, r_b), (m_a, m_b), (v_a, v_b), (xi_a, xi_b)):
        assert np.array_equal(a, b)
