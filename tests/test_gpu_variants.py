"""Variants of the method on the GPU against the oracle: the Adam gradient
in the SGHMC update of the means, and the Gaussian kernel (nu -> infinity)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_10148_gb300 import frame, inputs

from gpu_util import (DEV, adam_increment_mag, assert_step_close, f32, f32_scene, require_gpu,
                      step_mags)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("burn_in", [False, True])
def test_sghmc_with_the_adam_gradient_against_oracle(burn_in):
    require_gpu()
    n = 3000
    scene = f32_scene(inputs.scene_uniform_cube(n, seed=21))
    sl = oracle.theta_slices(n, 0)
    rng = np.random.default_rng(21)
    g0 = rng.normal(0, 1e-2, size=sl["sh"].stop).astype(np.float32)
    m_mu = rng.normal(0, 1e-3, size=(3, n)).astype(np.float32)
    v_mu = rng.uniform(1e-6, 1e-4, size=(3, n)).astype(np.float32)
    params = dict(eps=f32(2e-2), C=f32(0.6), k=f32(100.0), t0=f32(0.005), lr=f32((5e-3, 1e-3, 1e-2, 5e-2, 2.5e-3)),
                  beta1=f32(0.9), beta2=f32(0.999), adam_eps=f32(1e-8))
    step = 4
    sc = frame.Scene.from_numpy(scene, DEV)
    gsc = frame.Scene.zeros(n, 0, DEV)
    for f in frame.FIELDS:
        gsc.t[f].copy_(torch.as_tensor(g0[sl[f]].reshape(gsc.t[f].shape), device=DEV))
    st = frame.SamplerState(sc)
    mm = torch.as_tensor(m_mu, device=DEV)
    vv = torch.as_tensor(v_mu, device=DEV)
    sp = frame.step_params(eps=params["eps"], C=params["C"], burn_in=burn_in, seed=9, step=step, lr=params["lr"],
                           adam_eps=params["adam_eps"], mu_adam=(mm, vv))
    gpu_xi = torch.zeros(3, n, dtype=torch.float32, device=DEV)
    frame.sghmc_step(sc, gsc, st, sp, xi_out=gpu_xi)
    torch.cuda.synchronize()
    G, m2, v2 = oracle.adam_preconditioned(g0[sl["mean"]].reshape(3, n).astype(np.float64), m_mu, v_mu, step=step,
                                           beta1=params["beta1"], beta2=params["beta2"], adam_eps=params["adam_eps"])
    gpre = g0.astype(np.float64).copy()
    gpre[sl["mean"]] = G.reshape(-1)
    th, rr, _, _, _ = oracle.sghmc_step(oracle.theta_from_scene(scene), gpre, np.zeros(3 * n),
                                        np.zeros(sl["sh"].stop), np.zeros(sl["sh"].stop), n=n, sh_degree=0,
                                        params=params, burn_in=burn_in, seed=9, step=step)
    # m' = b1 m + (1 - b1) g can cancel: the sampler bar takes its rounding on
    # the magnitudes of the two terms
    g_mu = g0[sl["mean"]].reshape(3, n).astype(np.float64)
    b1, b2 = params["beta1"], params["beta2"]
    assert_step_close(mm.cpu().numpy(), m2, b1 * np.abs(m_mu) + (1 - b1) * np.abs(g_mu), "mu m")
    assert_step_close(vv.cpu().numpy(), v2, v2, "mu v")
    got = oracle.theta_from_scene(sc.to_numpy())
    sm = sl["mean"]
    G_mag = adam_increment_mag(m_mu, np.abs(g_mu), v2, 1.0, b1, b2, params["adam_eps"], step + 1)
    mu_mag, r_mag = step_mags(oracle.theta_from_scene(scene), G_mag, np.zeros(3 * n),
                              np.asarray(gpu_xi.cpu().numpy(), np.float64), n, 0, params, burn_in)
    rep = {"mean": assert_step_close(got[sm], th[sm], mu_mag, "mean"),
           "momentum": assert_step_close(st.r.cpu().numpy(), rr, r_mag, "momentum")}
    print("sampler bar, Adam gradient", burn_in, rep)


@pytest.mark.parametrize("tile", [(16, 16), (32, 32)])
def test_gaussian_kernel_forward_and_backward_against_oracle(tile):
    """kernel = 1 (T2D = exp(-h/2)): the forward within 1e-4 per channel and
    the gradient within the bar of the t kernel (nu gets none); one pixel
    per lane (16x16 tiles) and packed pixel pairs (32x32)."""
    from gpu_util import (assert_groups_close, gpu_forward, oracle_views, resolved_weights, scene_grads_flat,
                          sh_basis_bound)
    require_gpu()
    scene, cams = inputs.tiny_cube_2k()
    cfg = frame.make_cfg(kernel=1, tile_w=tile[0], tile_h=tile[1])
    fr, sc, cams = gpu_forward(scene, cams, cfg)
    cfgd = frame.cfg_dict(cfg)
    assert cfgd["kernel"] == 1
    s32 = f32_scene(scene)
    refs = oracle_views(s32, cams, cfgd)
    ws, flips, st = resolved_weights(fr, cams, cfgd, refs, seed=21)  # every pixel's forward compared
    assert np.isinf(fr.records().cpu().numpy()[:, 7]).all()  # records carry nu = inf
    dl = torch.as_tensor(np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32), device=DEV)
    g = sc.zeros_like()
    fr.backward(dl, [g])
    torch.cuda.synchronize()
    gflat = scene_grads_flat(g)
    gref, g2d, gabs, g2abs = oracle.backward(s32, cams, cfgd, ws, want_grad2d=True, want_abs=True, flip=flips)
    sl = oracle.theta_slices(scene["n"], 0)
    assert np.all(gflat[sl["nu"]] == 0.0) and np.all(gref[sl["nu"]] == 0.0)
    print(st, assert_groups_close(gflat, gref, scene["n"], 0, gabs, label="gauss",
                              extra=sh_basis_bound(scene["n"], 0, g2abs)))
