"""Variants of the method on the GPU against the oracle: the
Adam gradient in the SGHMC update of the means."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_10148_gb300 import frame, inputs

from gpu_util import DEV, f32_scene, require_gpu

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
    params = dict(eps=2e-2, C=0.6, k=100.0, t0=0.005, lr=(5e-3, 1e-3, 1e-2, 5e-2, 2.5e-3), beta1=0.9, beta2=0.999,
                  adam_eps=1e-8)
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
    frame.sghmc_step(sc, gsc, st, sp)
    torch.cuda.synchronize()
    G, m2, v2 = oracle.adam_preconditioned(g0[sl["mean"]].reshape(3, n).astype(np.float64), m_mu, v_mu, step=step,
                                           beta1=0.9, beta2=0.999, adam_eps=1e-8)
    gpre = g0.astype(np.float64).copy()
    gpre[sl["mean"]] = G.reshape(-1)
    th, rr, _, _, _ = oracle.sghmc_step(oracle.theta_from_scene(scene), gpre, np.zeros(3 * n),
                                        np.zeros(sl["sh"].stop), np.zeros(sl["sh"].stop), n=n, sh_degree=0,
                                        params=params, burn_in=burn_in, seed=9, step=step)
    assert np.allclose(mm.cpu().numpy(), m2, rtol=1e-6, atol=1e-12)
    assert np.allclose(vv.cpu().numpy(), v2, rtol=1e-6, atol=1e-14)
    got = oracle.theta_from_scene(sc.to_numpy())
    sm = sl["mean"]
    # G = m^/(sqrt(v^)+eps) is O(1): the FP32 step carries ~1e-6 of it
    assert np.all(np.abs(got[sm] - th[sm]) <= 2e-6 * np.maximum(np.abs(th[sm]), 1.0)), np.abs(got[sm] - th[sm]).max()
    assert np.allclose(st.r.cpu().numpy().reshape(-1), rr, rtol=1e-5, atol=2e-6)
