"""The torch.autograd.Function form (render, l1_loss) against the oracle.

The autograd backward is the same render_bwd + project_bwd launches as the
direct form, reached through torch.autograd; these tests check the wiring
(inputs, outputs, gradient routing, upstream scaling, graph capture) and the
resulting gradients against the oracle's FP64 analytic gradient and its
central finite differences."""
import numpy as np
import pytest
import torch

import oracle
from oracle import Magnitudes
from paper_2503_10148_gb300 import autograd as AG
from paper_2503_10148_gb300 import frame, inputs, train

from gpu_util import (DEV, GRAD_REL, assert_groups_close, check_forward_view, f32_scene, gpu_last_component, grad_den,
                      oracle_views,
                      require_gpu, scene_grads_flat)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _setup(scene_np, cams, cfg=None):
    cams = [frame.f32_camera(c) for c in cams]
    cfg = cfg or frame.make_cfg()
    sc = frame.Scene.from_numpy(scene_np, DEV)
    fr = frame.Frame([sc], cams, cfg=cfg, device=DEV)
    return sc, fr, cams


def _autograd_grads(sc, fr, ws):
    leaves = AG.leaves(sc)
    rgb = AG.render(fr, leaves)
    w = torch.as_tensor(np.concatenate([x.reshape(-1) for x in ws]).astype(np.float32), device=DEV)
    loss = (rgb * w).sum()
    grads = torch.autograd.grad(loss, leaves)
    torch.cuda.synchronize()
    return rgb, frame.Scene(dict(zip(frame.FIELDS, grads)), sc.n, sc.sh_degree)


def test_autograd_forward_and_gradient_against_oracle_analytic_and_fd():
    scene, cams = inputs.tiny_cube_2k()
    sc, fr, cams = _setup(scene, cams)
    cfgd = frame.cfg_dict(fr.cfg)
    s32 = f32_scene(scene)
    refs = oracle_views(s32, cams, cfgd)
    ws = inputs.linear_loss_weights(cams, 11)
    rgb, g = _autograd_grads(sc, fr, ws)
    img = fr.image_of(rgb.detach(), 0).reshape(3, -1).cpu().numpy().astype(np.float64)
    pb = fr.plan.jobs[0].pix_base
    T = fr.final_T()[pb:pb + cams[0].width * cams[0].height].cpu().numpy().astype(np.float64)
    chk = check_forward_view(refs[0][0], cams[0], cfgd, refs[0][1], img, T, last=gpu_last_component(fr, 0, cams[0]))
    if chk.unresolved.any():  # pixels whose image does not determine their decisions carry no weight
        ws = [w.reshape(3, -1) * (~chk.unresolved)[None, :] for w in ws]
        rgb, g = _autograd_grads(sc, fr, ws)
    gflat = scene_grads_flat(g)
    gref, gabs = oracle.backward(s32, cams, cfgd, ws, want_abs=True, flip=[chk.flip])
    print(chk.stats, assert_groups_close(gflat, gref, scene["n"], 0, gabs, label="autograd"))
    # central differences follow the oracle's own decisions: a second autograd
    # gradient with the flagged pixels weightless
    ws = [w.reshape(3, -1) * (refs[0][1]["flags"] == 0)[None, :] for w in ws]
    rgb, g = _autograd_grads(sc, fr, ws)
    gflat = scene_grads_flat(g)
    n = scene["n"]
    sl = oracle.theta_slices(n, 0)
    rng = np.random.default_rng(4)
    picks = []
    for name in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        cand = np.arange(sl[name].start, sl[name].stop)
        cand = cand[np.abs(gref[cand]) > 1e-3 * np.abs(gref[sl[name]]).max()]
        picks += list(rng.choice(cand, 10, replace=False))
    fd, smooth = oracle.fd_gradient(oracle.theta_from_scene(s32), n, 0, cams, cfgd, ws, picks)
    checked = 0
    for j, f, good in zip(picks, fd, smooth):
        if not good:
            continue
        den = grad_den(np.array([f]), Magnitudes(np.array([gabs.abs[j]]), np.array([gabs.absn[j]])))[0]
        assert abs(gflat[j] - f) <= GRAD_REL * den, (j, gflat[j], f)
        checked += 1
    assert checked >= 50


def test_autograd_equals_direct_form():
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 20))
    cams = [inputs.look_at(c.position, width=200, height=152) for c in cams[:3]]
    sc, fr, cams = _setup(scene, cams)
    ws = inputs.linear_loss_weights(cams, 12)
    _, g_ag = _autograd_grads(sc, fr, ws)
    # direct: same launches with caller-owned buffers
    fr2 = frame.Frame([sc], cams, cfg=fr.cfg, device=DEV)
    fr2.forward()
    dl = torch.as_tensor(np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32), device=DEV)
    g_d = sc.zeros_like()
    fr2.backward(dl, [g_d])
    torch.cuda.synchronize()
    for f in frame.FIELDS:
        a, b = g_ag.t[f], g_d.t[f]
        # the same kernels; only the order of the float atomics in render_bwd differs
        assert float((a - b).norm()) <= 1e-5 * float(b.norm()) + 1e-30, f


def test_l1_loss_function_value_gradient_and_upstream_scale():
    rng = np.random.default_rng(1)
    a = rng.uniform(size=50_001).astype(np.float32)
    b = rng.uniform(size=50_001).astype(np.float32)
    b[:7] = a[:7]
    pa = torch.as_tensor(a, device=DEV).requires_grad_(True)
    pb = torch.as_tensor(b, device=DEV)
    loss = AG.l1_loss(pa, pb)
    (g,) = torch.autograd.grad(loss * 3.0, [pa])
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(np.abs(a.astype(np.float64) - b).mean(), rel=1e-5)
    want = np.float32(3.0) * (np.sign(a - b) / np.float32(a.size)).astype(np.float32)
    assert np.allclose(g.cpu().numpy(), want, rtol=1e-6, atol=0)


def test_render_twice_before_backward_raises():
    scene, cams = inputs.tiny_cube_2k()
    sc, fr, cams = _setup(scene, cams)
    leaves = AG.leaves(sc)
    rgb1 = AG.render(fr, leaves)
    AG.render(fr, leaves)
    with pytest.raises(RuntimeError, match="rendered again"):
        torch.autograd.grad(rgb1.sum(), leaves)
    other = [t.detach().clone().requires_grad_(True) for t in leaves]
    with pytest.raises(ValueError, match="not the one"):
        AG.render(fr, other)


def test_trainstep_autograd_graph_gradients_equal_direct():
    """The graph-captured autograd step computes the same gradients as the
    direct step (one step from the same parameters)."""
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 25))
    cams = [frame.f32_camera(inputs.look_at(c.position, width=256, height=192)) for c in cams[:4]]
    targets = torch.as_tensor(np.concatenate([t.reshape(-1) for t in inputs.target_images(cams, seed=2)]),
                              device=DEV)
    grads = {}
    for form in ("autograd", "direct"):
        sc = frame.Scene.from_numpy(scene, DEV)
        ts = train.TrainStep(sc, cams, targets.clone(), device=DEV, form=form)
        ts.calibrate()
        if form == "autograd":
            ts.capture()  # the capture's warm-up step runs eagerly first
            torch.cuda.synchronize()
            before = {f: sc.t[f].detach().clone() for f in frame.FIELDS}
            ts.replay()
        else:
            ts.run()  # eager
        torch.cuda.synchronize()
        ts.check()
        grads[form] = {f: ts.grads.t[f].detach().clone() for f in frame.FIELDS}
        if form == "autograd":
            moved = sum(float((sc.t[f].detach() - before[f]).abs().max()) for f in frame.FIELDS)
            assert moved > 0.0  # the replay updated the parameters
    # the autograd replay saw parameters after one (eager warm-up) update; the
    # direct step saw the initial ones: compare the direct step against an
    # eager autograd step from the initial parameters instead
    sc = frame.Scene.from_numpy(scene, DEV)
    ts = train.TrainStep(sc, cams, targets.clone(), device=DEV, form="autograd")
    ts.calibrate()
    ts.run()
    torch.cuda.synchronize()
    for f in frame.FIELDS:
        a, b = ts.grads.t[f], grads["direct"][f]
        assert float((a - b).norm()) <= 1e-5 * float(b.norm()) + 1e-30, f


def test_trainstep_restart_replays_leave_the_scene_and_repeat_the_step():
    """With restart, captured replays read the configured scene, leave it
    unchanged and write the update beside it: with the sampler's step index
    and moments reset, two replays write the same parameters, and the
    gradients of every replay are those of the configured scene."""
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 50))
    cams = [frame.f32_camera(inputs.look_at(c.position, width=192, height=128)) for c in cams[:2]]
    targets = torch.as_tensor(np.concatenate([t.reshape(-1) for t in inputs.target_images(cams, seed=4)]),
                              device=DEV)
    sc = frame.Scene.from_numpy(scene, DEV)
    orig = {f: sc.t[f].detach().clone() for f in frame.FIELDS}
    ts = train.TrainStep(sc, cams, targets, device=DEV, form="autograd", loss="full", restart=True)
    ts.calibrate()
    ts.capture()
    outs, grads = [], []
    for _ in range(2):
        ts.step_counter.zero_()
        for x in (ts.state.r, ts.state.m, ts.state.v):
            x.zero_()
        ts.replay()
        torch.cuda.synchronize()
        ts.check()
        outs.append({f: ts.after.t[f].clone() for f in frame.FIELDS})
        grads.append({f: ts.grads.t[f].detach().clone() for f in frame.FIELDS})
    for f in frame.FIELDS:
        assert torch.equal(sc.t[f].detach(), orig[f]), f
        assert not torch.equal(outs[0][f], orig[f]), f
        # same parameters in: the same gradients up to the order of the float
        # atomics of render_bwd
        ga, gb = grads[0][f], grads[1][f]
        assert float((ga - gb).norm()) <= 1e-5 * float(gb.norm()) + 1e-30, f
    # same gradients, noise and moments: the same SGHMC update of the means
    # (linear in the gradient; the first Adam step of the other groups moves
    # by lr sign(g), which the atomics' order may flip where g is near 0)
    a, b = outs[0]["mean"], outs[1]["mean"]
    assert float((a - b).abs().max()) <= 1e-6 * max(float(a.abs().max()), 1.0)
