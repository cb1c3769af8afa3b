"""The training loss of Sec. 3.4 on the GPU (L1 + D-SSIM over a frame's
images, the opacity and scale regularisers) against the FP64 oracle.

Tolerances, from the arithmetic: SSIM's window statistics are FP32 sums of
121 products of values in [0, 1] (relative error ~121 u, u = 2^-24, about
7e-6), the variances subtract nearly equal numbers, and the per-pixel
partials multiply a handful of them; the gradient at a pixel is a further
121-term sum of those partials.  Loss values are accumulated in FP64.  Bars:
loss values 2e-5 relative; gradient elements 2e-4 of the largest element and
the whole gradient 1e-4 relative in the 2-norm."""
import numpy as np
import pytest
import torch

from oracle import image_loss as IL
from paper_2503_10148_gb300 import autograd as AG
from paper_2503_10148_gb300 import frame, inputs

from gpu_util import DEV, adam_increment_mag, assert_step_close, f32, f32_scene, require_gpu

pytestmark = pytest.mark.gpu

SIZES = ((100, 77), (64, 64), (33, 129), (250, 18))


@pytest.fixture(scope="module")
def fr():
    require_gpu()
    scene, _ = inputs.tiny_cube_2k()
    cams = [frame.f32_camera(inputs.look_at((0.0, 0.5, 3.0), width=w, height=h)) for w, h in SIZES]
    f = frame.Frame([frame.Scene.from_numpy(scene, DEV)], cams, device=DEV)
    return f


def _split(fr_, flat):
    out = []
    for j in range(fr_.plan.n_jobs):
        J = fr_.plan.jobs[j]
        n = 3 * J.cam.width * J.cam.height
        out.append(flat[3 * J.pix_base:3 * J.pix_base + n].reshape(3, J.cam.height, J.cam.width))
    return out


def _gpu_loss(fr_, pred, tgt, eps, dloss=None):
    p = torch.as_tensor(pred, device=DEV)
    t = torch.as_tensor(tgt, device=DEV)
    scratch = frame.loss_image_scratch(fr_)
    out = torch.zeros(3, device=DEV)
    frame.loss_image(fr_, p, t, eps, out, scratch)
    g = torch.empty_like(p)
    d = torch.tensor([dloss], device=DEV) if dloss is not None else None
    frame.loss_image_grad(fr_, p, t, eps, scratch, g, d)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)


def test_loss_scratch_covers_the_library_size(fr):
    from paper_2503_10148_gb300 import _abi
    need = _abi.sss_loss_image_scratch_bytes(fr.plan)
    buf = frame.loss_image_scratch(fr)
    assert need >= 9 * 4 * fr.plan.n_pixels + 16
    assert buf.numel() * buf.element_size() >= need and buf.data_ptr() % 16 == 0


def _check_grad(g, gref):
    scale = np.abs(gref).max()
    assert np.abs(g - gref).max() <= 2e-4 * scale, (np.abs(g - gref).max(), scale)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


@pytest.mark.parametrize("eps", [0.0, 0.2, 1.0])
def test_image_loss_value_and_gradient_against_oracle(fr, eps):
    rng = np.random.default_rng(10)
    n = 3 * fr.plan.n_pixels
    pred = rng.uniform(0, 1, n).astype(np.float32)
    tgt = np.clip(pred + rng.normal(0, 0.1, n), 0, 1).astype(np.float32)
    out, g = _gpu_loss(fr, pred, tgt, eps)
    L, l1, dssim, grads = IL.image_loss(_split(fr, pred.astype(np.float64)), _split(fr, tgt.astype(np.float64)), eps)
    assert out[0] == pytest.approx(L, rel=2e-5) and out[1] == pytest.approx(l1, rel=2e-5)
    assert out[2] == pytest.approx(dssim, rel=2e-5)
    gref = np.concatenate([x.reshape(-1) for x in grads])
    _check_grad(g, gref)


def test_image_loss_upstream_scale_and_rendered_images(fr):
    """A rendered frame (dark background, negative scooping contributions
    possible) against a target, with dL/dloss = -2.5 from upstream."""
    fr.forward()
    pred = fr.rgb.cpu().numpy().copy()
    rng = np.random.default_rng(11)
    tgt = rng.uniform(0, 1, pred.size).astype(np.float32)
    out, g = _gpu_loss(fr, pred, tgt, 0.2, dloss=-2.5)
    L, _, _, grads = IL.image_loss(_split(fr, pred.astype(np.float64)), _split(fr, tgt.astype(np.float64)), 0.2)
    assert out[0] == pytest.approx(L, rel=2e-5)
    _check_grad(g, -2.5 * np.concatenate([x.reshape(-1) for x in grads]))


def test_image_loss_degenerate_images(fr):
    n = 3 * fr.plan.n_pixels
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, n).astype(np.float32)
    out, g = _gpu_loss(fr, x, x, 0.2)
    assert abs(out[1]) == 0.0 and abs(out[2]) < 2e-6  # identical: L1 = 0, SSIM = 1
    assert np.abs(g).max() < 1e-6 * 0.2 / n * 100
    c = np.full(n, 0.25, np.float32)
    d = np.full(n, 0.75, np.float32)
    out, g = _gpu_loss(fr, c, d, 1.0)
    L, _, _, grads = IL.image_loss(_split(fr, c.astype(np.float64)), _split(fr, d.astype(np.float64)), 1.0)
    assert out[0] == pytest.approx(L, rel=2e-5)
    _check_grad(g, np.concatenate([x.reshape(-1) for x in grads]))


def test_image_loss_autograd_equals_direct(fr):
    n = 3 * fr.plan.n_pixels
    rng = np.random.default_rng(13)
    pred = torch.as_tensor(rng.uniform(0, 1, n).astype(np.float32), device=DEV).requires_grad_(True)
    tgt = torch.as_tensor(rng.uniform(0, 1, n).astype(np.float32), device=DEV)
    loss = AG.image_loss(fr, pred, tgt, 0.2)
    (g,) = torch.autograd.grad(loss * 3.0, [pred])
    out, gd = _gpu_loss(fr, pred.detach().cpu().numpy(), tgt.cpu().numpy(), 0.2, dloss=3.0)
    torch.cuda.synchronize()
    assert float(loss.detach()) == pytest.approx(out[0], rel=1e-6)
    assert np.array_equal(g.cpu().numpy().astype(np.float64), gd)


def test_regularizers_value_and_sghmc_gradient_against_oracle():
    require_gpu()
    import oracle
    scene = inputs.scene_uniform_cube(5000, seed=7)
    scene["sh"] = scene["sh"][:3]
    scene["sh_degree"] = 0
    sc = frame.Scene.from_numpy(scene, DEV)
    out = torch.zeros(1, device=DEV)
    frame.regularizers(sc, 0.01, 0.02, out)
    v, g_raw, g_ls = IL.regularizers(scene["opacity_raw"].astype(np.float32).astype(np.float64),
                                     scene["log_scale"].astype(np.float32).astype(np.float64), 0.01, 0.02)
    torch.cuda.synchronize()
    assert float(out) == pytest.approx(v, rel=1e-5)
    # one step with the regulariser weights = the oracle step with their gradients added
    n = scene["n"]
    rng = np.random.default_rng(8)
    g0 = rng.normal(0, 1e-3, size=oracle.theta_slices(n, 0)["sh"].stop).astype(np.float32)
    gsc = frame.Scene.zeros(n, 0, DEV)
    sl = oracle.theta_slices(n, 0)
    for f in frame.FIELDS:
        gsc.t[f].copy_(torch.as_tensor(g0[sl[f]].reshape(gsc.t[f].shape), device=DEV))
    st = frame.SamplerState(sc)
    params = dict(eps=f32(1e-3), C=f32(0.5), k=f32(100.0), t0=f32(0.005), lr=f32((5e-3, 1e-3, 1e-2, 5e-2, 2.5e-3)),
                  beta1=f32(0.9), beta2=f32(0.999), adam_eps=f32(1e-8))
    sp = frame.step_params(eps=params["eps"], C=params["C"], seed=3, step=0, lr=params["lr"],
                           adam_eps=params["adam_eps"], reg_opacity=0.01, reg_scale=0.02)
    theta0 = oracle.theta_from_scene(f32_scene(scene))
    frame.sghmc_step(sc, gsc, st, sp)
    torch.cuda.synchronize()
    greg = g0.astype(np.float64).copy()
    greg[sl["opacity_raw"]] += g_raw
    greg[sl["log_scale"]] += g_ls.reshape(-1)
    z = np.zeros(3 * n)
    th, _, _, vv, _ = oracle.sghmc_step(theta0, greg, z, np.zeros(sl["sh"].stop), np.zeros(sl["sh"].stop), n=n,
                                     sh_degree=0, params=params, seed=3, step=0)
    got = oracle.theta_from_scene(sc.to_numpy())
    # the regularisers' gradients are FP32 closed forms on the GPU: their
    # magnitudes join the gradient's in the sampler bar
    gmag = np.abs(g0.astype(np.float64))
    gmag[sl["opacity_raw"]] += np.abs(g_raw)
    gmag[sl["log_scale"]] += np.abs(g_ls.reshape(-1))
    for f, lr in zip(("log_scale", "quat", "nu", "opacity_raw", "sh"), params["lr"]):
        inc = adam_increment_mag(0.0, gmag[sl[f]], vv[sl[f]], lr, params["beta1"], params["beta2"],
                                 params["adam_eps"], 1)
        assert_step_close(got[sl[f]], th[sl[f]], inc, f)


def test_trainstep_full_loss_autograd_equals_direct():
    require_gpu()
    from paper_2503_10148_gb300 import train
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 25))
    cams = [frame.f32_camera(inputs.look_at(c.position, width=200, height=150)) for c in cams[:3]]
    targets = torch.as_tensor(np.concatenate([t.reshape(-1) for t in inputs.target_images(cams, seed=2)]),
                              device=DEV)
    res = {}
    for form in ("autograd", "direct"):
        sc = frame.Scene.from_numpy(scene, DEV)
        ts = train.TrainStep(sc, cams, targets.clone(), device=DEV, form=form, loss="full")
        ts.calibrate()
        ts.run()
        torch.cuda.synchronize()
        res[form] = ({f: ts.grads.t[f].detach().clone() for f in frame.FIELDS}, float(ts.loss.reshape(-1)[0]))
    for f in frame.FIELDS:
        a, b = res["autograd"][0][f], res["direct"][0][f]
        assert float((a - b).norm()) <= 1e-5 * float(b.norm()) + 1e-30, f
    assert res["autograd"][1] == pytest.approx(res["direct"][1], rel=1e-6)
