"""Helpers shared by the GPU parity tests (imported by test modules only)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2503_10148_gb300 import frame, inputs

DEV = "cuda:0"


def require_gpu():
    assert torch.cuda.is_available(), "GPU tests need CUDA (there is no CPU fallback)"
    from paper_2503_10148_gb300 import build
    build.build()


def f32_scene(scene: dict) -> dict:
    """Parameters rounded to float32 then widened: what both sides consume."""
    out = dict(scene)
    for k in frame.FIELDS:
        out[k] = np.asarray(scene[k], np.float32)
    return out


def gpu_forward(scene_np, cams, cfg=None, pair_capacity=None):
    cams = [frame.f32_camera(c) for c in cams]
    cfg = cfg or frame.make_cfg()
    sc = frame.Scene.from_numpy(scene_np, DEV)
    fr = frame.Frame([sc], cams, cfg=cfg, pair_capacity=pair_capacity, device=DEV)
    fr.forward()
    torch.cuda.synchronize()
    return fr, sc, cams


def oracle_views(scene_np, cams, cfgd, pix=None):
    """Oracle projection + render for every camera (pix: list of pixel index
    arrays or None)."""
    out = []
    for v, cam in enumerate(cams):
        proj = oracle.project(scene_np, cam, cfgd)
        out.append((proj, oracle.render(proj, cam, cfgd, None if pix is None else pix[v])))
    return out


def masked_weights(cams, refs, seed, pix=None):
    """Seeded dL/dC weights with the pixels the oracle flags as fragile (a
    discrete decision within rounding distance) set to zero, so neither side's
    gradient depends on them.  With pix given, only those pixels are nonzero."""
    ws = inputs.linear_loss_weights(cams, seed)
    out = []
    for v, (w, (_, ref)) in enumerate(zip(ws, refs)):
        w = w.reshape(3, -1).copy()
        if pix is None:
            w[:, ref["flags"] != 0] = 0.0
        else:
            keep = np.zeros(w.shape[1], bool)
            keep[pix[v][ref["flags"] == 0]] = True
            w[:, ~keep] = 0.0
        out.append(w)
    return out


def scene_grads_flat(g: frame.Scene) -> np.ndarray:
    return np.concatenate([g.t[f].detach().cpu().numpy().reshape(-1).astype(np.float64) for f in frame.FIELDS])


GRAD_REL = 1e-3     # per-element relative bar ...
GRAD_FLOOR = 1e-2   # ... against max(|g_ref|, GRAD_FLOOR * sum of |summands|)
GRAD_NORM = 1e-4    # and ||g - g_ref|| / ||g_ref|| per group


def grad_den(ref, absref, floor=GRAD_FLOOR):
    """Denominator of the relative error: |g_ref|, but at least GRAD_FLOOR of
    the magnitude summed into it (a sum of terms of both signs -- the gradient
    of a splat's position sums pixels on either side of it -- is only as
    accurate in FP32 as its summands, not as its result)."""
    scale = max(float(np.abs(ref).max()), 1e-30)
    return np.maximum(np.maximum(np.abs(ref), floor * absref), 1e-7 * scale)


def assert_groups_close(got, ref, n, sh_degree, absref, rel=GRAD_REL, norm=GRAD_NORM, label=""):
    """Per parameter group: every element within ``rel`` of grad_den and the
    group's relative L2 error within ``norm``."""
    sl = oracle.theta_slices(n, sh_degree)
    report = {}
    for name, s in sl.items():
        a, b = got[s], ref[s]
        scale = np.abs(b).max()
        if scale == 0:
            assert np.abs(a).max() == 0, (label, name)
            continue
        den = grad_den(b, absref[s])
        relerr = np.abs(a - b) / den
        l2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        report[name] = (float(relerr.max()), l2)
        bad = relerr > rel
        assert not bad.any(), (label, name, report[name], int(bad.sum()), a[bad][:5], b[bad][:5])
        assert l2 <= norm, (label, name, report[name])
    return report
