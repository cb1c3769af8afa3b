"""A frame at the limits of one launch sequence (GPU): the maximum number of
jobs (SSS_MAX_JOBS = 64) over the maximum number of scenes
(SSS_MAX_SCENES = 8), scenes of SH degree 0 and 3 side by side, and images
from a single pixel up to sizes that fill no tile, rendered and
differentiated against the oracle job by job and scene by scene."""
import numpy as np
import pytest
import torch

import oracle
from paper_2503_10148_gb300 import _abi, frame, inputs

from gpu_util import (DEV, assert_groups_close, f32_scene, oracle_views, require_gpu, resolved_weights,
                      scene_grads_flat, sh_basis_bound)

pytestmark = pytest.mark.gpu

SIZES = ((1, 1), (1, 9), (9, 1), (7, 5), (17, 16), (33, 18), (40, 23), (16, 17))  # (width, height)


def _limits(tile):
    scenes = []
    for s in range(_abi.SSS_MAX_SCENES):
        n = 150 + 37 * s
        if s % 2 == 0:
            scenes.append(inputs.scene_uniform_cube(n, seed=100 + s))  # SH degree 0
        else:
            shell = inputs.scene_sphere_shell(3 * n, seed=100 + s)  # SH degree 3
            scenes.append(inputs.subset_scene(shell, np.arange(0, 3 * n, 3)))
    rng = np.random.default_rng(5)
    cams, job_scene = [], []
    for j in range(_abi.SSS_MAX_JOBS):
        w, h = SIZES[j % len(SIZES)]
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cams.append(frame.f32_camera(inputs.look_at(3.0 * d, width=w, height=h, fov_x_deg=40.0 + 5.0 * (j % 5))))
        job_scene.append((j * 3) % _abi.SSS_MAX_SCENES)  # every scene, interleaved
    cfg = frame.make_cfg(tile_w=tile[0], tile_h=tile[1])
    scs = [frame.Scene.from_numpy(s, DEV) for s in scenes]
    fr = frame.Frame(scs, cams, job_scene=job_scene, cfg=cfg, device=DEV)
    fr.forward(grow=True)
    torch.cuda.synchronize()
    return fr, scenes, scs, cams, job_scene


@pytest.mark.parametrize("tile", [(16, 16), (64, 128)])
def test_max_jobs_and_scenes_forward_and_backward_against_oracle(tile):
    require_gpu()
    fr, scenes, scs, cams, job_scene = _limits(tile)
    assert fr.plan.n_jobs == _abi.SSS_MAX_JOBS and fr.plan.n_scenes == _abi.SSS_MAX_SCENES
    assert fr.status()[0] == 0
    cfgd = frame.cfg_dict(fr.cfg)
    s32 = [f32_scene(s) for s in scenes]
    # forward, job by job: every pixel (flagged ones against the admissible results)
    refs = []
    for j, cam in enumerate(cams):
        (proj, ref), = oracle_views(s32[job_scene[j]], [cam], cfgd)
        refs.append((proj, ref))
    ws, flips, st = resolved_weights(fr, cams, cfgd, refs, seed=9)
    print("forward", st)
    # backward: per scene, the gradient summed over that scene's jobs
    dl = torch.as_tensor(np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32), device=DEV)
    grads = [s.zeros_like() for s in scs]
    fr.backward(dl, grads)
    torch.cuda.synchronize()
    for s, sc in enumerate(scenes):
        jobs = [j for j in range(len(cams)) if job_scene[j] == s]
        gref, _, gabs, g2abs = oracle.backward(s32[s], [cams[j] for j in jobs], cfgd, [ws[j] for j in jobs],
                                               want_grad2d=True, want_abs=True, flip=[flips[j] for j in jobs])
        print(assert_groups_close(scene_grads_flat(grads[s]), gref, sc["n"], sc["sh_degree"], gabs,
                                  label=f"scene {s}", extra=sh_basis_bound(sc["n"], sc["sh_degree"], g2abs)))
