"""Runs the autotuner on a named workload and stores the choice.

    python -m paper_2503_10148_gb300.tune_main [workload] [--steps K]
    python -m paper_2503_10148_gb300.tune_main --serve   (list tile per serving resolution)
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import autotune, build, frame as F, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", nargs="?", default="clusters_1p5m_4views")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--out", default=autotune.CACHE)
    ap.add_argument("--serve", action="store_true", help="tune the serving list tile per resolution instead")
    args = ap.parse_args()
    build.build()
    if args.serve:
        dev = torch.device("cuda", 0)
        scenes = [F.Scene.from_numpy(s, dev) for s in inputs.serving_scenes()]
        print(autotune.tune_serve(scenes, inputs.SERVE_RESOLUTIONS, device=dev, path=args.out))
        return
    scene_np, cams = getattr(inputs, args.workload)()
    cams = [F.f32_camera(c) for c in cams]
    dev = torch.device("cuda", 0)
    scene = F.Scene.from_numpy(scene_np, dev)
    targets = torch.as_tensor(np.concatenate([t.reshape(-1) for t in inputs.target_images(cams, seed=3)]),
                              device=dev)
    # the step bench.py times: 0.8 L1 + 0.2 D-SSIM, opacity and scale
    # regularisers, every step from the configured scene
    step_kw = dict(loss="full", eps_dssim=0.2, reg_opacity=0.01, reg_scale=0.01, restart=True)
    choice = autotune.tune(args.workload, scene, cams, targets, steps=args.steps, device=dev, path=args.out,
                           step_kw=step_kw)
    print(choice)


if __name__ == "__main__":
    main()
