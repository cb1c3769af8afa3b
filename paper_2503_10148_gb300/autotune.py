"""Autotuner for the rasterizer's launch shape: the tile size, the staging
batch and the backward's warp box.

For a workload it times the whole captured train step (``train.TrainStep``)
for every (tile_w, tile_h, batch, bwd_box_h) candidate and keeps the
fastest.  Tile size
trades pair count (bigger tiles: fewer pairs to sort) against the render's
work per tile: a tile is rendered as sub-tiles of at most 32 x 32 pixels (32 x 64
in the backward with the taller box),
each walking the tile's whole list (its warps skip the records whose
ellipse misses their block).
The staging batch is the number of records a warp gathers per round, 32 or
64 (one or two per lane): deeper rounds mean fewer rounds, each with more
gathers in flight, at twice the shared memory.
The backward's warp box is 16 x 8 or 16 x 16 pixels (2 x 2 or 2 x 4 per
lane; the taller one on tiles at least 32 x 64): the taller box halves the
per-splat work (record setup, moments, the warp reduction) of splats larger
than the box, at a lower occupancy (128 registers a thread), so it pays on
scenes of large splats and not on small ones.

Results are stored per workload name in ``tuned.json`` next to this file;
``cached(name)`` returns the stored choice or None.
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuned.json")

TILES = ((16, 16), (32, 16), (16, 32), (32, 32), (64, 32), (32, 64), (64, 64), (128, 64), (64, 128), (128, 128))
BATCHES = (32, 64)


def default_candidates():
    """(tile_w, tile_h, batch, bwd_box_h) for every tile and batch, with the
    16-pixel backward box where the tile allows it."""
    out = []
    for tw, th in TILES:
        for b in BATCHES:
            out.append((tw, th, b, 8))
            if tw >= 32 and th >= 64:
                out.append((tw, th, b, 16))
    return out


def candidate_key(tw, th, b, box) -> str:
    return f"{tw}x{th}/{b}" + ("" if box == 8 else f"/box{box}")


def cached(name: str) -> dict | None:
    try:
        with open(CACHE) as f:
            return json.load(f).get(name)
    except (OSError, ValueError):
        return None


def store(name: str, choice: dict, path: str = CACHE):
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        pass
    data[name] = choice
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def tune(name: str, scene, cams, targets, candidates=None, steps: int = 5, finalists: int = 4, rounds: int = 3,
         device="cuda", log=print, path: str = CACHE, step_kw: dict | None = None) -> dict:
    """Times each candidate's captured step and stores the fastest, in two
    stages: every candidate for ``steps`` replays, then the ``finalists``
    fastest again, interleaved over ``rounds`` rounds of 4 x ``steps``
    replays each (the first stage's differences near the top are of the
    order of the run-to-run noise).  ``step_kw`` are the ``train.TrainStep``
    options of the step to tune (loss, regularisers, restart)."""
    import torch

    from . import frame as F
    from . import train

    candidates = candidates or default_candidates()
    snapshot = {f: scene.t[f].clone() for f in F.FIELDS}

    def build(tw, th, b, box):
        with torch.no_grad():  # every candidate starts from the same parameters
            for f in F.FIELDS:
                scene.t[f].copy_(snapshot[f])
        cfg = F.make_cfg(tile_w=tw, tile_h=th, batch=b, bwd_box_h=box)
        ts = train.TrainStep(scene, cams, targets, cfg=cfg, device=device, **(step_kw or {}))
        ts.calibrate()
        ts.capture()
        ts.replay()
        return ts

    def time_replays(ts, k):
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            ts.replay()
        e1.record()
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / k

    results = []
    for cand in candidates:
        ts = build(*cand)
        ms = time_replays(ts, steps)
        ts.check()
        results.append((ms, *cand))
        log(f"autotune {name}: tile {cand[0]}x{cand[1]} batch {cand[2]} backward box 16x{cand[3]}: {ms:.3f} ms/step")
        del ts
        torch.cuda.empty_cache()
    top = [r[1:] for r in sorted(results)[:max(1, finalists)]]
    steps_list = [build(*cand) for cand in top]
    sums = [0.0] * len(top)
    for _ in range(rounds):
        for i, ts in enumerate(steps_list):
            sums[i] += time_replays(ts, 4 * steps)
    for ts in steps_list:
        ts.check()
    del steps_list
    torch.cuda.empty_cache()
    refined = sorted((s / rounds, *cand) for s, cand in zip(sums, top))
    for m, *cand in refined:
        log(f"autotune {name}: finalist {candidate_key(*cand)}: {m:.3f} ms/step")
    with torch.no_grad():
        for f in F.FIELDS:
            scene.t[f].copy_(snapshot[f])
    ms, tw, th, b, box = refined[0]
    choice = {"tile_w": tw, "tile_h": th, "batch": b, "bwd_box_h": box, "ms_per_step": round(ms, 3),
              "candidates": {candidate_key(a, c, d, e): round(m, 3) for m, a, c, d, e in results},
              "finalists": {candidate_key(a, c, d, e): round(m, 3) for m, a, c, d, e in refined}}
    store(name, choice, path)
    return choice


# ---------------------------------------------------------------- serving
SERVE_TILES = (16, 32, 64, 128)
SERVE_KEY = "serving"


def tune_serve(scenes, resolutions, cams_per_res: int = 3, reps: int = 5, device="cuda", log=print,
               path: str = CACHE, seed: int = 5) -> dict:
    """For each serving resolution, the square list tile whose single-view
    frame (project -> bin -> sort -> render_fwd) is fastest, averaged over the
    resident scenes and a few seeded cameras on the radius-3 sphere.  A small
    view wants small tiles (more warps in flight, shorter lists per warp), a
    large one large tiles (fewer pairs to sort).  Stored under "serving"."""
    import numpy as np
    import torch

    from . import frame as F
    from . import inputs

    rng = np.random.default_rng(seed)
    table = {}
    for (w, h) in resolutions:
        cams = [F.f32_camera(inputs.random_sphere_camera(rng, width=w, height=h)) for _ in range(cams_per_res)]
        ms = {}
        for t in SERVE_TILES:
            cfg = F.make_cfg(tile_w=t, tile_h=t, batch=32)
            acc = []
            for sc in scenes:
                for cam in cams:
                    fr = F.Frame([sc], [cam], cfg=cfg, device=device)
                    fr.forward(grow=True)
                    torch.cuda.synchronize(device)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        fr.forward(grow=False)
                    e1.record()
                    torch.cuda.synchronize(device)
                    acc.append(e0.elapsed_time(e1) / reps)
                    del fr
            ms[t] = float(np.mean(acc))
            log(f"autotune serving {w}x{h}: tile {t}x{t}: {ms[t]:.3f} ms per view")
        best = min(ms, key=ms.get)
        table[f"{w}x{h}"] = {"tile": best, "ms": {str(k): round(v, 4) for k, v in ms.items()}}
    choice = {"tiles": table}
    store(SERVE_KEY, choice, path)
    return choice


def serve_tile(width: int, height: int, default: int = 32) -> int:
    """The tuned list tile (square side) for a view of width x height: that
    of the tuned resolution nearest in pixel count, or `default` when nothing
    is tuned."""
    c = cached(SERVE_KEY)
    if not c or not c.get("tiles"):
        return default
    px = width * height
    best = min(c["tiles"].items(), key=lambda kv: abs(int(kv[0].split("x")[0]) * int(kv[0].split("x")[1]) - px))
    return int(best[1]["tile"])
