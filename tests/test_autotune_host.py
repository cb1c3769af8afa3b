"""Host-side parts of the autotuner (no GPU): every candidate it would time
is a launch shape the planner accepts, and its cache keeps one choice per
workload."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2503_10148_gb300 import _abi, autotune, frame  # noqa: E402


def _scene(n):
    p = _abi.sss_params()
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        setattr(p, f, 0x1000)  # never dereferenced by the planner
    p.n, p.sh_degree = n, 3
    return p


def _cam(w, h):
    c = _abi.sss_camera()
    c.viewmat[0] = c.viewmat[5] = c.viewmat[10] = 1.0
    c.viewmat[11] = 3.0
    c.fx = c.fy = 1000.0
    c.cx, c.cy = w / 2, h / 2
    c.width, c.height = w, h
    return c


def test_every_candidate_plans_and_tiles_the_image():
    cands = [(tw, th, b) for (tw, th) in autotune.TILES for b in autotune.BATCHES]
    assert len(set(cands)) == len(cands) == 20
    for tw, th, b in cands:
        cfg = frame.make_cfg(tile_w=tw, tile_h=th, batch=b)
        plan = _abi.sss_plan_frame([_scene(1000)], [_cam(1297, 840), _cam(256, 256)], [0, 0], cfg, 1 << 20)
        want = sum(-(-w // tw) * -(-h // th) for w, h in ((1297, 840), (256, 256)))
        assert plan.n_tiles == want, (tw, th)
        assert plan.cfg.tile_w == tw and plan.cfg.tile_h == th and plan.cfg.batch == b


def test_store_keeps_one_choice_per_workload_and_cached_reads_it(tmp_path, monkeypatch):
    path = str(tmp_path / "tuned.json")
    monkeypatch.setattr(autotune, "CACHE", path)
    assert autotune.cached("a") is None  # no file yet
    autotune.store("a", {"tile_w": 64, "tile_h": 128, "batch": 32}, path)
    autotune.store("b", {"tile_w": 32, "tile_h": 32, "batch": 64}, path)
    autotune.store("a", {"tile_w": 64, "tile_h": 64, "batch": 32}, path)  # replaces a, keeps b
    with open(path) as f:
        data = json.load(f)
    assert set(data) == {"a", "b"}
    assert autotune.cached("a") == {"tile_w": 64, "tile_h": 64, "batch": 32}
    assert autotune.cached("b")["batch"] == 64
    with open(path, "w") as f:
        f.write("{ not json")
    assert autotune.cached("a") is None  # a damaged cache reads as no choice
    autotune.store("c", {"tile_w": 16, "tile_h": 16, "batch": 32}, path)  # and is rewritten
    assert autotune.cached("c")["tile_w"] == 16


def test_candidates_pair_the_tall_backward_box_with_tall_tiles():
    cands = autotune.default_candidates()
    assert len(cands) == len(autotune.TILES) * len(autotune.BATCHES) + 10
    assert all(box == 8 or (tw >= 32 and th >= 64) for tw, th, _, box in cands)
    assert len({autotune.candidate_key(*c) for c in cands}) == len(cands)


def test_the_shipped_choice_is_a_candidate():
    choice = autotune.cached("clusters_1p5m_4views")
    assert choice is not None
    assert (choice["tile_w"], choice["tile_h"]) in autotune.TILES and choice["batch"] in autotune.BATCHES
    key = autotune.candidate_key(choice["tile_w"], choice["tile_h"], choice["batch"], choice.get("bwd_box_h", 8))
    assert set(choice["candidates"]) == {autotune.candidate_key(*c) for c in autotune.default_candidates()}
    # the finalists are the fastest candidates of the first stage, re-timed
    fin = choice["finalists"]
    first = sorted(choice["candidates"], key=choice["candidates"].get)[:len(fin)]
    assert set(fin) == set(first) and key in fin
    assert choice["ms_per_step"] == min(fin.values()) == fin[key]
