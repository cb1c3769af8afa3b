"""Batched multi-scene, mixed-resolution frames and the render server."""
import numpy as np
import pytest
import torch

from paper_2503_10148_gb300 import frame, inputs, server

from gpu_util import DEV, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scenes():
    require_gpu()
    return [frame.Scene.from_numpy(inputs.scene_clusters_ground(n, seed=40 + i), DEV)
            for i, n in enumerate((20_000, 50_000, 30_000))]


def test_batched_frame_equals_single_frames(scenes):
    """Each job of a multi-scene, mixed-resolution frame renders exactly as
    the same request rendered alone (same kernels, per-job tile lists)."""
    reqs = server.poisson_requests(3, rate=50.0, duration=1.0, seed=7,
                                   resolutions=((64, 48), (200, 120), (256, 256), (97, 131)))[:12]
    assert len({r.scene for r in reqs}) == 3 and len({r.pixels for r in reqs}) > 2
    cfg = frame.make_cfg(tile_w=32, tile_h=32)
    used = sorted({r.scene for r in reqs})
    fr = frame.Frame([scenes[s] for s in used], [r.cam for r in reqs], [used.index(r.scene) for r in reqs], cfg=cfg,
                     device=DEV)
    fr.forward(grow=True)
    torch.cuda.synchronize()
    for j, r in enumerate(reqs):
        one = frame.Frame([scenes[r.scene]], [r.cam], cfg=cfg, device=DEV)
        one.forward(grow=True)
        torch.cuda.synchronize()
        assert torch.equal(fr.image(j), one.image(0)), j


def test_server_completes_every_request(scenes):
    cfg = frame.make_cfg(tile_w=32, tile_h=32)
    reqs = server.poisson_requests(3, rate=80.0, duration=1.5, seed=8,
                                   resolutions=((128, 128), (320, 240), (640, 360)))
    srv = server.RenderServer(scenes, cfg, hbm_budget_bytes=1 << 30, device=DEV)
    lat, overflow = srv.serve(reqs)
    assert lat.shape == (len(reqs),) and np.all(lat > 0) and np.all(np.isfinite(lat))
    assert np.percentile(lat, 99) < 1.0  # far below a second on this load
    plain, psrv = server.serve_plain(scenes, reqs[:20], cfg, hbm_budget_bytes=1 << 30, device=DEV)
    assert np.all(plain > 0) and psrv.frames == 20
    assert server.summarize(lat, reqs, srv)["mpix_s"] > 0


def test_server_batches_a_burst_within_its_budget(scenes):
    """Requests that all arrive at once are rendered in fewer frames than
    requests, each frame within the arena (admission by HBM budget)."""
    import dataclasses
    cfg = frame.make_cfg(tile_w=32, tile_h=32)
    reqs = server.poisson_requests(3, rate=200.0, duration=0.5, seed=9,
                                   resolutions=((128, 128), (320, 240), (640, 360)))
    burst = [dataclasses.replace(r, arrival=0.0) for r in reqs]
    budget = 64 << 20
    srv = server.RenderServer(scenes, cfg, hbm_budget_bytes=budget, device=DEV)
    sizes = []
    orig = srv.render

    def spy(batch, a):
        sizes.append(srv._plan_bytes(batch)[0])
        return orig(batch, a)

    srv.render = spy
    lat, _ = srv.serve(burst, warm=False)
    assert np.all(np.isfinite(lat)) and len(lat) == len(reqs)
    assert srv.frames < len(reqs)
    assert all(b <= budget // 2 for b in sizes[1:]), sizes


def test_served_mixed_frame_against_the_oracle(scenes):
    """A served frame holding 256x256, 800x800, 1297x840 and 1920x1080 jobs of
    two scenes, rendered by the server with the per-frame tile of its largest
    view: 300 seeded pixels per job compared with the FP64 oracle (flagged
    pixels against the admissible results)."""
    import oracle
    from gpu_util import check_forward_view, f32_scene, gpu_last_component, gpu_view, merge_stats
    rng = np.random.default_rng(3)
    res = ((256, 256), (800, 800), (1297, 840), (1920, 1080))
    reqs = [server.Request(i, 0.0, i % 2, frame.f32_camera(inputs.random_sphere_camera(rng, width=w, height=h)), w * h)
            for i, (w, h) in enumerate(res)]
    srv = server.RenderServer(scenes[:2], frame.make_cfg(), hbm_budget_bytes=2 << 30, device=DEV,
                              tile_of=lambda w, h: 16 if w * h < 100_000 else 64)
    fr, ev, used = srv.render(reqs, 0)
    ev.synchronize()
    srv.finish(fr, reqs, used, 0)
    assert fr.cfg.tile_w == 64
    cfgd = frame.cfg_dict(fr.cfg)
    stats = []
    for j, r in enumerate(reqs):
        s32 = f32_scene(scenes[r.scene].to_numpy())
        pix = rng.choice(r.pixels, 300, replace=False).astype(np.int64)
        proj = oracle.project(s32, r.cam, cfgd)
        ref = oracle.render(proj, r.cam, cfgd, pix)
        img, T = gpu_view(fr, j, r.cam, pix)
        stats.append(check_forward_view(proj, r.cam, cfgd, ref, img, T, pix,
                                        last=gpu_last_component(fr, j, r.cam, pix)).stats)
    print("served frame", merge_stats(stats))


def test_server_with_per_frame_tiles_matches_single_frames(scenes):
    """With a tile per frame (that of its largest view), every served image
    equals the same request rendered alone with its frame's tile."""
    import dataclasses
    reqs = server.poisson_requests(3, rate=200.0, duration=0.3, seed=12,
                                   resolutions=((128, 128), (320, 240), (640, 360)))
    burst = [dataclasses.replace(r, arrival=0.0) for r in reqs][:24]
    tile_of = lambda w, h: 16 if w * h <= 128 * 128 else 32
    srv = server.RenderServer(scenes, frame.make_cfg(), hbm_budget_bytes=1 << 30, device=DEV, tile_of=tile_of)
    seen = []
    orig = srv.finish

    def spy(fr, breqs, used, a):
        out = orig(fr, breqs, used, a)
        for j, r in enumerate(breqs):
            one = frame.Frame([scenes[r.scene]], [r.cam], cfg=fr.cfg, device=DEV)
            one.forward(grow=True)
            torch.cuda.synchronize()
            seen.append(torch.equal(fr.image(j), one.image(0)))
        return out

    srv.finish = spy
    lat, _ = srv.serve(burst, warm=False)
    assert len(seen) >= len(burst) and all(seen)
