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
