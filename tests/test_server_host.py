"""Host-side logic of the render server (no GPU): the pair model, the batch
choice (job and scene limits, longest fitting head by bisection, a head
too large for the arena alone is rejected), the seeded Poisson arrivals and
the latency summary.  The frame workspace size is replaced by a stand-in of known
growth, so that only the server's own logic is under test."""
import collections
import os
import sys
import types

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2503_10148_gb300 import _abi, inputs, server  # noqa: E402


def _req(rid, scene, t=0.0, w=256, h=256):
    cam = types.SimpleNamespace(width=w, height=h)
    return server.Request(rid, t, scene, cam, w * h)


def _server(bytes_per_request=100, max_jobs=_abi.SSS_MAX_JOBS):
    """A RenderServer without device state; its workspace size is
    bytes_per_request per request of the head."""
    srv = object.__new__(server.RenderServer)
    srv.max_jobs = max_jobs
    srv.tile_of = None
    srv.calls = []

    def plan_bytes(reqs):
        srv.calls.append(len(reqs))
        return bytes_per_request * len(reqs), None, None, None

    srv._plan_bytes = plan_bytes
    return srv


def test_pair_model_defaults_then_tracks_the_largest_recent_rate():
    pm = server.PairModel(default_per_entry=8.0)
    assert pm.estimate(0, 1000, 256, 256) == 8000
    pm.observe(0, 1000, 256, 256, 5000)      # first observation taken as is
    assert pm.estimate(0, 1000, 256, 256) == 5000
    pm.observe(0, 1000, 256, 256, 2000)      # a lower count decays slowly: 0.8 * 5 + 0.2 * 2
    assert pm.estimate(0, 1000, 256, 256) == pytest.approx(4400, abs=1)
    pm.observe(0, 1000, 256, 256, 9000)      # a higher count is taken at once
    assert pm.estimate(0, 1000, 256, 256) == 9000
    assert pm.estimate(0, 1000, 800, 800) == 8000  # per resolution
    assert pm.estimate(1, 1000, 256, 256) == 8000  # per scene


def test_take_batch_takes_the_longest_head_that_fits():
    srv = _server(bytes_per_request=100)
    q = collections.deque(_req(i, i % 3) for i in range(20))
    got = srv.take_batch(q, arena_bytes=750)
    assert [r.rid for r in got] == list(range(7))  # 7 x 100 <= 750 < 8 x 100
    assert len(q) == 13 and q[0].rid == 7
    assert max(srv.calls) <= 20 and len(srv.calls) <= 1 + int(np.ceil(np.log2(20))) + 1  # bisection


def test_take_batch_respects_the_job_and_scene_limits():
    srv = _server(bytes_per_request=1)
    q = collections.deque(_req(i, i) for i in range(12))  # every request a new scene
    got = srv.take_batch(q, arena_bytes=1 << 30)
    assert len(got) == _abi.SSS_MAX_SCENES
    srv = _server(bytes_per_request=1)
    q = collections.deque(_req(i, 0) for i in range(_abi.SSS_MAX_JOBS + 5))  # one scene
    assert len(srv.take_batch(q, arena_bytes=1 << 30)) == _abi.SSS_MAX_JOBS
    srv = _server(bytes_per_request=1, max_jobs=1)  # the plain server: one request per frame
    q = collections.deque(_req(i, 0) for i in range(4))
    assert [r.rid for r in srv.take_batch(q, arena_bytes=1 << 30)] == [0]


def test_take_batch_rejects_an_oversized_head_and_takes_nothing_from_an_empty_queue():
    """The HBM budget holds: a request whose frame alone exceeds the arena is
    rejected (counted), never rendered in memory of its own."""
    srv = _server(bytes_per_request=1000)
    srv.rejected = []
    q = collections.deque(_req(i, 0) for i in range(3))
    got = srv.take_batch(q, arena_bytes=500)
    assert got == [] and [r.rid for r in srv.rejected] == [0] and len(q) == 2
    assert srv.take_batch(collections.deque(), arena_bytes=500) == []


def test_poisson_requests_are_seeded_ordered_and_at_the_rate(monkeypatch):
    monkeypatch.setattr(server.F, "f32_camera", lambda c: c)
    a = server.poisson_requests(3, rate=200.0, duration=5.0, seed=7)
    b = server.poisson_requests(3, rate=200.0, duration=5.0, seed=7)
    assert [(r.arrival, r.scene, r.pixels) for r in a] == [(r.arrival, r.scene, r.pixels) for r in b]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 5.0
    assert abs(len(a) - 1000) < 4 * np.sqrt(1000)  # Poisson count, 4 sigma
    assert {r.scene for r in a} == {0, 1, 2}
    res = {(r.cam.width, r.cam.height) for r in a}
    assert res == set(inputs.SERVE_RESOLUTIONS)
    assert all(r.pixels == r.cam.width * r.cam.height for r in a)
    assert [r.rid for r in a] == list(range(len(a)))


def test_summarize_reports_percentiles_and_throughput_over_the_span():
    reqs = [_req(i, 0, w=100, h=100) for i in range(100)]
    lat = np.arange(1, 101, dtype=np.float64) * 1e-3  # 1 .. 100 ms
    srv = types.SimpleNamespace(frames=40, span_s=2.0, rejected=[], outside_allocs=0, outside_bytes_max=0)
    s = server.summarize(lat, reqs, srv)
    assert s["requests"] == 100 and s["frames"] == 40 and s["requests_per_frame"] == 2.5
    assert s["rejected"] == 0 and s["outside_arena_frames"] == 0
    assert s["p50_ms"] == pytest.approx(50.5) and s["p99_ms"] == pytest.approx(99.01)
    assert s["mean_ms"] == pytest.approx(50.5)
    assert s["mpix_s"] == pytest.approx(100 * 100 * 100 / 2.0 / 1e6)


def test_summarize_counts_rejected_requests_out_of_the_throughput():
    reqs = [_req(i, 0, w=100, h=100) for i in range(10)]
    srv = types.SimpleNamespace(frames=3, span_s=1.0, rejected=reqs[:2], outside_allocs=1, outside_bytes_max=3 << 20)
    s = server.summarize(np.full(8, 1e-3), reqs, srv)
    assert s["rejected"] == 2 and s["mpix_s"] == pytest.approx(8 * 100 * 100 / 1e6)
    assert s["requests_per_frame"] == pytest.approx(8 / 3, abs=1e-3)
    assert s["outside_arena_frames"] == 1 and s["outside_arena_mb_max"] == 3.0


def test_frame_tile_follows_the_largest_view():
    srv = object.__new__(server.RenderServer)
    srv.cfg = _abi.sss_default_cfg()
    srv.tile_of = lambda w, h: 16 if w * h < 100_000 else 64
    small, big = _req(0, 0, w=256, h=256), _req(1, 0, w=1920, h=1080)
    assert srv.frame_cfg([small]).tile_w == 16 and srv.frame_cfg([small]).tile_h == 16
    assert srv.frame_cfg([small, big]).tile_w == 64
    assert srv.frame_cfg([small]).batch == srv.cfg.batch  # the rest of the options kept
    srv.tile_of = None
    assert srv.frame_cfg([small]) is srv.cfg


def test_serve_tile_reads_the_tuned_table(tmp_path, monkeypatch):
    from paper_2503_10148_gb300 import autotune
    path = str(tmp_path / "tuned.json")
    monkeypatch.setattr(autotune, "CACHE", path)
    assert autotune.serve_tile(800, 800) == 32  # nothing tuned: the default
    autotune.store(autotune.SERVE_KEY, {"tiles": {"256x256": {"tile": 16}, "800x800": {"tile": 32},
                                                   "1920x1080": {"tile": 64}}}, path)
    assert autotune.serve_tile(256, 256) == 16 and autotune.serve_tile(300, 300) == 16
    assert autotune.serve_tile(1297, 840) == 32 and autotune.serve_tile(1920, 1080) == 64


def test_take_batch_keeps_to_the_head_tile_class():
    """With a tile policy a frame holds only requests of its head's tile
    class, in arrival order, from the first `lookahead` queued requests; the
    others keep their places."""
    srv = _server(bytes_per_request=1)
    srv.tile_of = lambda w, h: 16 if w * h < 100_000 else 64
    q = collections.deque([_req(0, 0, w=256, h=256), _req(1, 1, w=256, h=256), _req(2, 0, w=1920, h=1080),
                           _req(3, 0, w=256, h=256), _req(4, 0, w=1920, h=1080)])
    assert [r.rid for r in srv.take_batch(q, arena_bytes=1 << 30)] == [0, 1, 3]
    assert [r.rid for r in q] == [2, 4]
    assert [r.rid for r in srv.take_batch(q, arena_bytes=1 << 30)] == [2, 4]
    q = collections.deque([_req(0, 0, w=256, h=256), _req(1, 0, w=1920, h=1080), _req(2, 0, w=256, h=256)])
    assert [r.rid for r in srv.take_batch(q, arena_bytes=1 << 30, lookahead=2)] == [0]
