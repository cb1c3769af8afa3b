"""Render server: batches novel-view requests as they arrive.

Scenes stay resident on the device.  Requests (scene, camera, resolution)
queue in arrival order; whenever a workspace arena is free, the server takes
the queued requests in order while the frame's estimated workspace fits the
arena (the HBM budget is split between two arenas so one batch renders while
the next is assembled), at most SSS_MAX_JOBS jobs and SSS_MAX_SCENES scenes,
and renders them as ONE multi-scene, mixed-resolution frame (project + bin +
sort + render_fwd in four launches).  A request's latency runs from its
arrival to the device completion of its frame, read from CUDA events recorded
on the rendering stream.

The pair count of a frame is estimated from the pairs per (scene, view) seen
so far (per scene and resolution); a frame that still overflows its capacity
is re-rendered with the measured count (the device status word reports it).

HBM budget: the arenas hold every workspace.  A request whose frame alone
does not fit an arena is rejected at admission (counted, not rendered).  An
overflow re-render whose larger plan no longer fits its arena is split into
single-request frames rendered one after another in the arena; a single
request that still does not fit is rendered in a frame-owned workspace, and
such allocations are counted and reported (they are the only device memory
beyond the budget).

``serve_plain`` is the reference form: the same server, the same two arenas
and streams, with one request per frame (one launch sequence per request), so
the two differ only in batching.  Images stay in their arena until the
arena's next frame.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import _abi as abi
from . import frame as F
from . import inputs


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float  # seconds from the start of the run
    scene: int
    cam: object
    pixels: int


def poisson_requests(n_scenes: int, rate: float, duration: float, seed: int, resolutions=inputs.SERVE_RESOLUTIONS):
    """Seeded Poisson arrivals; uniform scene, uniform resolution, uniform
    camera direction on the radius-3 sphere."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        w, h = resolutions[rng.integers(len(resolutions))]
        cam = F.f32_camera(inputs.random_sphere_camera(rng, width=w, height=h))
        out.append(Request(len(out), t, int(rng.integers(n_scenes)), cam, w * h))
    return out


class PairModel:
    """Pairs per (scene, view) seen so far, by scene, resolution and list
    tile."""

    def __init__(self, default_per_entry: float = 8.0):
        self.rate = {}
        self.default = default_per_entry

    def estimate(self, scene_idx: int, n: int, w: int, h: int, tile: int = 0) -> int:
        r = self.rate.get((scene_idx, w, h, tile), self.default)
        return int(r * n)

    def observe(self, scene_idx: int, n: int, w: int, h: int, pairs: int, tile: int = 0):
        key = (scene_idx, w, h, tile)
        old = self.rate.get(key)
        val = pairs / max(n, 1)
        self.rate[key] = val if old is None else max(val, 0.8 * old + 0.2 * val)


class RenderServer:
    def __init__(self, scenes, cfg=None, hbm_budget_bytes: int = 8 << 30, headroom: float = 1.6, device="cuda",
                 max_jobs: int = abi.SSS_MAX_JOBS, n_arenas: int = 2, tile_of=None):
        """``tile_of``: optional (width, height) -> square list tile side; a
        frame then takes the tile of its largest view (small views render
        faster on small tiles, large ones on large tiles), else ``cfg``'s."""
        self.scenes = list(scenes)
        self.cfg = cfg if cfg is not None else F.make_cfg()
        self.tile_of = tile_of
        self.device = torch.device(device)
        self.max_jobs = max(1, min(int(max_jobs), abi.SSS_MAX_JOBS))
        per = hbm_budget_bytes // n_arenas
        self.arenas = [torch.empty(per, dtype=torch.uint8, device=self.device) for _ in range(n_arenas)]
        self.arena_busy = [None] * n_arenas  # event of the frame using the arena
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_arenas)]  # one per arena
        self.pairs = PairModel()
        self.headroom = headroom
        self.frames = 0
        self.rejected = []  # requests whose frame alone exceeds an arena
        self.outside_allocs = 0  # frames that had to allocate beyond the arenas
        self.outside_bytes_max = 0
        self.span_s = 0.0  # first arrival to last completion of the last serve()

    # ------------------------------------------------------------ batches
    def frame_cfg(self, reqs):
        """The raster options of a frame of ``reqs``."""
        if self.tile_of is None:
            return self.cfg
        big = max(reqs, key=lambda r: r.cam.width * r.cam.height)
        t = int(self.tile_of(big.cam.width, big.cam.height))
        c = type(self.cfg).from_buffer_copy(self.cfg)
        c.tile_w = c.tile_h = t
        return c

    def _plan_bytes(self, reqs):
        used = sorted({r.scene for r in reqs})
        remap = {s: i for i, s in enumerate(used)}
        cfg = self.frame_cfg(reqs)
        cap = 4096 + int(self.headroom * sum(
            self.pairs.estimate(r.scene, self.scenes[r.scene].n, r.cam.width, r.cam.height, cfg.tile_w) for r in reqs))
        plan = abi.sss_plan_frame([self.scenes[s].params() for s in used], [F.camera_struct(r.cam) for r in reqs],
                                  [remap[r.scene] for r in reqs], cfg, min(cap, 0x7fffffff))
        return F.Frame.bytes_needed(plan), used, remap, cap

    def tile_class(self, r) -> int:
        """The list tile a request renders best on (0 without a tile policy)."""
        return int(self.tile_of(r.cam.width, r.cam.height)) if self.tile_of is not None else 0

    def take_batch(self, queue: collections.deque, arena_bytes: int, lookahead: int = 2 * abi.SSS_MAX_JOBS):
        """The longest run of queued requests whose frame fits the arena (at
        most SSS_MAX_JOBS jobs and SSS_MAX_SCENES scenes), found by
        bisection: the workspace grows with every request added, so the
        fitting runs are a prefix of the lengths.  With a tile policy the
        run holds only requests of the head's tile class (no view renders on
        a tile chosen for another size), taken in arrival order from the
        first ``lookahead`` queued requests; the others keep their places.
        A head request whose frame alone does not fit the arena is rejected
        (moved to ``self.rejected``) and an empty batch returned."""
        if not queue:
            return []
        cls = self.tile_class(queue[0])
        picked, scenes = [], set()
        for i, r in enumerate(queue):
            if i == lookahead or len(picked) == self.max_jobs:
                break
            if self.tile_class(r) != cls or (r.scene not in scenes and len(scenes) == abi.SSS_MAX_SCENES):
                continue
            scenes.add(r.scene)
            picked.append(i)
        head = [queue[i] for i in picked]
        if self._plan_bytes(head[:1])[0] > arena_bytes:
            self.rejected.append(queue.popleft())
            return []
        lo, hi = 1, len(head)  # lo: known to fit, hi: upper bound
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if self._plan_bytes(head[:mid])[0] <= arena_bytes:
                lo = mid
            else:
                hi = mid - 1
        take = set(picked[:lo])
        rest = [r for i, r in enumerate(queue) if i not in take]
        queue.clear()
        queue.extend(rest)
        return head[:lo]

    def _count_outside(self, fr):
        if fr.outside_bytes:
            self.outside_allocs += 1
            self.outside_bytes_max = max(self.outside_bytes_max, int(fr.outside_bytes))

    def render(self, reqs, arena_idx: int):
        """Enqueue one frame for ``reqs`` on the server stream; returns
        (frame, done event)."""
        _, used, remap, cap = self._plan_bytes(reqs)
        st = self.streams[arena_idx]
        with torch.cuda.stream(st):
            fr = F.Frame([self.scenes[s] for s in used], [r.cam for r in reqs], [remap[r.scene] for r in reqs],
                         cfg=self.frame_cfg(reqs), pair_capacity=cap, device=self.device,
                         arena=self.arenas[arena_idx])
            fr.forward(st, grow=False)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        self._count_outside(fr)
        return fr, ev, used

    def finish(self, fr, reqs, used, arena_idx: int):
        """Check the frame's status; re-render it on overflow.  Updates the
        pair model from the device counts (needs the frame complete)."""
        st_ = self.streams[arena_idx]
        st, need, _ = fr.status(st_)
        if st & abi.SSS_STATUS_PAIR_OVERFLOW:
            cap = int(need * 1.1) + 4096
            arena = self.arenas[arena_idx]
            plan = abi.sss_plan_frame([s.params() for s in fr.scenes], [F.camera_struct(c) for c in fr.cams],
                                      fr.job_scene, fr.cfg, min(cap, 0x7fffffff))
            if len(reqs) > 1 and F.Frame.bytes_needed(plan) > arena.numel():
                # split: one request per frame, in turn, in the arena
                for r in reqs:
                    one, _, _ = self.render([r], arena_idx)
                    self.frames += 1
                    self.finish(one, [r], [r.scene], arena_idx)
                return True
            fr.pair_capacity = cap
            fr._replan()
            self._count_outside(fr)
            with torch.cuda.stream(st_):
                fr.forward(st_, grow=False)
            st_.synchronize()
        P = fr.plan
        cum = torch.cumsum(fr.ntiles(), 0, dtype=torch.int64)
        ends = torch.tensor([P.jobs[j].entry_base + self.scenes[r.scene].n - 1 for j, r in enumerate(reqs)],
                            device=cum.device)
        ends_np = cum[ends].cpu().numpy()
        counts = np.diff(np.concatenate([[0], ends_np]))
        for r, c in zip(reqs, counts):
            self.pairs.observe(r.scene, self.scenes[r.scene].n, r.cam.width, r.cam.height, int(c), fr.cfg.tile_w)
        return bool(st & abi.SSS_STATUS_PAIR_OVERFLOW)

    # ------------------------------------------------------------ serving loop
    def serve(self, requests, warm=True):
        """Replay ``requests`` in real time.  Returns per-request latency (s).
        The warm-up, outside the timed run, renders one request of every
        (scene, resolution) alone -- every launch and host path, and the pair
        model's first count of each -- alternating the arenas."""
        if warm:
            first = {}
            for r in requests:
                first.setdefault((r.scene, r.cam.width, r.cam.height), r)
            for i, r in enumerate(first.values()):
                a = i % len(self.arenas)
                fr, ev, used = self.render([r], a)
                ev.synchronize()
                self.finish(fr, [r], used, a)
            torch.cuda.synchronize(self.device)
        reqs = sorted(requests, key=lambda r: r.arrival)
        start_ev = torch.cuda.Event(enable_timing=True)
        start_ev.record(self.streams[0])
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        pending = collections.deque(reqs)
        queue = collections.deque()
        inflight = []  # (arena, frame, event, reqs, used)
        latency = {}
        overflow = 0
        last_done = 0.0
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # retire finished frames
            for item in list(inflight):
                a, fr, ev, breqs, used = item
                if ev.query():
                    if self.finish(fr, breqs, used, a):
                        overflow += 1
                        ev = torch.cuda.Event(enable_timing=True)
                        ev.record(self.streams[a])
                        self.streams[a].synchronize()
                    done = start_ev.elapsed_time(ev) / 1e3
                    last_done = max(last_done, done)
                    for r in breqs:
                        latency[r.rid] = done - r.arrival
                    inflight.remove(item)
                    self.arena_busy[a] = None
            free = [a for a in range(len(self.arenas)) if self.arena_busy[a] is None]
            if queue and free:
                a = free[0]
                batch = self.take_batch(queue, self.arenas[a].numel())
                if not batch:  # the head request was rejected
                    continue
                fr, ev, used = self.render(batch, a)
                self.frames += 1
                self.arena_busy[a] = ev
                inflight.append((a, fr, ev, batch, used))
                continue
            if not queue and pending and not inflight:
                time.sleep(max(0.0, min(pending[0].arrival - now, 0.002)))
            else:
                time.sleep(0.0002)
        lat = np.array([latency[r.rid] for r in reqs if r.rid in latency])
        self.span_s = last_done - (reqs[0].arrival if reqs else 0.0)
        return lat, overflow


def serve_plain(scenes, requests, cfg=None, hbm_budget_bytes: int = 8 << 30, device="cuda", tile_of=None):
    """One frame per request, in arrival order, on the same two arenas,
    streams and tile policy as the batched server (only the batching
    differs).  Returns (latency, server)."""
    srv = RenderServer(scenes, cfg, hbm_budget_bytes=hbm_budget_bytes, device=device, max_jobs=1, n_arenas=2,
                       tile_of=tile_of)
    lat, _ = srv.serve(requests)
    return lat, srv


def summarize(lat, requests, srv: RenderServer) -> dict:
    """Latency percentiles and throughput (pixels over the span from the
    first arrival to the last completion)."""
    rejected = {r.rid for r in srv.rejected}
    px = sum(r.pixels for r in requests if r.rid not in rejected)
    served = len(requests) - len(rejected)
    return {"requests": len(requests), "frames": srv.frames,
            "requests_per_frame": round(served / max(srv.frames, 1), 3), "rejected": len(rejected),
            "outside_arena_frames": srv.outside_allocs, "outside_arena_mb_max": round(srv.outside_bytes_max / 2 ** 20, 1),
            "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
            "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3), "mean_ms": round(float(lat.mean()) * 1e3, 3),
            "mpix_s": round(px / max(srv.span_s, 1e-9) / 1e6, 2), "span_s": round(srv.span_s, 3)}
