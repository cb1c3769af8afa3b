"""Device-side objects around the C ABI: scenes, cameras, frames.

PyTorch only provides device memory and streams here; every step of the
rasterizer runs in libsss.  A Frame owns one plan and its workspace and
enqueues the entry points in order:

    forward:  sss_project -> sss_bin -> sss_sort -> sss_render_fwd
    backward: sss_render_bwd -> sss_project_bwd

Pair capacity: the number of (tile, splat) pairs is only known on the device.
``Frame.forward(grow=True)`` reads it back once after binning and, if the
capacity was too small, re-plans with 25% headroom and re-runs the frame.
Graph-captured use (see ``graph.py``) sizes the capacity up front and checks
the device status word afterwards instead.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi as abi

FIELDS = ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh")


def _rows(field: str, sh_degree: int) -> int:
    return {"mean": 3, "log_scale": 3, "quat": 4, "nu": 1, "opacity_raw": 1,
            "sh": 3 * (sh_degree + 1) ** 2}[field]


class Scene:
    """Planar float32 parameters [rows][n] of one mixture, resident on a device."""

    def __init__(self, tensors: dict, n: int, sh_degree: int):
        self.t = tensors
        self.n = int(n)
        self.sh_degree = int(sh_degree)
        for f in FIELDS:
            x = self.t[f]
            assert x.dtype == torch.float32 and x.is_contiguous(), f
            assert x.numel() == _rows(f, sh_degree) * self.n, (f, x.shape)

    @classmethod
    def from_numpy(cls, scene: dict, device="cuda") -> "Scene":
        t = {f: torch.as_tensor(np.ascontiguousarray(scene[f], np.float32), device=device).reshape(
            _rows(f, scene["sh_degree"]), scene["n"]) for f in FIELDS}
        return cls(t, scene["n"], scene["sh_degree"])

    @classmethod
    def zeros(cls, n: int, sh_degree: int, device="cuda") -> "Scene":
        t = {f: torch.zeros(_rows(f, sh_degree), n, dtype=torch.float32, device=device) for f in FIELDS}
        return cls(t, n, sh_degree)

    def zeros_like(self) -> "Scene":
        return Scene.zeros(self.n, self.sh_degree, self.t["mean"].device)

    def params(self) -> abi.sss_params:
        p = abi.sss_params()
        for f in FIELDS:
            setattr(p, f, self.t[f].data_ptr())
        p.n = self.n
        p.sh_degree = self.sh_degree
        return p

    def to_numpy(self) -> dict:
        out = {f: self.t[f].detach().cpu().numpy() for f in FIELDS}
        out["nu"] = out["nu"].reshape(-1)
        out["opacity_raw"] = out["opacity_raw"].reshape(-1)
        out["n"] = self.n
        out["sh_degree"] = self.sh_degree
        return out


def camera_struct(cam) -> abi.sss_camera:
    c = abi.sss_camera()
    vm = np.asarray(cam.viewmat, np.float32).reshape(-1)
    for k in range(12):
        c.viewmat[k] = float(vm[k])
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def f32_camera(cam):
    """The camera with every parameter rounded to float32 (what the GPU sees);
    tests hand this to the oracle so both sides start from the same numbers."""
    from .inputs import Camera
    return Camera(np.asarray(cam.viewmat, np.float32).astype(np.float64),
                  float(np.float32(cam.fx)), float(np.float32(cam.fy)), float(np.float32(cam.cx)),
                  float(np.float32(cam.cy)), int(cam.width), int(cam.height))


def make_cfg(**kw) -> abi.sss_raster_cfg:
    c = abi.sss_default_cfg()
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                c.bg[i] = float(v[i])
        else:
            setattr(c, k, v)
    return c


def cfg_dict(c: abi.sss_raster_cfg) -> dict:
    """The options as the oracle's dictionary (float64 of the FP32 values)."""
    return dict(tau=float(c.tau), t_min=float(c.t_min), alpha_max=float(c.alpha_max), znear=float(c.znear),
                lowpass=float(c.lowpass), bg=tuple(float(c.bg[i]) for i in range(3)), tile_w=int(c.tile_w),
                tile_h=int(c.tile_h), nu_grad_mode=int(c.nu_grad_mode), kernel=int(c.kernel))


class Frame:
    """One batch of (scene, camera) jobs with its plan and workspace."""

    def __init__(self, scenes, cams, job_scene=None, cfg: abi.sss_raster_cfg | None = None,
                 pair_capacity: int | None = None, device="cuda", arena: torch.Tensor | None = None):
        """``arena``: optional uint8 device buffer holding the workspace and
        the output image (a resident buffer reused across frames); a fresh
        one is allocated when it is missing or too small."""
        self.scenes = list(scenes)
        self.cams = list(cams)
        self.job_scene = list(job_scene) if job_scene is not None else [0] * len(self.cams)
        self.cfg = cfg if cfg is not None else abi.sss_default_cfg()
        self.device = torch.device(device)
        self.arena = arena
        n_entries = sum(self.scenes[s].n for s in self.job_scene)
        self.pair_capacity = int(pair_capacity or max(1 << 16, 16 * n_entries))
        self.generation = 0  # forwards run through the autograd form
        # optional {"render_fwd" | "render_bwd": (start, end)} CUDA events
        # recorded around those launches (also inside a captured graph when
        # the events are external), for kernel timing
        self.timing = None
        self._replan()

    @staticmethod
    def bytes_needed(plan) -> int:
        return ((int(plan.ws_bytes) + 255) & ~255) + 12 * int(plan.n_pixels)

    def _replan(self):
        self.plan = abi.sss_plan_frame([s.params() for s in self.scenes], [camera_struct(c) for c in self.cams],
                                       self.job_scene, self.cfg, self.pair_capacity)
        need = self.bytes_needed(self.plan)
        if self.arena is not None and self.arena.numel() >= need:
            wsb = (int(self.plan.ws_bytes) + 255) & ~255
            self.ws = self.arena[:int(self.plan.ws_bytes)]
            self.rgb = self.arena[wsb:wsb + 12 * int(self.plan.n_pixels)].view(torch.float32)
            self.outside_bytes = 0
        else:
            self.ws = torch.empty(int(self.plan.ws_bytes), dtype=torch.uint8, device=self.device)
            self.rgb = torch.empty(3 * int(self.plan.n_pixels), dtype=torch.float32, device=self.device)
            # bytes held outside a caller's arena (a server counts them against its budget)
            self.outside_bytes = need if self.arena is not None else 0

    # ------------------------------------------------------------ steps
    @property
    def ws_ptr(self) -> int:
        return self.ws.data_ptr()

    def project(self, stream=None):
        abi.sss_project(self.plan, self.ws_ptr, stream)

    def bin(self, stream=None):
        abi.sss_bin(self.plan, self.ws_ptr, stream)

    def sort(self, stream=None):
        abi.sss_sort(self.plan, self.ws_ptr, stream)

    def _mark(self, name: str, i: int, stream):
        if self.timing and name in self.timing:
            ev = self.timing[name][i]
            ev.record(stream) if stream is not None else ev.record()

    def render_fwd(self, stream=None, out: torch.Tensor | None = None):
        if out is None:
            out = self.rgb
        assert out.dtype == torch.float32 and out.is_contiguous() and out.numel() == 3 * int(self.plan.n_pixels)
        self._mark("render_fwd", 0, stream)
        abi.sss_render_fwd(self.plan, self.ws_ptr, out.data_ptr(), stream)
        self._mark("render_fwd", 1, stream)

    def render_bwd(self, dl_drgb: torch.Tensor, stream=None):
        assert dl_drgb.dtype == torch.float32 and dl_drgb.is_contiguous()
        assert dl_drgb.numel() == self.rgb.numel()
        self._mark("render_bwd", 0, stream)
        abi.sss_render_bwd(self.plan, self.ws_ptr, dl_drgb.data_ptr(), stream)
        self._mark("render_bwd", 1, stream)

    def project_bwd(self, grads, stream=None):
        abi.sss_project_bwd(self.plan, self.ws_ptr, [g.params() for g in grads], stream)

    def status(self, stream=None):
        """(status bits, pairs needed, pairs sorted); synchronises the stream."""
        return abi.sss_read_status(self.plan, self.ws_ptr, stream)

    def forward(self, stream=None, grow: bool = True, out: torch.Tensor | None = None):
        """project -> bin -> sort -> render_fwd; the images go to ``out``
        (flat float32 [3 * n_pixels]) or to the frame's own buffer."""
        self.project(stream)
        self.bin(stream)
        if grow:
            st, need, _ = self.status(stream)
            if need > self.pair_capacity:
                self.pair_capacity = int(need * 1.25) + 1024
                self._replan()
                self.project(stream)
                self.bin(stream)
        self.sort(stream)
        self.render_fwd(stream, out)
        return self.rgb if out is None else out

    def count_pairs(self, stream=None) -> tuple[int, int]:
        """One forward with pair counting on (``cfg.count_pairs``); returns
        the frame's contributing and evaluated (splat, pixel) pairs."""
        self.plan.cfg.count_pairs = 1
        try:
            self.forward(stream, grow=False)
        finally:
            self.plan.cfg.count_pairs = 0
        ctrl = self.ws_view(self.plan.ws_off_ctrl, torch.int64, 4).cpu()
        return int(ctrl[2]), int(ctrl[3])

    def backward(self, dl_drgb: torch.Tensor, grads, stream=None):
        self.render_bwd(dl_drgb, stream)
        self.project_bwd(grads, stream)

    # ------------------------------------------------------------ views
    def ws_view(self, off: int, dtype: torch.dtype, count: int) -> torch.Tensor:
        nbytes = torch.empty((), dtype=dtype).element_size() * int(count)
        return self.ws[int(off):int(off) + nbytes].view(dtype)

    def image(self, j: int) -> torch.Tensor:
        return self.image_of(self.rgb, j)

    def image_of(self, flat: torch.Tensor, j: int) -> torch.Tensor:
        """Job j's [3][H][W] image inside a flat [3 * n_pixels] buffer."""
        J = self.plan.jobs[j]
        H, W = J.cam.height, J.cam.width
        b = 3 * J.pix_base
        return flat[b:b + 3 * H * W].view(3, H, W)

    def image_slices(self):
        return [self.image(j) for j in range(self.plan.n_jobs)]

    def records(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_rec, torch.float32, 12 * self.plan.n_entries).view(-1, 12)

    def depth_keys(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_dkey, torch.int32, self.plan.n_entries)

    def ntiles(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_ntiles, torch.int32, self.plan.n_entries)

    def rects(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_rect, torch.int32, 2 * self.plan.n_entries).view(-1, 2)

    def sorted_pairs(self, count: int):
        cap = self.plan.pair_capacity
        slot = self.plan.pair_slot
        k = self.ws_view(self.plan.ws_off_pkey, torch.int32, 2 * cap)[slot * cap:slot * cap + count]
        v = self.ws_view(self.plan.ws_off_pval, torch.int32, 2 * cap)[slot * cap:slot * cap + count]
        return k, v

    def ranges(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_ranges, torch.int32, 2 * self.plan.n_tiles).view(-1, 2)

    def final_T(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_T, torch.float32, self.plan.n_pixels)

    def last_contrib(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_last, torch.int32, self.plan.n_pixels)

    def grad2d(self) -> torch.Tensor:
        return self.ws_view(self.plan.ws_off_grad2d, torch.float32, 12 * self.plan.n_entries).view(-1, 12)


def step_params(eps=1e-3, C=0.5, k=100.0, t0=0.005, burn_in=False, seed=0, step=0,
                lr=(5e-3, 1e-3, 1e-2, 5e-2, 2.5e-3), beta1=0.9, beta2=0.999, adam_eps=1e-15,
                step_counter: torch.Tensor | None = None, reg_opacity=0.0, reg_scale=0.0,
                mu_adam: tuple | None = None, philox_out: torch.Tensor | None = None) -> abi.sss_step_params:
    """Sampler options.  With ``step_counter`` (a 1-element int64 device
    tensor) the step index is read from and advanced on the device, so a
    CUDA-graph replay of the step draws fresh noise.  ``reg_opacity`` and
    ``reg_scale`` are the loss's regulariser weights, whose gradients the
    step adds.  ``mu_adam`` = (m, v), two float32 [3][n] device tensors:
    the SGHMC gradient becomes Adam's normalised gradient of dL/dmu.
    ``philox_out``, an int32 or uint32 [4][n] device tensor, receives the
    Philox words the noise of each component was drawn from."""
    sp = abi.sss_step_params()
    if step_counter is not None:
        assert step_counter.dtype == torch.int64 and step_counter.numel() == 1
        sp.step_counter = step_counter.data_ptr()
    sp.eps, sp.C, sp.k, sp.t0 = eps, C, k, t0
    sp.burn_in = int(bool(burn_in))
    sp.seed, sp.step = int(seed), int(step)
    for i in range(5):
        sp.lr[i] = float(lr[i])
    sp.beta1, sp.beta2, sp.adam_eps = beta1, beta2, adam_eps
    sp.reg_opacity, sp.reg_scale = float(reg_opacity), float(reg_scale)
    if mu_adam is not None:
        sp.mu_adam_m, sp.mu_adam_v = mu_adam[0].data_ptr(), mu_adam[1].data_ptr()
    if philox_out is not None:
        assert philox_out.element_size() == 4 and philox_out.is_contiguous()
        sp.philox_out = philox_out.data_ptr()
    return sp


class SamplerState:
    """Momentum (3 x n) and Adam moments ((9 + 3K) x n) of one scene."""

    def __init__(self, scene: Scene):
        dev = scene.t["mean"].device
        K = (scene.sh_degree + 1) ** 2
        self.r = torch.zeros(3, scene.n, dtype=torch.float32, device=dev)
        self.m = torch.zeros(9 + 3 * K, scene.n, dtype=torch.float32, device=dev)
        self.v = torch.zeros(9 + 3 * K, scene.n, dtype=torch.float32, device=dev)


def sghmc_step(scene: Scene, grads: Scene, state: SamplerState, sp: abi.sss_step_params, xi_out=None,
               stream=None, out: Scene | None = None):
    """One sampler step on ``scene``, in place, or into ``out`` (a scene of
    the same size and degree, in separate memory) leaving ``scene`` as it was."""
    xi = xi_out.data_ptr() if xi_out is not None else 0
    if out is None:
        abi.sss_sghmc_step(scene.params(), grads.params(), state.r.data_ptr(), state.m.data_ptr(),
                           state.v.data_ptr(), sp, xi, stream)
    else:
        abi.sss_sghmc_step_to(scene.params(), out.params(), grads.params(), state.r.data_ptr(), state.m.data_ptr(),
                              state.v.data_ptr(), sp, xi, stream)


def loss_l1(pred: torch.Tensor, target: torch.Tensor, grad_out: torch.Tensor, loss_out: torch.Tensor, stream=None):
    abi.sss_loss_l1(pred.data_ptr(), target.data_ptr(), pred.numel(), grad_out.data_ptr(), loss_out.data_ptr(),
                    stream)


def loss_image_scratch(frame: Frame) -> torch.Tensor:
    """Device scratch for sss_loss_image on this frame's plan."""
    nbytes = abi.sss_loss_image_scratch_bytes(frame.plan)
    # float64 elements, two per 16 bytes: at least nbytes, 16-byte aligned
    buf = torch.empty(2 * ((nbytes + 15) // 16), dtype=torch.float64, device=frame.device)
    assert buf.numel() * buf.element_size() >= nbytes and buf.data_ptr() % 16 == 0
    return buf


def loss_image(frame: Frame, pred: torch.Tensor, target: torch.Tensor, eps_dssim: float, loss_out: torch.Tensor,
               scratch: torch.Tensor, stream=None):
    abi.sss_loss_image(frame.plan, pred.data_ptr(), target.data_ptr(), eps_dssim, loss_out.data_ptr(),
                       scratch.data_ptr(), stream)


def loss_image_grad(frame: Frame, pred: torch.Tensor, target: torch.Tensor, eps_dssim: float,
                    scratch: torch.Tensor, grad_out: torch.Tensor, dloss: torch.Tensor | None = None, stream=None):
    abi.sss_loss_image_grad(frame.plan, pred.data_ptr(), target.data_ptr(), eps_dssim,
                            dloss.data_ptr() if dloss is not None else 0, scratch.data_ptr(), grad_out.data_ptr(),
                            stream)


def regularizers(scene: Scene, reg_opacity: float, reg_scale: float, loss_out: torch.Tensor, stream=None):
    abi.sss_regularizers(scene.params(), reg_opacity, reg_scale, loss_out.data_ptr(), stream)


def relocate(scene: Scene, state: SamplerState, dead_opacity=0.005, max_fraction=0.05, n_max=32, seed=0, step=0,
             moved_out: torch.Tensor | None = None, scratch: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Component recycling in place (sss_relocate); returns the device count
    of moved components (int32 tensor of one element)."""
    rp = abi.sss_relocate_params()
    rp.dead_opacity, rp.max_fraction, rp.n_max = float(dead_opacity), float(max_fraction), int(n_max)
    rp.seed, rp.step = int(seed), int(step)
    dev = scene.t["mean"].device
    if scratch is None:
        nbytes = abi.sss_relocate_scratch_bytes(scene.n, max_fraction)
        scratch = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    off = (-scratch.data_ptr()) % 256
    moved = moved_out if moved_out is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    abi.sss_relocate(scene.params(), state.r.data_ptr(), state.m.data_ptr(), state.v.data_ptr(), rp,
                     moved.data_ptr(), scratch.data_ptr() + off, stream)
    return moved
