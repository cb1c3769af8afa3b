"""One training step of the method, plain or captured into a CUDA graph.

A step on one scene with V views is: project, bin, sort and forward-render
all V views as one frame; L1 loss against the V target images (value and
dL/dC); backward render and projection backward (gradients summed over the
views); SGHMC on the means and Adam on the rest.  Every step is a libsss
entry point; nothing is computed in Python.

Two forms of the same launches: ``form="autograd"`` (default) goes through
the torch.autograd.Functions of ``autograd.py`` (render, l1_loss,
torch.autograd.grad), ``form="direct"`` calls the entry points one after
the other with buffers the step owns.

``TrainStep.capture()`` records the whole step (about 40 kernels) into one
CUDA graph.  The number of (tile, splat) pairs is data dependent, so the
frame is planned with a pair capacity measured on an eager step plus
headroom; the device status word (checked with ``check()``) reports an
overflow instead of a host sync inside the step.

``PlainStep`` is the reference form the batched one is compared with: one
frame per view, launched eagerly one after the other.
"""
from __future__ import annotations

import torch

from . import autograd as AG
from . import frame as F


class TrainStep:
    def __init__(self, scene: F.Scene, cams, targets: torch.Tensor, cfg=None, sampler: dict | None = None,
                 headroom: float = 1.5, device="cuda", form: str = "autograd", loss: str = "l1",
                 eps_dssim: float = 0.2, reg_opacity: float = 0.01, reg_scale: float = 0.01,
                 restart: bool = False):
        """``loss="l1"``: the L1 term alone; ``loss="full"``: the loss of
        Sec. 3.4, (1 - eps_dssim) L1 + eps_dssim D-SSIM plus the opacity and
        scale regularisers (their gradients added by the sampler step).
        ``restart=True`` starts every step from the parameters the step was
        built with: the sampler writes its update into a second parameter set
        (``self.after``, through sss_sghmc_step_to) and leaves the scene as
        it was, so repeated steps run the same workload instead of a scene
        that drifts under the sampler (for timing), with no copy back."""
        if form not in ("autograd", "direct") or loss not in ("l1", "full"):
            raise ValueError((form, loss))
        self.form = form
        self.loss_kind, self.eps_dssim = loss, float(eps_dssim)
        self.scene = scene
        self.cams = list(cams)
        self.device = torch.device(device)
        self.cfg = cfg if cfg is not None else F.make_cfg()
        self.frame = F.Frame([scene], self.cams, cfg=self.cfg, device=self.device)
        assert targets.numel() == self.frame.rgb.numel() and targets.dtype == torch.float32
        self.targets = targets
        self.grads = scene.zeros_like()
        self.state = F.SamplerState(scene)
        self.dl = torch.zeros_like(self.frame.rgb)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step_counter = torch.zeros(1, dtype=torch.int64, device=self.device)
        regs = dict(reg_opacity=reg_opacity, reg_scale=reg_scale) if loss == "full" else {}
        self.sp = F.step_params(step_counter=self.step_counter, **{**regs, **(sampler or {})})
        if loss == "full":
            self.scratch = F.loss_image_scratch(self.frame)
            self.loss3 = torch.zeros(3, dtype=torch.float32, device=self.device)  # [L, L1, 1 - SSIM]
            self.loss = self.loss3[0:1]
        self.headroom = headroom
        self.graph = None
        self.after = scene.zeros_like() if restart else None  # the sampler's output with restart
        if form == "autograd":
            self.leaves = AG.leaves(scene)
            self.one = torch.ones((), dtype=torch.float32, device=self.device)

    def calibrate(self):
        """Eager forward with capacity growth, then re-plan with headroom."""
        self.frame.forward(grow=True)
        _, need, _ = self.frame.status()
        cap = max(int(need * self.headroom) + 4096, 1 << 16)
        if cap != self.frame.pair_capacity:
            self.frame.pair_capacity = cap
            self.frame._replan()
        return need

    def run(self):
        """Enqueue one step on the current stream (no host synchronisation)."""
        st = torch.cuda.current_stream(self.device)
        fr = self.frame
        if self.form == "autograd":
            rgb = AG.render(fr, self.leaves, grow=False)
            if self.loss_kind == "full":
                loss = AG.image_loss(fr, rgb, self.targets, self.eps_dssim)
            else:
                loss = AG.l1_loss(rgb, self.targets)
            grads = torch.autograd.grad(loss, self.leaves, grad_outputs=self.one)
            self.rgb_out, self.loss = rgb, loss
            self.grads = F.Scene(dict(zip(F.FIELDS, grads)), self.scene.n, self.scene.sh_degree)
            self.sample(st)
            return
        fr.project(st)
        fr.bin(st)
        fr.sort(st)
        fr.render_fwd(st)
        if self.loss_kind == "full":
            F.loss_image(fr, fr.rgb, self.targets, self.eps_dssim, self.loss3, self.scratch, st)
            F.loss_image_grad(fr, fr.rgb, self.targets, self.eps_dssim, self.scratch, self.dl, stream=st)
        else:
            F.loss_l1(fr.rgb, self.targets, self.dl, self.loss, st)
        fr.render_bwd(self.dl, st)
        fr.project_bwd([self.grads], st)
        self.sample(st)

    def sample(self, stream=None):
        """The sampler step on this step's gradients: in place, or with
        ``restart`` into ``self.after``."""
        F.sghmc_step(self.scene, self.grads, self.state, self.sp, stream=stream, out=self.after)

    def time_kernels(self, names=("render_fwd", "render_bwd")) -> bool:
        """Record CUDA events around these launches in every later step,
        captured ones included (external events become record nodes of the
        graph).  Returns False when this PyTorch has no external events."""
        try:
            self.frame.timing = {n: (torch.cuda.Event(enable_timing=True, external=True),
                                     torch.cuda.Event(enable_timing=True, external=True)) for n in names}
        except TypeError:
            self.frame.timing = None
            return False
        return True

    def kernel_ms(self, name: str) -> float:
        """Duration of the named launch in the last completed step."""
        e0, e1 = self.frame.timing[name]
        return e0.elapsed_time(e1)

    def capture(self, pool=None, warmup: int = 2):
        """Warm-up steps on a side stream (the autograd engine must not have
        run this backward on the legacy stream before a capture: it would
        touch that stream during the capture), then one captured step.
        ``pool``: the memory pool of an earlier capture of this step (copies
        of the step, replayed one after another, share its temporaries)."""
        cur = torch.cuda.current_stream(self.device)
        side = torch.cuda.Stream(self.device)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.run()
        cur.wait_stream(side)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g, pool=pool):
                self.run()
        except BaseException:
            torch.cuda.set_stream(cur)  # a failed capture_end leaves the capture stream current
            raise
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def check(self):
        """(status bits, pairs needed, pairs sorted); raises on overflow."""
        st, need, done = self.frame.status()
        if st:
            raise RuntimeError(f"pair capacity {self.frame.pair_capacity} exceeded: {need} pairs needed")
        return st, need, done


class PlainStep:
    """Same step with one frame per view, launched eagerly view after view."""

    def __init__(self, scene: F.Scene, cams, targets: torch.Tensor, cfg=None, sampler: dict | None = None,
                 device="cuda", loss: str = "l1", eps_dssim: float = 0.2, reg_opacity: float = 0.01,
                 reg_scale: float = 0.01, restart: bool = False):
        """Same options as TrainStep; each view's loss is a mean over that
        view's pixels (the per-view gradients are summed by a PyTorch
        reduction before the sampler step)."""
        self.scene = scene
        self.device = torch.device(device)
        self.cfg = cfg if cfg is not None else F.make_cfg()
        self.loss_kind, self.eps_dssim = loss, float(eps_dssim)
        self.frames = [F.Frame([scene], [c], cfg=self.cfg, device=self.device) for c in cams]
        self.targets = []
        off = 0
        for fr in self.frames:
            n = fr.rgb.numel()
            self.targets.append(targets[off:off + n])
            off += n
        self.grads = [scene.zeros_like() for _ in self.frames]
        self.total = scene.zeros_like()
        self.state = F.SamplerState(scene)
        self.dl = [torch.zeros_like(fr.rgb) for fr in self.frames]
        self.loss = torch.zeros(3 * len(self.frames), dtype=torch.float32, device=self.device)  # per view
        self.step_counter = torch.zeros(1, dtype=torch.int64, device=self.device)
        regs = dict(reg_opacity=reg_opacity, reg_scale=reg_scale) if loss == "full" else {}
        self.sp = F.step_params(step_counter=self.step_counter, **{**regs, **(sampler or {})})
        self.scratch = [F.loss_image_scratch(fr) for fr in self.frames] if loss == "full" else None
        self.after = scene.zeros_like() if restart else None  # the sampler's output with restart

    def run(self):
        for v, (fr, tgt, dl, g) in enumerate(zip(self.frames, self.targets, self.dl, self.grads)):
            fr.forward(grow=True)
            if self.loss_kind == "full":
                F.loss_image(fr, fr.rgb, tgt, self.eps_dssim, self.loss[3 * v:3 * v + 3], self.scratch[v])
                F.loss_image_grad(fr, fr.rgb, tgt, self.eps_dssim, self.scratch[v], dl)
            else:
                F.loss_l1(fr.rgb, tgt, dl, self.loss[v:v + 1])
            fr.backward(dl, [g])
        for f in F.FIELDS:
            self.total.t[f].copy_(torch.stack([g.t[f] for g in self.grads]).sum(0))
        F.sghmc_step(self.scene, self.total, self.state, self.sp, out=self.after)
