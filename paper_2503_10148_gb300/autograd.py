"""The rasterizer and the image losses as torch.autograd.Functions.

    leaves = autograd.leaves(scene)                # six tensors, requires_grad
    images = autograd.render(frame, leaves)        # flat [3 * n_pixels]
    loss = autograd.l1_loss(images, target)        # or image_loss(frame, ...)
    grads = torch.autograd.grad(loss, leaves)      # or loss.backward()

``frame`` is a Frame built on the scenes whose parameter tensors are passed
(six per scene, in FIELDS order: mean, log_scale, quat, nu, opacity_raw,
sh).  The forward enqueues project, bin, sort and render_fwd; the backward
enqueues render_bwd and project_bwd (Sec. 3.4 and the closed-form backward
of the supplementary material).  render_bwd recomputes every pixel's
transmittance front to back within its tile from the final transmittance
the forward left in the workspace (T_k = T_{k+1} / (1 - alpha_k)), so no
per-pixel contributor lists are stored.  Every step is a libsss entry point
on the current stream; PyTorch allocates the outputs and runs nothing.

The workspace holds the forward state until the backward has run, so a
frame has one forward in flight: rendering the same frame again before the
backward of the previous render is detected (eagerly) and raises.
"""
from __future__ import annotations

import torch

from . import _abi as abi
from . import frame as F


def leaves(*scenes: F.Scene):
    """The parameter tensors of ``scenes`` (six per scene), marked as
    requiring gradients."""
    out = []
    for sc in scenes:
        for f in F.FIELDS:
            out.append(sc.t[f].requires_grad_(True))
    return out


def _check_binding(frame: F.Frame, tensors):
    if len(tensors) != len(F.FIELDS) * len(frame.scenes):
        raise ValueError(f"expected {len(F.FIELDS) * len(frame.scenes)} parameter tensors, got {len(tensors)}")
    for s, sc in enumerate(frame.scenes):
        for i, f in enumerate(F.FIELDS):
            t = tensors[len(F.FIELDS) * s + i]
            if t.data_ptr() != sc.t[f].data_ptr() or t.numel() != sc.t[f].numel():
                raise ValueError(f"tensor {f} of scene {s} is not the one the frame was planned on")


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame: F.Frame, grow: bool, *tensors):
        _check_binding(frame, tensors)
        st = torch.cuda.current_stream(frame.device)
        out = torch.empty(3 * int(frame.plan.n_pixels), dtype=torch.float32, device=frame.device)
        frame.forward(st, grow=grow, out=out)
        frame.generation += 1
        ctx.frame = frame
        ctx.generation = frame.generation
        return out

    @staticmethod
    def backward(ctx, grad_rgb):
        frame = ctx.frame
        if frame.generation != ctx.generation:
            raise RuntimeError("the frame was rendered again before the backward of an earlier render")
        if grad_rgb.dtype != torch.float32:
            grad_rgb = grad_rgb.float()
        grad_rgb = grad_rgb.contiguous()
        st = torch.cuda.current_stream(frame.device)
        grads = [F.Scene({f: torch.empty_like(sc.t[f], requires_grad=False) for f in F.FIELDS}, sc.n, sc.sh_degree)
                 for sc in frame.scenes]
        frame.backward(grad_rgb, grads, st)
        return (None, None, *[g.t[f] for g in grads for f in F.FIELDS])


class L1LossFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pred, target):
        if pred.dtype != torch.float32 or target.dtype != torch.float32:
            raise TypeError("l1_loss takes float32 tensors")
        if pred.numel() != target.numel() or not pred.is_contiguous() or not target.is_contiguous():
            raise ValueError("l1_loss takes contiguous tensors of equal size")
        st = torch.cuda.current_stream(pred.device)
        loss = torch.empty((), dtype=torch.float32, device=pred.device)
        abi.sss_loss_l1(pred.data_ptr(), target.data_ptr(), pred.numel(), 0, loss.data_ptr(), st)
        ctx.save_for_backward(pred, target)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        pred, target = ctx.saved_tensors
        g = grad_loss.float().contiguous()
        st = torch.cuda.current_stream(pred.device)
        out = torch.empty_like(pred)
        abi.sss_loss_l1_grad(pred.data_ptr(), target.data_ptr(), pred.numel(), g.data_ptr(), out.data_ptr(), st)
        return out, None


class ImageLossFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame: F.Frame, eps_dssim: float, pred, target):
        n = 3 * int(frame.plan.n_pixels)
        if pred.dtype != torch.float32 or target.dtype != torch.float32 or pred.numel() != n or target.numel() != n:
            raise ValueError("image_loss takes float32 images in the frame's layout")
        if not pred.is_contiguous() or not target.is_contiguous():
            raise ValueError("image_loss takes contiguous tensors")
        st = torch.cuda.current_stream(frame.device)
        scratch = F.loss_image_scratch(frame)
        out = torch.empty(3, dtype=torch.float32, device=frame.device)
        F.loss_image(frame, pred, target, eps_dssim, out, scratch, st)
        frame.loss_parts = out  # [L, L1, 1 - SSIM] of the last evaluation
        ctx.frame, ctx.eps, ctx.scratch = frame, eps_dssim, scratch
        ctx.save_for_backward(pred, target)
        return out[0]

    @staticmethod
    def backward(ctx, grad_loss):
        pred, target = ctx.saved_tensors
        g = grad_loss.float().contiguous()
        st = torch.cuda.current_stream(pred.device)
        grad = torch.empty_like(pred)
        F.loss_image_grad(ctx.frame, pred, target, ctx.eps, ctx.scratch, grad, g, st)
        return None, None, grad, None


def image_loss(frame: F.Frame, pred: torch.Tensor, target: torch.Tensor, eps_dssim: float = 0.2):
    """(1 - eps) L1 + eps (1 - SSIM) over the frame's images (Sec. 3.4) as a
    0-d tensor; ``frame.loss_parts`` then holds [L, L1, 1 - SSIM]."""
    return ImageLossFunction.apply(frame, eps_dssim, pred, target)


def render(frame: F.Frame, tensors, grow: bool = True) -> torch.Tensor:
    """Images of every job of ``frame`` as one flat float32 tensor (job j's
    [3][H][W] image at 3 * pix_base[j]; ``frame.image_of(out, j)`` slices
    it).  ``grow=False`` keeps the planned pair capacity (no host
    synchronisation; needed under CUDA-graph capture)."""
    return RenderFunction.apply(frame, grow, *tensors)


def l1_loss(pred: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """mean |pred - target| as a 0-d tensor, with its gradient in libsss."""
    return L1LossFunction.apply(pred, target)
