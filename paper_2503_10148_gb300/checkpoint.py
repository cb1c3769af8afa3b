"""Checkpoint and resume of a sampler run.

One file holds what the next sampler step reads besides the gradients: the
scene's parameters, the SGHMC momentum, the Adam moments (and, when the
Adam gradient drives SGHMC, the moments of dL/dmu), the step index that
keys the sampler's noise, and its seed.  The noise is Philox4x32-10 on
(component, 0, step) under the seed and every update is elementwise, so a
step taken after a resume, from the same gradients, writes bit for bit what
the uninterrupted run wrote.

The file is a NumPy ``.npz`` archive of plain arrays (nothing pickled). It is
written under a temporary name in the target's directory and renamed into
place, so a reader sees the previous checkpoint or the new one, never a
partial file.

``load`` builds a new scene and sampler state; ``load_into`` copies into
existing tensors, keeping their memory, which a captured train step needs
(a CUDA graph holds the addresses of the tensors it was captured on).
"""
from __future__ import annotations

import os
import tempfile

import numpy as np
import torch

from . import frame as F

FORMAT = 1


def _step_value(step) -> int:
    if isinstance(step, torch.Tensor):
        return int(step.item())
    return int(step)


def save(path: str, scene: F.Scene, state: F.SamplerState, step, seed: int = 0,
         mu_adam: tuple | None = None) -> None:
    """Writes the checkpoint.  ``step`` is the index of the next sampler step
    (an int or the one-element device counter of ``frame.step_params``);
    ``mu_adam`` the (m, v) moments of dL/dmu when the run uses them."""
    step_v = _step_value(step)
    if not (0 <= step_v < 1 << 64) or not (0 <= int(seed) < 1 << 64):
        raise ValueError("step and seed must fit in 64 unsigned bits")
    arrays = {f"param_{f}": scene.t[f].detach().cpu().numpy() for f in F.FIELDS}
    arrays["sampler_r"] = state.r.detach().cpu().numpy()
    arrays["sampler_m"] = state.m.detach().cpu().numpy()
    arrays["sampler_v"] = state.v.detach().cpu().numpy()
    if mu_adam is not None:
        arrays["sampler_mu_m"] = mu_adam[0].detach().cpu().numpy()
        arrays["sampler_mu_v"] = mu_adam[1].detach().cpu().numpy()
    arrays["meta_format"] = np.array(FORMAT, dtype=np.int64)
    arrays["meta_n"] = np.array(scene.n, dtype=np.int64)
    arrays["meta_sh_degree"] = np.array(scene.sh_degree, dtype=np.int64)
    arrays["meta_step"] = np.array(step_v, dtype=np.uint64)
    arrays["meta_seed"] = np.array(int(seed), dtype=np.uint64)
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".ckpt-", suffix=".npz", dir=d)
    try:
        with os.fdopen(fd, "wb") as f:
            np.savez(f, **arrays)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        try:
            os.unlink(tmp)
        except OSError:
            pass
        raise


def _read(path: str) -> dict:
    with np.load(path, allow_pickle=False) as z:
        data = {k: z[k] for k in z.files}
    if int(data.get("meta_format", -1)) != FORMAT:
        raise ValueError(f"{path}: not a checkpoint of format {FORMAT}")
    n, deg = int(data["meta_n"]), int(data["meta_sh_degree"])
    K = (deg + 1) ** 2
    want = {f"param_{f}": (F._rows(f, deg), n) for f in F.FIELDS}
    want.update(sampler_r=(3, n), sampler_m=(9 + 3 * K, n), sampler_v=(9 + 3 * K, n))
    if "sampler_mu_m" in data:
        want.update(sampler_mu_m=(3, n), sampler_mu_v=(3, n))
    for k, shape in want.items():
        if k not in data or data[k].shape != shape or data[k].dtype != np.float32:
            raise ValueError(f"{path}: {k} missing or not float32 {shape}")
    return data


def load(path: str, device="cuda") -> dict:
    """Reads a checkpoint: {"scene", "state", "step", "seed", "mu_adam"}
    (``mu_adam`` None when it was saved without)."""
    data = _read(path)
    n, deg = int(data["meta_n"]), int(data["meta_sh_degree"])
    scene = F.Scene({f: torch.as_tensor(data[f"param_{f}"], device=device).contiguous() for f in F.FIELDS}, n, deg)
    state = F.SamplerState(scene)
    state.r.copy_(torch.as_tensor(data["sampler_r"]))
    state.m.copy_(torch.as_tensor(data["sampler_m"]))
    state.v.copy_(torch.as_tensor(data["sampler_v"]))
    mu = None
    if "sampler_mu_m" in data:
        mu = (torch.as_tensor(data["sampler_mu_m"], device=device).contiguous(),
              torch.as_tensor(data["sampler_mu_v"], device=device).contiguous())
    return {"scene": scene, "state": state, "step": int(data["meta_step"]), "seed": int(data["meta_seed"]),
            "mu_adam": mu}


def load_into(path: str, scene: F.Scene, state: F.SamplerState, step_counter: torch.Tensor | None = None,
              mu_adam: tuple | None = None) -> dict:
    """Copies a checkpoint into existing tensors of the same sizes (their
    memory is kept); sets ``step_counter`` when given.  Returns
    {"step", "seed"}."""
    data = _read(path)
    if int(data["meta_n"]) != scene.n or int(data["meta_sh_degree"]) != scene.sh_degree:
        raise ValueError(f"{path}: saved for n={int(data['meta_n'])}, degree {int(data['meta_sh_degree'])}; "
                         f"the scene has n={scene.n}, degree {scene.sh_degree}")
    if (mu_adam is None) != ("sampler_mu_m" not in data):
        raise ValueError(f"{path}: the Adam moments of dL/dmu are "
                         f"{'absent' if mu_adam is not None else 'present'} in the checkpoint")
    with torch.no_grad():
        for f in F.FIELDS:
            scene.t[f].copy_(torch.as_tensor(data[f"param_{f}"]))
        state.r.copy_(torch.as_tensor(data["sampler_r"]))
        state.m.copy_(torch.as_tensor(data["sampler_m"]))
        state.v.copy_(torch.as_tensor(data["sampler_v"]))
        if mu_adam is not None:
            mu_adam[0].copy_(torch.as_tensor(data["sampler_mu_m"]))
            mu_adam[1].copy_(torch.as_tensor(data["sampler_mu_v"]))
        if step_counter is not None:
            # the device counter is int64; the step index's bits are kept
            step_counter.fill_(int(np.array(data["meta_step"], dtype=np.uint64).view(np.int64)))
    return {"step": int(data["meta_step"]), "seed": int(data["meta_seed"])}
