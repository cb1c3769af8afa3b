"""Helpers shared by the GPU parity tests (imported by test modules only)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2503_10148_gb300 import frame, inputs

DEV = "cuda:0"


def require_gpu():
    assert torch.cuda.is_available(), "GPU tests need CUDA (there is no CPU fallback)"
    from paper_2503_10148_gb300 import build
    build.build()


def f32_scene(scene: dict) -> dict:
    """Parameters rounded to float32 then widened: what both sides consume."""
    out = dict(scene)
    for k in frame.FIELDS:
        out[k] = np.asarray(scene[k], np.float32)
    return out


def gpu_forward(scene_np, cams, cfg=None, pair_capacity=None):
    cams = [frame.f32_camera(c) for c in cams]
    cfg = cfg or frame.make_cfg()
    sc = frame.Scene.from_numpy(scene_np, DEV)
    fr = frame.Frame([sc], cams, cfg=cfg, pair_capacity=pair_capacity, device=DEV)
    fr.forward()
    torch.cuda.synchronize()
    return fr, sc, cams


def oracle_views(scene_np, cams, cfgd, pix=None):
    """Oracle projection + render for every camera (pix: list of pixel index
    arrays or None)."""
    out = []
    for v, cam in enumerate(cams):
        proj = oracle.project(scene_np, cam, cfgd)
        out.append((proj, oracle.render(proj, cam, cfgd, None if pix is None else pix[v])))
    return out


def masked_weights(cams, refs, seed, pix=None):
    """Seeded dL/dC weights with the pixels the oracle flags as fragile (a
    discrete decision within rounding distance) set to zero, so neither side's
    gradient depends on them.  With pix given, only those pixels are nonzero."""
    ws = inputs.linear_loss_weights(cams, seed)
    out = []
    for v, (w, (_, ref)) in enumerate(zip(ws, refs)):
        w = w.reshape(3, -1).copy()
        if pix is None:
            w[:, ref["flags"] != 0] = 0.0
        else:
            keep = np.zeros(w.shape[1], bool)
            keep[pix[v][ref["flags"] == 0]] = True
            w[:, ~keep] = 0.0
        out.append(w)
    return out


def scene_grads_flat(g: frame.Scene) -> np.ndarray:
    return np.concatenate([g.t[f].detach().cpu().numpy().reshape(-1).astype(np.float64) for f in frame.FIELDS])


GRAD_REL = 1e-3   # relative bar per element ...
U32 = 2.0 ** -24  # FP32 unit roundoff
# ... unless the difference is within the FP32 rounding bound of the sums:
# u * (16 * sum |term| n + 256 * sum |term|), n the contributor count of each
# term's pixel (the transmittance is recovered by one division per contributor,
# so its rounding grows with n) and 256 u for the per-term evaluation (MUFU
# lg2/ex2 approximations times the exponent (nu+2)/2, mean2D rounding).
GRAD_NORM = 1e-4  # and ||g - g_ref|| / ||g_ref|| per group


def grad_den(ref, mag, extra=0.0):
    """Per-element scale of the bar: max(|g_ref|, FP32 bound / GRAD_REL)."""
    bound = U32 * (16.0 * mag.absn + 256.0 * mag.abs) + extra
    scale = max(float(np.abs(ref).max()), 1e-30)
    return np.maximum(np.maximum(np.abs(ref), bound / GRAD_REL), 1e-9 * scale)


def sh_basis_bound(n, sh_degree, mag2d):
    """Extra FP32 bound of the SH-coefficient gradients dL/dsh_kc =
    sum_views dL/drgb_c Y_k(dir): a degree <= 3 basis value at an FP32 unit
    direction (coefficients <= 3) carries up to ~64 u of absolute rounding,
    which matters where Y_k(dir) itself is near zero.  Returns a theta-sized
    array (zero outside the SH rows)."""
    K = (sh_degree + 1) ** 2
    sl = oracle.theta_slices(n, sh_degree)
    extra = np.zeros(sl["sh"].stop)
    rgb_mag = sum(mag2d.abs[j][:, 7:10] for j in range(mag2d.abs.shape[0]))  # [n][3]
    for k in range(K):
        for c in range(3):
            r = 3 * k + c
            extra[sl["sh"].start + r * n:sl["sh"].start + (r + 1) * n] = 64.0 * U32 * rgb_mag[:, c]
    return extra


def assert_groups_close(got, ref, n, sh_degree, mag, rel=GRAD_REL, norm=GRAD_NORM, label="", extra=None):
    """Per parameter group: every element within ``rel`` of grad_den (1e-3
    relative, or the FP32 rounding bound of its sums) and the group's relative
    L2 error within ``norm``."""
    sl = oracle.theta_slices(n, sh_degree)
    report = {}
    for name, s in sl.items():
        a, b = got[s], ref[s]
        scale = np.abs(b).max()
        if scale == 0:
            assert np.abs(a).max() == 0, (label, name)
            continue
        den = grad_den(b, mag[s], 0.0 if extra is None else extra[s])
        relerr = np.abs(a - b) / den
        l2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        report[name] = (float(relerr.max()), l2)
        bad = relerr > rel
        assert not bad.any(), (label, name, report[name], int(bad.sum()), a[bad][:5], b[bad][:5])
        assert l2 <= norm, (label, name, report[name])
    return report


# ---------------------------------------------------------------- sampler step bar
# An updated value (parameter, momentum, Adam moment) must be within 1e-6 of
# the oracle's value relative to that value, or -- where the increment's own
# terms are larger than the value or cancel -- within the FP32 rounding of
# those terms: |got - ref| <= 1e-6 |ref| + 16 u D, D the sum of the
# magnitudes of the increment's terms (for Adam, taken on the terms of m').
# 16 bounds the FP32 roundings along one element's update (tanh, exp and the
# division of the gate; log, sqrt and sincospi of Box-Muller; expm1 of the bias
# corrections; the products and sums of the update), each at most an ulp of
# its operands.  Both sides get the same FP32 hyper-parameters.
STEP_REL = 1e-6
STEP_ROUNDINGS = 16.0


def f32(x):
    """The FP32 value the kernel sees for a hyper-parameter (scalar or tuple)."""
    if isinstance(x, (tuple, list)):
        return tuple(float(np.float32(v)) for v in x)
    return float(np.float32(x))


def adam_increment_mag(m0, g_mag, v_new, lr, beta1, beta2, adam_eps, t):
    """lr m^/(sqrt(v^) + eps) with m^ taken on the magnitudes of its terms."""
    bc1 = 1.0 - beta1 ** t
    bc2 = 1.0 - beta2 ** t
    return lr * (beta1 * np.abs(m0) + (1.0 - beta1) * g_mag) / bc1 / (np.sqrt(np.abs(v_new) / bc2) + adam_eps)


def _rotations(quat):
    """[n][3][3] rotation matrices of (w, x, y, z) quaternions [4][n]."""
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=0, keepdims=True)
    w, x, y, z = q
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def noise_mag(theta0, xi, n, sh_degree, burn_in):
    """Per mean element, the magnitude of the noise term's factors: |xi| or,
    in burn-in, sum_k |R_ak| s_k^2 sum_b |R_bk| |xi_b| (Sigma xi evaluated as
    R (s^2 (R^T xi)))."""
    xi = np.asarray(xi, np.float64).reshape(3, n)
    if not burn_in:
        return np.abs(xi)
    sl = oracle.theta_slices(n, sh_degree)
    R = np.abs(_rotations(theta0[sl["quat"]].reshape(4, n)))  # [n][a][k]
    s2 = np.exp(2.0 * theta0[sl["log_scale"]].reshape(3, n)).T  # [n][k]
    inner = np.einsum("nbk,bn->nk", R, np.abs(xi)) * s2
    return np.einsum("nak,nk->an", R, inner)


def step_mags(theta0, G_mag, r0, xi, n, sh_degree, p, burn_in):
    """(mean increment magnitude, momentum increment magnitude), [3][n] each,
    of mu' = mu - eps^2 G + g eps (1 - eps C) r + g eps sqrt(2 eps C) (xi or
    Sigma xi) and r' = (1 - eps C) r - eps G + sqrt(2 eps C) xi."""
    sl = oracle.theta_slices(n, sh_degree)
    o = np.tanh(theta0[sl["opacity_raw"]])
    gate = 1.0 / (1.0 + np.exp(np.minimum(p["k"] * (np.abs(o) - p["t0"]), 700.0)))
    eps, C = p["eps"], p["C"]
    sq = np.sqrt(2.0 * eps * C)
    fr = abs(1.0 - eps * C)
    r0 = np.abs(np.asarray(r0, np.float64).reshape(3, n))
    G = np.asarray(G_mag, np.float64).reshape(3, n)
    nm = noise_mag(theta0, xi, n, sh_degree, burn_in)
    mu = eps * eps * G + gate * eps * sq * nm + (0.0 if burn_in else 1.0) * gate * eps * fr * r0
    r = fr * r0 + eps * G + sq * np.abs(np.asarray(xi, np.float64).reshape(3, n))
    return mu, r


def assert_step_close(got, ref, mag, label="", rel=STEP_REL):
    """|got - ref| <= rel |ref| + 16 u mag elementwise; returns the largest
    ratio of error to bound and the fraction of elements whose bound is set by
    the rounding term rather than rel |ref|."""
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    floor = STEP_ROUNDINGS * U32 * np.asarray(mag, np.float64).reshape(-1)
    bound = rel * np.abs(ref) + floor
    ratio = np.abs(got - ref) / np.maximum(bound, 1e-300)
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 1.0, (label, float(ratio[worst]), got[worst], ref[worst], float(bound[worst]))
    return {"max_ratio": round(float(ratio.max()), 4), "floor_frac": round(float(np.mean(floor > rel * np.abs(ref))), 4)}
