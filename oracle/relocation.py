"""FP64 oracle of component recycling (Sec. 3.4 "Adding and Recycling
Components", Eq. relocation; SM "Component Recycling"; Implementation
Details).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

Readings (the paper leaves these open):
- dead: |o| = |tanh(opacity_raw)| < dead_opacity (0.005, the opacity below
  which the sampler's gate opens); at most floor(max_fraction * n) dead
  components move per call (5 %), the first ones in index order.
- targets: a multinomial over the live components with probability
  proportional to |o|.  Weights are quantised, w = floor(|o| 2^12), and the
  draw is exact integer arithmetic: v = (x * W) >> 32 with x the first word
  of Philox4x32-10 on counter (dead rank, 1, step_lo, step_hi), key (seed_lo,
  seed_hi), W the weight total; the target is the first index whose
  inclusive weight prefix exceeds v.
- a target receives at most n_max - 1 copies (the first ones in dead-rank
  order); N = 1 + copies.
- o_new = 1 - (1 - |o_old|)^(1/N) with the sign of o_old; nu_new = nu_old;
  Sigma_new = F Sigma_old with
      F = o_old^2 (nu_old / nu_new) (B(1/2, (nu_old + 2)/2) / K)^2,
      K = sum_{i=1..N} sum_{k=0..i-1} C(i-1, k) (-1)^k o_new^(k+1)
          B(1/2, ((k+1)(nu_new + 3) - 1)/2),
  all with |o|, so log_scale grows by ln(F)/2; the Beta function through
  ln Gamma, as the paper computes it.
- copies take the target's mean, quaternion, nu, SH and the new opacity and
  scale; their momentum and Adam moments restart from zero.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox4x32_10

WEIGHT_BITS = 12
STREAM_WORD = 1  # counter word 1 of the draws (the sampler's noise uses 0)


def beta(x: float, y: float) -> float:
    return math.exp(math.lgamma(x) + math.lgamma(y) - math.lgamma(x + y))


def relocated_opacity(o_old: float, N: int) -> float:
    """(1 - o_new)^N = 1 - o_old, on |o|, sign kept."""
    a = 1.0 - (1.0 - abs(o_old)) ** (1.0 / N)
    return math.copysign(a, o_old)


def k_sum(o_new: float, nu_new: float, N: int) -> float:
    """The double sum K of Eq. relocation, term by term."""
    o = abs(o_new)
    total = 0.0
    for i in range(1, N + 1):
        for k in range(i):
            total += math.comb(i - 1, k) * (-1) ** k * o ** (k + 1) * beta(0.5, ((k + 1) * (nu_new + 3.0) - 1.0) / 2.0)
    return total


def scale_factor(o_old: float, nu_old: float, N: int, nu_new: float | None = None) -> float:
    """F with Sigma_new = F Sigma_old (Eq. relocation)."""
    nu_new = nu_old if nu_new is None else nu_new
    o_new = relocated_opacity(o_old, N)
    K = k_sum(o_new, nu_new, N)
    return o_old * o_old * (nu_old / nu_new) * (beta(0.5, (nu_old + 2.0) / 2.0) / K) ** 2


def weights(opacity_raw, dead_opacity: float) -> tuple[np.ndarray, np.ndarray]:
    """(dead flags, quantised weights of the live components)."""
    o = np.abs(np.tanh(np.asarray(opacity_raw, np.float64)))
    dead = o < dead_opacity
    w = np.where(dead, 0, np.floor(o * (1 << WEIGHT_BITS))).astype(np.int64)
    return dead, w


def draw_targets(w: np.ndarray, n_draws: int, seed: int, step: int) -> np.ndarray:
    """Target index of draws 0..n_draws-1 (all -1 when the live weight is 0)."""
    prefix = np.cumsum(w)
    W = int(prefix[-1]) if len(prefix) else 0
    out = np.full(n_draws, -1, np.int64)
    if W == 0:
        return out
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    for r in range(n_draws):
        x = int(philox4x32_10((r, STREAM_WORD, step & 0xFFFFFFFF, (step >> 32) & 0xFFFFFFFF), key)[0])
        v = (x * W) >> 32
        out[r] = int(np.searchsorted(prefix, v, side="right"))
    return out


def relocate(scene: dict, momentum, adam_m, adam_v, *, dead_opacity=0.005, max_fraction=0.05, n_max=32, seed=0,
             step=0):
    """One recycling call on a planar scene dict (FP64 copies).  Returns
    (scene, momentum, m, v, moved, targets): moved[r] is the component index
    of the r-th recycled component, targets[r] its target."""
    sc = {k: (np.array(v, np.float64, copy=True) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    r_ = np.array(momentum, np.float64, copy=True)
    m_ = np.array(adam_m, np.float64, copy=True)
    v_ = np.array(adam_v, np.float64, copy=True)
    n = sc["n"]
    dead, w = weights(sc["opacity_raw"], dead_opacity)
    dead_idx = np.flatnonzero(dead)[: int(math.floor(max_fraction * n))]
    targets = draw_targets(w, len(dead_idx), seed, step)
    if len(dead_idx) == 0 or targets[0] < 0:
        return sc, r_, m_, v_, np.zeros(0, np.int64), np.zeros(0, np.int64)
    # copies per target in dead-rank order, capped
    taken = {}
    moved, moved_t = [], []
    for d, t in zip(dead_idx, targets):
        c = taken.get(int(t), 0)
        if c < n_max - 1:
            taken[int(t)] = c + 1
            moved.append(int(d))
            moved_t.append(int(t))
    old_o = np.tanh(sc["opacity_raw"])
    new_raw, new_ls = {}, {}
    for t, c in taken.items():
        N = c + 1
        o_new = relocated_opacity(old_o[t], N)
        F = scale_factor(old_o[t], float(sc["nu"][t]), N)
        new_raw[t] = math.atanh(o_new)
        new_ls[t] = sc["log_scale"][:, t] + 0.5 * math.log(F)
    for d, t in zip(moved, moved_t):
        for f in ("mean", "quat", "sh"):
            sc[f][:, d] = sc[f][:, t]
        sc["nu"][d] = sc["nu"][t]
        sc["opacity_raw"][d] = new_raw[t]
        sc["log_scale"][:, d] = new_ls[t]
        r_[:, d] = 0.0
        m_[:, d] = 0.0
        v_[:, d] = 0.0
    for t in taken:
        sc["opacity_raw"][t] = new_raw[t]
        sc["log_scale"][:, t] = new_ls[t]
    return sc, r_, m_, v_, np.array(moved, np.int64), np.array(moved_t, np.int64)
