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


# ---------------------------------------------------------------- forward bar
# Every pixel is compared.  Where the oracle met no ambiguous decision (an
# |alpha| or a T' within the FP32 rounding window of tau or t_min), the GPU
# pixel must equal the oracle's within FWD_TOL per channel and in T.  Where it
# met k of them, both outcomes of each are correct results: the GPU pixel
# must equal, within FWD_TOL, one of the oracle's renders with those decisions
# taken either way (all 2^(k+1) combinations of the first k + 1 decisions met,
# the extra bit for a decision met only on another path).
FWD_TOL = 1e-4
FLIP_BITS = 10


class ForwardCheck:
    """Result of check_forward_view: flip[k] is the oracle's choice of
    ambiguous decisions that the GPU's pixel k matched best (0 where none was
    met); unresolved[k] is True where two different admissible results both
    match the GPU's pixel within tol, so its image does not determine which
    decisions it took (a gradient through it cannot be attributed);
    [nc_lo, nc_hi] bounds the contributor count over the admissible results
    within tol; alts[k] (unresolved pixels only) lists one decision mask per
    distinct admissible result the GPU's pixel matched; stats summarises the
    view."""

    def __init__(self, flip, unresolved, nc_lo, nc_hi, stats, alts=None):
        self.flip, self.unresolved, self.nc_lo, self.nc_hi, self.stats = flip, unresolved, nc_lo, nc_hi, stats
        self.alts = alts or {}


def check_forward_view(proj, cam, cfgd, ref, img, T, pix=None, tol=FWD_TOL, last=None) -> ForwardCheck:
    """Compares one view's GPU image [3][npix] and transmittance [npix] (the
    pixels `pix`, or all) with the oracle render `ref` of the same pixels.
    With `last` (the GPU's last contributor per pixel, component index or
    -1), it must equal the oracle's too, and an admissible result matches
    only with the same last contributor."""
    img = np.asarray(img, np.float64)
    T = np.asarray(T, np.float64)
    npix = T.size
    fl = ref["flags"] != 0
    ok = ~fl
    worst = 0.0
    if ok.any():
        worst = max(float(np.abs(img[:, ok] - ref["rgb"][:, ok]).max()), float(np.abs(T[ok] - ref["T"][ok]).max()))
    assert worst <= tol, ("unflagged pixel", worst)
    if last is not None:
        last = np.asarray(last, np.int64)
        assert np.array_equal(last[ok], ref["last"][ok]), int(np.sum(last[ok] != ref["last"][ok]))
    flip = np.zeros(npix, np.uint32)
    unresolved = np.zeros(npix, bool)
    nc_lo = np.asarray(ref["n_contrib"], np.int64).copy()
    nc_hi = nc_lo.copy()
    idx = np.flatnonzero(fl)
    worst_fl, primary = 0.0, 0
    alts = {}
    if idx.size:
        k = ref["n_amb"][idx]
        assert int(k.max()) < FLIP_BITS, ("ambiguous decisions per pixel", int(k.max()))
        reps = 1 << (k + 1)
        lin = (np.arange(npix) if pix is None else np.asarray(pix, np.int64))[idx]
        rep_pos = np.repeat(np.arange(idx.size), reps)
        masks = np.concatenate([np.arange(r) for r in reps]).astype(np.uint32)
        alt = oracle.render(proj, cam, cfgd, lin[rep_pos], flip=masks)
        err = np.maximum(np.abs(alt["rgb"] - img[:, idx[rep_pos]]).max(axis=0), np.abs(alt["T"] - T[idx[rep_pos]]))
        if last is not None:  # a different last contributor is a different result
            err = np.where(alt["last"] == last[idx[rep_pos]], err, np.inf)
        starts = np.concatenate([[0], np.cumsum(reps)[:-1]])
        best = np.minimum.reduceat(err, starts)
        bad = best > tol
        assert not bad.any(), ("flagged pixel matches no admissible result", int(bad.sum()), float(best.max()))
        for i, (s0, r) in enumerate(zip(starts, reps)):
            pick = s0 + int(np.argmin(err[s0:s0 + r]))  # the first combination reaching the best error
            flip[idx[i]] = masks[pick]
            good = np.flatnonzero(err[s0:s0 + r] <= tol) + s0
            res = np.concatenate([alt["rgb"][:, good], alt["T"][None, good], alt["n_contrib"][None, good]])
            _, first = np.unique(res, axis=1, return_index=True)
            unresolved[idx[i]] = first.size > 1
            if first.size > 1:
                alts[int(idx[i])] = [int(masks[good[f]]) for f in sorted(first)]
            nc_lo[idx[i]] = alt["n_contrib"][good].min()
            nc_hi[idx[i]] = alt["n_contrib"][good].max()
        worst_fl = float(best.max())
        primary = int((flip[idx] == 0).sum())
    stats = {"pixels": int(npix), "flagged": int(idx.size), "flagged_frac": round(idx.size / max(npix, 1), 5),
             "near_tau": int(np.sum((ref["flags"] & oracle.F_NEAR_TAU) != 0)),
             "near_tmin": int(np.sum((ref["flags"] & oracle.F_NEAR_TMIN) != 0)),
             "flagged_as_primary": primary, "unresolved": int(unresolved.sum()), "max_err_unflagged": worst,
             "max_err_flagged": worst_fl}
    return ForwardCheck(flip, unresolved, nc_lo, nc_hi, stats, alts)


def merge_stats(stats):
    out = {"pixels": 0, "flagged": 0, "near_tau": 0, "near_tmin": 0, "flagged_as_primary": 0, "unresolved": 0,
           "max_err_unflagged": 0.0, "max_err_flagged": 0.0}
    for st in stats:
        for k in ("pixels", "flagged", "near_tau", "near_tmin", "flagged_as_primary", "unresolved"):
            out[k] += st[k]
        for k in ("max_err_unflagged", "max_err_flagged"):
            out[k] = max(out[k], st[k])
    out["flagged_frac"] = round(out["flagged"] / max(out["pixels"], 1), 5)
    return out


def gpu_view(fr, j, cam, pix=None):
    """GPU image [3][npix] and final T [npix] of job j (float64)."""
    img = fr.image(j).reshape(3, -1).cpu().numpy().astype(np.float64)
    pb = fr.plan.jobs[j].pix_base
    T = fr.final_T()[pb:pb + cam.width * cam.height].cpu().numpy().astype(np.float64)
    if pix is not None:
        img, T = img[:, pix], T[pix]
    return img, T


def gpu_last_component(fr, j, cam, pix=None):
    """Component index of each pixel's last contributor in job j (-1 when
    none), from the GPU's list positions, tile ranges and sorted pairs."""
    J = fr.plan.jobs[j]
    hw = cam.width * cam.height
    last = fr.last_contrib()[J.pix_base:J.pix_base + hw].cpu().numpy().astype(np.int64)
    rng = fr.ranges().cpu().numpy().astype(np.int64)
    _, vals = fr.sorted_pairs(fr.status()[1])
    vals = vals.cpu().numpy().astype(np.int64)
    ys, xs = np.divmod(np.arange(hw), cam.width)
    tile = J.tile_base + (ys // fr.cfg.tile_h) * J.tiles_x + xs // fr.cfg.tile_w
    comp = np.where(last > 0, vals[np.maximum(rng[tile, 0] + last - 1, 0)] - J.entry_base, -1)
    return comp if pix is None else comp[pix]


def check_forward_frame(fr, cams, cfgd, refs, pix=None, tol=FWD_TOL, alts_out=None):
    """check_forward_view for every job of a frame; returns (flips per view,
    merged stats, unresolved masks per view).  With alts_out (a list), every
    unresolved pixel is appended as (view, linear pixel, admissible masks)."""
    flips, stats, unres = [], [], []
    for j, (cam, (proj, ref)) in enumerate(zip(cams, refs)):
        pj = None if pix is None else pix[j]
        img, T = gpu_view(fr, j, cam, pj)
        c = check_forward_view(proj, cam, cfgd, ref, img, T, pj, tol, last=gpu_last_component(fr, j, cam, pj))
        flips.append(c.flip)
        stats.append(c.stats)
        unres.append(c.unresolved)
        if alts_out is not None:
            lin = np.arange(cam.width * cam.height) if pj is None else np.asarray(pj, np.int64)
            alts_out.extend((j, int(lin[k]), m) for k, m in sorted(c.alts.items()))
    return flips, merge_stats(stats), unres


def resolved_weights(fr, cams, cfgd, refs, seed, pix=None, alts_out=None):
    """Seeded dL/dC weights and, per view, the oracle's choice of ambiguous
    decisions that the GPU's forward matched, so that the oracle
    differentiates the same admissible forward.  Only the pixels whose image
    matches two different admissible results (its decisions are then not
    determined; counted in stats["unresolved"]) carry no weight.  With pix
    given, only those pixels carry weight.  alts_out as in
    check_forward_frame."""
    flips, stats, unres = check_forward_frame(fr, cams, cfgd, refs, pix, alts_out=alts_out)
    ws = inputs.linear_loss_weights(cams, seed)
    out = []
    for v, w in enumerate(ws):
        w = w.reshape(3, -1).copy()
        if pix is None:
            w[:, unres[v]] = 0.0
        else:
            keep = np.zeros(w.shape[1], bool)
            keep[np.asarray(pix[v])[~unres[v]]] = True
            w[:, ~keep] = 0.0
        out.append(w)
    return out, flips, stats


def scene_grads_flat(g: frame.Scene) -> np.ndarray:
    return np.concatenate([g.t[f].detach().cpu().numpy().reshape(-1).astype(np.float64) for f in frame.FIELDS])


def check_unresolved_gradients(fr, sc, s32, cams, cfgd, unresolved, seed, sh_degree, max_pixels=48):
    """Pixels whose image matches two different admissible results carry no
    weight in the frame-wide gradient tests; here each is differentiated on
    its own.  unresolved: list of (view j, linear pixel p, masks), the masks
    the admissible results the GPU's pixel matched (ForwardCheck.alts).  For
    each (at most max_pixels, in order) the GPU runs its full backward with a
    seeded dL/dC on that pixel alone, and its gradient must pass the gradient
    bar against the oracle's differentiated through one of the admissible
    results.  Returns (pixels checked, how many matched their first mask)."""
    rng = np.random.default_rng(seed)
    n = s32["n"]
    checked = first = 0
    for j, p, masks in unresolved[:max_pixels]:
        w = rng.uniform(-1, 1, size=3).astype(np.float32).astype(np.float64)
        dl = [np.zeros((3, c.width * c.height), np.float32) for c in cams]
        dl[j][:, p] = w
        g = sc.zeros_like()
        fr.backward(torch.as_tensor(np.concatenate([d.reshape(-1) for d in dl]), device=DEV), [g])
        torch.cuda.synchronize()
        got = scene_grads_flat(g)
        errors = []
        for k, m in enumerate(masks):
            gref, _, gabs, g2abs = oracle.backward(s32, [cams[j]], cfgd, [w[:, None]], [np.array([p], np.int64)],
                                                   want_grad2d=True, want_abs=True, flip=[np.array([m], np.uint32)])
            try:
                assert_groups_close(got, gref, n, sh_degree, gabs, label=f"unresolved pixel {j}:{p}",
                                    extra=sh_basis_bound(n, sh_degree, g2abs))
            except AssertionError as e:
                errors.append(e)
                continue
            first += k == 0
            break
        else:
            raise AssertionError(("unresolved pixel matches none of its admissible gradients", j, p, errors[:2]))
        checked += 1
    return checked, first



GRAD_REL = 1e-3   # the gradient bar: |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max_group |g_ref|) ...
U32 = 2.0 ** -24  # FP32 unit roundoff
# ... or, for an element where the terms of its sum cancel, within the FP32
# rounding bound of that sum: u (16 A_n + 256 A), A = sum |term| (taken on the
# operands of the subtractions inside a term), A_n the same with every
# pixel's terms weighted by its contributor count (the transmittance is
# recovered by one division per contributor, so its rounding grows with the
# count), 256 u for the per-term evaluation (MUFU lg2/ex2 times the exponent,
# the stored mean); SH coefficients add the basis bound of sh_basis_bound.
# At most FLOOR_FRAC of the touched elements of a group (at least one) may
# rest on it.
FLOOR_N, FLOOR_A = 16.0, 256.0
FLOOR_FRAC = 0.01
GRAD_NORM = 1e-4  # and ||g - g_ref|| / ||g_ref|| per group


def grad_floor(mag, extra=0.0):
    """The FP32 rounding bound of each element's sum."""
    return U32 * (FLOOR_N * mag.absn + FLOOR_A * mag.abs) + extra


def grad_den(ref, mag, extra=0.0):
    """Per-element scale: the gradient bar divided by GRAD_REL, or the FP32
    bound divided by GRAD_REL where that is larger (|g - g_ref| <= GRAD_REL x
    this is the element's test)."""
    scale = max(float(np.abs(ref).max()), 1e-30)
    lit = np.maximum(np.abs(ref), 1e-3 * scale)
    return np.maximum(lit, grad_floor(mag, extra) / GRAD_REL)


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
    """Per parameter group: every element within the gradient bar
    rel max(|g_ref|, 1e-3 max_group |g_ref|) or within the FP32 rounding
    bound of its sum; at most FLOOR_FRAC of the touched elements (those with a
    nonzero reference or summand) resting on the latter; and the group's
    relative L2 error within ``norm``.  Returns per group: the largest ratio
    of error to bar, the relative L2 error, the number of touched elements,
    how many of them fail the 1e-3 bar (and so rest on the FP32 bound),
    and that fraction."""
    sl = oracle.theta_slices(n, sh_degree)
    report = {}
    for name, s in sl.items():
        a, b = got[s], ref[s]
        scale = np.abs(b).max()
        if scale == 0:
            assert np.abs(a).max() == 0, (label, name)
            continue
        ex = 0.0 if extra is None else extra[s]
        den = grad_den(b, mag[s], ex)
        err = np.abs(a - b)
        relerr = err / den
        l2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        touched = (b != 0) | (mag[s].abs > 0)
        literal = touched & (err > rel * np.maximum(np.abs(b), 1e-3 * scale))
        frac = float(literal.sum()) / max(int(touched.sum()), 1)
        report[name] = {"max_ratio": round(float(relerr.max()) / rel, 4), "l2": float(f"{l2:.3g}"),
                        "touched": int(touched.sum()), "literal_fail": int(literal.sum()),
                        "floor_frac": round(frac, 5)}
        bad = relerr > rel
        assert not bad.any(), (label, name, report[name], int(bad.sum()), a[bad][:5], b[bad][:5])
        assert l2 <= norm, (label, name, report[name])
        assert literal.sum() <= max(1.0, FLOOR_FRAC * touched.sum()), (label, name, report[name])
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


# ---------------------------------------------------------------- the windows, checked
def projection_error_ratio(fr, j, cam, proj, seed=0):
    """The GPU projection's error of h on the ellipse h = h_max (where
    alpha = tau), against the part of the oracle's ambiguity window that
    models it, 8 u h + 64 u^2 E h + u q + 2 u (|m - origin| + 1) |dh/dm|
    (scales, double-float conic, its FP32 rounding, the stored mean; E the
    record's error scale, q the sum of the magnitudes of h's terms): one
    random point of the ring per valid entry of job j.  Returns the ratios
    |dh| / window (all must be <= 1)."""
    n = proj.shape[0]
    eb = fr.plan.jobs[j].entry_base
    recs = fr.records()[eb:eb + n].cpu().numpy().astype(np.float64)
    dkey = fr.depth_keys()[eb:eb + n].cpu().numpy().view(np.uint32)
    ok = (proj[:, oracle.P["valid"]] != 0) & (dkey != 0xFFFFFFFF) & (proj[:, oracle.P["ntiles"]] > 0)
    r, f = recs[ok], proj[ok]
    org = r[:, 11].astype(np.float32).view(np.uint32)
    ox, oy = (org & 0xFFFF).astype(np.float64), (org >> 16).astype(np.float64)
    A, B, C = f[:, oracle.P["cov_a"]], f[:, oracle.P["cov_b"]], f[:, oracle.P["cov_c"]]
    l11 = np.sqrt(A)
    l21 = B / l11
    l22 = np.sqrt(np.maximum(C - l21 ** 2, 0.0))
    th = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, len(f))
    hm = f[:, oracle.P["hmax"]]
    dx = np.sqrt(hm) * l11 * np.cos(th)
    dy = np.sqrt(hm) * (l21 * np.cos(th) + l22 * np.sin(th))
    ca, cb, cc = f[:, oracle.P["con_a"]], f[:, oracle.P["con_b"]], f[:, oracle.P["con_c"]]
    h = ca * dx * dx + 2 * cb * dx * dy + cc * dy * dy
    px, py = f[:, oracle.P["mx"]] + dx, f[:, oracle.P["my"]] + dy
    gx, gy = px - (r[:, 0] + ox), py - (r[:, 1] + oy)
    hg = r[:, 2] * gx * gx + 2 * r[:, 3] * gx * gy + r[:, 4] * gy * gy
    gm = (2 * np.abs(ca * dx + cb * dy) * 2 * U32 * (np.abs(f[:, oracle.P["mx"]] - ox) + 1)
          + 2 * np.abs(cb * dx + cc * dy) * 2 * U32 * (np.abs(f[:, oracle.P["my"]] - oy) + 1))
    q = np.abs(ca) * dx * dx + 2 * np.abs(cb * dx * dy) + np.abs(cc) * dy * dy
    return np.abs(hg - h) / (8 * U32 * h + 64 * U32 * U32 * f[:, oracle.P["es"]] * h + U32 * q + gm)
