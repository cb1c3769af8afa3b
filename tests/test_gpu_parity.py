"""GPU parity of every hot-path step against the FP64 oracle, through the C ABI.

Bars: tile lists and sorted keys bit-exact; forward <= 1e-4 max-abs per pixel
channel and in T on every pixel (where the oracle met a decision within the
FP32 rounding window of tau or t_min, against the admissible result -- those
decisions taken either way -- that the GPU matched; the flagged fraction is
reported); gradients, through the same admissible forward: every element
within 1e-3 relative or within the FP32 rounding bound of its sums (derived
from the magnitudes of its summands and the contributor counts of their
pixels), and <= 1e-4 relative L2 per group; sampler: Philox words bit for
bit, updates within 1e-6 relative or the FP32 rounding of the increment.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_10148_gb300 import _abi, frame, inputs

from gpu_util import (DEV, FWD_TOL, GRAD_NORM, GRAD_REL, U32, adam_increment_mag, assert_groups_close,
                      assert_step_close, check_forward_frame, check_forward_view, check_unresolved_gradients, f32,
                      f32_scene, gpu_forward,
                      gpu_last_component, gpu_view, grad_den, oracle_views, projection_error_ratio, require_gpu,
                      resolved_weights, scene_grads_flat,
                      sh_basis_bound, step_mags)
from oracle import Magnitudes

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


# ---------------------------------------------------------------- a1 project

def _check_projection(fr, scene, cams, cfgd):
    recs = fr.records().cpu().numpy().astype(np.float64)
    dkey = _u32(fr.depth_keys())
    nt = fr.ntiles().cpu().numpy()
    rect = _u32(fr.rects())
    n = scene["n"]
    for j, cam in enumerate(cams):
        ref = oracle.project(scene, cam, cfgd)
        eb = fr.plan.jobs[j].entry_base
        sl = slice(eb, eb + n)
        valid_ref = ref[:, oracle.P["valid"]] != 0
        valid_gpu = dkey[sl] != 0xFFFFFFFF
        assert np.array_equal(valid_ref, valid_gpu), int((valid_ref != valid_gpu).sum())
        # FP32 depth keys: same FMA chain on both sides -> bit-exact
        ref_bits = ref[valid_ref, oracle.P["depth"]].astype(np.float32).view(np.uint32)
        assert np.array_equal(ref_bits, dkey[sl][valid_ref])
        r = recs[sl][valid_ref]
        rf = ref[valid_ref]
        org = recs[sl][valid_ref][:, 11].astype(np.float32).view(np.uint32)
        ox, oy = (org & 0xFFFF).astype(np.float64), (org >> 16).astype(np.float64)
        # the origin is the integer pixel nearest to the mean's FP32 high part
        # (either one within that part's spacing of a half-integer), limited
        # to [0, 16384]; the stored offset is the ~46-bit mean rounded once
        for col, key, o in ((0, "mx", ox), (1, "my", oy)):
            m = rf[:, oracle.P[key]]
            near = np.clip(np.rint(m), 0, 16384)
            half = np.abs(np.abs(m - np.floor(m)) - 0.5) <= 2.0 ** -23 * np.maximum(np.abs(m), 1.0)
            okn = (o == near) | half
            assert okn.all(), (key, int((~okn).sum()), m[~okn][:4].tolist(), o[~okn][:4].tolist())
            dm = np.abs(r[:, col] + o - m) / (U32 * np.abs(m - o) + 1e-9)
            assert dm.max() <= 1.0, (key, float(dm.max()))
        # the conic: double-float, rounded once to FP32 (u relative); the FP32
        # scales exp(log_scale) (2 ulp each) perturb Sigma2D by at most 8 u of
        # itself, so entry (i, j) of its inverse by 8 u sqrt(con_ii con_jj);
        # the double-float chain's own error, 64 u^2 E on Sigma2D relative to
        # lambda_min, is at most 128 u^2 E times the conic's largest diagonal
        # entry (E the record's error scale)
        ca_r, cc_r = rf[:, oracle.P["con_a"]], rf[:, oracle.P["con_c"]]
        scale = np.maximum(np.abs(ca_r), np.abs(cc_r))
        es = rf[:, oracle.P["es"]]
        for col, key, geo in ((2, "con_a", ca_r), (3, "con_b", np.sqrt(ca_r * cc_r)), (4, "con_c", cc_r)):
            ref_c = rf[:, oracle.P[key]]
            bound = 1.01 * U32 * np.abs(ref_c) + 8.1 * U32 * geo + 128 * U32 * U32 * es * scale
            assert np.all(np.abs(r[:, col] - ref_c) <= bound), (key, float(np.max(np.abs(r[:, col] - ref_c) / bound)))
        assert np.allclose(r[:, 5], rf[:, oracle.P["o"]], rtol=0, atol=2e-6)
        assert np.allclose(r[:, 6], rf[:, oracle.P["hmax"]], rtol=2e-5, atol=1e-5)
        assert np.allclose(r[:, 7], rf[:, oracle.P["nu"]], rtol=1e-6)
        for col, key in ((8, "r"), (9, "g"), (10, "b")):
            assert np.allclose(r[:, col], rf[:, oracle.P[key]], rtol=0, atol=2e-5), key
        # tile rectangles: equal except where a box edge sits within 1e-3 px of
        # a pixel-centre boundary (FP32 ceil/floor there is a coin toss)
        ex = np.sqrt(rf[:, oracle.P["cov_a"]] * rf[:, oracle.P["hmax"]])
        ey = np.sqrt(rf[:, oracle.P["cov_c"]] * rf[:, oracle.P["hmax"]])
        edges = np.stack([rf[:, oracle.P["mx"]] - ex - 0.5, rf[:, oracle.P["mx"]] + ex - 0.5,
                          rf[:, oracle.P["my"]] - ey - 0.5, rf[:, oracle.P["my"]] + ey - 0.5], 1)
        fragile = np.any(np.abs(edges - np.round(edges)) < 1e-3, axis=1)
        rg = rect[sl][valid_ref]
        tx0, tx1 = rg[:, 0] & 0xFFFF, rg[:, 0] >> 16
        ty0, ty1 = rg[:, 1] & 0xFFFF, rg[:, 1] >> 16
        ntr = rf[:, oracle.P["ntiles"]]
        has = ntr > 0
        same = (nt[sl][valid_ref] == ntr) & (~has | ((tx0 == rf[:, oracle.P["tx0"]]) & (tx1 == rf[:, oracle.P["tx1"]])
                                                      & (ty0 == rf[:, oracle.P["ty0"]]) & (ty1 == rf[:, oracle.P["ty1"]])))
        assert np.all(same | fragile), int((~same & ~fragile).sum())
        assert fragile.mean() < 0.03, fragile.mean()


def test_project_tiny():
    scene, cams = inputs.tiny_cube_2k()
    fr, _, cams = gpu_forward(scene, cams)
    _check_projection(fr, f32_scene(scene), cams, frame.cfg_dict(fr.cfg))


def test_project_shell_sh3_multiview():
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 5))
    fr, _, cams = gpu_forward(scene, cams)
    _check_projection(fr, f32_scene(scene), cams, frame.cfg_dict(fr.cfg))


# ---------------------------------------------------------------- a2 + a3

def _check_bin_sort(fr):
    st, need, done = fr.status()
    assert st == 0 and need == done
    P = fr.plan
    nt = fr.ntiles().cpu().numpy().astype(np.int64)
    rect = _u32(fr.rects())
    dkey = _u32(fr.depth_keys())
    assert int(nt.sum()) == need
    tiles_x = np.zeros(P.n_entries, np.int64)
    tile_base = np.zeros(P.n_entries, np.int64)
    for j in range(P.n_jobs):
        J = P.jobs[j]
        n = P.scenes[J.scene].n
        tiles_x[J.entry_base:J.entry_base + n] = J.tiles_x
        tile_base[J.entry_base:J.entry_base + n] = J.tile_base
    r = np.stack([rect[:, 0] & 0xFFFF, rect[:, 0] >> 16, rect[:, 1] & 0xFFFF, rect[:, 1] >> 16], 1).astype(np.int64)
    r[nt == 0] = (0, -1, 0, -1)
    # reference fed the GPU's own rectangles and depth-key bits
    ref_tiles, ref_ents = oracle.bin_sort_reference(r, dkey, tiles_x, tile_base)
    k, v = fr.sorted_pairs(need)
    assert np.array_equal(k.cpu().numpy().astype(np.int64), ref_tiles)
    assert np.array_equal(v.cpu().numpy().astype(np.int64), ref_ents)
    rng = fr.ranges().cpu().numpy().astype(np.int64)
    t = np.arange(P.n_tiles)
    lo = np.searchsorted(ref_tiles, t, "left")
    hi = np.searchsorted(ref_tiles, t, "right")
    empty = lo == hi
    assert np.array_equal(rng[~empty, 0], lo[~empty]) and np.array_equal(rng[~empty, 1], hi[~empty])
    assert np.all(rng[empty, 0] == rng[empty, 1])


def test_bin_sort_bit_exact_tiny():
    scene, cams = inputs.tiny_cube_2k()
    fr, _, _ = gpu_forward(scene, cams)
    _check_bin_sort(fr)


@pytest.mark.parametrize("tile", [(16, 16), (32, 16), (16, 32), (32, 32), (64, 32), (64, 64)])
def test_bin_sort_bit_exact_multiview(tile):
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 3))
    cams = [inputs.look_at(c.position, width=300 + 7 * i, height=211 + 3 * i) for i, c in enumerate(cams[:5])]
    fr, _, _ = gpu_forward(scene, cams, frame.make_cfg(tile_w=tile[0], tile_h=tile[1]))
    _check_bin_sort(fr)


def test_projection_error_within_the_ambiguity_window():
    """The FP32 projection's error in h, on the ellipse where alpha = tau,
    stays inside the part of the oracle's ambiguity window that models it
    (shell workload, every valid entry of every view)."""
    scene, cams = inputs.shell_100k_8views()
    fr, _, cams = gpu_forward(scene, cams)
    cfgd = frame.cfg_dict(fr.cfg)
    ratios = np.concatenate([projection_error_ratio(fr, j, cam, oracle.project(f32_scene(scene), cam, cfgd), seed=j)
                             for j, cam in enumerate(cams)])
    print("projection error / window:", {q: float(np.quantile(ratios, q)) for q in (0.5, 0.99, 0.9999, 1.0)})
    assert ratios.max() <= 1.0


def test_depth_ties_break_by_component_index():
    """Identical components (same depth key) must keep index order."""
    base = inputs.scene_uniform_cube(64, seed=7)
    idx = np.repeat(np.arange(64), 3)  # each component three times
    scene = inputs.subset_scene(base, idx)
    fr, _, _ = gpu_forward(scene, [inputs.look_at((0, 0, 3), width=64, height=64)])
    _check_bin_sort(fr)


# ---------------------------------------------------------------- a4 forward

def _check_forward(fr, scene, cams, cfgd, pix=None, max_flagged=None):
    refs = oracle_views(scene, cams, cfgd, pix)
    flips, st, _ = check_forward_frame(fr, cams, cfgd, refs, pix)
    print("forward", st)
    if max_flagged is not None:
        assert st["flagged_frac"] <= max_flagged, st
    return st


@pytest.mark.parametrize("tile,batch", [((16, 16), 32), ((32, 16), 32), ((16, 32), 32), ((32, 32), 32),
                                        ((64, 32), 32), ((32, 64), 32), ((64, 64), 32), ((64, 16), 32),
                                        ((128, 64), 32), ((128, 128), 32), ((16, 16), 64), ((32, 32), 64),
                                        ((64, 128), 64)])
def test_forward_tiny_all_tile_configs(tile, batch):
    scene, cams = inputs.tiny_cube_2k()
    cfg = frame.make_cfg(tile_w=tile[0], tile_h=tile[1], batch=batch)
    fr, _, cams = gpu_forward(scene, cams, cfg)
    _check_forward(fr, f32_scene(scene), cams, frame.cfg_dict(cfg))


def test_forward_last_contributor_matches_oracle():
    """Every pixel's last contributor equals the oracle's (flagged pixels:
    that of the admissible result they match)."""
    scene, cams = inputs.tiny_cube_2k()
    fr, _, cams = gpu_forward(scene, cams)
    cfgd = frame.cfg_dict(fr.cfg)
    proj = oracle.project(f32_scene(scene), cams[0], cfgd)
    ref = oracle.render(proj, cams[0], cfgd)
    img, T = gpu_view(fr, 0, cams[0])
    comp = gpu_last_component(fr, 0, cams[0])
    chk = check_forward_view(proj, cams[0], cfgd, ref, img, T, last=comp)
    alt = oracle.render(proj, cams[0], cfgd, flip=chk.flip)  # the admissible result the GPU matched
    assert np.array_equal(comp, alt["last"]) and (comp >= 0).sum() > 1000


def test_pair_counters_match_oracle():
    """cfg.count_pairs: the forward counts contributing (splat, pixel) pairs
    (the oracle's n_contrib summed over pixels, each pixel through the
    admissible forward the GPU matched) and evaluated pairs (at least the
    contributing ones); a forward without counting adds nothing."""
    scene, cams = inputs.tiny_cube_2k()
    fr, _, cams = gpu_forward(scene, cams)
    cfgd = frame.cfg_dict(fr.cfg)
    nc, ne = fr.count_pairs()
    lo = hi = 0
    for j, cam in enumerate(cams):
        proj = oracle.project(f32_scene(scene), cam, cfgd)
        ref = oracle.render(proj, cam, cfgd)
        img, T = gpu_view(fr, j, cam)
        chk = check_forward_view(proj, cam, cfgd, ref, img, T, last=gpu_last_component(fr, j, cam))
        lo += int(chk.nc_lo.sum())
        hi += int(chk.nc_hi.sum())
    assert lo <= nc <= hi and hi - lo <= 20, (nc, lo, hi)
    assert lo > 0 and ne >= nc
    fr.forward(grow=False)
    torch.cuda.synchronize()
    ctrl = fr.ws_view(fr.plan.ws_off_ctrl, torch.int64, 4).cpu()
    assert (int(ctrl[2]), int(ctrl[3])) == (0, 0)


def test_forward_shell_8views_800_sampled():
    """Shell workload at full size (100k components, 8 x 800x800, SH degree 3),
    2,000 sampled pixels per view computed one by one by the oracle."""
    scene, cams = inputs.shell_100k_8views()
    fr, _, cams = gpu_forward(scene, cams)
    rng = np.random.default_rng(0)
    pix = [rng.choice(c.width * c.height, 2000, replace=False) for c in cams]
    _check_forward(fr, f32_scene(scene), cams, frame.cfg_dict(fr.cfg), pix, max_flagged=0.005)


@pytest.mark.parametrize("case", ["ragged", "no_termination", "lowpass", "background", "large_nu", "clamped_alpha",
                                  "sh1", "sh2", "large_nu_packed", "no_termination_packed"])
def test_forward_edge_cases(case):
    scene = inputs.scene_uniform_cube(1500, seed=11)
    cam = inputs.look_at((0.3, -0.2, 3.0), width=100, height=60)
    kw = dict(tile_w=16, tile_h=16)  # one pixel per lane (scalar FP32)
    if case.endswith("_packed"):  # 32x32 tiles: pixels in packed pairs
        case = case[:-len("_packed")]
        kw.update(tile_w=32, tile_h=32)
    if case == "no_termination":
        kw["t_min"] = 0.0
    elif case == "lowpass":
        kw["lowpass"] = 0.3
    elif case == "background":
        kw["bg"] = (0.2, 0.5, 1.0)
    elif case == "large_nu":
        scene["nu"] = np.exp(np.random.default_rng(1).uniform(math.log(40), math.log(1e4), 1500)).astype(np.float32)
    elif case == "clamped_alpha":
        scene["opacity_raw"] = np.sign(scene["opacity_raw"]) * np.float32(4.0)
    elif case in ("sh1", "sh2"):
        deg = 1 if case == "sh1" else 2
        K = (deg + 1) ** 2
        sh = np.random.default_rng(2).normal(0, 0.3, (3 * K, 1500)).astype(np.float32)
        sh[:3] = scene["sh"]
        scene["sh"], scene["sh_degree"] = sh, deg
    cfg = frame.make_cfg(**kw)
    fr, _, cams = gpu_forward(scene, [cam], cfg)
    _check_forward(fr, f32_scene(scene), cams, frame.cfg_dict(cfg))


def test_forward_empty_and_culled_scenes():
    cam = inputs.look_at((0, 0, 3), width=48, height=40)
    cfg = frame.make_cfg(bg=(0.1, 0.2, 0.3))
    behind = inputs.scene_uniform_cube(50, seed=1)
    behind["mean"] = behind["mean"] + np.array([[0], [0], [5.0]], np.float32)  # all behind the camera
    for sc in (inputs.subset_scene(inputs.scene_uniform_cube(10, seed=1), np.arange(0)), behind):
        fr, _, _ = gpu_forward(sc, [cam], cfg)
        img = fr.image(0).cpu().numpy()
        assert np.allclose(img, np.array([0.1, 0.2, 0.3], np.float32)[:, None, None])
        assert fr.status()[1] == 0


@pytest.mark.parametrize("shape,tile", [((16384, 24), (16, 16)), ((24, 16384), (32, 32))])
def test_forward_and_backward_at_the_largest_image_extent(shape, tile):
    """Images 16,384 pixels wide or high, the plan's limit: 1,024 tiles along
    a row (16-pixel tiles), record origins up to the 16,384 limit and pixel
    offsets from them at the largest magnitudes; every pixel's forward and the
    gradient of a seeded linear loss over all of them against the oracle."""
    w, h = shape
    scene = inputs.scene_uniform_cube(3000, seed=17)
    fx = 17567.0 if w > h else 14000.0  # a strip of the cube seen at a usual pixel scale
    cam = inputs.look_at((0.2, -0.1, 3.0), width=w, height=h, fov_x_deg=math.degrees(2 * math.atan(w / 2 / fx)))
    cfg = frame.make_cfg(tile_w=tile[0], tile_h=tile[1])
    fr, sc, cams = gpu_forward(scene, [cam], cfg)
    cfgd = frame.cfg_dict(cfg)
    s32 = f32_scene(scene)
    assert fr.status()[1] > 10000  # the strip holds many splats
    st = _check_forward(fr, s32, cams, cfgd, max_flagged=0.01)
    refs = oracle_views(s32, cams, cfgd)
    unresolved = []
    ws, flips, fst = resolved_weights(fr, cams, cfgd, refs, seed=18, alts_out=unresolved)
    g = _gpu_backward(fr, sc, ws)
    gref, gabs = oracle.backward(s32, cams, cfgd, ws, want_abs=True, flip=flips)
    print(st, assert_groups_close(scene_grads_flat(g), gref, scene["n"], 0, gabs, label=f"{w}x{h}"))
    checked, _ = check_unresolved_gradients(fr, sc, s32, cams, cfgd, unresolved, seed=19, sh_degree=0)
    assert checked == min(len(unresolved), 48)


# ---------------------------------------------------------------- a5 + a6 backward

def _gpu_backward(fr, sc, ws):
    dl = torch.as_tensor(np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32), device=DEV)
    g = sc.zeros_like()
    fr.backward(dl, [g])
    torch.cuda.synchronize()
    return g


def _grad2d_report(fr, g2d_ref, g2d_abs, cams, scene):
    g2 = fr.grad2d().cpu().numpy().astype(np.float64)[:, :10]
    n = scene["n"]
    for j in range(len(cams)):
        eb = fr.plan.jobs[j].entry_base
        got = g2[eb:eb + n]
        ref = g2d_ref[j]
        for c, name in enumerate(oracle.G_FIELDS):
            scale = np.abs(ref[:, c]).max()
            if scale == 0:
                continue
            tol = GRAD_REL * grad_den(ref[:, c], Magnitudes(g2d_abs.abs[j][:, c], g2d_abs.absn[j][:, c]))
            bad = np.abs(got[:, c] - ref[:, c]) > tol
            assert not bad.any(), (j, name, int(bad.sum()), got[bad, c][:4], ref[bad, c][:4])
            assert np.linalg.norm(got[:, c] - ref[:, c]) <= GRAD_NORM * np.linalg.norm(ref[:, c]), (j, name)


@pytest.mark.parametrize("nu_mode,tile", [(0, (16, 16)), (1, (16, 16)), (0, (32, 16)), (0, (16, 32)), (1, (32, 32)),
                                          (0, (64, 32)), (1, (32, 64)), (0, (64, 64)), (1, (128, 128)),
                                          (0, (16, 16, 64)), (1, (64, 128, 64)),
                                          (0, (32, 64, 32, 16)), (1, (64, 64, 64, 16)), (0, (128, 128, 32, 16))])
def test_backward_tiny_against_oracle_analytic(nu_mode, tile):
    """tile = (tile_w, tile_h[, records per warp and staging round[, height
    of the backward's warp box]])."""
    scene, cams = inputs.tiny_cube_2k()
    batch = tile[2] if len(tile) > 2 else 32
    box = tile[3] if len(tile) > 3 else 8
    cfg = frame.make_cfg(nu_grad_mode=nu_mode, tile_w=tile[0], tile_h=tile[1], batch=batch, bwd_box_h=box)
    fr, sc, cams = gpu_forward(scene, cams, cfg)
    cfgd = frame.cfg_dict(cfg)
    s32 = f32_scene(scene)
    refs = oracle_views(s32, cams, cfgd)
    ws, flips, fst = resolved_weights(fr, cams, cfgd, refs, seed=5)
    g = _gpu_backward(fr, sc, ws)
    gref, g2d, gabs, g2abs = oracle.backward(s32, cams, cfgd, ws, want_grad2d=True, want_abs=True, flip=flips)
    _grad2d_report(fr, g2d, g2abs, cams, scene)
    print(fst, assert_groups_close(scene_grads_flat(g), gref, scene["n"], 0, gabs, label="tiny",
                              extra=sh_basis_bound(scene["n"], 0, g2abs)))


def test_backward_shell_sh3_multiview_against_oracle_analytic():
    scene, cams = inputs.shell_100k_8views()
    scene = inputs.subset_scene(scene, np.arange(0, 100_000, 10))
    cams = [inputs.look_at(c.position, width=160, height=128) for c in cams[:3]]
    fr, sc, cams = gpu_forward(scene, cams)
    cfgd = frame.cfg_dict(fr.cfg)
    s32 = f32_scene(scene)
    refs = oracle_views(s32, cams, cfgd)
    unresolved = []
    ws, flips, fst = resolved_weights(fr, cams, cfgd, refs, seed=6, alts_out=unresolved)
    g = _gpu_backward(fr, sc, ws)
    gref, g2d, gabs, g2abs = oracle.backward(s32, cams, cfgd, ws, want_grad2d=True, want_abs=True, flip=flips)
    _grad2d_report(fr, g2d, g2abs, cams, scene)
    print(fst, assert_groups_close(scene_grads_flat(g), gref, scene["n"], 3, gabs, label="shell",
                              extra=sh_basis_bound(scene["n"], 3, g2abs)))
    checked, first = check_unresolved_gradients(fr, sc, s32, cams, cfgd, unresolved, seed=9, sh_degree=3)
    print(f"unresolved pixels: {len(unresolved)}, checked one by one {checked}, matching the first admissible "
          f"result {first}")
    assert checked == min(len(unresolved), 48)


def test_backward_gradcheck_50k_against_oracle_fd_and_analytic():
    """Gradient check: 50k components, 256x256; GPU gradient against the
    oracle's FP64 central differences (h = 1e-6) on 200 parameters spread
    over all six groups, and against the full analytic FP64 gradient."""
    scene, cams = inputs.gradcheck_cube_50k()
    fr, sc, cams = gpu_forward(scene, cams)
    cfgd = frame.cfg_dict(fr.cfg)
    s32 = f32_scene(scene)
    refs = oracle_views(s32, cams, cfgd)
    unresolved = []
    ws, flips, fst = resolved_weights(fr, cams, cfgd, refs, seed=7, alts_out=unresolved)
    g = scene_grads_flat(_gpu_backward(fr, sc, ws))
    gref, gabs = oracle.backward(s32, cams, cfgd, ws, want_abs=True, flip=flips)
    print(fst, assert_groups_close(g, gref, scene["n"], 0, gabs, label="gradcheck"))
    # the pixels whose image leaves their decisions open, each on its own
    checked, first = check_unresolved_gradients(fr, sc, s32, cams, cfgd, unresolved, seed=8, sh_degree=0)
    print(f"unresolved pixels: {len(unresolved)}, checked one by one {checked}, matching the first admissible "
          f"result {first}")
    assert checked == min(len(unresolved), 48)
    # central differences follow the oracle's own decisions: compare them with
    # a GPU gradient whose flagged pixels carry no weight
    ws = [w * (ref["flags"] == 0)[None, :] for w, (_, ref) in zip(ws, refs)]
    g = scene_grads_flat(_gpu_backward(fr, sc, ws))
    # finite differences on parameters that influence the loss
    n = scene["n"]
    sl = oracle.theta_slices(n, 0)
    rng = np.random.default_rng(3)
    theta = oracle.theta_from_scene(s32)
    picks = []
    per = {"mean": 34, "log_scale": 34, "quat": 34, "nu": 33, "opacity_raw": 33, "sh": 32}
    for name, k in per.items():
        cand = np.arange(sl[name].start, sl[name].stop)
        cand = cand[np.abs(gref[cand]) > 1e-4 * np.abs(gref[sl[name]]).max()]
        picks += list(rng.choice(cand, k, replace=False))
    fd, smooth = oracle.fd_gradient(theta, n, 0, cams, cfgd, ws, picks)
    checked = 0
    for j, f, ok in zip(picks, fd, smooth):
        if not ok:
            continue
        group = next(k for k, s in sl.items() if s.start <= j < s.stop)
        den = grad_den(np.array([f]), Magnitudes(np.array([gabs.abs[j]]), np.array([gabs.absn[j]])))[0]
        assert abs(g[j] - f) <= GRAD_REL * den, (group, j, g[j], f, gabs[j])
        checked += 1
    assert checked >= 180


@pytest.mark.parametrize("tile", [(16, 16), (32, 32), (64, 64, 16)])
def test_backward_edge_cases_large_nu_and_clamp(tile):
    """Large nu (the log1pf/expf path) and clamped alpha, one pixel per lane
    (16x16 tiles), two packed pixel pairs per lane (32x32) and four (64x64
    with 16-pixel-high backward boxes)."""
    scene = inputs.scene_uniform_cube(1200, seed=13)
    rng = np.random.default_rng(4)
    scene["nu"] = np.exp(rng.uniform(0, math.log(2e4), 1200)).astype(np.float32)  # some beyond the 1e4 limit
    scene["opacity_raw"][:100] = np.float32(3.5)  # |o| > alpha_max: clamped alpha
    cam = inputs.look_at((0.1, 0.2, 3.0), width=96, height=72)
    cfg = frame.make_cfg(bg=(0.3, 0.1, 0.6), lowpass=0.3, tile_w=tile[0], tile_h=tile[1],
                         bwd_box_h=tile[2] if len(tile) > 2 else 8)
    fr, sc, cams = gpu_forward(scene, [cam], cfg)
    cfgd = frame.cfg_dict(cfg)
    s32 = f32_scene(scene)
    refs = oracle_views(s32, cams, cfgd)
    ws, flips, fst = resolved_weights(fr, cams, cfgd, refs, seed=8)
    g = _gpu_backward(fr, sc, ws)
    gref, gabs = oracle.backward(s32, cams, cfgd, ws, want_abs=True, flip=flips)
    print(fst, assert_groups_close(scene_grads_flat(g), gref, 1200, 0, gabs, label="edge"))


# ---------------------------------------------------------------- a7 step

@pytest.mark.parametrize("burn_in,step,n_comp", [(False, 0, 3000), (True, 3, 3000), (False, (1 << 32) + 5, 3000),
                                                  (True, (1 << 33) + 1, 3000), (False, 2, 2999), (True, 1, 2999)])
def test_sghmc_step_against_oracle(burn_in, step, n_comp):
    """The step's Philox words equal the oracle's bit for bit (every
    component, step indices above 2^32); every updated value is within the
    sampler bar (1e-6 relative, or the FP32 rounding of the increment's
    terms).  n_comp = 2999 (not a multiple of 4) takes the Adam rows' strided
    path, 3000 their 16-byte path."""
    scene = inputs.scene_sphere_shell(n_comp, seed=9)
    n = scene["n"]
    rng = np.random.default_rng(10)
    sc = frame.Scene.from_numpy(scene, DEV)
    grads = sc.zeros_like()
    for f in frame.FIELDS:
        grads.t[f].copy_(torch.as_tensor(rng.normal(size=tuple(grads.t[f].shape)).astype(np.float32)))
    grads.t["opacity_raw"][0, :200] = 0.0
    sc.t["opacity_raw"][0, :300] = torch.as_tensor(rng.uniform(-0.01, 0.01, 300).astype(np.float32))
    st = frame.SamplerState(sc)
    st.r.copy_(torch.as_tensor(rng.normal(size=(3, n)).astype(np.float32) * 0.1))
    st.m.copy_(torch.as_tensor(rng.normal(size=tuple(st.m.shape)).astype(np.float32) * 0.01))
    st.v.copy_(torch.as_tensor(np.abs(rng.normal(size=tuple(st.v.shape))).astype(np.float32) * 0.01))
    theta0 = oracle.theta_from_scene(sc.to_numpy())
    g0 = scene_grads_flat(grads)
    r0 = st.r.cpu().numpy().astype(np.float64).reshape(-1)
    m0 = st.m.cpu().numpy().astype(np.float64)
    v0 = st.v.cpu().numpy().astype(np.float64)
    # oracle moments use theta's layout: mean rows unused
    mo = np.concatenate([np.zeros(3 * n), m0.reshape(-1)])
    vo = np.concatenate([np.zeros(3 * n), v0.reshape(-1)])
    params = dict(eps=f32(2e-2), C=f32(0.6), k=f32(100.0), t0=f32(0.005), lr=f32((5e-3, 1e-3, 1e-2, 5e-2, 2.5e-3)),
                  beta1=f32(0.9), beta2=f32(0.999), adam_eps=f32(1e-8))
    words = torch.zeros(4, n, dtype=torch.int32, device=DEV)
    sp = frame.step_params(eps=params["eps"], C=params["C"], burn_in=burn_in, seed=77, step=step,
                           lr=params["lr"], adam_eps=params["adam_eps"], philox_out=words)
    xi = torch.zeros(3, n, dtype=torch.float32, device=DEV)
    frame.sghmc_step(sc, grads, st, sp, xi_out=xi)
    torch.cuda.synchronize()
    th, rr, mm, vv, xir = oracle.sghmc_step(theta0, g0, r0, mo, vo, n=n, sh_degree=3, params=params,
                                             burn_in=burn_in, seed=77, step=step)
    # the generator, bit for bit: counter (i, 0, step_lo, step_hi), key (seed_lo, seed_hi)
    got_w = words.cpu().numpy().view(np.uint32)
    key = (77, 0)
    want_w = np.stack([oracle.philox4x32_10((i, 0, step & 0xFFFFFFFF, step >> 32), key) for i in range(n)], axis=1)
    assert np.array_equal(got_w, want_w)
    # the normals: FP32 Box-Muller of identical uniforms
    assert np.all(np.abs(xi.cpu().numpy() - xir) <= 8 * U32 * np.maximum(np.abs(xir), 1.0))
    got = oracle.theta_from_scene(sc.to_numpy())
    sl = oracle.theta_slices(n, 3)
    mu_mag, r_mag = step_mags(theta0, np.abs(g0[sl["mean"]]), r0, xir, n, 3, params, burn_in)
    rep = {"mean": assert_step_close(got[sl["mean"]], th[sl["mean"]], mu_mag, "mean"),
           "momentum": assert_step_close(st.r.cpu().numpy(), rr, r_mag, "momentum")}
    t = step + 1  # beta^t is 0 in both precisions above 2^24
    b1, b2 = params["beta1"], params["beta2"]
    for f, lr in zip(("log_scale", "quat", "nu", "opacity_raw", "sh"), params["lr"]):
        j = sl[f]
        ga = np.abs(g0[j])
        inc = adam_increment_mag(mo[j], ga, vv[j], lr, b1, b2, params["adam_eps"], t)
        rep[f] = assert_step_close(got[j], th[j], inc, f)
        jm = slice(j.start - 3 * n, j.stop - 3 * n)
        assert_step_close(st.m.cpu().numpy().reshape(-1)[jm], mm[j], b1 * np.abs(mo[j]) + (1 - b1) * ga, f + " m")
        assert_step_close(st.v.cpu().numpy().reshape(-1)[jm], vv[j], vv[j], f + " v")
    print("sampler bar", burn_in, step, rep)


@pytest.mark.parametrize("burn_in,n_comp", [(False, 5000), (True, 5000), (False, 4999)])
def test_sghmc_step_to_matches_the_step_in_place(burn_in, n_comp):
    """sss_sghmc_step_to writes bit for bit the parameters the in-place step
    leaves (regularisers on), updates momentum and moments identically, and
    leaves its input parameters as they were (both Adam row paths)."""
    scene = inputs.scene_sphere_shell(n_comp, seed=11)
    rng = np.random.default_rng(12)
    a, b, orig = (frame.Scene.from_numpy(scene, DEV) for _ in range(3))
    grads = a.zeros_like()
    for f in frame.FIELDS:
        grads.t[f].copy_(torch.as_tensor(rng.normal(size=tuple(grads.t[f].shape)).astype(np.float32)))
    sa, sb = frame.SamplerState(a), frame.SamplerState(b)
    r0 = torch.as_tensor(rng.normal(size=tuple(sa.r.shape)).astype(np.float32) * 0.1, device=DEV)
    m0 = torch.as_tensor(rng.normal(size=tuple(sa.m.shape)).astype(np.float32) * 0.01, device=DEV)
    v0 = torch.as_tensor(np.abs(rng.normal(size=tuple(sa.v.shape))).astype(np.float32) * 0.01, device=DEV)
    for s in (sa, sb):
        s.r.copy_(r0)
        s.m.copy_(m0)
        s.v.copy_(v0)
    kw = dict(eps=2e-2, C=0.6, burn_in=burn_in, seed=3, step=7, reg_opacity=0.01, reg_scale=0.01)
    out = b.zeros_like()
    frame.sghmc_step(a, grads, sa, frame.step_params(**kw))
    frame.sghmc_step(b, grads, sb, frame.step_params(**kw), out=out)
    torch.cuda.synchronize()
    for f in frame.FIELDS:
        assert torch.equal(out.t[f], a.t[f]), f
        assert torch.equal(b.t[f], orig.t[f]), f
        assert not torch.equal(a.t[f], orig.t[f]), f  # the step moved every group
    for x, y in ((sa.r, sb.r), (sa.m, sb.m), (sa.v, sb.v)):
        assert torch.equal(x, y)
    bad = frame.Scene.zeros(b.n - 1, b.sh_degree, DEV)
    with pytest.raises(_abi.SSSError):
        frame.sghmc_step(b, grads, sb, frame.step_params(**kw), out=bad)


def test_sghmc_noise_moments_on_gpu():
    n = 1_000_000
    scene = inputs.scene_uniform_cube(n, seed=2)
    sc = frame.Scene.from_numpy(scene, DEV)
    st = frame.SamplerState(sc)
    xi = torch.zeros(3, n, dtype=torch.float32, device=DEV)
    frame.sghmc_step(sc, sc.zeros_like(), st, frame.step_params(seed=5, step=1), xi_out=xi)
    z = xi.double()
    assert float(z.mean(1).abs().max()) < 5e-3
    assert float((z.var(1) - 1).abs().max()) < 6e-3
    # spot-check individual normals against the oracle's Philox + Box-Muller
    for i in (0, 1, 12345, n - 1):
        assert np.allclose(xi[:, i].cpu().numpy(), oracle.normals3(5, 1, i), atol=2e-5)


# ---------------------------------------------------------------- loss, capacity

def test_loss_l1():
    rng = np.random.default_rng(0)
    a = rng.uniform(size=100_003).astype(np.float32)
    b = rng.uniform(size=100_003).astype(np.float32)
    b[:10] = a[:10]
    pa, pb = torch.as_tensor(a, device=DEV), torch.as_tensor(b, device=DEV)
    g = torch.empty_like(pa)
    loss = torch.zeros(1, device=DEV)
    frame.loss_l1(pa, pb, g, loss)
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(np.abs(a.astype(np.float64) - b).mean(), rel=1e-5)
    assert np.array_equal(g.cpu().numpy(), (np.sign(a - b) / a.size).astype(np.float32))


def test_pair_capacity_overflow_is_reported_and_recovered():
    scene, cams = inputs.tiny_cube_2k()
    cams = [frame.f32_camera(c) for c in cams]
    sc = frame.Scene.from_numpy(scene, DEV)
    fr = frame.Frame([sc], cams, pair_capacity=1000, device=DEV)
    fr.project()
    fr.bin()
    fr.sort()
    fr.render_fwd()
    st, need, done = fr.status()
    assert st & _abi.SSS_STATUS_PAIR_OVERFLOW and need > 1000 and done == 1000
    fr2 = frame.Frame([sc], cams, pair_capacity=1000, device=DEV)
    fr2.forward(grow=True)
    st2, need2, done2 = fr2.status()
    assert st2 == 0 and need2 == need == done2


# ---------------------------------------------------------------- persistent launches, captured frames

def test_persistent_render_queue_resets_between_launches():
    """The render kernels take their work items from a counter in the
    workspace: after every launch it is back at 0 (control words 8 and 9), and
    repeated renders of a frame are bit for bit the first one."""
    scene, cams = inputs.tiny_cube_2k()
    fr, sc, cams = gpu_forward(scene, cams)
    ctrl = lambda: fr.ws_view(fr.plan.ws_off_ctrl, torch.int32, 16)[8:10].cpu().tolist()
    assert ctrl() == [0, 0]
    first = fr.rgb.clone()
    w = torch.as_tensor(np.concatenate([x.reshape(-1) for x in inputs.linear_loss_weights(cams, 3)]).astype(np.float32),
                        device=DEV)
    grads = []
    for _ in range(3):
        fr.render_fwd()
        g = sc.zeros_like()
        fr.backward(w, [g])
        torch.cuda.synchronize()
        assert ctrl() == [0, 0]
        assert torch.equal(fr.rgb, first)
        grads.append(g)
    for f in frame.FIELDS:  # the backward's float atomics may add in another order
        a, b = grads[0].t[f], grads[2].t[f]
        assert float((a - b).norm()) <= 1e-5 * float(b.norm()) + 1e-30, f


def test_multi_scene_frame_captured_in_a_cuda_graph():
    """A frame of two scenes and mixed resolutions -- projection, binning,
    sorting, forward and backward -- captured once into a CUDA graph and
    replayed: the replays equal the eager frame (images bit for bit)."""
    a = inputs.scene_uniform_cube(3000, seed=31)
    b = inputs.subset_scene(inputs.scene_sphere_shell(100_000, seed=32), np.arange(0, 100_000, 20))
    scs = [frame.Scene.from_numpy(x, DEV) for x in (a, b)]
    cams = [frame.f32_camera(inputs.look_at((0.2, 0.1, 3.0), width=160, height=120)),
            frame.f32_camera(inputs.look_at((2.0, 1.0, 2.0), width=97, height=203)),
            frame.f32_camera(inputs.look_at((-1.0, 2.5, 1.2), width=256, height=256))]
    job_scene = [0, 1, 1]
    fr = frame.Frame(scs, cams, job_scene=job_scene, device=DEV)
    fr.forward(grow=True)
    torch.cuda.synchronize()
    eager = fr.rgb.clone()
    dl = torch.as_tensor(np.random.default_rng(4).uniform(-1, 1, fr.rgb.numel()).astype(np.float32), device=DEV)
    ge = [s.zeros_like() for s in scs]
    fr.backward(dl, ge)
    torch.cuda.synchronize()
    gg = [s.zeros_like() for s in scs]
    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up off the capture
        fr.forward(side, grow=False)
        fr.backward(dl, gg, side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = torch.cuda.current_stream()
        fr.forward(st, grow=False)
        fr.backward(dl, gg, st)
    for _ in range(2):
        fr.rgb.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(fr.rgb, eager)
        for x, y in zip(gg, ge):
            for f in frame.FIELDS:  # float atomics: the order of the additions may differ
                assert float((x.t[f] - y.t[f]).norm()) <= 1e-5 * float(y.t[f].norm()) + 1e-30, f
    assert fr.status()[0] == 0
