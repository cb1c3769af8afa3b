"""Parity at the benchmark's full size and launch configuration:
1.5M components, 4 views at 1297x840, the tile/batch choice bench.py uses.

The oracle cannot render the whole frame, so it checks sampled outputs one by
one: seeded pixels of every view (forward), whole tile lists of seeded tiles
(binning and sorting, bit-exact), and the gradient of a loss restricted to
seeded pixels (the GPU runs its full backward with dL/dC zero elsewhere).
"""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_2503_10148_gb300 import frame, inputs

from gpu_util import DEV, assert_groups_close, f32_scene, require_gpu, scene_grads_flat, sh_basis_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    require_gpu()

    class A:
        tile = batch = None
    cfg, _ = bench._cfg(A)
    scene, cams = inputs.clusters_1p5m_4views()
    cams = [frame.f32_camera(c) for c in cams]
    sc = frame.Scene.from_numpy(scene, DEV)
    fr = frame.Frame([sc], cams, cfg=cfg, device=DEV)
    fr.forward(grow=True)
    torch.cuda.synchronize()
    return dict(scene=scene, s32=f32_scene(scene), cams=cams, sc=sc, fr=fr, cfgd=frame.cfg_dict(cfg))


def test_fullsize_forward_sampled_pixels(full):
    fr, cams = full["fr"], full["cams"]
    rng = np.random.default_rng(11)
    worst, flagged, total = 0.0, 0, 0
    for j, cam in enumerate(cams):
        pix = rng.choice(cam.width * cam.height, 250, replace=False).astype(np.int64)
        ref = oracle.render(oracle.project(full["s32"], cam, full["cfgd"]), cam, full["cfgd"], pix)
        img = fr.image(j).reshape(3, -1)[:, torch.as_tensor(pix, device=DEV)].cpu().numpy().astype(np.float64)
        ok = ref["flags"] == 0
        flagged += int((~ok).sum())
        total += ok.size
        worst = max(worst, float(np.abs(img[:, ok] - ref["rgb"][:, ok]).max()))
    print(f"full-size forward: max-abs {worst:.3e}, flagged {flagged}/{total}")
    assert worst <= 1e-4
    assert flagged <= 0.1 * total


def test_fullsize_tile_lists_sampled_tiles(full):
    """Whole lists of 40 seeded tiles against (depth key, entry)-sorted brute
    force over all 6M entries, using the GPU's rectangles and depth keys."""
    fr = full["fr"]
    P = fr.plan
    st, need, done = fr.status()
    assert st == 0 and need == done
    rect = fr.rects().cpu().numpy().view(np.uint32)
    nt = fr.ntiles().cpu().numpy()
    dkey = fr.depth_keys().cpu().numpy().view(np.uint32)
    assert int(nt.astype(np.int64).sum()) == need
    rng_t = fr.ranges().cpu().numpy().astype(np.int64)
    _, vals = fr.sorted_pairs(need)
    rng = np.random.default_rng(12)
    tx0, tx1 = rect[:, 0] & 0xFFFF, rect[:, 0] >> 16
    ty0, ty1 = rect[:, 1] & 0xFFFF, rect[:, 1] >> 16
    for t in rng.choice(P.n_tiles, 40, replace=False):
        j = max(k for k in range(P.n_jobs) if P.jobs[k].tile_base <= t)
        J = P.jobs[j]
        lt = int(t) - J.tile_base
        tx, ty = lt % J.tiles_x, lt // J.tiles_x
        e = np.arange(J.entry_base, J.entry_base + P.scenes[J.scene].n)
        cover = (nt[e] > 0) & (tx0[e] <= tx) & (tx <= tx1[e]) & (ty0[e] <= ty) & (ty <= ty1[e])
        ee = e[cover]
        expect = ee[np.lexsort((ee, dkey[ee]))]
        a, b = rng_t[t]
        got = vals[a:b].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, expect), int(t)


def test_fullsize_backward_on_pixel_subset(full):
    fr, sc, cams = full["fr"], full["sc"], full["cams"]
    rng = np.random.default_rng(13)
    pix, dl_sub, dl_full = [], [], []
    for j, cam in enumerate(cams):
        p = rng.choice(cam.width * cam.height, 120, replace=False).astype(np.int64)
        ref = oracle.render(oracle.project(full["s32"], cam, full["cfgd"]), cam, full["cfgd"], p)
        w = rng.uniform(-1, 1, size=(3, p.size))
        w[:, ref["flags"] != 0] = 0.0
        img = np.zeros((3, cam.width * cam.height), np.float32)
        img[:, p] = w
        pix.append(p)
        dl_sub.append(w)
        dl_full.append(img)
    g = sc.zeros_like()
    fr.backward(torch.as_tensor(np.concatenate([d.reshape(-1) for d in dl_full]), device=DEV), [g])
    torch.cuda.synchronize()
    gref, _, gabs, g2abs = oracle.backward(full["s32"], cams, full["cfgd"], dl_sub, pix, want_grad2d=True,
                                           want_abs=True)
    got = scene_grads_flat(g)
    n = full["scene"]["n"]
    touched = np.count_nonzero(gref[:n])
    assert touched > 1000
    print(assert_groups_close(got, gref, n, 3, gabs, label="full-size", extra=sh_basis_bound(n, 3, g2abs)))
