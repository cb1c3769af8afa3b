"""Pins of the loss oracle (oracle/image_loss.py, Sec. 3.4 loss) against
closed forms, brute force and finite differences -- nothing here re-calls the
oracle to check itself."""
import numpy as np
import pytest

from oracle import image_loss as IL


def _rand_img(rng, c, h, w):
    return rng.uniform(0.0, 1.0, size=(c, h, w))


def test_window_is_the_normalised_gaussian():
    w = IL.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    g = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g /= g.sum()
    assert np.allclose(w, np.outer(g, g), rtol=0, atol=1e-17)
    # ratio of the centre to its neighbour is exp(1 / (2 sigma^2)) per axis
    assert w[5, 5] / w[5, 4] == pytest.approx(np.exp(1.0 / (2 * 1.5 ** 2)), rel=1e-12)


def _brute_window_sum(img, w):
    h, wd = img.shape
    r = w.shape[0] // 2
    out = np.zeros_like(img)
    for i in range(h):
        for j in range(wd):
            acc = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < h and 0 <= jj < wd:  # zero padding
                        acc += w[a + r, b + r] * img[ii, jj]
            out[i, j] = acc
    return out


def test_ssim_map_equals_brute_force_windows():
    rng = np.random.default_rng(0)
    x, y = _rand_img(rng, 2, 9, 13), _rand_img(rng, 2, 9, 13)
    w = IL.gaussian_window()
    want = np.empty_like(x)
    for c in range(2):
        mx, my = _brute_window_sum(x[c], w), _brute_window_sum(y[c], w)
        sx2 = _brute_window_sum(x[c] ** 2, w) - mx ** 2
        sy2 = _brute_window_sum(y[c] ** 2, w) - my ** 2
        sxy = _brute_window_sum(x[c] * y[c], w) - mx * my
        want[c] = ((2 * mx * my + 1e-4) * (2 * sxy + 9e-4)) / ((mx ** 2 + my ** 2 + 1e-4) * (sx2 + sy2 + 9e-4))
    assert np.allclose(IL.ssim_map(x, y), want, rtol=0, atol=1e-13)


def test_identical_images_have_ssim_one_and_zero_gradient():
    rng = np.random.default_rng(1)
    x = _rand_img(rng, 3, 20, 17)
    assert np.allclose(IL.ssim_map(x, x), 1.0, atol=1e-12)
    assert np.abs(IL.ssim_grad_sum(x, x)).max() < 1e-10


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.3, 0.7
    x, y = np.full((1, 30, 31), a), np.full((1, 30, 31), b)
    s = IL.ssim_map(x, y)[0]
    want = (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)  # the variance factor is C2 / C2
    assert np.allclose(s[5:-5, 5:-5], want, rtol=1e-12)
    # at the border the zero padding darkens the windowed means
    assert not np.isclose(s[0, 0], want)


def test_ssim_is_symmetric():
    rng = np.random.default_rng(2)
    x, y = _rand_img(rng, 3, 15, 11), _rand_img(rng, 3, 15, 11)
    assert np.allclose(IL.ssim_map(x, y), IL.ssim_map(y, x), rtol=0, atol=1e-14)


def test_ssim_gradient_against_central_differences():
    rng = np.random.default_rng(3)
    x, y = _rand_img(rng, 3, 12, 14), _rand_img(rng, 3, 12, 14)
    g = IL.ssim_grad_sum(x, y)
    h = 1e-6
    for _ in range(40):
        c, i, j = rng.integers(3), rng.integers(12), rng.integers(14)
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (IL.ssim_map(xp, y).sum() - IL.ssim_map(xm, y).sum()) / (2 * h)
        assert g[c, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_loss_mixing_limits_and_multi_image_averaging():
    rng = np.random.default_rng(4)
    preds = [_rand_img(rng, 3, 10, 12), _rand_img(rng, 3, 7, 5)]
    tgts = [_rand_img(rng, 3, 10, 12), _rand_img(rng, 3, 7, 5)]
    count = 3 * (120 + 35)
    l1_want = (np.abs(preds[0] - tgts[0]).sum() + np.abs(preds[1] - tgts[1]).sum()) / count
    loss0, l1, dssim, g0 = IL.image_loss(preds, tgts, 0.0)
    assert loss0 == pytest.approx(l1_want, rel=1e-14) and l1 == pytest.approx(l1_want, rel=1e-14)
    assert np.array_equal(g0[1], np.sign(preds[1] - tgts[1]) / count)
    loss1, _, dssim1, g1 = IL.image_loss(preds, tgts, 1.0)
    s_mean = (IL.ssim_map(preds[0], tgts[0]).sum() + IL.ssim_map(preds[1], tgts[1]).sum()) / count
    assert loss1 == pytest.approx(1.0 - s_mean, rel=1e-14) and dssim1 == pytest.approx(1.0 - s_mean, rel=1e-14)
    # mixed loss is the affine combination, and so is its gradient
    lm, _, _, gm = IL.image_loss(preds, tgts, 0.2)
    assert lm == pytest.approx(0.8 * loss0 + 0.2 * loss1, rel=1e-13)
    assert np.allclose(gm[0], 0.8 * g0[0] + 0.2 * g1[0], rtol=0, atol=1e-16)


def test_regularizers_closed_forms_and_differences():
    rng = np.random.default_rng(5)
    raw = rng.normal(size=50)
    ls = rng.normal(-3.0, 0.5, size=(3, 50))
    v, g_raw, g_ls = IL.regularizers(raw, ls, 0.01, 0.02)
    assert v == pytest.approx(0.01 * np.abs(np.tanh(raw)).sum() + 0.02 * np.exp(ls).sum(), rel=1e-14)
    # sqrt of the eigenvalues of R S S^T R^T are the scales, for any rotation
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    wq, xq, yq, zq = q
    R = np.array([[1 - 2 * (yq * yq + zq * zq), 2 * (xq * yq - wq * zq), 2 * (xq * zq + wq * yq)],
                  [2 * (xq * yq + wq * zq), 1 - 2 * (xq * xq + zq * zq), 2 * (yq * zq - wq * xq)],
                  [2 * (xq * zq - wq * yq), 2 * (yq * zq + wq * xq), 1 - 2 * (xq * xq + yq * yq)]])
    Sg = R @ np.diag(np.exp(2 * ls[:, 0])) @ R.T
    assert np.allclose(np.sort(np.sqrt(np.linalg.eigvalsh(Sg))), np.sort(np.exp(ls[:, 0])), rtol=1e-10)
    h = 1e-6
    for k in range(5):
        rp, rm = raw.copy(), raw.copy()
        rp[k] += h
        rm[k] -= h
        fd = (IL.regularizers(rp, ls, 0.01, 0.02)[0] - IL.regularizers(rm, ls, 0.01, 0.02)[0]) / (2 * h)
        assert g_raw[k] == pytest.approx(fd, rel=1e-6)
        lp, lm = ls.copy(), ls.copy()
        lp[1, k] += h
        lm[1, k] -= h
        fd = (IL.regularizers(raw, lp, 0.01, 0.02)[0] - IL.regularizers(raw, lm, 0.01, 0.02)[0]) / (2 * h)
        assert g_ls[1, k] == pytest.approx(fd, rel=1e-6)
