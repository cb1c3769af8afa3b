"""FP64 oracle of the training loss of Sec. 3.4 and its gradients.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by the
tests, the smoke check and the benchmark's CPU legs, never by the product.

The loss (Sec. 3.4, after the cited 3DGS-MCMC loss):

    L = (1 - eps_d) L1 + eps_d L_D-SSIM + eps_o sum_i |o_i| + eps_s sum_i sum_j sqrt(lambda_ij)

- L1 = mean |x - y| over every pixel and channel of every image.
- L_D-SSIM = 1 - mean SSIM over every pixel and channel, SSIM as in 3DGS:
  11 x 11 Gaussian window, sigma 1.5, weights normalised to sum 1, zero
  padding outside the image ("same" size), C1 = 0.01^2, C2 = 0.03^2,

      S = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx2 + sy2 + C2))

  with mx = w * x, sx2 = w * x^2 - mx^2, sxy = w * (x y) - mx my (* the
  windowed sum, a library correlation here).
- lambda_ij are the eigenvalues of Sigma_i = R S S^T R^T, so sqrt(lambda_ij)
  = exp(log_scale_ij); o_i = tanh(opacity_raw_i).

Gradient of the D-SSIM term: with a = dS/dmx - 2 mx dS/dsx2 - my dS/dsxy,
b = dS/dsx2, c = dS/dsxy at every output pixel (the partials holding the
other statistics fixed), dS_total/dx(q) = (w * a)(q) + 2 x(q) (w * b)(q) +
y(q) (w * c)(q), the window being symmetric.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WINDOW = 11
SIGMA = 1.5


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """2D window: outer product of the normalised 1D Gaussian."""
    k = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def window_sum(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Windowed weighted sum of a 2D image, zero outside ("same" size)."""
    return correlate(np.asarray(img, np.float64), w, mode="constant", cval=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray, w=None) -> np.ndarray:
    """Per-pixel SSIM of two [C][H][W] images."""
    w = gaussian_window() if w is None else w
    out = np.empty(x.shape, np.float64)
    for c in range(x.shape[0]):
        xc, yc = np.asarray(x[c], np.float64), np.asarray(y[c], np.float64)
        mx, my = window_sum(xc, w), window_sum(yc, w)
        sx2 = window_sum(xc * xc, w) - mx * mx
        sy2 = window_sum(yc * yc, w) - my * my
        sxy = window_sum(xc * yc, w) - mx * my
        out[c] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx2 + sy2 + C2))
    return out


def ssim_grad_sum(x: np.ndarray, y: np.ndarray, w=None) -> np.ndarray:
    """d(sum over pixels and channels of SSIM)/dx for one [C][H][W] image."""
    w = gaussian_window() if w is None else w
    g = np.empty(x.shape, np.float64)
    for c in range(x.shape[0]):
        xc, yc = np.asarray(x[c], np.float64), np.asarray(y[c], np.float64)
        mx, my = window_sum(xc, w), window_sum(yc, w)
        sx2 = window_sum(xc * xc, w) - mx * mx
        sy2 = window_sum(yc * yc, w) - my * my
        sxy = window_sum(xc * yc, w) - mx * my
        A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
        B1, B2 = mx * mx + my * my + C1, sx2 + sy2 + C2
        S = A1 * A2 / (B1 * B2)
        dS_dmx = S * (2 * my / A1 - 2 * mx / B1)
        dS_dsx2 = -S / B2
        dS_dsxy = 2 * S / A2
        a = dS_dmx - 2 * mx * dS_dsx2 - my * dS_dsxy
        g[c] = window_sum(a, w) + 2 * xc * window_sum(dS_dsx2, w) + yc * window_sum(dS_dsxy, w)
    return g


def image_loss(preds, targets, eps_d: float):
    """(1 - eps_d) L1 + eps_d (1 - mean SSIM) over a list of [C][H][W] images
    (means over all their pixels and channels together) and its gradient
    with respect to every prediction.  Returns (loss, l1, dssim, [grads])."""
    count = sum(p.size for p in preds)
    l1 = sum(np.abs(np.asarray(p, np.float64) - t).sum() for p, t in zip(preds, targets)) / count
    s_sum = sum(ssim_map(p, t).sum() for p, t in zip(preds, targets))
    dssim = 1.0 - s_sum / count
    grads = []
    for p, t in zip(preds, targets):
        g1 = np.sign(np.asarray(p, np.float64) - t) / count
        gs = -ssim_grad_sum(p, t) / count
        grads.append((1.0 - eps_d) * g1 + eps_d * gs)
    return (1.0 - eps_d) * l1 + eps_d * dssim, l1, dssim, grads


def regularizers(opacity_raw, log_scale, eps_o: float, eps_s: float):
    """eps_o sum |tanh(raw)| + eps_s sum exp(log_scale) and its gradients
    (d/draw = eps_o sign(o) (1 - o^2), d/dlog_scale = eps_s exp(log_scale))."""
    o = np.tanh(np.asarray(opacity_raw, np.float64))
    s = np.exp(np.asarray(log_scale, np.float64))
    value = eps_o * np.abs(o).sum() + eps_s * s.sum()
    return value, eps_o * np.sign(o) * (1.0 - o * o), eps_s * s
