"""Voronoi initialisation of tonal optimisation (paper Sec. 5.3), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The mask pixels are asked to interpolate local averages of f rather than f
itself: with a weight matrix W whose row for mask pixel s averages over an
"influence zone" of s,

    C W A^{-1} C g = C W u = C W f                 (Sec. 5.3, average interpolation)

solved by the modified Richardson iteration

    C g^{k+1} = C g^k + tau C W (f - A^{-1} C g^k),

one inpainting per step, stopped as soon as the MSE of the inpainting rises
(the surrogate is not the tonal problem itself); the best iterate is kept.

Readings (the paper does not print them):
  * the residual of the Richardson step is C W f - C W u (the printed "C f"
    would not have the average-interpolation system as its fixed point, and
    only C W f reproduces the error-balancing rule of Galic et al. for tau = 1);
  * influence zones, `mode`:
      0  the Voronoi cell of s (exact labels, ties to the lowest site index),
         weight 1 / (1 + ln(1 + d)) with d the Euclidean distance from the
         pixel to s ("inverse logarithmic distance weighting");
      1  the Voronoi cell of s, constant weight;
      2  the 3x3 neighbourhood of s clipped to the image, constant weight
         (error balancing, Galic et al., the paper's "direct neighbours"
         including s itself);
    every row of W is normalised to sum 1;
  * colour: W acts on every channel separately; the stopping test uses the
    MSE over all channels;
  * tau = 1 (the error-balancing step); a rising MSE stops the iteration.
"""

from __future__ import annotations

import numpy as np

from .densify import voronoi_labels
from .laplace import _as_channels
from .tonal import B_apply


def zone_weights(c: np.ndarray, mode: int = 0):
    """(V, w): the Voronoi label V(p) (linear site index) and the weight w_p
    of every pixel for modes 0 and 1."""
    cb = np.asarray(c, dtype=bool)
    H, W = cb.shape
    V = voronoi_labels(cb)
    if mode == 1:
        return V, np.ones((H, W))
    py, px = np.divmod(np.arange(H * W), W)
    sy, sx = np.divmod(V.ravel(), W)
    d = np.sqrt((px - sx) ** 2.0 + (py - sy) ** 2.0).reshape(H, W)
    return V, 1.0 / (1.0 + np.log1p(d))


def apply_W(e: np.ndarray, c: np.ndarray, mode: int = 0, zones=None) -> np.ndarray:
    """(W e)_s at every mask pixel s (zero elsewhere), per channel."""
    e3 = _as_channels(e).astype(np.float64)
    cb = np.asarray(c, dtype=bool)
    H, Wd = cb.shape
    out = np.zeros_like(e3)
    if mode == 2:
        for y, x in zip(*np.nonzero(cb)):
            y0, y1, x0, x1 = max(y - 1, 0), min(y + 2, H), max(x - 1, 0), min(x + 2, Wd)
            out[:, y, x] = e3[:, y0:y1, x0:x1].mean(axis=(1, 2))
    else:
        V, w = zones if zones is not None else zone_weights(cb, mode)
        lab = V.ravel()
        den = np.bincount(lab, weights=w.ravel(), minlength=H * Wd)
        for ch in range(e3.shape[0]):
            num = np.bincount(lab, weights=(w * e3[ch]).ravel(), minlength=H * Wd)
            sites = np.flatnonzero(cb.ravel())
            o = np.zeros(H * Wd)
            o[sites] = num[sites] / den[sites]
            out[ch] = o.reshape(H, Wd)
    return out if np.ndim(e) == 3 else out[0]


def voronoi_init(f: np.ndarray, c: np.ndarray, max_iter: int = 20, tau: float = 1.0, mode: int = 0,
                 stop_on_rise: bool = True):
    """Richardson iteration on the average-interpolation system from g = f on
    the mask. Returns (g, history): g the iterate with the lowest MSE reached
    before the MSE first rose (all max_iter steps without stop_on_rise),
    history["mse"] the MSE of every computed inpainting (the last one may be
    the rejected step) and history["accepted"] the number of steps kept."""
    f3 = _as_channels(f).astype(np.float64)
    cb = np.asarray(c, dtype=bool)
    zones = None if mode == 2 else zone_weights(cb, mode)
    g = f3 * cb
    u = B_apply(g, cb)
    err = float(np.mean((f3 - u) ** 2))
    hist = {"mse": [err], "accepted": 0}
    for _ in range(max_iter):
        r = apply_W(f3 - u, cb, mode, zones)
        g_new = (g + tau * r) * cb
        u_new = B_apply(g_new, cb)
        err_new = float(np.mean((f3 - u_new) ** 2))
        hist["mse"].append(err_new)
        if stop_on_rise and err_new > err:
            break
        g, u, err = g_new, u_new, err_new
        hist["accepted"] += 1
    return (g if np.ndim(f) == 3 else g[0]), hist
