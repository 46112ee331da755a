"""Oracle computations for the full-size parity tests, run in worker
processes started with `spawn` (never forked from a process that has
touched the GPU). Every function here calls only `oracle/` and `synthdata/`;
the GPU results they check arrive as NumPy arrays.

Inputs are regenerated in the worker from their seeds (cheaper than sending
them) and cached per process.
"""

from __future__ import annotations

import numpy as np

_cache: dict = {}


def _image(H: int, W: int, seed: int) -> np.ndarray:
    """One FP32 channel of the synthetic generator, widened to FP64 (the
    GPU solves the FP32 image exactly as stored)."""
    from synthdata import synth_image
    key = ("img", H, W, seed)
    if key not in _cache:
        _cache[key] = synth_image(H, W, seed, np.float32).astype(np.float64)
    return _cache[key]


def _rgb(H: int, W: int, seeds) -> np.ndarray:
    from synthdata import synth_rgb
    key = ("rgb", H, W, tuple(seeds))
    if key not in _cache:
        _cache[key] = synth_rgb(H, W, seeds=tuple(seeds), dtype=np.float32).astype(np.float64)
    return _cache[key]


def _mask(H: int, W: int, density: float, seed: int) -> np.ndarray:
    from synthdata import random_mask
    key = ("mask", H, W, density, seed)
    if key not in _cache:
        _cache[key] = random_mask(H, W, density, seed)
    return _cache[key]


def inpaint_channel(H: int, W: int, seed: int, density: float, mask_seed: int) -> np.ndarray:
    """u* = A^{-1} C f for one channel (Sec. 2.1), FP64 CG to 1e-13 above
    the oracle's direct-solver size."""
    from oracle import inpaint
    return inpaint(_image(H, W, seed), _mask(H, W, density, mask_seed))


def tonal_channel_direct(H: int, W: int, seed: int, density: float, mask_seed: int) -> np.ndarray:
    """g* of one channel (Sec. 5): CG on (I + S^T S) g_K = f_K - S^T f_U to
    1e-14, every S / S^T application through one SuperLU factor of L_UU
    (the oracle's direct solver, allowed up to this image size here)."""
    import oracle.laplace as lp
    from oracle import tonal
    lp.DIRECT_MAX = max(lp.DIRECT_MAX, H * W)
    return tonal(_image(H, W, seed), _mask(H, W, density, mask_seed))


def normal_residual_channel(f_args: tuple, c: np.ndarray, g: np.ndarray) -> float:
    """||B^T (f - B g)|| / ||B^T f|| of one channel (Sec. 5.1), each B and
    B^T application an FP64 solve of the oracle. f_args = (H, W, seed)."""
    from oracle import normal_residual
    f = _image(*f_args)
    return float(normal_residual(f, c, np.asarray(g, np.float64))[0])


def densify_check(rgb_args: tuple, c: np.ndarray, u: np.ndarray | None, k: int, seed: int) -> np.ndarray:
    """One densification step of the oracle (Sec. 4.1, Alg. 1; the dithered
    initial mask of Sec. 4.2 when c is empty) on the given mask and
    inpainting. rgb_args = (H, W, seeds)."""
    from oracle.densify import densify_step, initial_mask
    f = _rgb(*rgb_args)
    if u is None:
        return initial_mask(f, k, seed)
    out, _ = densify_step(f, c, np.asarray(u, np.float64), k, seed)
    return out


def normal_residual_direct(f_args: tuple, c: np.ndarray, g: np.ndarray):
    """(relative normal residual of g, ||B^T f||_2) for one channel, every
    solve through one SuperLU factor of L_UU. f_args = (H, W, seed)."""
    import oracle.laplace as lp
    from oracle import normal_residual, Bt_apply
    H, W = f_args[0], f_args[1]
    lp.DIRECT_MAX = max(lp.DIRECT_MAX, H * W)
    f = _image(*f_args)
    nr = float(normal_residual(f, c, np.asarray(g, np.float64))[0])
    btf = float(np.sqrt(np.sum(Bt_apply(f, c) ** 2)))
    return nr, btf
