"""Parity of the CUDA CGNR tonal optimisation (Sec. 5.1, "Improvements") and
of the MSE-gain stopping rule (Sec. 6) against the FP64 oracle, called
through the C ABI (tonal_method = 1, tonal_mse_gain)."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import tonal as tonal_ref, tonal_cgnr as cgnr_ref, normal_residual, B_apply, inpaint, mse
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu


def run(f, c, tol, allow_not_converged=False, **params):
    need_gpu()
    k = ctx(**params)
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    st = k.tonal_opt(fd, cd, out, tol=tol, allow_not_converged=allow_not_converged)
    return out.cpu().numpy(), st


@pytest.mark.parametrize("H,W,d,seed", [(77, 131, 0.04, 1), (130, 60, 0.1, 2), (40, 33, 0.02, 3)])
def test_cgnr_ragged_rgb_fp32(H, W, d, seed):
    f = synth_rgb(H, W, seeds=(seed, seed + 10, seed + 20), dtype=np.float32)
    c = random_mask(H, W, d, seed + 100)
    g, st = run(f, c, 1e-6, tonal_method=1)
    f64 = f.astype(np.float64)
    ref = tonal_ref(f64, c)
    assert st["rel_res"] <= 1e-6
    assert normal_residual(f64, c, g.astype(np.float64)).max() <= 2e-6
    assert np.abs(g - ref).max() <= 0.05
    assert np.all(g[:, c == 0] == 0)
    assert mse(B_apply(g.astype(np.float64), c), f64) <= mse(inpaint(f64, c), f64)
    assert abs(st["mse"] - mse(B_apply(ref, c), f64)) <= 1e-3 * st["mse"] + 1e-6


def test_cgnr_gray_fp64_tight():
    """128x128 grey FP64, 4% mask: CGNR to relative normal residual 1e-9."""
    f = synth_image(128, 128, 4)
    c = random_mask(128, 128, 0.04, 5)
    g, st = run(f, c, 1e-9, tonal_method=1)
    assert st["rel_res"] <= 1e-9
    assert normal_residual(f, c, g)[0] <= 5e-9
    assert np.abs(g - tonal_ref(f, c)).max() <= 1e-4


def test_cgnr_recovers_generating_values():
    c = random_mask(64, 64, 0.05, 6)
    g0 = np.where(c.astype(bool), synth_image(64, 64, 7), 0.0)
    g, _ = run(B_apply(g0, c), c, 1e-9, tonal_method=1)
    assert np.abs(g - g0).max() <= 1e-4


def test_cgnr_and_ras_reach_the_same_minimiser():
    f = synth_rgb(96, 128, seeds=(11, 12, 13), dtype=np.float32)
    c = random_mask(96, 128, 0.04, 14)
    g_cg, _ = run(f, c, 1e-7, tonal_method=1)
    g_ras, _ = run(f, c, 1e-7)
    assert np.abs(g_cg - g_ras).max() <= 0.02


def test_cgnr_first_iterations_follow_oracle():
    """With inner solves far below the outer residual, the MSE after each of
    the first CGNR iterations matches the oracle's CGNR (exact solves)."""
    f = synth_image(80, 96, 21)
    c = random_mask(80, 96, 0.04, 22)
    _, hist = cgnr_ref(f, c, max_iter=3, rtol=0.0)
    for k in (1, 2, 3):
        _, st = run(f, c, 1e-12, allow_not_converged=True, tonal_method=1, tonal_max_iter=k,
                    tonal_inner_ratio=1e-6, tonal_inner_max=1e-9)
        assert st["iterations"] == k
        assert abs(st["mse"] - hist["mse"][k]) <= 1e-5 * hist["mse"][k]


@pytest.mark.parametrize("method", [0, 1])
def test_mse_gain_stop(method):
    """0.1% MSE-gain rule (Sec. 6): the call stops early, returns success, and
    its MSE is within a few tenths of a percent of the optimum."""
    f = synth_rgb(96, 112, seeds=(31, 32, 33), dtype=np.float32)
    c = random_mask(96, 112, 0.04, 34)
    g, st = run(f, c, 1e-12, tonal_method=method, tonal_mse_gain=1e-3)
    f64 = f.astype(np.float64)
    e_opt = mse(B_apply(tonal_ref(f64, c), c), f64)
    e = mse(B_apply(g.astype(np.float64), c), f64)
    assert st["rel_res"] > 1e-12            # stopped by the MSE rule, not the tolerance
    assert e_opt <= e <= 1.01 * e_opt
    assert abs(st["mse"] - e) <= 1e-3 * e
    if method == 1:
        _, hist = cgnr_ref(f64, c, max_iter=400, rtol=1e-13, mse_gain=1e-3)
        assert abs(st["iterations"] - (len(hist["mse"]) - 1)) <= 1
