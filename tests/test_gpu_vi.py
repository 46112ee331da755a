"""Parity of the CUDA Voronoi initialisation of tonal optimisation (Sec. 5.3)
against the FP64 oracle, called through the C ABI (tonal_init = 1)."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import tonal as tonal_ref, B_apply, mse
from oracle.vi import voronoi_init
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu


def run(f, c, tol=1e-6, **params):
    need_gpu()
    k = ctx(**params)
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    st = k.tonal_opt(fd, cd, out, tol=tol)
    return out.cpu().numpy(), st


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("H,W,d,seed", [(77, 131, 0.04, 1), (130, 60, 0.1, 2), (33, 40, 0.02, 3)])
def test_vi_steps_match_oracle(mode, H, W, d, seed):
    """Three Richardson steps with near-exact inpaintings: the same g as the
    oracle (FP32 arithmetic of the weights and errors aside)."""
    f = synth_rgb(H, W, seeds=(seed, seed + 10, seed + 20), dtype=np.float32)
    c = random_mask(H, W, d, seed + 100)
    f64 = f.astype(np.float64)
    ref, hist = voronoi_init(f64, c, max_iter=3, mode=mode, stop_on_rise=True)
    g, st = run(f, c, tonal_init=1, tonal_max_iter=0, vi_max_iter=3, vi_weight=mode, vi_inner_tol=1e-9)
    assert st["init_steps"] == hist["accepted"]
    assert np.abs(g - ref).max() <= 2e-3
    assert np.all(g[:, c == 0] == 0)
    assert abs(st["mse"] - mse(B_apply(ref, c), f64)) <= 1e-4 * st["mse"]


def test_vi_gray_fp64_default_tolerance():
    """Default inner tolerance, run to the stop-on-rise rule: the kept MSE
    matches the oracle's best to 0.1% and the step count to one."""
    f = synth_image(96, 128, 4)
    c = random_mask(96, 128, 0.05, 5)
    ref, hist = voronoi_init(f, c, max_iter=20, mode=0)
    g, st = run(f, c, tonal_init=1, tonal_max_iter=0)
    e_ref = mse(B_apply(ref, c), f)
    e = mse(B_apply(g, c), f)
    assert abs(st["init_steps"] - hist["accepted"]) <= 1
    assert abs(e - e_ref) <= 1e-3 * e_ref
    assert e < hist["mse"][0]


def test_vi_fixed_point_on_generated_data():
    c = random_mask(64, 64, 0.05, 6)
    g0 = np.where(c.astype(bool), synth_image(64, 64, 7), 0.0)
    g, st = run(B_apply(g0, c), c, tonal_init=1, tonal_max_iter=0, vi_inner_tol=1e-10)
    assert np.abs(g - g0).max() <= 1e-5


@pytest.mark.parametrize("method", [0, 1])
def test_vi_then_outer_solver_reaches_the_optimum(method):
    """VI followed by RAS or CGNR to 1e-6: the optimum of the oracle, in no
    more outer iterations than from f."""
    f = synth_rgb(96, 112, seeds=(31, 32, 33), dtype=np.float32)
    c = random_mask(96, 112, 0.04, 34)
    f64 = f.astype(np.float64)
    ref = tonal_ref(f64, c)
    g, st = run(f, c, tonal_init=1, tonal_method=method)
    _, st0 = run(f, c, tonal_method=method)
    assert st["rel_res"] <= 1e-6
    assert np.abs(g - ref).max() <= 0.05
    assert st["iterations"] <= st0["iterations"]
    assert st["init_steps"] >= 1
