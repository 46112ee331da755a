"""Staged row loads (stage_loads bits: the level-0 refinement residual and
restriction copy their next rows into shared memory with cp.async while
they compute the current ones) read the same addresses and do the same
arithmetic as the unstaged loops, so every result is bit-identical:
inpainting, tonal optimisation (both residual forms of Sec. 5.1) and the
batched engine."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu

SIZES = [(77, 131, 3, 0.04), (300, 200, 3, 0.02), (520, 97, 1, 0.05), (1, 40, 1, 0.2), (33, 33, 3, 0.1),
         (260, 390, 3, 0.04)]


def data(H, W, ch, d, seed):
    f = synth_rgb(H, W, seeds=(seed, seed + 1, seed + 2)) if ch == 3 else synth_image(H, W, seed)[None]
    return f.astype(np.float32), random_mask(H, W, d, seed + 7)


@pytest.mark.parametrize("H,W,ch,d", SIZES)
def test_inpaint_staged_equals_unstaged(H, W, ch, d):
    need_gpu()
    f, c = data(H, W, ch, d, 31)
    fd, cd = dev(f), dev(c)
    outs, stats = [], []
    for st in (0, 3):
        o = torch.empty_like(fd)
        stats.append(ctx(stage_loads=st).inpaint(fd, cd, o, tol=1e-7))
        outs.append(o.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    assert stats[0]["iterations"] == stats[1]["iterations"]
    assert stats[0]["rel_res"] == stats[1]["rel_res"]


@pytest.mark.parametrize("method", [0, 1])
def test_tonal_staged_equals_unstaged(method):
    need_gpu()
    f, c = data(180, 250, 3, 0.04, 41)
    fd, cd = dev(f), dev(c)
    outs, stats = [], []
    for st in (0, 3):
        o = torch.empty_like(fd)
        stats.append(ctx(stage_loads=st, tonal_method=method).tonal_opt(fd, cd, o, tol=1e-6))
        outs.append(o.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    assert stats[0]["iterations"] == stats[1]["iterations"] and stats[0]["mse"] == stats[1]["mse"]


def test_engine_staged_equals_unstaged():
    need_gpu()
    import paper_2401_06747_b300 as hdi
    items = [data(*s, 51 + i) for i, s in enumerate(SIZES)]
    res = []
    for st in (0, 3):
        e = hdi.Engine(0, budget_gb=4.0, stage_loads=st)
        outs = []
        for i, (f, c) in enumerate(items):
            o = torch.empty_like(dev(f))
            assert e.submit(dev(f), dev(c), o, tol=1e-7, tag=i)
            outs.append(o)
        n = 0
        while n < len(items):
            n += len(e.step())
        res.append([o.cpu().numpy() for o in outs])
        e.close()
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)
