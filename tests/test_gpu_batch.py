"""Batched inpainting (hdi_inpaint_batch): images of uneven size, channel count
and mask density in one call; each result is checked against the oracle and
against the single-image entry point."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import inpaint as inpaint_ref, rel_residual
from synthdata import synth_image, synth_rgb, random_mask, batch_specs

pytestmark = pytest.mark.gpu


def make(spec):
    H, W, ch = spec["height"], spec["width"], spec["channels"]
    s = spec["seed"]
    f = synth_rgb(H, W, seeds=(s, s + 1000, s + 2000)) if ch == 3 else synth_image(H, W, s)[None]
    return f.astype(np.float32), random_mask(H, W, spec["density"], s + 5000)


def test_uneven_batch_matches_oracle():
    need_gpu()
    specs = [dict(height=h, width=w, channels=c, density=d, seed=i)
             for i, (h, w, c, d) in enumerate([(96, 128, 3, 0.04), (96, 128, 1, 0.08), (50, 70, 1, 0.02),
                                               (96, 128, 3, 0.01), (200, 64, 3, 0.05), (33, 33, 1, 0.1),
                                               (50, 70, 3, 0.05), (1, 40, 1, 0.2)])]
    data = [make(s) for s in specs]
    k = ctx()
    fs = [dev(f) for f, _ in data]
    ms = [dev(c) for _, c in data]
    outs = [torch.empty_like(x) for x in fs]
    st = k.inpaint_batch(fs, ms, outs, tol=1e-6)
    for (f, c), o, s in zip(data, outs, st):
        u = o.cpu().numpy().astype(np.float64)
        ref = inpaint_ref(f.astype(np.float64), c)
        assert s["rel_res"] <= 1e-6
        assert rel_residual(u, f.astype(np.float64), c).max() <= 1.5e-6
        assert np.abs(u - ref).max() <= 1e-3
    # same answers as one-by-one solves, within the solver tolerance
    for (f, c), o in zip(data, outs):
        single = torch.empty_like(o)
        k.inpaint(dev(f), dev(c), single, tol=1e-6)
        assert (single - o).abs().max().item() <= 1e-3


def test_batch_specs_sample_host_buffers():
    """A sample of the 64-image workload (sizes, grey/RGB, densities 1-10%),
    passed as host arrays."""
    need_gpu()
    specs = [s for s in batch_specs(64, 200) if s["width"] * s["height"] <= 1024 * 768][:6]
    data = [make(s) for s in specs]
    k = ctx()
    outs = [np.empty_like(f) for f, _ in data]
    st = k.inpaint_batch([f for f, _ in data], [c for _, c in data], outs, tol=1e-6)
    for (f, c), o, s in zip(data, outs, st):
        assert s["rel_res"] <= 1e-6
        assert rel_residual(o.astype(np.float64), f.astype(np.float64), c).max() <= 1.5e-6


def test_batch_mixed_dtypes_keep_fp64_data_exact():
    """FP32 and FP64 images of one size class in one batch: the FP64 image's
    data words below FP32 precision are used (its known pixels come back
    bit for bit, its residual meets the tolerance) although the other images
    of the system are FP32."""
    need_gpu()
    H, W = 96, 128
    a = synth_rgb(H, W, seeds=(71, 72, 73))                    # FP32
    b = synth_image(H, W, 74)[None]                            # FP64, not FP32-representable
    c = synth_image(H, W, 75).astype(np.float32)[None]         # FP32
    ms = [random_mask(H, W, 0.05, s) for s in (76, 77, 78)]
    assert np.any(b != b.astype(np.float32))
    k = ctx()
    fs = [dev(a), dev(b), dev(c)]
    outs = [torch.empty_like(x) for x in fs]
    st = k.inpaint_batch(fs, [dev(m) for m in ms], outs, tol=1e-6)
    for f, m, o, s in zip((a, b, c), ms, outs, st):
        u = o.cpu().numpy().astype(np.float64)
        assert s["rel_res"] <= 1e-6
        assert rel_residual(u, f.astype(np.float64), m).max() <= 1.5e-6
        assert np.abs(u - inpaint_ref(f.astype(np.float64), m)).max() <= 1e-3
    ub = outs[1].cpu().numpy()
    known = ms[1].astype(bool)
    assert np.array_equal(ub[0][known], b[0][known])
