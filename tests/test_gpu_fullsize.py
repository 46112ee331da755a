"""Full-size checks on the workload bench.py times (3840x2160 RGB FP32, 4%
random mask, seeds as in the bench) in the same launch configuration (one
context, device buffers, tol 1e-6).

The oracle cannot solve 8.3M-unknown problems in seconds, so the solver
outputs are checked by properties that hold at any size, evaluated on the CPU
with the oracle's own operator: the relative residual of the returned u,
exact data on the mask, the discrete maximum principle, and for tonal
optimisation the support of g, the residual of its inpainting and an MSE not
above that of the untuned data. Densification steps are cheap for the oracle
at full size and are compared bit for bit (Sec. 4.1, Alg. 1)."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import rel_residual
from oracle.densify import initial_mask as initial_ref, densify_step as densify_ref
from synthdata import synth_rgb, random_mask

pytestmark = pytest.mark.gpu

H, W = 2160, 3840
SEEDS = (1, 2, 3)
MASK_SEED = 1001
DENSITY = 0.04
TOL = 1e-6
# the FP32 output adds its own rounding to the FP64-accurate solve
RES_TOL = 1.5e-6


@pytest.fixture(scope="module")
def workload():
    need_gpu()
    f = synth_rgb(H, W, seeds=SEEDS, dtype=np.float32)
    c = random_mask(H, W, DENSITY, MASK_SEED)
    return f, c


def inpaint_gpu(k, f, c):
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    st = k.inpaint(fd, cd, out, tol=TOL)
    return out.cpu().numpy(), st


def test_inpaint_4k_rgb(workload):
    f, c = workload
    k = ctx()
    u, st = inpaint_gpu(k, f, c)
    assert st["rel_res"] <= TOL
    assert np.all(rel_residual(u.astype(np.float64), f.astype(np.float64), c) <= RES_TOL)
    known = c.astype(bool)
    np.testing.assert_array_equal(u[:, known], f[:, known])
    for ch in range(3):
        lo, hi = f[ch][known].min(), f[ch][known].max()
        assert u[ch].min() >= lo - 1e-3 and u[ch].max() <= hi + 1e-3


def test_tonal_4k_rgb(workload):
    f, c = workload
    k = ctx()
    fd, cd = dev(f), dev(c)
    g = torch.empty_like(fd)
    st = k.tonal_opt(fd, cd, g, tol=TOL)
    assert st["rel_res"] <= TOL
    g = g.cpu().numpy()
    known = c.astype(bool)
    assert np.all(g[:, ~known] == 0.0)
    ug, _ = inpaint_gpu(k, g, c)
    assert np.all(rel_residual(ug.astype(np.float64), g.astype(np.float64), c) <= RES_TOL)
    uf, _ = inpaint_gpu(k, f, c)
    mse_g = float(np.mean((ug.astype(np.float64) - f) ** 2))
    mse_f = float(np.mean((uf.astype(np.float64) - f) ** 2))
    assert mse_g < mse_f
    assert abs(mse_g - st["mse"]) <= 1e-4 * mse_g


def test_densify_4k_rgb_bit_exact(workload):
    """Initial dithered mask and one densification step at full size; the
    step takes the GPU's own inpainting as u on both sides."""
    f, _ = workload
    k = ctx()
    n = int(round(0.005 * H * W))
    fd = dev(f)
    md = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    k.densify_step(fd, md, None, n, 300)
    m1 = md.cpu().numpy()
    np.testing.assert_array_equal(m1, initial_ref(f.astype(np.float64), n, 300))
    u1, _ = inpaint_gpu(k, f, m1)
    k.densify_step(fd, md, dev(u1), n, 300)
    m2 = md.cpu().numpy()
    ref, _ = densify_ref(f.astype(np.float64), m1, u1.astype(np.float64), n, 300)
    np.testing.assert_array_equal(m2, ref)
    assert m2.sum() > m1.sum()
