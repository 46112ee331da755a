"""Parity at the headline size, element by element against the FP64 oracle.

The bench workload (3840x2160 RGB FP32, 4% random mask, channel seeds 1/2/3,
mask seed 1001) in the bench's launch configuration:
  - inpainting (Sec. 2.1) to relative residual 1e-7: max |u - u*| <= 1e-3 on
    every channel, u* from the oracle's FP64 CG (at this size a residual of
    1e-6 alone left 1.4e-3 on channel 0, so the workload solves to 1e-7 to
    meet both gates);
  - tonal optimisation (Sec. 5): the oracle-evaluated relative normal
    residual ||B^T (f - B g)|| / ||B^T f|| of the GPU's g on channel 0;
  - tonal optimisation at 1920x1080 (grey, same generator and density):
    max |g - g*| against the oracle optimum (CG on the normal equations with
    a direct factor of L_UU), within the bound that the oracle-evaluated
    normal residual implies: B^T B = I + S^T S has eigenvalues >= 1, so
    ||g - g*||_2 <= ||B^T (f - B g)||_2 = rel * ||B^T f||_2;
  - the densification loop of the C4 workload (Sec. 4, Alg. 1): eight steps of
    0.5% from the empty mask, each followed by a warm-started re-inpainting;
    after every step the GPU's mask equals, bit for bit, the oracle's step on
    the same previous mask and the same GPU inpainting; then tonal
    optimisation on the final 4% mask, checked by the oracle's normal
    residual on channel 0.

The oracle's solves take minutes at these sizes, so they run in a pool of
worker processes started with `spawn` while the GPU works, and each test
waits for its own result.
"""

import multiprocessing
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
import oracle_jobs as jobs
from synthdata import synth_rgb, synth_image, random_mask

pytestmark = pytest.mark.gpu

H, W = 2160, 3840
SEEDS = (1, 2, 3)
MASK_SEED = 1001
DENSITY = 0.04
TOL = 1e-6
INPAINT_TOL = 1e-7
# tolerances of the accuracy gates; the FP32 output of a 1e-6 solve adds
# its own rounding to the normal residual (as in the smaller tonal tests)
U_TOL = 1e-3
NR_TOL = 2e-6
H2, W2 = 1080, 1920
STEP_SEED = 300
STEPS = 8
ORACLE_TIMEOUT = 1500


@pytest.fixture(scope="module")
def headline():
    """Runs every GPU solve of the module once and submits the oracle jobs
    that check them; returns the GPU results and the oracle futures."""
    need_gpu()
    workers = max(2, min(10, (os.cpu_count() or 2)))
    pool = ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn"))
    fut = {}
    # independent of the GPU: start first
    for ch, s in enumerate(SEEDS):
        fut[("u*", ch)] = pool.submit(jobs.inpaint_channel, H, W, s, DENSITY, MASK_SEED)
    fut["g*1080"] = pool.submit(jobs.tonal_channel_direct, H2, W2, SEEDS[0], DENSITY, MASK_SEED)

    f = synth_rgb(H, W, seeds=SEEDS, dtype=np.float32)
    c = random_mask(H, W, DENSITY, MASK_SEED)
    k = ctx()
    fd, cd = dev(f), dev(c)
    out = {}
    u = torch.empty_like(fd)
    out["inpaint_st"] = k.inpaint(fd, cd, u, tol=INPAINT_TOL)
    out["u"] = u.cpu().numpy()
    g = torch.empty_like(fd)
    out["tonal_st"] = k.tonal_opt(fd, cd, g, tol=TOL)
    out["g"] = g.cpu().numpy()
    fut["nr4k"] = pool.submit(jobs.normal_residual_channel, (H, W, SEEDS[0]), c, out["g"][0])

    # 1920x1080 grey
    f2 = synth_image(H2, W2, SEEDS[0], np.float32)[None]
    c2 = random_mask(H2, W2, DENSITY, MASK_SEED)
    g2 = torch.empty_like(dev(f2))
    out["tonal1080_st"] = k.tonal_opt(dev(f2), dev(c2), g2, tol=TOL)
    out["g1080"] = g2.cpu().numpy()[0]
    out["c1080"] = c2
    fut["nr1080"] = pool.submit(jobs.normal_residual_direct, (H2, W2, SEEDS[0]), c2, out["g1080"])

    # the densification loop, recording every step's input and output
    n = int(round(0.005 * H * W))
    md = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    ud = torch.empty_like(fd)
    masks, added = [], []
    for s in range(STEPS):
        prev = md.cpu().numpy()
        u_prev = None if s == 0 else ud.cpu().numpy()
        added.append(k.densify_step(fd, md, None if s == 0 else ud, n, STEP_SEED))
        new = md.cpu().numpy()
        masks.append(new)
        fut[("step", s)] = pool.submit(jobs.densify_check, (H, W, SEEDS), prev, u_prev, n, STEP_SEED)
        k.inpaint(fd, md, ud, u0=None if s == 0 else ud, tol=TOL)
    gd = torch.empty_like(fd)
    out["c4_tonal_st"] = k.tonal_opt(fd, md, gd, tol=TOL)
    out["c4_g"] = gd.cpu().numpy()
    out["c4_masks"] = masks
    out["c4_added"] = added
    fut["nr_c4"] = pool.submit(jobs.normal_residual_channel, (H, W, SEEDS[0]), masks[-1], out["c4_g"][0])
    torch.cuda.synchronize()
    yield out, fut
    pool.shutdown(wait=False, cancel_futures=True)


def test_inpaint_4k_rgb_matches_oracle(headline):
    out, fut = headline
    assert out["inpaint_st"]["rel_res"] <= INPAINT_TOL
    for ch in range(3):
        ustar = fut[("u*", ch)].result(timeout=ORACLE_TIMEOUT)
        err = float(np.abs(out["u"][ch].astype(np.float64) - ustar).max())
        assert err <= U_TOL, (ch, err)


def test_tonal_4k_rgb_normal_residual_by_oracle(headline):
    out, fut = headline
    assert out["tonal_st"]["rel_res"] <= TOL
    nr = fut["nr4k"].result(timeout=ORACLE_TIMEOUT)
    assert nr <= NR_TOL, nr
    c = random_mask(H, W, DENSITY, MASK_SEED).astype(bool)
    assert np.all(out["g"][:, ~c] == 0.0)


def test_tonal_1080p_matches_oracle_optimum(headline):
    out, fut = headline
    assert out["tonal1080_st"]["rel_res"] <= TOL
    gstar = fut["g*1080"].result(timeout=ORACLE_TIMEOUT)
    nr, btf = fut["nr1080"].result(timeout=ORACLE_TIMEOUT)
    assert nr <= NR_TOL, nr
    diff = out["g1080"].astype(np.float64) - gstar
    # eigenvalues of B^T B are >= 1: ||g - g*||_2 <= nr * ||B^T f||_2
    assert float(np.sqrt(np.sum(diff ** 2))) <= nr * btf * (1 + 1e-6) + 1e-9, (np.sqrt(np.sum(diff ** 2)), nr, btf)
    assert float(np.abs(diff).max()) <= 0.2, float(np.abs(diff).max())
    assert np.all(out["g1080"][out["c1080"] == 0] == 0.0)


def test_densify_loop_4k_bit_exact_every_step(headline):
    out, fut = headline
    n = int(round(0.005 * H * W))
    for s in range(STEPS):
        ref = fut[("step", s)].result(timeout=ORACLE_TIMEOUT)
        np.testing.assert_array_equal(out["c4_masks"][s], ref, err_msg=f"step {s}")
        # the first step dithers (about n pixels); later ones add at most n
        assert out["c4_added"][s] > 0 and (s == 0 or out["c4_added"][s] <= n)


def test_densify_loop_4k_final_tonal_by_oracle(headline):
    out, fut = headline
    assert out["c4_tonal_st"]["rel_res"] <= TOL
    nr = fut["nr_c4"].result(timeout=ORACLE_TIMEOUT)
    assert nr <= NR_TOL, nr
