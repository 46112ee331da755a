"""Parity of the CUDA tonal optimisation (RAS, Alg. 2) against the FP64
oracle (CG on the normal equations), called through the C ABI."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import tonal as tonal_ref, normal_residual, B_apply, inpaint, mse
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu


def run(f, c, tol, g0=None, **params):
    need_gpu()
    k = ctx(**params)
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    st = k.tonal_opt(fd, cd, out, g0=None if g0 is None else dev(g0), tol=tol)
    return out.cpu().numpy(), st


def test_c1_256_gray_fp64_tight():
    """256x256 grey FP64, 4% mask: normal equations to relative residual 1e-10."""
    f = synth_image(256, 256, 0)
    c = random_mask(256, 256, 0.04, 1000)
    g, st = run(f, c, 1e-10)
    ref = tonal_ref(f, c)
    assert st["rel_res"] <= 1e-10
    assert normal_residual(f, c, g)[0] <= 2e-10
    assert np.abs(g - ref).max() <= 1e-5
    assert np.all(g[c == 0] == 0)


@pytest.mark.parametrize("H,W,d,seed", [(77, 131, 0.04, 1), (130, 60, 0.1, 2), (40, 33, 0.02, 3)])
def test_ragged_rgb_fp32(H, W, d, seed):
    f = synth_rgb(H, W, seeds=(seed, seed + 10, seed + 20), dtype=np.float32)
    c = random_mask(H, W, d, seed + 100)
    g, st = run(f, c, 1e-6)
    f64 = f.astype(np.float64)
    ref = tonal_ref(f64, c)
    assert st["rel_res"] <= 1e-6
    assert normal_residual(f64, c, g.astype(np.float64)).max() <= 2e-6
    assert np.abs(g - ref).max() <= 0.05
    # never worse than the unoptimised values (Sec. 5)
    assert mse(B_apply(g.astype(np.float64), c), f64) <= mse(inpaint(f64, c), f64)
    assert abs(st["mse"] - mse(B_apply(ref, c), f64)) <= 1e-3 * st["mse"] + 1e-6


def test_generated_data_is_recovered():
    c = random_mask(64, 64, 0.05, 6)
    g0 = np.where(c.astype(bool), synth_image(64, 64, 7), 0.0)
    fb = B_apply(g0, c)
    g, _ = run(fb, c, 1e-9)
    assert np.abs(g - g0).max() <= 1e-4


def test_bitwise_determinism_across_contexts_and_history():
    """Same input, different contexts and call histories: identical g. The
    89 x 158 size makes the border subdomains overlap their same-parity
    neighbours, which the local-phase colouring must keep race-free."""
    need_gpu()
    f = synth_rgb(89, 158, seeds=(7, 8, 9), dtype=np.float32)
    c = random_mask(89, 158, 0.05, 10)
    a = ctx()
    g1 = torch.empty_like(dev(f))
    a.tonal_opt(dev(f), dev(c), g1, tol=1e-6)
    b = ctx()
    other = dev(synth_rgb(37, 61, seeds=(1, 2, 3), dtype=np.float32))
    b.tonal_opt(other, dev(random_mask(37, 61, 0.05, 3)), torch.empty_like(other), tol=1e-6)
    g2 = torch.empty_like(g1)
    b.tonal_opt(dev(f), dev(c), g2, tol=1e-6)
    g3 = torch.empty_like(g1)
    a.tonal_opt(dev(f), dev(c), g3, tol=1e-6)
    assert torch.equal(g1, g2) and torch.equal(g1, g3)


@pytest.mark.parametrize("H,W,d,block", [(96, 128, 0.15, 0), (90, 110, 0.05, 40)])
def test_dense_subdomains(H, W, d, block):
    """Subdomains above 128 mask pixels take the global-memory factorisation:
    15% density (the top of the paper's range), and a fully known 40 x 40
    block (subdomains with up to all 1024 pixels on the mask)."""
    f = synth_rgb(H, W, seeds=(31, 32, 33), dtype=np.float32)
    c = random_mask(H, W, d, 77)
    if block:
        c[20:20 + block, 30:30 + block] = 1
    g, st = run(f, c, 1e-6)
    f64 = f.astype(np.float64)
    ref = tonal_ref(f64, c)
    assert st["rel_res"] <= 1e-6
    assert normal_residual(f64, c, g.astype(np.float64)).max() <= 2e-6
    assert np.abs(g - ref).max() <= 0.05
    assert np.all(g[:, c == 0] == 0)


@pytest.mark.parametrize("H,W,d,seed", [(150, 210, 0.005, 31), (77, 131, 0.02, 32), (130, 60, 0.1, 33),
                                        (40, 50, 0.05, 34)])
def test_block64_reaches_the_optimum(H, W, d, seed):
    """RAS on 64x64 subdomains (the paper's block size, tonal_block = 64): the
    same minimiser as the oracle, including images narrower than a block."""
    f = synth_rgb(H, W, seeds=(seed, seed + 10, seed + 20), dtype=np.float32)
    c = random_mask(H, W, d, seed + 100)
    if c.sum() == 0:
        c[H // 2, W // 2] = 1
    g, st = run(f, c, 1e-6, tonal_block=64)
    f64 = f.astype(np.float64)
    ref = tonal_ref(f64, c)
    assert st["rel_res"] <= 1e-6
    assert normal_residual(f64, c, g.astype(np.float64)).max() <= 2e-6
    assert np.abs(g - ref).max() <= 0.05
    assert np.all(g[:, c == 0] == 0)


def test_block64_gray_fp64_tight():
    f = synth_image(200, 180, 35)
    c = random_mask(200, 180, 0.01, 36)
    g, st = run(f, c, 1e-10, tonal_block=64)
    assert st["rel_res"] <= 1e-10
    assert np.abs(g - tonal_ref(f, c)).max() <= 1e-5


def test_block64_falls_back_on_a_densely_known_block():
    """A fully known 70x70 region at 1% density elsewhere: some 64x64 block holds
    more than 1024 mask pixels, so the call runs on 32x32 blocks; the result is
    still the optimum."""
    H, W = 160, 200
    f = synth_rgb(H, W, seeds=(41, 42, 43), dtype=np.float32)
    c = random_mask(H, W, 0.01, 44)
    c[40:110, 60:130] = 1
    g, st = run(f, c, 1e-6, tonal_block=64)
    f64 = f.astype(np.float64)
    assert st["rel_res"] <= 1e-6
    assert np.abs(g - tonal_ref(f64, c)).max() <= 0.05


@pytest.mark.parametrize("d,seed", [(0.02, 12), (0.04, 13)])
def test_plain_alg2_64x64_reaches_the_optimum_at_the_oracle_rate(d, seed):
    """The paper's RAS iteration without acceleration (tonal_anderson = 0,
    Sec. 5.2, Alg. 2) on its 64x64 blocks with overlap 6: the GPU reaches the
    oracle optimum, in the number of iterations the oracle's Alg. 2 (exact
    local solves, exact B and B^T) needs for the same tolerance, give or take
    the effect of the GPU's inexact inner solves."""
    from oracle.ras import RASTonal
    H, W = 200, 180
    f = synth_image(H, W, 11)
    c = random_mask(H, W, d, seed)
    tol = 1e-9
    g, st = run(f, c, tol, tonal_anderson=0, tonal_block=64)
    ref = tonal_ref(f, c)
    assert st["rel_res"] <= tol
    assert normal_residual(f, c, g)[0] <= 2 * tol
    assert np.abs(g - ref).max() <= 1e-4
    assert np.all(g[c == 0] == 0)
    _, hist = RASTonal(c, size=64).run(f, 80)
    need = int(np.argmax(hist[:, 0] <= tol))
    assert hist[need, 0] <= tol
    assert abs(st["iterations"] - need) <= 2, (st["iterations"], need)


@pytest.mark.parametrize("oras_warp", [0, 1])
@pytest.mark.parametrize("H,W,d,seed", [(150, 210, 0.04, 21), (31, 70, 0.05, 22)])
def test_echo_layouts_reach_the_optimum(oras_warp, H, W, d, seed):
    """The local echoes S e_k of Sec. 5.2 (Neumann subdomain solves on 32x32
    RAS blocks, 3% density and above) in both kernel layouts -- one warp per
    echo (oras_warp = 1) and two warps (0) -- including images lower than
    one block: RAS reaches the oracle optimum with either, FP64 to 1e-10."""
    f = synth_image(H, W, seed)
    c = random_mask(H, W, d, seed + 100)
    g, st = run(f, c, 1e-10, oras_warp=oras_warp, tonal_block=32)
    assert st["rel_res"] <= 1e-10
    assert normal_residual(f, c, g)[0] <= 2e-10
    assert np.abs(g - tonal_ref(f, c)).max() <= 1e-5
    assert np.all(g[c == 0] == 0)


@pytest.mark.parametrize("method", [0, 1])
def test_host_buffers_equal_device_buffers(method):
    """Tonal optimisation from host memory: f (pageable NumPy or pinned) is
    copied on a side stream while the local factors (mask only) are computed;
    the result equals the one from device buffers bit for bit, and a second
    call on the same context reuses the staging correctly."""
    need_gpu()
    f = synth_rgb(160, 230, seeds=(71, 72, 73), dtype=np.float32)
    c = random_mask(160, 230, 0.04, 74)
    k = ctx(tonal_method=method)
    ref = torch.empty((3, 160, 230), dtype=torch.float32, device="cuda")
    k.tonal_opt(dev(f), dev(c), ref, tol=1e-6)
    ref = ref.cpu().numpy()
    for host_f in (f, torch.from_numpy(f).pin_memory()):
        out = np.zeros_like(f)
        k.tonal_opt(host_f, c, out, tol=1e-6)
        np.testing.assert_array_equal(out, ref)
