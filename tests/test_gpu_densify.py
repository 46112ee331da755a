"""Parity of the CUDA densification step (Sec. 4.1, Alg. 1; initial mask of
Sec. 4.2) against the oracle: new mask bits must match exactly."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import inpaint as inpaint_ref
from oracle.densify import densify_step as densify_ref, initial_mask
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu


def gpu_step(f, c, u, k, seed=0, host=False):
    need_gpu()
    kx = ctx()
    if host:
        m = np.ascontiguousarray(c.copy())
        added = kx.densify_step(f, m, u, k, seed)
        return m, added
    md = dev(c.copy())
    added = kx.densify_step(dev(f), md, None if u is None else dev(u), k, seed)
    return md.cpu().numpy(), added


@pytest.mark.parametrize("H,W,ch,dtype,k,seed", [(77, 131, 3, np.float32, 60, 5), (200, 150, 1, np.float64, 300, 9),
                                                 (33, 40, 3, np.float32, 2000, 1), (1, 64, 1, np.float64, 5, 2)])
def test_initial_mask_bit_exact(H, W, ch, dtype, k, seed):
    f = synth_rgb(H, W, seeds=tuple(range(seed, seed + ch)), dtype=dtype) if ch == 3 else synth_image(H, W, seed).astype(dtype)
    c = np.zeros((H, W), np.uint8)
    m, added = gpu_step(f, c, None, k, seed)
    ref = initial_mask(f.astype(np.float64), k, seed)
    np.testing.assert_array_equal(m, ref)
    assert added == int(ref.sum())


@pytest.mark.parametrize("H,W,ch,dtype,d,k", [(96, 128, 3, np.float32, 0.02, 40), (300, 200, 1, np.float64, 0.005, 150),
                                              (64, 80, 3, np.float32, 0.05, 10000), (130, 70, 1, np.float32, 0.01, 0)])
def test_step_bit_exact(H, W, ch, dtype, d, k):
    f = synth_rgb(H, W, seeds=(4, 5, 6), dtype=dtype) if ch == 3 else synth_image(H, W, 4).astype(dtype)
    c = random_mask(H, W, d, 17)
    u = inpaint_ref(f.astype(np.float64), c).astype(dtype)
    m, added = gpu_step(f, c, u, k)
    ref, ref_added = densify_ref(f.astype(np.float64), c, u.astype(np.float64), k)
    np.testing.assert_array_equal(m, ref)
    assert added == ref_added
    assert np.all(m >= c)


def test_edge_cases():
    f = synth_image(40, 30, 3)
    one = np.zeros((40, 30), np.uint8)
    one[10, 12] = 1
    u = np.full_like(f, f[10, 12])
    m, a = gpu_step(f, one, u, 7)
    ref, ra = densify_ref(f, one, u, 7)
    np.testing.assert_array_equal(m, ref)
    assert a == ra
    full = np.ones((40, 30), np.uint8)
    m, a = gpu_step(f, full, f, 5)
    assert a == 0 and np.all(m == 1)
    row = synth_image(1, 50, 8)
    cr = random_mask(1, 50, 0.1, 3)
    ur = inpaint_ref(row, cr)
    m, a = gpu_step(row, cr, ur, 3)
    ref, ra = densify_ref(row, cr, ur, 3)
    np.testing.assert_array_equal(m, ref)


def test_host_buffers():
    f = synth_rgb(50, 60, seeds=(1, 2, 3), dtype=np.float32)
    c = random_mask(50, 60, 0.03, 2)
    u = inpaint_ref(f.astype(np.float64), c).astype(np.float32)
    m, a = gpu_step(f, c, u, 12, host=True)
    ref, ra = densify_ref(f.astype(np.float64), c, u.astype(np.float64), 12)
    np.testing.assert_array_equal(m, ref)


def test_densify_loop_matches_oracle_loop():
    """Empty mask -> 0.5% steps up to 3%, re-inpainting after each step on
    each side (GPU solver vs oracle solver, FP64 data, tight tolerance)."""
    need_gpu()
    H, W = 192, 256
    f = synth_rgb(H, W, seeds=(1, 2, 3)).astype(np.float64)
    N = H * W
    kx = ctx()
    fd = dev(f)
    cg = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    co = np.zeros((H, W), np.uint8)
    ug = torch.empty_like(fd)
    uo = None
    for s in range(1, 7):
        k = int(s * 0.005 * N) - int(co.sum())
        kx.densify_step(fd, cg, None if s == 1 else ug, k, 300)
        co, _ = densify_ref(f, co, uo, k, 300)
        np.testing.assert_array_equal(cg.cpu().numpy(), co, err_msg=f"step {s}")
        kx.inpaint(fd, cg, ug, tol=1e-12)
        uo = inpaint_ref(f, co)


# ---- jump flooding and the full densification loop (Sec. 4.2) -------------

from oracle.densify import densify as densify_loop_ref, densify_counts, jfa_first_step, label_max_dist2, jfa_labels


@pytest.mark.parametrize("H,W,d,k", [(77, 131, 0.02, 40), (150, 200, 0.05, 300), (64, 33, 0.1, 20)])
def test_jfa_step_bit_exact(H, W, d, k):
    """A densification step on jump-flooding labels (full schedule, and the
    schedule shortened to the bound of a sparser mask's labels)."""
    need_gpu()
    f = synth_rgb(H, W, seeds=(4, 5, 6)).astype(np.float64)
    c = random_mask(H, W, d, 7)
    u = inpaint_ref(f, c)
    sparse = random_mask(H, W, d / 2, 7) & c
    sparse[0, 0] = 1
    bound = jfa_first_step(label_max_dist2(jfa_labels(sparse)))
    for first in (0, bound):
        want, added_ref = densify_ref(f, c, u, k, 0, voronoi="jfa", first_step=first or None)
        kx = ctx(densify_voronoi=1, jfa_first_step=first)
        md = dev(c.copy())
        added = kx.densify_step(dev(f), md, dev(u), k, 0)
        assert added == added_ref
        np.testing.assert_array_equal(md.cpu().numpy(), want)


@pytest.mark.parametrize("voronoi", [0, 1])
def test_densify_loop_bit_exact(voronoi):
    """hdi_densify against the oracle loop (each side inpaints with its own
    solver, tight tolerance): the same mask after the same schedule."""
    need_gpu()
    H, W = 120, 160
    f = synth_rgb(H, W, seeds=(8, 9, 10)).astype(np.float64)
    n, t, d = 6, 1.03, 0.05
    want, _, hist = densify_loop_ref(f, n, t, d, 300, "jfa" if voronoi else "exact")
    kx = ctx(densify_voronoi=voronoi, densify_tol=1e-12)
    m = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    u = torch.empty_like(dev(f))
    sizes = kx.densify(dev(f), m, u, n, t, d, 300)
    assert sizes == hist["sizes"]
    assert sizes[-1] == densify_counts(int(np.floor(d * H * W + 0.5)), n, t)[-1]
    np.testing.assert_array_equal(m.cpu().numpy(), want)
    np.testing.assert_allclose(u.cpu().numpy(), inpaint_ref(f, want), atol=1e-6)


def test_jfa_loop_quality_matches_exact():
    """The paper's setting (20 iterations to 5%, t = 1): jump flooding costs
    at most a few hundredths of a dB against exact labels."""
    need_gpu()
    H, W = 240, 320
    f = synth_rgb(H, W, seeds=(11, 12, 13), dtype=np.float32)
    psnr = {}
    for vor in (0, 1):
        kx = ctx(densify_voronoi=vor)
        m = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        u = torch.empty_like(dev(f))
        kx.densify(dev(f), m, u, 20, 1.0, 0.05, 300)
        err = float(((u.cpu().numpy().astype(np.float64) - f) ** 2).mean())
        psnr[vor] = 10 * np.log10(255.0 ** 2 / err)
    assert abs(psnr[1] - psnr[0]) <= 0.05


@pytest.mark.parametrize("H,W,ch,dtype,d,k", [(96, 128, 3, np.float32, 0.02, 40), (300, 200, 1, np.float64, 0.005, 150),
                                              (64, 80, 3, np.float32, 0.05, 10000), (1, 90, 1, np.float64, 0.1, 3)])
def test_voronoi_partition_step_bit_exact(H, W, ch, dtype, d, k):
    """Voronoi-cell densification (densify_partition = 1, the variant of the
    Sec. 6.2 comparison) against the oracle's partition = "voronoi" step."""
    need_gpu()
    f = synth_rgb(H, W, seeds=(4, 5, 6), dtype=dtype) if ch == 3 else synth_image(H, W, 4).astype(dtype)
    c = random_mask(H, W, d, 17)
    u = inpaint_ref(f.astype(np.float64), c).astype(dtype)
    kx = ctx(densify_partition=1)
    md = dev(c.copy())
    added = kx.densify_step(dev(f), md, dev(u), k, 0)
    ref, ref_added = densify_ref(f.astype(np.float64), c, u.astype(np.float64), k, partition="voronoi")
    np.testing.assert_array_equal(md.cpu().numpy(), ref)
    assert added == ref_added


def test_voronoi_partition_loop_bit_exact():
    """hdi_densify with Voronoi cells against the oracle loop with the same
    partition (each side inpaints with its own solver, tight tolerance)."""
    need_gpu()
    from oracle.densify import densify as densify_oracle
    H, W = 120, 160
    f = synth_rgb(H, W, seeds=(8, 9, 10)).astype(np.float64)
    n, t, d = 6, 1.03, 0.05
    want, _, hist = densify_oracle(f, n, t, d, 300, "exact", partition="voronoi")
    kx = ctx(densify_partition=1, densify_tol=1e-12)
    m = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    u = torch.empty_like(dev(f))
    sizes = kx.densify(dev(f), m, u, n, t, d, 300)
    assert sizes == hist["sizes"]
    np.testing.assert_array_equal(m.cpu().numpy(), want)
