"""Parity of the CUDA inpainting path (multigrid ORAS, FP64 refinement)
against the FP64 oracle, called through the C ABI."""

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from oracle import inpaint as inpaint_ref, rel_residual
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu


def run(f, c, tol, u0=None, **params):
    need_gpu()
    k = ctx(**params)
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    st = k.inpaint(fd, cd, out, u0=None if u0 is None else dev(u0), tol=tol)
    return out.cpu().numpy(), st


def test_c1_256_gray_fp64_tight():
    """256x256 grey FP64, 4% mask, relative residual 1e-10."""
    f = synth_image(256, 256, 0)
    c = random_mask(256, 256, 0.04, 1000)
    u, st = run(f, c, 1e-10)
    ref = inpaint_ref(f, c)
    assert st["rel_res"] <= 1e-10
    assert rel_residual(u, f, c)[0] <= 1e-10
    assert np.abs(u - ref).max() <= 1e-6
    assert st["iterations"] <= 12


@pytest.mark.parametrize("H,W,d,seed", [(77, 131, 0.04, 1), (300, 200, 0.1, 2), (33, 33, 0.02, 3),
                                        (1, 40, 0.1, 4), (41, 1, 0.1, 5), (70, 3, 0.05, 6),
                                        (520, 97, 0.01, 7)])
def test_ragged_rgb_fp32(H, W, d, seed):
    """Ragged sizes spanning several subdomains and a partial last tile."""
    f = synth_rgb(H, W, seeds=(seed, seed + 10, seed + 20), dtype=np.float32)
    c = random_mask(H, W, d, seed + 100)
    u, st = run(f, c, 1e-6)
    ref = inpaint_ref(f.astype(np.float64), c)
    assert st["rel_res"] <= 1e-6
    assert rel_residual(u.astype(np.float64), f.astype(np.float64), c).max() <= 1.5e-6
    assert np.abs(u - ref).max() <= 1e-3


@pytest.mark.parametrize("layout", [dict(oras_warp=1, oras_warp_waves=0), dict(oras_warp=0), {}])
@pytest.mark.parametrize("H,W,d,seed", [(77, 131, 0.04, 11), (300, 200, 0.1, 12), (33, 33, 0.02, 13),
                                        (1, 40, 0.1, 14), (520, 97, 0.01, 15)])
def test_oras_layouts(layout, H, W, d, seed):
    """The ORAS sweep (Sec. 3.1) in each kernel layout: one warp per
    subdomain on every level (oras_warp_waves = 0), two warps on every level
    (oras_warp = 0), and the default choice by sweep size; each reaches the
    oracle's solution."""
    f = synth_rgb(H, W, seeds=(seed, seed + 10, seed + 20), dtype=np.float32)
    c = random_mask(H, W, d, seed + 100)
    u, st = run(f, c, 1e-6, **layout)
    ref = inpaint_ref(f.astype(np.float64), c)
    assert st["rel_res"] <= 1e-6
    assert rel_residual(u.astype(np.float64), f.astype(np.float64), c).max() <= 1.5e-6
    assert np.abs(u - ref).max() <= 1e-3


def test_full_mask_and_single_pixel():
    f = synth_image(40, 50, 9)
    u, _ = run(f, np.ones((40, 50), np.uint8), 1e-8)
    np.testing.assert_array_equal(u, f)
    c = np.zeros((40, 50), np.uint8)
    c[17, 33] = 1
    u, _ = run(f, c, 1e-9)
    assert np.abs(u - f[17, 33]).max() <= 1e-6


def test_warm_start_and_host_buffers():
    need_gpu()
    f = synth_rgb(96, 128, dtype=np.float32)
    c = random_mask(96, 128, 0.05, 11)
    ref = inpaint_ref(f.astype(np.float64), c)
    k = ctx()
    out = np.empty_like(f)
    st = k.inpaint(f, c, out, tol=1e-6)          # host buffers
    assert np.abs(out - ref).max() <= 1e-3
    out2 = np.empty_like(f)
    st2 = k.inpaint(f, c, out2, u0=out, tol=1e-6)
    assert st2["iterations"] <= 1 and np.abs(out2 - ref).max() <= 1e-3


def test_determinism():
    f = synth_rgb(130, 90, dtype=np.float32)
    c = random_mask(130, 90, 0.04, 12)
    u1, _ = run(f, c, 1e-6)
    u2, _ = run(f, c, 1e-6)
    np.testing.assert_array_equal(u1, u2)


@pytest.mark.parametrize("H,W", [(130, 90), (540, 960)])
def test_programmatic_launch_matches_plain_launch(H, W):
    """The multigrid kernels launched with programmatic stream serialisation
    (each overlapping its predecessor's tail) give bit-identical inpaintings
    and tonal values to plain launches, so no kernel reads its predecessor's
    output before pdl_wait()."""
    need_gpu()
    f = dev(synth_rgb(H, W, seeds=(3, 4, 5), dtype=np.float32))
    c = dev(random_mask(H, W, 0.04, 13))
    outs = []
    for pdl in (0, 1):
        k = ctx(pdl=pdl)
        u = torch.empty_like(f)
        g = torch.empty_like(f)
        k.inpaint(f, c, u, tol=1e-6)
        k.tonal_opt(f, c, g, tol=1e-6)
        outs.append((u, g))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_errors():
    need_gpu()
    import paper_2401_06747_b300 as hdi
    k = ctx()
    f = dev(synth_image(20, 20, 1))
    out = torch.empty_like(f)
    with pytest.raises(hdi.HdiError) as e:
        k.inpaint(f, dev(np.zeros((20, 20), np.uint8)), out)
    assert e.value.code == -2
    bad = np.zeros((20, 20), np.uint8)
    bad[3, 3] = 2
    with pytest.raises(hdi.HdiError) as e:
        k.inpaint(f, dev(bad), out)
    assert e.value.code == -1
    fn = f.clone()
    fn[2, 2] = float("nan")
    with pytest.raises(hdi.HdiError) as e:
        k.inpaint(fn, dev(random_mask(20, 20, 0.1, 1)), out)
    assert e.value.code == -6


def test_timing_classes_and_algorithmic_bytes():
    """The per-class event timing and the library's algorithmic byte counts:
    one inpainting and one tonal optimisation with timing on; every
    streaming class reports the bytes its launches must move (13.125 B per
    value for the prolongation, 9.125 for the restriction, 8.125-12.125 for
    the ORAS sweeps, 24.125 for the inpainting residual update and up to
    40.125 for the tonal adjoint residual), the others none."""
    need_gpu()
    H, W = 200, 260
    f = synth_rgb(H, W, seeds=(61, 62, 63), dtype=np.float32)
    c = random_mask(H, W, 0.04, 64)
    k = ctx()
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    values = 3 * H * W
    k.timing(enable=True, reset=True)
    k.inpaint(fd, cd, out, tol=1e-6)
    b, t = k.timing_bytes(), k.timing(enable=True, reset=True)
    for name, bpv in (("prolong_fine", 13.125), ("restrict_fine", 9.125)):
        assert t[name][1] > 0 and b[name] == pytest.approx(bpv * values * t[name][1], rel=1e-12)
    n = t["oras_fine"][1]
    assert n > 0 and 8.125 * values * n <= b["oras_fine"] <= 12.125 * values * n
    n = t["residual_fine"][1]
    assert n > 0 and 12.125 * values * n <= b["residual_fine"] <= 24.125 * values * n
    assert all(b[x] == 0.0 for x in ("tonal_echo", "tonal_gram", "tonal_local", "anderson"))
    k.tonal_opt(fd, cd, out, tol=1e-6)
    b, t = k.timing_bytes(), k.timing(enable=False, reset=True)
    n = t["residual_fine"][1]
    assert b["residual_fine"] > 24.125 * values * n / 2 and b["residual_fine"] <= 40.125 * values * n
    assert t["tonal_echo"][1] > 0 and b["tonal_echo"] == 0.0
    assert all(v[0] > 0 for x, v in t.items() if v[1] > 0)


def test_plain_fp32_form():
    """inpaint_fp32 = 1: FP32 iterate, residual and update without the
    double-float refinement (the per-image baseline of the mixed-precision
    path). It reaches a loose tolerance with the oracle's solution and stops
    with NOT_CONVERGED once V-cycles no longer gain (FP32 rounding level)."""
    need_gpu()
    H, W = 300, 200
    f = synth_rgb(H, W, seeds=(61, 62, 63), dtype=np.float32)
    c = random_mask(H, W, 0.04, 64)
    k = ctx(inpaint_fp32=1)
    fd, cd = dev(f), dev(c)
    out = torch.empty_like(fd)
    st = k.inpaint(fd, cd, out, tol=1e-5)
    u = out.cpu().numpy().astype(np.float64)
    f64 = f.astype(np.float64)
    assert st["rel_res"] <= 1e-5
    assert np.all(rel_residual(u, f64, c) <= 3e-5)
    assert np.abs(u - inpaint_ref(f64, c)).max() <= 0.02
    np.testing.assert_array_equal(out.cpu().numpy()[:, c == 1], f[:, c == 1])
    st = k.inpaint(fd, cd, out, tol=1e-10, allow_not_converged=True)
    assert st["status"] == -3 and 1e-10 < st["rel_res"] < 1e-4
    assert st["iterations"] < 20   # stopped by the stall rule, not the cap


def test_hierarchy_truncation_is_exact():
    """mg_truncate = 1 ends the hierarchy at its first fully known level (at
    4% density the any-of-4 mask restriction leaves no unknown pixel from
    the fifth level on): the same results bit for bit as the full hierarchy,
    for inpainting and tonal optimisation, with fewer launches."""
    need_gpu()
    H, W = 768, 1024
    f = synth_rgb(H, W, seeds=(91, 92, 93), dtype=np.float32)
    c = random_mask(H, W, 0.04, 94)
    fd, cd = dev(f), dev(c)
    res, launches = [], []
    for tr in (0, 1):
        k = ctx(mg_truncate=tr)
        u = torch.empty_like(fd)
        g = torch.empty_like(fd)
        s1 = k.inpaint(fd, cd, u, tol=1e-7)
        s2 = k.tonal_opt(fd, cd, g, tol=1e-6)
        res.append((u.cpu().numpy(), g.cpu().numpy(), s1, s2))
        launches.append(k.launch_count())
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])
    assert res[0][2]["local_iters"] == res[1][2]["local_iters"]
    assert res[0][3]["vcycles"] == res[1][3]["vcycles"]
    assert launches[1] < launches[0]
