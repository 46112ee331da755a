"""Pins for the tonal-optimisation oracle (paper Sec. 5) against facts fixed by
the paper and by the mathematics."""

import numpy as np
import pytest

from oracle import (B_apply, Bt_apply, tonal, tonal_projection, normal_residual, tonal_cgnr, mse_gain_stop,
                    inpaint, mse, laplacian)
from synthdata import synth_image, random_mask


def test_full_mask_gives_f():
    f = synth_image(10, 13, 1)
    c = np.ones((10, 13), np.uint8)
    np.testing.assert_allclose(tonal(f, c), f, atol=1e-10)


def test_constant_data():
    c = random_mask(18, 21, 0.05, 2)
    f = np.full((18, 21), 77.0)
    np.testing.assert_allclose(tonal(f, c), 77.0 * c, atol=1e-9)


def test_recovers_generating_values():
    """If f is itself an inpainting B g0, the optimum is g0 with zero error."""
    H, W = 20, 17
    c = random_mask(H, W, 0.07, 3)
    g0 = np.where(c.astype(bool), synth_image(H, W, 4), 0.0)
    f = B_apply(g0, c)
    g = tonal(f, c)
    np.testing.assert_allclose(g, g0, atol=1e-8)
    assert mse(B_apply(g, c), f) < 1e-16


def test_single_pixel_gives_mean():
    """One mask pixel: B g = g * 1, so the optimum is the mean of f."""
    f = synth_image(13, 9, 5)
    c = np.zeros((13, 9), np.uint8)
    c[4, 2] = 1
    g = tonal(f, c)
    assert abs(g[4, 2] - f.mean()) < 1e-9
    assert np.count_nonzero(g) == 1


def test_never_raises_mse_and_is_optimal():
    """Tonal optimisation never increases the MSE (Sec. 5) and small
    perturbations of the optimum cannot lower it."""
    H, W = 32, 28
    f = synth_image(H, W, 6)
    c = random_mask(H, W, 0.05, 7)
    g = tonal(f, c)
    e_opt = mse(B_apply(g, c), f)
    e_plain = mse(inpaint(f, c), f)
    assert e_opt <= e_plain
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(size=(H, W)) * c
        assert mse(B_apply(g + 1e-2 * d, c), f) >= e_opt


def test_adjoint_dot_product():
    """<B x, y> = <x, B^T y> for x supported on the mask."""
    H, W = 19, 23
    c = random_mask(H, W, 0.06, 8)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(H, W)) * c
    y = rng.normal(size=(H, W))
    lhs = float(np.sum(B_apply(x, c) * y))
    rhs = float(np.sum(x * Bt_apply(y, c)))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    bx = B_apply(x, c)
    np.testing.assert_allclose(bx[c.astype(bool)], x[c.astype(bool)], atol=0)


def test_bt_matches_dense_adjoint():
    """B^T = C A^{-T} built densely from the definition (Sec. 5.1)."""
    H, W = 7, 9
    c = random_mask(H, W, 0.15, 9)
    L = laplacian(H, W).toarray()
    C = np.diag(c.ravel().astype(float))
    A = C + (np.eye(H * W) - C) @ L
    B = np.linalg.solve(A, C)
    y = np.random.default_rng(2).normal(size=(H, W))
    np.testing.assert_allclose(Bt_apply(y, c).ravel(), B.T @ y.ravel(), atol=1e-10)


@pytest.mark.parametrize("H,W,seed", [(8, 8, 1), (12, 15, 2), (16, 16, 3), (1, 20, 4)])
def test_dense_lstsq(H, W, seed):
    """LAPACK least squares on the dense operator B = A^{-1} C."""
    f = synth_image(H, W, seed)
    c = random_mask(H, W, 0.12, seed + 10)
    L = laplacian(H, W).toarray()
    C = np.diag(c.ravel().astype(float))
    A = C + (np.eye(H * W) - C) @ L
    B = np.linalg.solve(A, C)
    K = np.flatnonzero(c.ravel())
    gK, *_ = np.linalg.lstsq(B[:, K], f.ravel(), rcond=None)
    g = np.zeros(H * W)
    g[K] = gK
    np.testing.assert_allclose(tonal(f, c).ravel(), g, atol=1e-8)


def test_projection_formulation_agrees():
    H, W = 48, 40
    f = np.stack([synth_image(H, W, 11), synth_image(H, W, 12)])
    c = random_mask(H, W, 0.04, 13)
    g1 = tonal(f, c)
    g2 = tonal_projection(f, c)
    scale = np.abs(g1).max()
    assert np.abs(g1 - g2).max() <= 1e-9 * scale
    assert normal_residual(f, c, g1).max() < 1e-12


def test_normal_residual_of_unoptimised_values_is_large():
    H, W = 40, 40
    f = synth_image(H, W, 14)
    c = random_mask(H, W, 0.04, 15)
    assert normal_residual(f, c, f * c)[0] > 1e-3


# ---- CGNR (Sec. 5.1, "Improvements") and the MSE-gain stopping rule ----------

def _tiny_case(H=9, W=11, d=0.12, seed=21):
    f = np.stack([synth_image(H, W, seed), synth_image(H, W, seed + 1)])
    c = random_mask(H, W, d, seed + 2)
    return f, c


def test_cgnr_finite_termination():
    """CG on the m x m normal equations reaches the exact minimiser within m
    steps; compared with the independent projection formulation."""
    f, c = _tiny_case()
    m = int(c.sum())
    g, hist = tonal_cgnr(f, c, max_iter=m, rtol=0.0)
    gp = tonal_projection(f, c)
    assert np.abs(g - gp).max() <= 1e-7 * np.abs(gp).max()
    assert hist["rel"][-1] < 1e-7


def test_cgnr_first_step_is_exact_line_search():
    """The first CGNR step minimises ||f - B(g0 + t z0)|| over t: the
    minimiser of the quadratic through three samples t = 0, 1, 2."""
    f, c = _tiny_case(seed=31)
    f = f[0]
    g0 = f * c
    z0 = Bt_apply(f - B_apply(g0, c), c)
    q = [float(np.sum((f - B_apply(g0 + t * z0, c)) ** 2)) for t in (0.0, 1.0, 2.0)]
    a2 = (q[2] - 2 * q[1] + q[0]) / 2.0
    b1 = q[1] - q[0] - a2
    t_star = -b1 / (2 * a2)
    g1, _ = tonal_cgnr(f, c, max_iter=1, rtol=0.0)
    np.testing.assert_allclose(g1, g0 + t_star * z0, atol=1e-9 * np.abs(g0).max())


def test_cgnr_residual_never_increases():
    """CGNR minimises ||f - B g|| over a growing Krylov space: the MSE
    history is non-increasing and ends at the optimum."""
    f = synth_image(24, 20, 41)
    c = random_mask(24, 20, 0.06, 42)
    g, hist = tonal_cgnr(f, c, max_iter=200, rtol=1e-12)
    m = np.asarray(hist["mse"])
    assert np.all(np.diff(m) <= 1e-12 * m[0])
    e_opt = mse(B_apply(tonal(f, c), c), f)
    assert abs(m[-1] - e_opt) <= 1e-9 * e_opt
    np.testing.assert_allclose(g, tonal(f, c), atol=1e-7 * np.abs(f).max())


def test_cgnr_mse_gain_stop():
    """With the 0.1% rule the run stops at the first iteration whose MSE gain
    is below 0.1%, and not before."""
    f = np.stack([synth_image(32, 30, 51), synth_image(32, 30, 52)])
    c = random_mask(32, 30, 0.04, 53)
    _, full = tonal_cgnr(f, c, max_iter=300, rtol=1e-13)
    _, hist = tonal_cgnr(f, c, max_iter=300, rtol=1e-13, mse_gain=1e-3)
    m = full["mse"]
    k = len(hist["mse"]) - 1
    assert 1 <= k < len(m) - 1
    assert mse_gain_stop(m[k - 1], m[k], 1e-3)
    assert not any(mse_gain_stop(m[j - 1], m[j], 1e-3) for j in range(1, k))
    np.testing.assert_allclose(hist["mse"], m[:k + 1], rtol=1e-12)
