"""Pins for the Voronoi-initialisation oracle (paper Sec. 5.3) against facts
fixed by the paper and by the mathematics."""

import numpy as np
import pytest

from oracle import B_apply, inpaint, mse
from oracle.densify import voronoi_labels
from oracle.vi import apply_W, voronoi_init, zone_weights
from synthdata import synth_image, synth_rgb, random_mask


def test_error_balancing_is_the_one_step_neighbour_case():
    """Galic et al.'s rule as printed in Sec. 5.3, written out with loops:
    g_i = u_i + mean over the 3x3 neighbourhood (with i) of (f - u)."""
    H, W = 14, 17
    f = synth_image(H, W, 1)
    c = random_mask(H, W, 0.08, 2)
    u = inpaint(f, c)
    want = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            if not c[y, x]:
                continue
            acc, n = 0.0, 0
            for yy in range(y - 1, y + 2):
                for xx in range(x - 1, x + 2):
                    if 0 <= yy < H and 0 <= xx < W:
                        acc += f[yy, xx] - u[yy, xx]
                        n += 1
            want[y, x] = u[y, x] + acc / n
    g, hist = voronoi_init(f, c, max_iter=1, tau=1.0, mode=2, stop_on_rise=False)
    np.testing.assert_allclose(g, want, atol=1e-10)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_rows_of_W_average(mode):
    """Every row of W sums to one: a constant error is reproduced at every
    mask pixel, so constant data stay a fixed point."""
    H, W = 20, 23
    c = random_mask(H, W, 0.06, 3)
    r = apply_W(np.full((H, W), 3.25), c, mode)
    np.testing.assert_allclose(r[c.astype(bool)], 3.25, rtol=1e-14)
    assert np.all(r[~c.astype(bool)] == 0)
    f = np.full((H, W), 42.0)
    g, _ = voronoi_init(f, c, max_iter=3, mode=mode, stop_on_rise=False)
    np.testing.assert_allclose(g, 42.0 * c, atol=1e-9)


@pytest.mark.parametrize("mode", [0, 1])
def test_voronoi_zones_partition_the_image(mode):
    """Modes 0/1: each pixel feeds exactly the mask pixel whose Voronoi cell
    holds it, with weight 1 at the site and less further out (mode 0)."""
    H, W = 16, 19
    c = random_mask(H, W, 0.07, 4)
    V, w = zone_weights(c, mode)
    np.testing.assert_array_equal(V, voronoi_labels(c))
    rng = np.random.default_rng(5)
    for p in rng.choice(H * W, 12, replace=False):
        e = np.zeros(H * W)
        e[p] = 1.0
        r = apply_W(e.reshape(H, W), c, mode).ravel()
        assert np.count_nonzero(r) == 1 and r[V.ravel()[p]] > 0
    sites = np.flatnonzero(c.ravel())
    assert np.all(w.ravel()[sites] == 1.0)
    if mode == 0:
        py, px = np.divmod(np.arange(H * W), W)
        sy, sx = np.divmod(V.ravel(), W)
        d = np.hypot(px - sx, py - sy)
        order = np.argsort(d)
        assert np.all(np.diff(w.ravel()[order]) <= 1e-15)


def test_generated_data_are_a_fixed_point():
    """If f is itself an inpainting B g0, then u = f and g stays g0."""
    H, W = 24, 20
    c = random_mask(H, W, 0.06, 6)
    g0 = np.where(c.astype(bool), synth_image(H, W, 7), 0.0)
    f = B_apply(g0, c)
    g, hist = voronoi_init(f, c, max_iter=4, mode=0, stop_on_rise=False)
    np.testing.assert_allclose(g, g0, atol=1e-9)
    assert hist["mse"][-1] < 1e-18


def test_richardson_converges_to_the_average_interpolation_solution():
    """Without the stopping rule the iteration solves C W A^-1 C g = C W f
    (Sec. 5.3): compared with a dense solve of that m x m system, whenever
    tau = 1 contracts on it."""
    H, W = 10, 12
    f = synth_image(H, W, 8)
    c = random_mask(H, W, 0.15, 9)
    K = np.flatnonzero(c.ravel())
    m = K.size
    # dense M = (W B)_KK column by column from unit data on each mask pixel
    M = np.zeros((m, m))
    for j, k in enumerate(K):
        x = np.zeros(H * W)
        x[k] = 1.0
        M[:, j] = apply_W(B_apply(x.reshape(H, W), c), c, 0).ravel()[K]
    rho = np.abs(np.linalg.eigvals(np.eye(m) - M)).max()
    assert rho < 0.999
    rhs = apply_W(f, c, 0).ravel()[K]
    g_direct = np.linalg.solve(M, rhs)
    g, _ = voronoi_init(f, c, max_iter=4000, mode=0, stop_on_rise=False)
    np.testing.assert_allclose(g.ravel()[K], g_direct, atol=1e-6 * np.abs(g_direct).max())


def test_stop_on_rise_keeps_the_best_iterate():
    """The iteration stops at the first MSE increase and returns the iterate
    before it; the MSE never exceeds the untuned one."""
    f = synth_rgb(40, 36, seeds=(11, 12, 13))
    c = random_mask(40, 36, 0.05, 14)
    g, hist = voronoi_init(f, c, max_iter=30, mode=0)
    _, full = voronoi_init(f, c, max_iter=30, mode=0, stop_on_rise=False)
    k = hist["accepted"]
    m = full["mse"]
    assert all(m[j + 1] <= m[j] for j in range(k))
    if k < 30:
        assert m[k + 1] > m[k]
    assert mse(B_apply(g, c), f) == pytest.approx(m[k], rel=1e-12)
    assert m[k] < m[0]
