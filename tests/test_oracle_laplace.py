"""Pins for the inpainting oracle (paper Sec. 2.1) against facts fixed by the
paper and by the mathematics, not against the oracle itself."""

import numpy as np
import pytest

import oracle.laplace as lp
from oracle import laplacian, inpaint, solve_A, rel_residual, apply_A
from synthdata import synth_image, random_mask


def dct_mode(H, W, p, q):
    x = np.arange(W) + 0.5
    y = np.arange(H) + 0.5
    return np.cos(np.pi * q * y / H)[:, None] * np.cos(np.pi * p * x / W)[None, :]


@pytest.mark.parametrize("H,W", [(7, 11), (16, 16), (1, 9), (5, 1)])
def test_laplacian_dct2_eigenpairs(H, W):
    """Reflecting 5-point L has the DCT-II basis as eigenvectors (Sec. 2.1)
    with eigenvalues 4 sin^2(pi p / 2W) + 4 sin^2(pi q / 2H)."""
    L = laplacian(H, W)
    for p in range(W):
        for q in range(H):
            phi = dct_mode(H, W, p, q)
            lam = 4 * np.sin(np.pi * p / (2 * W)) ** 2 + 4 * np.sin(np.pi * q / (2 * H)) ** 2
            np.testing.assert_allclose((L @ phi.ravel()).reshape(H, W), lam * phi, atol=1e-12)


def test_laplacian_constants_and_symmetry():
    L = laplacian(9, 13)
    assert np.abs(L @ np.ones(9 * 13)).max() == 0.0
    assert abs(L - L.T).max() == 0.0


def test_full_mask_gives_f():
    f = synth_image(12, 17, 3)
    c = np.ones((12, 17), np.uint8)
    np.testing.assert_array_equal(inpaint(f, c), f)


def test_constant_data_gives_constant():
    c = random_mask(20, 23, 0.05, 7)
    f = np.full((20, 23), 42.5)
    np.testing.assert_allclose(inpaint(f, c), 42.5, rtol=0, atol=1e-10)


def test_single_mask_pixel_gives_flat_image():
    """One mask pixel -> u is constant, equal to that pixel's value (Sec. 2.1)."""
    f = synth_image(15, 21, 4)
    c = np.zeros((15, 21), np.uint8)
    c[6, 13] = 1
    np.testing.assert_allclose(inpaint(f, c), f[6, 13], atol=1e-9)


def test_two_columns_linear_interpolation():
    """Two fully known columns with constant values alpha, beta: the discrete
    solution is linear between them and constant outside (reflecting BCs)."""
    H, W, x0, x1 = 9, 20, 4, 15
    alpha, beta = 10.0, 200.0
    f = np.zeros((H, W))
    f[:, x0] = alpha
    f[:, x1] = beta
    c = np.zeros((H, W), np.uint8)
    c[:, x0] = 1
    c[:, x1] = 1
    u = inpaint(f, c)
    xs = np.arange(W, dtype=float)
    expect = np.where(xs <= x0, alpha,
                      np.where(xs >= x1, beta, alpha + (beta - alpha) * (xs - x0) / (x1 - x0)))
    np.testing.assert_allclose(u, np.broadcast_to(expect, (H, W)), atol=1e-9)


def test_maximum_principle():
    f = synth_image(40, 33, 5)
    c = random_mask(40, 33, 0.03, 11)
    u = inpaint(f, c)
    fk = f[c.astype(bool)]
    assert u.min() >= fk.min() - 1e-9 and u.max() <= fk.max() + 1e-9


def test_maximum_principle_nonbinary_mask():
    """A = C + (I - C) L is an M-matrix for c in [0, 1] with c != 0, so
    u = A^{-1} C f obeys min f <= u <= max f for f >= 0 (Sec. 2.1 cites the
    matrix structure). Solved densely from the definition."""
    rng = np.random.default_rng(3)
    H, W = 9, 10
    f = rng.uniform(20, 230, (H, W))
    c = np.where(rng.uniform(size=(H, W)) < 0.2, rng.uniform(0.05, 1.0, (H, W)), 0.0)
    L = laplacian(H, W).toarray()
    C = np.diag(c.ravel())
    A = C + (np.eye(H * W) - C) @ L
    u = np.linalg.solve(A, C @ f.ravel())
    assert u.min() >= f.min() - 1e-9 and u.max() <= f.max() + 1e-9


def test_linearity_and_channel_independence():
    c = random_mask(24, 18, 0.06, 2)
    f1 = synth_image(24, 18, 8)
    f2 = synth_image(24, 18, 9)
    u1, u2 = inpaint(f1, c), inpaint(f2, c)
    np.testing.assert_allclose(inpaint(2.0 * f1 - 0.5 * f2, c), 2.0 * u1 - 0.5 * u2, atol=1e-9)
    u3 = inpaint(np.stack([f1, f2]), c)
    np.testing.assert_allclose(u3[0], u1, atol=1e-12)
    np.testing.assert_allclose(u3[1], u2, atol=1e-12)


@pytest.mark.parametrize("H,W,seed", [(8, 8, 1), (16, 16, 2), (5, 13, 3), (1, 16, 4)])
def test_dense_brute_force(H, W, seed):
    """Dense numpy solve of (C + (I - C) L) u = C f on tiny images."""
    f = synth_image(H, W, seed)
    c = random_mask(H, W, 0.15, seed + 50)
    L = laplacian(H, W).toarray()
    C = np.diag(c.ravel().astype(float))
    A = C + (np.eye(H * W) - C) @ L
    u = np.linalg.solve(A, C @ f.ravel()).reshape(H, W)
    np.testing.assert_allclose(inpaint(f, c), u, atol=1e-9)


def test_symmetrised_system_same_solution():
    """A~ = C + (I-C) L (I-C), C~ = C - (I-C) L C: A~^{-1} C~ f = A^{-1} C f (Sec. 5.1)."""
    H, W = 11, 12
    f = synth_image(H, W, 21)
    c = random_mask(H, W, 0.1, 22)
    L = laplacian(H, W).toarray()
    C = np.diag(c.ravel().astype(float))
    I = np.eye(H * W)
    At = C + (I - C) @ L @ (I - C)
    Ct = C - (I - C) @ L @ C
    assert np.abs(At - At.T).max() == 0.0
    assert np.linalg.eigvalsh(At).min() > 0
    u = np.linalg.solve(At, Ct @ f.ravel()).reshape(H, W)
    np.testing.assert_allclose(inpaint(f, c), u, atol=1e-9)


def test_cg_branch_matches_direct(monkeypatch):
    """The FP64 CG branch used for large images agrees with SuperLU."""
    H, W = 48, 40
    f = synth_image(H, W, 31)
    c = random_mask(H, W, 0.04, 32)
    u_direct = inpaint(f, c)
    lp._cache.clear()
    monkeypatch.setattr(lp, "DIRECT_MAX", 0)
    u_cg = inpaint(f, c)
    lp._cache.clear()
    np.testing.assert_allclose(u_cg, u_direct, atol=1e-9)


def test_general_rhs_and_residual():
    H, W = 14, 19
    c = random_mask(H, W, 0.08, 41)
    rng = np.random.default_rng(5)
    b = rng.normal(size=(H, W))
    u = solve_A(b, c)
    np.testing.assert_allclose(apply_A(u, c), b, atol=1e-10)
    f = synth_image(H, W, 42)
    assert rel_residual(inpaint(f, c), f, c)[0] < 1e-12


def test_empty_mask_rejected():
    with pytest.raises(ValueError):
        inpaint(np.ones((4, 4)), np.zeros((4, 4), np.uint8))
