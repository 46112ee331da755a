"""Pins for the decomposition geometry and the RAS iteration (Sec. 3, Sec. 5.2, Alg. 2)."""

import json
import os

import numpy as np

from oracle import tonal
from oracle.ras import block_count, block_origins, multiplicity, RASTonal
from synthdata import synth_image, random_mask

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def test_block_count_matches_paper():
    g = json.load(open(GOLD))["oras_local_problems_4k_rgb"]
    assert block_count(g["height"], g["width"], g["channels"], g["block"], g["overlap"]) == g["value"]


def test_dense_normal_matrix_size_matches_paper():
    g = json.load(open(GOLD))["dense_normal_matrix_bytes_4k_5pct"]
    m = 0.05 * 3840 * 2160
    assert abs(m - g["mask_pixels_approx"]) / g["mask_pixels_approx"] < 0.05
    assert abs(g["mask_pixels_approx"] ** 2 * g["bytes_per_entry"] - g["bytes_approx"]) < 1e9


def test_partition_of_unity():
    """sum_i R_i^T D_i R_i = I with D_i = 1/multiplicity (Sec. 3.1)."""
    for (H, W, B, ov) in [(100, 77, 32, 6), (3840 // 16, 2160 // 16, 64, 6), (31, 5, 32, 6)]:
        m = multiplicity(H, W, B, ov)
        acc = np.zeros((H, W))
        for y0, y1 in block_origins(H, B, ov):
            for x0, x1 in block_origins(W, B, ov):
                acc[y0:y1, x0:x1] += 1.0 / m[y0:y1, x0:x1]
        np.testing.assert_allclose(acc, 1.0, atol=1e-15)
        assert m.min() >= 1


def test_ras_converges_to_the_tonal_optimum():
    """Alg. 2 is a convergent iteration whose fixed point is the optimum."""
    H, W = 64, 64
    f = synth_image(H, W, 3)
    c = random_mask(H, W, 0.05, 4)
    g_ref = tonal(f, c)
    g, hist = RASTonal(c, 32, 6).run(f, 60)
    assert hist[-1][0] < 1e-9 and hist[-1][0] < hist[0][0] * 1e-6
    assert np.abs(g - g_ref).max() < 1e-5 * np.abs(g_ref).max()
