"""Pins for the densification oracle (Sec. 4.1, Alg. 1; Sec. 4.2)."""

import json
import os

import numpy as np
import pytest

from oracle.densify import (voronoi_labels, triangles, ownership, densify_step, initial_mask, error_map,
                            quantise_error, laplace_weight, _orient)
from oracle.splitmix import splitmix64, splitmix64_scalar
from synthdata import synth_image, synth_rgb, random_mask

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")


def test_splitmix64_published_outputs():
    g = json.load(open(GOLD))
    want = [int(h, 16) for h in g["outputs_hex"]]
    assert [splitmix64_scalar(g["seed"], i) for i in range(3)] == want
    assert [int(v) for v in splitmix64(g["seed"], np.arange(3))] == want


def brute_labels(c):
    H, W = c.shape
    sy, sx = np.nonzero(c)
    s = sy * W + sx
    out = np.empty((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            d2 = (sx - x) ** 2 + (sy - y) ** 2
            out[y, x] = s[d2 == d2.min()].min()
    return out


@pytest.mark.parametrize("H,W,d,seed", [(9, 11, 0.1, 1), (16, 16, 0.05, 2), (1, 13, 0.2, 3), (20, 7, 0.15, 4)])
def test_voronoi_matches_brute_force(H, W, d, seed):
    c = random_mask(H, W, d, seed).astype(bool)
    np.testing.assert_array_equal(voronoi_labels(c), brute_labels(c))


def test_voronoi_ties_go_to_lowest_index():
    c = np.zeros((5, 5), bool)
    c[0, 0] = c[0, 4] = True        # pixel (2, 0) is equidistant from both
    V = voronoi_labels(c)
    assert V[0, 2] == 0 and V[4, 2] == 0


def test_three_sites_one_triangle():
    c = np.zeros((30, 30), bool)
    c[3, 4] = c[5, 25] = c[24, 12] = True
    T, I = triangles(voronoi_labels(c))
    assert T.shape[0] == 1
    assert sorted(T[0]) == sorted([3 * 30 + 4, 5 * 30 + 25, 24 * 30 + 12])


def test_four_cocircular_sites_split_by_cyclic_rule():
    """Square corners: the centre quad sees four labels; the rule gives the
    triangles {TL,TR,BR} and {TL,BR,BL} of that quad."""
    W = 10
    c = np.zeros((10, W), bool)
    for (y, x) in [(2, 2), (2, 7), (7, 7), (7, 2)]:
        c[y, x] = True
    V = voronoi_labels(c)
    T, I = triangles(V)
    # quad (4,4)-(5,5) sees TL=(2,2) TR=(2,7) BR=(7,7) BL=(7,2)
    q = 4 * (W - 1) + 4
    a, b, cc, d = 2 * W + 2, 2 * W + 7, 7 * W + 7, 7 * W + 2
    got = {tuple(t): i for t, i in zip(T.tolist(), I.tolist())}
    assert got[tuple(sorted([a, b, cc]))] == 2 * q
    assert got[tuple(sorted([a, cc, d]))] == 2 * q + 1
    assert len(got) == 2


def incircle(ax, ay, bx, by, cx, cy, dx, dy):
    """> 0 iff d lies strictly inside the circumcircle of counter-clockwise a, b, c (exact ints)."""
    m = np.array([[ax - dx, ay - dy, (ax - dx) ** 2 + (ay - dy) ** 2],
                  [bx - dx, by - dy, (bx - dx) ** 2 + (by - dy) ** 2],
                  [cx - dx, cy - dy, (cx - dx) ** 2 + (cy - dy) ** 2]], dtype=object)
    return (m[0, 0] * (m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1]) - m[0, 1] * (m[1, 0] * m[2, 2] - m[1, 2] * m[2, 0])
            + m[0, 2] * (m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0]))


def test_triangles_are_delaunay_for_scattered_sites():
    """Dual of the discrete Voronoi diagram vs the empty-circumcircle property."""
    H = W = 160
    rng = np.random.default_rng(5)
    c = np.zeros((H, W), bool)
    c[rng.integers(0, H, 40), rng.integers(0, W, 40)] = True
    T, _ = triangles(voronoi_labels(c))
    sy, sx = np.nonzero(c)
    good = 0
    for t in T:
        (ay, ax), (by, bx), (cy, cx) = [divmod(int(v), W) for v in t]
        if _orient(ax, ay, bx, by, cx, cy) < 0:
            bx, by, cx, cy = cx, cy, bx, by
        ok = all(incircle(ax, ay, bx, by, cx, cy, int(x), int(y)) <= 0 for x, y in zip(sx, sy))
        good += ok
    assert T.shape[0] >= 40
    assert good >= 0.95 * T.shape[0]


def brute_owner(c, V, T, I):
    H, W = c.shape
    out = np.full((H, W), -1, np.int64)
    for y in range(H):
        for x in range(W):
            if c[y, x]:
                continue
            best = None
            for t, i in zip(T, I):
                (ay, ax), (by, bx), (cy, cx) = [divmod(int(v), W) for v in t]
                o = _orient(ax, ay, bx, by, cx, cy)
                s = 1 if o > 0 else -1
                if (s * _orient(ax, ay, bx, by, x, y) >= 0 and s * _orient(bx, by, cx, cy, x, y) >= 0
                        and s * _orient(cx, cy, ax, ay, x, y) >= 0):
                    best = i if best is None else min(best, i)
            out[y, x] = best if best is not None else 2 * (W - 1) * (H - 1) + V[y, x]
    return out


@pytest.mark.parametrize("H,W,seed", [(12, 14, 1), (20, 9, 2)])
def test_ownership_matches_brute_force(H, W, seed):
    c = random_mask(H, W, 0.1, seed).astype(bool)
    V = voronoi_labels(c)
    T, I = triangles(V)
    np.testing.assert_array_equal(ownership(c, V, T, I), brute_owner(c, V, T, I))


def test_densify_step_invariants_and_brute_force_selection():
    H, W = 40, 52
    f = synth_rgb(H, W, seeds=(1, 2, 3))
    c = random_mask(H, W, 0.02, 9)
    from oracle import inpaint
    u = inpaint(f, c)
    k = 15
    new, added = densify_step(f, c, u, k)
    cb = c.astype(bool)
    e = error_map(u, f)
    eq = quantise_error(e)
    V = voronoi_labels(cb)
    T, I = triangles(V)
    own = brute_owner(cb, V, T, I)
    cells = {}
    for y in range(H):
        for x in range(W):
            if own[y, x] >= 0:
                cells.setdefault(int(own[y, x]), []).append((y * W + x))
    E = {i: int(sum(eq.ravel()[p] for p in px)) for i, px in cells.items()}
    ranked = sorted([i for i in E if E[i] > 0], key=lambda i: (-E[i], i))[:k]
    expect = cb.ravel().copy()
    for i in ranked:
        px = cells[i]
        best = max(px, key=lambda p: (e.ravel()[p], -p))
        expect[best] = True
    np.testing.assert_array_equal(new.ravel().astype(bool), expect)
    assert added == min(k, sum(1 for v in E.values() if v > 0))
    assert np.all(new.astype(bool) >= cb)
    assert int(new.sum()) == int(c.sum()) + added


def test_initial_mask_dithering():
    f = synth_image(120, 90, 4)
    k = 300
    m1 = initial_mask(f, k, 7)
    m2 = initial_mask(f, k, 7)
    m3 = initial_mask(f, k, 8)
    np.testing.assert_array_equal(m1, m2)
    assert np.any(m1 != m3)
    w = laplace_weight(f)
    assert np.all(m1[w == 0] == 0)
    p = np.minimum(1.0, k * w / w.sum())
    mean, var = p.sum(), (p * (1 - p)).sum()
    assert abs(int(m1.sum()) - mean) < 5 * np.sqrt(var) + 1
    new, added = densify_step(f, np.zeros((120, 90), np.uint8), None, k, seed=7)
    np.testing.assert_array_equal(new, m1)
    assert added == int(m1.sum())


def test_laplace_weight_is_abs_of_laplacian():
    from oracle import laplacian
    f = synth_rgb(17, 23, seeds=(4, 5, 6))
    L = laplacian(17, 23)
    w = sum(np.abs(L @ f[ch].ravel()) for ch in range(3)).reshape(17, 23)
    np.testing.assert_allclose(laplace_weight(f), w, rtol=0, atol=1e-9)


# ---- jump flooding, the growth schedule and the full loop (Sec. 4.2) -------

from oracle.densify import jfa_labels, label_max_dist2, jfa_first_step, densify_counts, densify


def _brute_labels(c):
    H, W = c.shape
    sy, sx = np.nonzero(c)
    sites = sy * W + sx
    py, px = np.divmod(np.arange(H * W), W)
    d2 = (px[:, None] - sx[None]) ** 2 + (py[:, None] - sy[None]) ** 2
    m = d2.min(axis=1)
    lab = np.where(d2 == m[:, None], sites[None], 10 ** 9).min(axis=1)
    return lab.reshape(H, W), m.reshape(H, W)


def test_jfa_single_seed_is_exact():
    c = np.zeros((37, 53), np.uint8)
    c[20, 7] = 1
    assert np.all(jfa_labels(c) == 20 * 53 + 7)


@pytest.mark.parametrize("H,W,d,seed", [(48, 64, 0.01, 1), (61, 47, 0.04, 2), (33, 90, 0.1, 3)])
def test_jfa_close_to_exact_and_never_closer(H, W, d, seed):
    """JFA labels are seeds, are never nearer than the true nearest seed, and
    agree with the exact diagram on nearly every pixel; the same holds with
    the first step cut down to the distance bound."""
    c = random_mask(H, W, d, seed)
    lab_b, m = _brute_labels(c)
    for first in (None, jfa_first_step(int(m.max()))):
        V = jfa_labels(c, first)
        assert np.all(c.ravel()[V.ravel()] == 1)
        py, px = np.divmod(np.arange(H * W), W)
        sy, sx = np.divmod(V.ravel(), W)
        dj = ((px - sx) ** 2 + (py - sy) ** 2).reshape(H, W)
        assert np.all(dj >= m)
        assert (V == lab_b).mean() >= 0.99
        assert label_max_dist2(V) >= m.max()


def test_jfa_distance_bound_from_an_earlier_mask():
    """The bound taken from a sparser mask's labels still covers a denser
    superset: every pixel gets a label."""
    c1 = random_mask(70, 90, 0.01, 4)
    bound = jfa_first_step(label_max_dist2(jfa_labels(c1)))
    c2 = np.maximum(c1, random_mask(70, 90, 0.02, 5))
    V = jfa_labels(c2, bound)
    assert V.min() >= 0
    assert (V == voronoi_labels(c2)).mean() >= 0.99


@pytest.mark.parametrize("total,n,t", [(1000, 8, 1.0), (41472 * 8, 8, 1.0), (5000, 20, 1.03), (777, 5, 0.9)])
def test_densify_counts(total, n, t):
    """Cumulative targets end at the total; the increments grow by t
    (equal for t = 1) up to the rounding of the targets."""
    c = densify_counts(total, n, t)
    assert c[-1] == total and len(c) == n
    k = np.diff([0] + c)
    assert np.all(k >= 0)
    k1 = total * (t - 1) / (t ** n - 1) if t != 1.0 else total / n
    want = k1 * t ** np.arange(n)
    assert np.all(np.abs(k - want) <= 1.0 + 1e-9)


def test_densify_loop_reaches_the_density():
    f = synth_rgb(40, 52, seeds=(1, 2, 3))
    for vor in ("exact", "jfa"):
        c, u, hist = densify(f, n=6, t=1.03, density=0.05, seed=7, voronoi=vor)
        total = int(np.floor(0.05 * 40 * 52 + 0.5))
        assert hist["sizes"][-1] == total == int(c.sum())
        assert all(b >= a for a, b in zip(hist["sizes"], hist["sizes"][1:]))
        np.testing.assert_allclose(u[:, c == 1], f[:, c == 1], atol=1e-9)


@pytest.mark.parametrize("H,W,d,k,seed", [(40, 52, 0.02, 15, 9), (1, 30, 0.1, 2, 3), (17, 23, 0.05, 100, 4)])
def test_voronoi_partition_step_brute_force(H, W, d, k, seed):
    """Voronoi-cell densification (Sec. 6.2): cells from brute-force nearest
    sites (ties to the lowest index), integer cell sums, top-k by (E desc,
    site asc), one new pixel per selected cell at its largest error."""
    f = synth_rgb(H, W, seeds=(seed, seed + 1, seed + 2))
    c = random_mask(H, W, d, seed + 10)
    from oracle import inpaint
    u = inpaint(f, c)
    new, added = densify_step(f, c, u, k, partition="voronoi")
    cb = c.astype(bool)
    e = error_map(u, f).ravel()
    eq = quantise_error(error_map(u, f)).ravel()
    lab = brute_labels(cb).ravel()
    cells = {}
    for p in range(H * W):
        if not cb.ravel()[p]:
            cells.setdefault(int(lab[p]), []).append(p)
    E = {s: int(sum(eq[p] for p in px)) for s, px in cells.items()}
    ranked = sorted([s for s in E if E[s] > 0], key=lambda s: (-E[s], s))[:k]
    expect = cb.ravel().copy()
    for s in ranked:
        expect[max(cells[s], key=lambda p: (e[p], -p))] = True
    np.testing.assert_array_equal(new.ravel().astype(bool), expect)
    assert added == min(k, sum(1 for v in E.values() if v > 0))
    # at most one new pixel per Voronoi cell of the old mask
    newpix = np.flatnonzero(new.ravel().astype(bool) & ~cb.ravel())
    assert len(set(lab[newpix].tolist())) == newpix.size


def test_voronoi_and_delaunay_partitions_differ_but_add_alike():
    """The two partitions pick different pixels on a natural image, but each
    adds min(k, non-empty cells) pixels outside the old mask."""
    H, W = 48, 64
    f = synth_image(H, W, 5)
    c = random_mask(H, W, 0.02, 6)
    from oracle import inpaint
    u = inpaint(f, c)
    a, na = densify_step(f, c, u, 20, partition="delaunay")
    b, nb = densify_step(f, c, u, 20, partition="voronoi")
    assert na == nb == 20
    assert not np.array_equal(a, b)
    for m in (a, b):
        assert np.all(m.astype(bool) >= c.astype(bool))
    with pytest.raises(ValueError):
        densify_step(f, c, u, 5, partition="square")
