"""One Delaunay densification step (paper Sec. 4.1, Alg. 1) and the
random-dithering initial mask (Sec. 4.2), with exact integer geometry.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Given f, the current mask c, its inpainting u and a count k:
  1. error map e_p = sum_ch (u_p - f_p)^2 in FP64 (Sec. 4.1, e = |u - f|^2,
     summed over colour channels);
  2. Voronoi labels V(p) = the mask pixel s minimising (dx^2 + dy^2), ties
     to the lowest linear index y*W + x of s (exact integers);
  3. Delaunay triangles as the dual of the label map (Sec. 4.2, Delaunay
     from the Voronoi diagram): every 2x2 block of pixel centres (a "quad",
     index q = y*(W-1) + x) whose labels TL, TR, BR, BL hold 3 distinct sites
     gives the triangle of those sites; with 4 distinct sites a, b, c, d in
     that cyclic order it gives {a, b, c} and {a, c, d}. Collinear triples are
     dropped. A triangle's id is the smallest 2*q + sub over the quads that
     produce it (sub = 0 for the first, 1 for the second triangle of a quad);
  4. ownership: each non-mask pixel belongs to the lowest-id triangle whose
     closed triangle (vertices at pixel centres) contains its centre, else to
     the "hull cell" of its label, id 2*(W-1)*(H-1) + V(p);
  5. cell error E_T = sum of e over the owned pixels, accumulated exactly as
     integers after quantising e to multiples of 2^-20 (order-independent);
  6. the cells with E_T > 0 are ranked by (E_T desc, id asc); in each of the
     first k the pixel of largest e (ties: lowest linear index) is added
     (Alg. 1: at most one new pixel per triangle, placed at the maximum
     pointwise error, triangles in order of decreasing error).
Voronoi-cell partition (partition = "voronoi"; the Voronoi-based
densification the paper compares against in Sec. 6.2, after Daropoulos et
al.): the same step with the triangles of 3.-4. replaced by the Voronoi
cells of the current mask pixels: every non-mask pixel p belongs to the cell
of its label V(p), the cell id is V(p) itself (the site's linear index), and
5.-6. are unchanged (cells ranked by (E desc, site index asc), one new pixel
per selected cell at its largest e).
With an empty mask the step draws the initial mask instead (Sec. 4.2):
  w_i = sum_ch |(L f)_i| (FP64, (L f)_i = sum of (f_i - f_n) over the in-image
  neighbours in the order left, right, up, down), quantised to
  wq_i = rint(w_i * 2^24); pixel i is taken when
  (splitmix64(seed, i) >> 11) < min(1, k * wq_i / sum(wq)) * 2^53
  (random dithering: a biased coin per pixel with probability proportional to
  the Laplacian magnitude). If sum(wq) = 0 the probability is min(1, k/N).
"""

from __future__ import annotations

import numpy as np

from .splitmix import splitmix64

E_SCALE = float(2 ** 20)
W_SCALE = float(2 ** 24)


def _as3(a):
    a = np.asarray(a)
    return a[None] if a.ndim == 2 else a


def error_map(u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """e_p = sum over channels (in channel order) of (u - f)^2, FP64."""
    u3 = _as3(u).astype(np.float64)
    f3 = _as3(f).astype(np.float64)
    e = np.zeros(u3.shape[1:])
    for ch in range(u3.shape[0]):
        d = u3[ch] - f3[ch]
        e = e + d * d
    return e


def quantise_error(e: np.ndarray) -> np.ndarray:
    return np.rint(e * E_SCALE).astype(np.int64)


def voronoi_labels(c: np.ndarray) -> np.ndarray:
    """Exact nearest mask pixel (linear index) of every pixel, ties to the
    lowest linear index. Candidates come from a k-d tree; the decision is
    made on exact int64 squared distances, and k grows until every site tied
    at the minimum is among the candidates."""
    from scipy.spatial import cKDTree
    cb = np.asarray(c, dtype=bool)
    H, W = cb.shape
    sy, sx = np.nonzero(cb)
    sites = sy.astype(np.int64) * W + sx
    if sites.size == 0:
        raise ValueError("empty mask has no Voronoi diagram")
    tree = cKDTree(np.stack([sx, sy], 1).astype(np.float64))
    py, px = np.divmod(np.arange(H * W, dtype=np.int64), W)
    out = np.empty(H * W, dtype=np.int64)
    todo = np.arange(H * W)
    k = min(8, sites.size)
    while todo.size:
        _, cand = tree.query(np.stack([px[todo], py[todo]], 1).astype(np.float64), k=k)
        cand = cand.reshape(todo.size, k)
        d2 = (sx[cand] - px[todo, None]) ** 2 + (sy[cand] - py[todo, None]) ** 2
        dmin = d2.min(axis=1)
        lab = np.where(d2 == dmin[:, None], sites[cand], np.iinfo(np.int64).max).min(axis=1)
        if k < sites.size:
            # all minimal sites are guaranteed among the candidates only if the
            # farthest candidate is strictly farther than the minimum
            safe = d2.max(axis=1) > dmin
        else:
            safe = np.ones(todo.size, bool)
        out[todo[safe]] = lab[safe]
        todo = todo[~safe]
        k = min(2 * k, sites.size)
    return out.reshape(H, W)


def jfa_labels(c: np.ndarray, first_step: int | None = None) -> np.ndarray:
    """Approximate Voronoi labels by jump flooding (Rong and Tan 2006; the
    paper's speed mode, Sec. 4.2): every seed starts with its own label, and
    for step k = first_step, first_step / 2, ..., 1 every pixel takes, among
    its own label and the labels of the 8 pixels at offsets (+-k or 0,
    +-k or 0), the site of least (d^2, linear index); each pass reads the
    labels of the previous one. first_step defaults to half the smallest
    power of two >= max(H, W) (the full schedule); a smaller first step
    (a power of two at least the largest pixel-to-site distance) saves passes
    once the mask is dense."""
    cb = np.asarray(c, dtype=bool)
    H, W = cb.shape
    if not cb.any():
        raise ValueError("empty mask has no Voronoi diagram")
    N = H * W
    idx = np.arange(N, dtype=np.int64)
    lab = np.where(cb.ravel(), idx, -1)
    py, px = np.divmod(idx, W)
    if first_step is None:
        n2 = 1
        while n2 < max(H, W):
            n2 *= 2
        first_step = max(n2 // 2, 1)
    k = int(first_step)
    while k >= 1:
        best_d2 = np.full(N, np.iinfo(np.int64).max)
        best_s = np.full(N, -1, dtype=np.int64)
        for dy in (-k, 0, k):
            for dx in (-k, 0, k):
                ny, nx = py + dy, px + dx
                inside = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
                s = np.full(N, -1, dtype=np.int64)
                s[inside] = lab[ny[inside] * W + nx[inside]]
                ok = s >= 0
                sy, sx = np.divmod(np.where(ok, s, 0), W)
                d2 = (px - sx) ** 2 + (py - sy) ** 2
                better = ok & ((d2 < best_d2) | ((d2 == best_d2) & (s < best_s)))
                best_d2 = np.where(better, d2, best_d2)
                best_s = np.where(better, s, best_s)
        lab = best_s
        k //= 2
    return lab.reshape(H, W)


def label_max_dist2(V: np.ndarray) -> int:
    """Largest squared distance from a pixel to the site of its label."""
    H, W = V.shape
    py, px = np.divmod(np.arange(H * W, dtype=np.int64), W)
    sy, sx = np.divmod(V.ravel().astype(np.int64), W)
    return int(((px - sx) ** 2 + (py - sy) ** 2).max())


def jfa_first_step(max_dist2: int) -> int:
    """Smallest power of two >= the distance bound sqrt(max_dist2) (>= 1)."""
    k = 1
    while k * k < max_dist2:
        k *= 2
    return k


def densify_counts(total: int, n: int, t: float) -> list:
    """Pixels to have after each of the n densification iterations (Sec. 4.2,
    "Number of New Pixels per Iteration"): the count added in iteration i is
    t times that of iteration i - 1, and the first count is chosen so that
    the n iterations add `total` pixels. Cumulative targets are rounded
    (floor(x + 0.5)) so that the last one is exactly `total`."""
    out = []
    for i in range(1, n + 1):
        if t == 1.0:
            frac = i / n
        else:
            frac = (t ** i - 1.0) / (t ** n - 1.0)
        out.append(int(np.floor(total * frac + 0.5)))
    out[-1] = int(total)
    return out


def _orient(ax, ay, bx, by, cx, cy):
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)


def triangles(V: np.ndarray):
    """Triangles of the label map. Returns (verts [n,3] sorted site indices,
    ids [n]) with one row per distinct triangle."""
    H, W = V.shape
    if H < 2 or W < 2:
        return np.zeros((0, 3), np.int64), np.zeros(0, np.int64)
    a = V[:-1, :-1].ravel()   # TL
    b = V[:-1, 1:].ravel()    # TR
    c = V[1:, 1:].ravel()     # BR
    d = V[1:, :-1].ravel()    # BL
    q = np.arange(a.size, dtype=np.int64)
    lab = np.stack([a, b, c, d], 1)
    srt = np.sort(lab, axis=1)
    ndist = 1 + (srt[:, 1] != srt[:, 0]) + (srt[:, 2] != srt[:, 1]) + (srt[:, 3] != srt[:, 2])
    tris, ids = [], []
    m3 = ndist == 3
    if m3.any():
        s3 = srt[m3]
        # distinct values of the sorted row
        u3 = np.where(s3[:, 1:2] == s3[:, 0:1], s3[:, [0, 2, 3]], np.where(s3[:, 2:3] == s3[:, 1:2], s3[:, [0, 1, 3]], s3[:, [0, 1, 2]]))
        tris.append(u3)
        ids.append(2 * q[m3])
    m4 = ndist == 4
    if m4.any():
        l4 = lab[m4]
        tris.append(np.sort(l4[:, [0, 1, 2]], axis=1))
        ids.append(2 * q[m4])
        tris.append(np.sort(l4[:, [0, 2, 3]], axis=1))
        ids.append(2 * q[m4] + 1)
    if not tris:
        return np.zeros((0, 3), np.int64), np.zeros(0, np.int64)
    T = np.concatenate(tris)
    I = np.concatenate(ids)
    y, x = np.divmod(T, W)
    o = _orient(x[:, 0], y[:, 0], x[:, 1], y[:, 1], x[:, 2], y[:, 2])
    keep = o != 0
    T, I = T[keep], I[keep]
    order = np.lexsort((I, T[:, 2], T[:, 1], T[:, 0]))
    T, I = T[order], I[order]
    first = np.ones(T.shape[0], bool)
    first[1:] = np.any(T[1:] != T[:-1], axis=1)
    return T[first], I[first]


def ownership(c: np.ndarray, V: np.ndarray, T: np.ndarray, I: np.ndarray, chunk: int = 200_000) -> np.ndarray:
    """Owner cell id of every pixel (-1 for mask pixels)."""
    cb = np.asarray(c, dtype=bool)
    H, W = cb.shape
    big = np.iinfo(np.int64).max
    owner = np.full(H * W, big, dtype=np.int64)
    if T.shape[0]:
        ty, tx = np.divmod(T, W)
        # counter-clockwise orientation in (x, y) with y down is fine as long as
        # all three tests use the same sign convention
        o = _orient(tx[:, 0], ty[:, 0], tx[:, 1], ty[:, 1], tx[:, 2], ty[:, 2])
        sw = o < 0
        tx[sw, 1], tx[sw, 2] = tx[sw, 2].copy(), tx[sw, 1].copy()
        ty[sw, 1], ty[sw, 2] = ty[sw, 2].copy(), ty[sw, 1].copy()
        for s in range(0, T.shape[0], chunk):
            e = slice(s, s + chunk)
            X, Y, ID = tx[e], ty[e], I[e]
            x0, x1 = X.min(1), X.max(1)
            y0, y1 = Y.min(1), Y.max(1)
            bw, bh = x1 - x0 + 1, y1 - y0 + 1
            n = bw * bh
            rep = np.repeat(np.arange(X.shape[0]), n)
            start = np.concatenate([[0], np.cumsum(n)[:-1]])
            off = np.arange(rep.size) - start[rep]
            qx = x0[rep] + off % bw[rep]
            qy = y0[rep] + off // bw[rep]
            ax, ay, bx_, by_, cx, cy = X[rep, 0], Y[rep, 0], X[rep, 1], Y[rep, 1], X[rep, 2], Y[rep, 2]
            inside = ((_orient(ax, ay, bx_, by_, qx, qy) >= 0) & (_orient(bx_, by_, cx, cy, qx, qy) >= 0)
                      & (_orient(cx, cy, ax, ay, qx, qy) >= 0))
            pix = (qy * W + qx)[inside]
            np.minimum.at(owner, pix, ID[rep][inside])
    hull = 2 * (W - 1) * (H - 1) + V.ravel().astype(np.int64)
    owner = np.where(owner == big, hull, owner)
    owner[cb.ravel()] = -1
    return owner.reshape(H, W)


def laplace_weight(f: np.ndarray) -> np.ndarray:
    """w_i = sum_ch |(L f)_i| with the neighbour differences added in the
    order left, right, up, down (FP64)."""
    f3 = _as3(f).astype(np.float64)
    H, W = f3.shape[1:]
    w = np.zeros((H, W))
    for ch in range(f3.shape[0]):
        g = f3[ch]
        acc = np.zeros((H, W))
        acc[:, 1:] = acc[:, 1:] + (g[:, 1:] - g[:, :-1])      # left neighbour
        acc[:, :-1] = acc[:, :-1] + (g[:, :-1] - g[:, 1:])    # right neighbour
        acc[1:, :] = acc[1:, :] + (g[1:, :] - g[:-1, :])      # up neighbour
        acc[:-1, :] = acc[:-1, :] + (g[:-1, :] - g[1:, :])    # down neighbour
        w = w + np.abs(acc)
    return w


def initial_mask(f: np.ndarray, k: int, seed: int) -> np.ndarray:
    """Random dithering of |L f| (Sec. 4.2) with the counter-based SplitMix64."""
    f3 = _as3(f)
    H, W = f3.shape[1:]
    wq = np.rint(laplace_weight(f3) * W_SCALE).astype(np.int64).ravel()
    total = int(wq.sum())
    if total > 0:
        p = np.minimum(1.0, (float(k) * wq.astype(np.float64)) / float(np.float64(total)))
    else:
        p = np.full(wq.shape, min(1.0, float(k) / float(H * W)))
    h = splitmix64(seed, np.arange(H * W, dtype=np.uint64))
    take = (h >> np.uint64(11)).astype(np.float64) < p * float(2 ** 53)
    return take.reshape(H, W).astype(np.uint8)


def voronoi_ownership(c: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Owner cell of every pixel for the Voronoi-cell partition: the label
    V(p) of each non-mask pixel (its nearest mask pixel), -1 on the mask."""
    cb = np.asarray(c, dtype=bool)
    own = np.asarray(V, dtype=np.int64).copy()
    own[cb] = -1
    return own


def densify_step(f: np.ndarray, c: np.ndarray, u: np.ndarray | None, k: int, seed: int = 0,
                 voronoi: str = "exact", first_step: int | None = None, info: dict | None = None,
                 partition: str = "delaunay"):
    """Returns (new mask uint8, number of pixels added). voronoi = "jfa" uses
    jump-flooding labels (first pass step `first_step`) instead of the exact
    ones; `info`, if given, receives the labels' largest squared
    pixel-to-site distance ("max_dist2"). partition = "voronoi" selects one
    pixel per Voronoi cell of the current mask instead of per Delaunay
    triangle."""
    if partition not in ("delaunay", "voronoi"):
        raise ValueError("partition must be 'delaunay' or 'voronoi'")
    cb = np.asarray(c, dtype=bool)
    H, W = cb.shape
    if k < 0:
        raise ValueError("k must be >= 0")
    if not cb.any():
        m = initial_mask(f, k, seed)
        return m, int(m.sum())
    e = error_map(u, f)
    eq = quantise_error(e).ravel()
    if voronoi == "exact":
        V = voronoi_labels(cb)
    else:
        V = jfa_labels(cb, first_step)
        if V.min() < 0:   # a shortened schedule that missed pixels: the full one
            V = jfa_labels(cb, None)
    if info is not None:
        info["max_dist2"] = label_max_dist2(V)
    if partition == "voronoi":
        own = voronoi_ownership(cb, V).ravel()
    else:
        T, I = triangles(V)
        own = ownership(cb, V, T, I).ravel()
    free = own >= 0
    ids, inv = np.unique(own[free], return_inverse=True)
    E = np.zeros(ids.size, dtype=np.int64)
    np.add.at(E, inv, eq[free])
    # argmax of e per cell, ties to the lowest linear index
    pix = np.flatnonzero(free)
    order = np.lexsort((pix, -e.ravel()[pix], inv))      # by cell, then e desc, then index asc
    first = np.ones(order.size, bool)
    first[1:] = inv[order][1:] != inv[order][:-1]
    best = np.empty(ids.size, dtype=np.int64)
    best[inv[order][first]] = pix[order][first]
    pos = np.flatnonzero(E > 0)
    rank = pos[np.lexsort((ids[pos], -E[pos]))][:k]
    new = cb.ravel().copy()
    new[best[rank]] = True
    return new.reshape(H, W).astype(np.uint8), int(rank.size)


def densify(f: np.ndarray, n: int, t: float, density: float, seed: int, voronoi: str = "exact", solve=None,
            partition: str = "delaunay"):
    """Delaunay densification from an empty mask (Sec. 4, Alg. 1 with the
    image-adaptive initial mask and the growth factor t of Sec. 4.2): n
    iterations, each a densification step to the cumulative target of
    densify_counts(floor(density * N + 0.5), n, t) followed by an inpainting.
    The first iteration draws the initial mask. With voronoi = "jfa" every
    step after the first uses jump flooding whose first step comes from the
    previous labels' largest distance (the mask only grows, so that bound
    holds for the next mask); the first JFA step runs the full schedule.
    `solve(f, c)` computes the inpainting (default: the exact one).
    partition = "voronoi" runs the Voronoi-cell variant of every step.
    Returns (mask, u, history) with the mask size after every iteration."""
    from .laplace import inpaint
    solve = solve or inpaint
    f3 = _as3(f)
    H, W = f3.shape[1:]
    total = int(np.floor(density * H * W + 0.5))
    targets = densify_counts(total, n, t)
    c = np.zeros((H, W), np.uint8)
    u = None
    first = None
    sizes = []
    for i in range(n):
        k = max(targets[i] - int(c.sum()), 0)
        info = {}
        c, _ = densify_step(f3, c, u, k, seed, voronoi, first, info, partition)
        if voronoi == "jfa" and "max_dist2" in info:
            first = jfa_first_step(info["max_dist2"])
        u = solve(f3, c)
        sizes.append(int(c.sum()))
    if np.ndim(f) == 2:
        u = u[0] if np.ndim(u) == 3 else u
    return c, u, {"sizes": sizes, "targets": targets}
