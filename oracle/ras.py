"""Overlapping decomposition and restricted additive Schwarz for tonal
optimisation (paper Sec. 3.1 and Sec. 5.2, Alg. 2), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Decomposition (Sec. 3.1, Sec. 3.3, Sec. 5.2): square subdomains of side B
with overlap ov are placed at stride s = B - ov from the top-left corner;
n_x = ceil((W - ov) / s) per row (the last one is cut at the image border),
likewise n_y. For B = 32, ov = 6 on 3840x2160 this gives 148 x 83 subdomains
per channel, i.e. the 36,852 local problems per ORAS iteration that Sec. 3.3
reports for a 4K colour image.

Alg. 2 (one iteration):
  1. r = B^T (f - B g)
  2. for every subdomain i solve B_i^T B_i v_i = R_i r, where B_i is the
     inpainting operator of the subdomain with homogeneous Neumann
     conditions at all subdomain boundaries (Sec. 5.2 "Local Normal
     Equations"; read here as the reflecting 5-point L rebuilt on the
     subdomain rectangle) and the unknowns are the mask pixels in it;
  3. g <- g + sum_i R_i^T D_i v_i with D_i = 1 / (number of subdomains
     containing the pixel), the "simple averaging" of Sec. 5.2.
The local systems are solved exactly here (dense Cholesky). The iterates are
not a parity target ("parity unpinned" for intermediate iterates by design);
the fixed point is the tonal optimum, which is pinned.
"""

from __future__ import annotations

import numpy as np

from .laplace import laplacian, _as_channels
from .tonal import B_apply, Bt_apply


def block_origins(n: int, size: int, overlap: int) -> list[tuple[int, int]]:
    """(start, stop) of each subdomain along one axis."""
    stride = size - overlap
    count = max(1, -(-(n - overlap) // stride))
    return [(i * stride, min(i * stride + size, n)) for i in range(count)]


def block_count(height: int, width: int, channels: int, size: int = 32,
                overlap: int = 6) -> int:
    return (len(block_origins(width, size, overlap)) *
            len(block_origins(height, size, overlap)) * channels)


def multiplicity(height: int, width: int, size: int, overlap: int) -> np.ndarray:
    m = np.zeros((height, width))
    for y0, y1 in block_origins(height, size, overlap):
        for x0, x1 in block_origins(width, size, overlap):
            m[y0:y1, x0:x1] += 1
    return m


def _local_gram(c_block: np.ndarray):
    """Cholesky factor of B_i^T B_i = I + S_i^T S_i, S_i = L_UU^{-1} L_UK on
    the subdomain with reflecting (Neumann) boundaries."""
    h, w = c_block.shape
    L = laplacian(h, w).toarray()
    cf = c_block.ravel().astype(bool)
    K = np.flatnonzero(cf)
    U = np.flatnonzero(~cf)
    if K.size == 0:
        return K, None
    if U.size:
        S = np.linalg.solve(L[np.ix_(U, U)], L[np.ix_(U, K)])
    else:
        S = np.zeros((0, K.size))
    G = np.eye(K.size) + S.T @ S
    return K, np.linalg.cholesky(G)


class RASTonal:
    """Alg. 2 with exact local solves, for small images."""

    def __init__(self, c: np.ndarray, size: int = 32, overlap: int = 6):
        self.c = np.asarray(c, dtype=bool)
        H, W = self.c.shape
        self.mult = multiplicity(H, W, size, overlap)
        self.blocks = []
        for y0, y1 in block_origins(H, size, overlap):
            for x0, x1 in block_origins(W, size, overlap):
                K, Lc = _local_gram(self.c[y0:y1, x0:x1])
                if Lc is not None:
                    self.blocks.append((y0, y1, x0, x1, K, Lc))

    def local_phase(self, r: np.ndarray) -> np.ndarray:
        """sum_i R_i^T D_i (B_i^T B_i)^{-1} R_i r for one channel."""
        out = np.zeros_like(r)
        for y0, y1, x0, x1, K, Lc in self.blocks:
            rl = r[y0:y1, x0:x1].ravel()[K]
            v = np.linalg.solve(Lc.T, np.linalg.solve(Lc, rl))
            d = self.mult[y0:y1, x0:x1].ravel()[K]
            blk = out[y0:y1, x0:x1].ravel()
            blk[K] += v / d
            out[y0:y1, x0:x1] = blk.reshape(y1 - y0, x1 - x0)
        return out

    def run(self, f: np.ndarray, iterations: int, g0: np.ndarray | None = None):
        f3 = _as_channels(f)
        g = (f3 * self.c) if g0 is None else _as_channels(g0) * self.c
        hist = []
        den = np.sqrt(np.sum(Bt_apply(f3, self.c) ** 2, axis=(1, 2)))
        for _ in range(iterations):
            r = Bt_apply(f3 - B_apply(g, self.c), self.c)
            hist.append(np.sqrt(np.sum(r ** 2, axis=(1, 2))) / den)
            g = g + np.stack([self.local_phase(r[k]) for k in range(r.shape[0])])
        return (g if np.ndim(f) == 3 else g[0]), np.array(hist)
