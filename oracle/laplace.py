"""Discrete homogeneous diffusion inpainting (paper Sec. 2.1, Eq. "inp-discrete-lsi").

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Model. Pixels are indexed i = y*W + x. L is the 5-point stencil of the
negated Laplacian with reflecting boundary conditions (Sec. 2.1): the
difference to every in-image 4-neighbour is kept and out-of-image neighbours
are dropped (mirror ghost), so L_ii = number of in-image neighbours and
L_ij = -1 for each neighbour j. Grid spacing h = 1. Its eigenvectors are the
DCT-II basis images (Sec. 2.1, last paragraph of "Image Edges").

  A = C + (I - C) L,   b = C f,   A u = b                        (Sec. 2.1)

With K = {c = 1} and U = {c = 0} this is u_K = f_K and
L_UU u_U = -L_UK f_K; L_UU is SPD whenever K is non-empty (the grid graph is
connected), which is the uniqueness statement of Sec. 2.1. Colour channels
are independent systems with the same matrix (Sec. 2.1).

Solvers: SuperLU (scipy.sparse.linalg.splu) for images up to DIRECT_MAX
pixels; above that, textbook conjugate gradients in FP64 to a relative
residual of 1e-13 (the L_UU system is SPD).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

DIRECT_MAX = 300_000
CG_RTOL = 1e-13


def laplacian(height: int, width: int) -> sp.csr_matrix:
    """5-point negated Laplacian with reflecting boundaries, h = 1."""
    H, W = int(height), int(width)
    n = H * W
    idx = np.arange(n).reshape(H, W)
    pairs = [(idx[:, :-1], idx[:, 1:]), (idx[:-1, :], idx[1:, :])]
    rows, cols = [], []
    for a, b in pairs:
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    off = sp.csr_matrix((-np.ones(r.size), (r, c)), shape=(n, n))
    deg = -np.asarray(off.sum(axis=1)).ravel()
    return (off + sp.diags(deg)).tocsr()


def _as_channels(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    return f[None] if f.ndim == 2 else f


def apply_A(u: np.ndarray, c: np.ndarray) -> np.ndarray:
    """A u = C u + (I - C) L u, per channel (Sec. 2.1)."""
    u3 = _as_channels(u)
    H, W = u3.shape[1:]
    L = laplacian(H, W)
    cf = np.asarray(c, dtype=bool).ravel()
    out = np.empty_like(u3)
    for k in range(u3.shape[0]):
        x = u3[k].ravel()
        Lx = L @ x
        out[k] = np.where(cf, x, Lx).reshape(H, W)
    return out if np.ndim(u) == 3 else out[0]


class _Split:
    """Index split into K (known) and U (unknown) with the blocks of L."""

    def __init__(self, c: np.ndarray):
        c = np.asarray(c, dtype=bool)
        self.H, self.W = c.shape
        self.cflat = c.ravel()
        self.K = np.flatnonzero(self.cflat)
        self.U = np.flatnonzero(~self.cflat)
        if self.K.size == 0:
            raise ValueError("empty mask: A is singular (Sec. 2.1)")
        L = laplacian(self.H, self.W)
        self.L = L
        self.L_UU = L[self.U][:, self.U].tocsc()
        self.L_UK = L[self.U][:, self.K].tocsr()
        self.L_KU = L[self.K][:, self.U].tocsr()
        self._lu = None
        if self.U.size and self.U.size <= DIRECT_MAX:
            self._lu = spl.splu(self.L_UU)

    def solve_UU(self, rhs: np.ndarray) -> np.ndarray:
        """x = L_UU^{-1} rhs (direct for small images, FP64 CG otherwise)."""
        if self.U.size == 0:
            return np.zeros(0)
        if self._lu is not None:
            return self._lu.solve(rhs)
        return cg(self.L_UU, rhs, rtol=CG_RTOL)


_cache: dict = {}


def split_for(c: np.ndarray) -> _Split:
    """Factorisation cache keyed by the mask bytes (one factor per mask)."""
    c = np.asarray(c, dtype=bool)
    key = (c.shape, c.tobytes())
    s = _cache.get(key)
    if s is None:
        if len(_cache) > 8:
            _cache.clear()
        s = _Split(c)
        _cache[key] = s
    return s


def cg(M, rhs: np.ndarray, rtol: float = CG_RTOL, maxiter: int = 100000,
       x0: np.ndarray | None = None) -> np.ndarray:
    """Textbook conjugate gradients (Hestenes & Stiefel) for SPD M, FP64."""
    x = np.zeros_like(rhs) if x0 is None else x0.copy()
    r = rhs - M @ x
    p = r.copy()
    rr = float(r @ r)
    stop = (rtol * float(np.linalg.norm(rhs))) ** 2
    for _ in range(maxiter):
        if rr <= stop:
            break
        q = M @ p
        alpha = rr / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def solve_A(b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """General right-hand side: A u = b, i.e. u_K = b_K and
    L_UU u_U = b_U - L_UK b_K. With b = C f this is the inpainting."""
    b3 = _as_channels(b)
    s = split_for(c)
    out = np.empty_like(b3)
    for k in range(b3.shape[0]):
        bb = b3[k].ravel()
        u = np.empty_like(bb)
        u[s.K] = bb[s.K]
        u[s.U] = s.solve_UU(bb[s.U] - s.L_UK @ bb[s.K])
        out[k] = u.reshape(s.H, s.W)
    return out if np.ndim(b) == 3 else out[0]


def inpaint(f: np.ndarray, c: np.ndarray) -> np.ndarray:
    """u = A^{-1} C f (Sec. 2.1), per channel, FP64."""
    f3 = _as_channels(f)
    cb = np.asarray(c, dtype=bool)
    b = np.where(cb[None], f3, 0.0)
    u = solve_A(b, cb)
    return u if np.ndim(f) == 3 else u[0]


def inpaint_residual(u: np.ndarray, f: np.ndarray, c: np.ndarray) -> np.ndarray:
    """r = C f - A u, per channel, evaluated in FP64."""
    u3 = _as_channels(u)
    f3 = _as_channels(f)
    cb = np.asarray(c, dtype=bool)
    r = np.where(cb[None], f3, 0.0) - apply_A(u3, cb)
    return r if np.ndim(u) == 3 else r[0]


def rel_residual(u: np.ndarray, f: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Per-channel ||C f - A u||_2 / ||C f||_2 (FP64)."""
    u3 = _as_channels(u)
    f3 = _as_channels(f)
    cb = np.asarray(c, dtype=bool)
    r = inpaint_residual(u3, f3, cb)
    den = np.sqrt(np.sum(np.where(cb[None], f3, 0.0) ** 2, axis=(1, 2)))
    num = np.sqrt(np.sum(r ** 2, axis=(1, 2)))
    return num / np.where(den > 0, den, 1.0)
