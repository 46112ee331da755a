"""Tonal optimisation (paper Sec. 5, Eqs. "tonal-opt-minimisation" and
"tonal-normal-equations"), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  min_g || f - B g ||_2^2,   B = A^{-1} C,   g = 0 off the mask     (Sec. 5)
  normal equations  B^T B g = B^T f                                 (Sec. 5.1)

In (K, U) coordinates the inpainting of data x is (B x)_K = x_K and
(B x)_U = -S x_K with S = L_UU^{-1} L_UK, so B = [I; -S] and
B^T y = y_K - S^T y_U with S^T = L_KU L_UU^{-1} (L is symmetric). This is the
symmetrised form of Sec. 5.1: with A~ = C + (I-C) L (I-C) and
C~ = C - (I-C) L C one has A~^{-1} C~ = A^{-1} C, so
B^T = C~^T A~^{-1}, and A~ acts on U as L_UU.

The normal equations on K read (I + S^T S) g_K = f_K - S^T f_U. The matrix
has all eigenvalues >= 1, so plain CG converges; it is run to a relative
residual of 1e-14 in FP64.

CGNR (Sec. 5.1, "Improvements") runs conjugate gradients on the same
normal equations through B and B^T, with the MSE-gain stopping rule of the
paper's experiments as an option.

Cross-check (independent formulation): the optimum u* = B g* is the
orthogonal projection of f onto H_K = {u : (L u)_U = 0}. Its complement is
spanned by the rows U of L, so u* = f - L_{U.}^T lam with
(L_{U.} L_{U.}^T) lam = L_{U.} f, and g*_K = u*_K.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .laplace import _as_channels, split_for, laplacian, cg

TONAL_RTOL = 1e-14


def B_apply(x: np.ndarray, c: np.ndarray) -> np.ndarray:
    """B x = A^{-1} C x: the inpainting with data x on the mask."""
    x3 = _as_channels(x)
    s = split_for(c)
    out = np.zeros_like(x3)
    for k in range(x3.shape[0]):
        xx = x3[k].ravel()
        y = np.zeros_like(xx)
        y[s.K] = xx[s.K]
        y[s.U] = -s.solve_UU(s.L_UK @ xx[s.K])
        out[k] = y.reshape(s.H, s.W)
    return out if np.ndim(x) == 3 else out[0]


def Bt_apply(y: np.ndarray, c: np.ndarray) -> np.ndarray:
    """B^T y = C~^T A~^{-1} y: zero off the mask, y_K - L_KU L_UU^{-1} y_U on it."""
    y3 = _as_channels(y)
    s = split_for(c)
    out = np.zeros_like(y3)
    for k in range(y3.shape[0]):
        yy = y3[k].ravel()
        z = np.zeros_like(yy)
        w_U = s.solve_UU(yy[s.U])
        z[s.K] = yy[s.K] - s.L_KU @ w_U
        out[k] = z.reshape(s.H, s.W)
    return out if np.ndim(y) == 3 else out[0]


class _NormalOp(spl.LinearOperator):
    """g_K -> (I + S^T S) g_K."""

    def __init__(self, s):
        self.s = s
        super().__init__(dtype=np.float64, shape=(s.K.size, s.K.size))

    def _matvec(self, gK):
        s = self.s
        gK = np.ravel(gK)
        z = s.solve_UU(s.L_UK @ gK)          # z = S g_K
        return gK + s.L_KU @ s.solve_UU(z)   # g_K + S^T S g_K

    def __matmul__(self, v):
        return self._matvec(v)


def tonal(f: np.ndarray, c: np.ndarray, rtol: float = TONAL_RTOL) -> np.ndarray:
    """Minimiser g of ||f - B g||, zero off the mask (Sec. 5), FP64 CG."""
    f3 = _as_channels(f)
    s = split_for(c)
    op = _NormalOp(s)
    out = np.zeros_like(f3)
    for k in range(f3.shape[0]):
        ff = f3[k].ravel()
        rhs = ff[s.K] - s.L_KU @ s.solve_UU(ff[s.U])   # B^T f restricted to K
        gK = cg(op, rhs, rtol=rtol, x0=ff[s.K].copy())
        g = np.zeros_like(ff)
        g[s.K] = gK
        out[k] = g.reshape(s.H, s.W)
    return out if np.ndim(f) == 3 else out[0]


def tonal_projection(f: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Same minimiser via the projection onto H_K (independent cross-check;
    direct sparse solve, small images only)."""
    f3 = _as_channels(f)
    cb = np.asarray(c, dtype=bool)
    H, W = cb.shape
    L = laplacian(H, W)
    U = np.flatnonzero(~cb.ravel())
    K = np.flatnonzero(cb.ravel())
    LU = L[U]                                   # rows U of L
    M = (LU @ LU.T).tocsc()
    lu = spl.splu(M) if U.size else None
    out = np.zeros_like(f3)
    for k in range(f3.shape[0]):
        ff = f3[k].ravel()
        if lu is not None:
            lam = lu.solve(LU @ ff)
            ustar = ff - LU.T @ lam
        else:
            ustar = ff.copy()
        g = np.zeros_like(ff)
        g[K] = ustar[K]
        out[k] = g.reshape(H, W)
    return out if np.ndim(f) == 3 else out[0]


def normal_residual(f: np.ndarray, c: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Per-channel ||B^T (f - B g)||_2 / ||B^T f||_2 (FP64)."""
    f3 = _as_channels(f)
    g3 = _as_channels(g)
    r = Bt_apply(f3 - B_apply(g3, c), c)
    d = Bt_apply(f3, c)
    num = np.sqrt(np.sum(r ** 2, axis=(1, 2)))
    den = np.sqrt(np.sum(d ** 2, axis=(1, 2)))
    return num / np.where(den > 0, den, 1.0)


def mse_gain_stop(mse_prev: float, mse_now: float, gain: float) -> bool:
    """The stopping rule of the paper's tonal runtime experiments (Sec. 6,
    runtime scaling): stop once an iteration improved the MSE by less than the
    relative amount `gain` (0.1% there). A rising MSE also stops."""
    return (mse_prev - mse_now) < gain * mse_prev


def tonal_cgnr(f: np.ndarray, c: np.ndarray, max_iter: int = 1000, rtol: float = 1e-12,
               g0: np.ndarray | None = None, mse_gain: float = 0.0):
    """CGNR for tonal optimisation (Sec. 5.1, "Improvements"): conjugate
    gradients on the normal equations B^T B g = B^T f, carried on the
    inpainting residual r = f - B g, so the MSE is known in every iteration:

        r = f - B g,  z = B^T r,  p = z
        repeat:  w = B p;  alpha = <z, z> / <w, w>
                 g <- g + alpha p;  r <- r - alpha w
                 z' = B^T r;  beta = <z', z'> / <z, z>;  p <- z' + beta p

    Each channel is its own least-squares problem (own alpha and beta); the
    channels stop together: when every channel has |z| <= rtol |B^T f|, after
    max_iter iterations, or, with mse_gain > 0, when the MSE over all channels
    improved by less than mse_gain (relative) in the last iteration.
    g0 defaults to f on the mask. Returns (g, history) with history["mse"]
    the MSE of B g before the first and after every iteration and
    history["rel"] the largest relative normal residual at the same points."""
    f3 = _as_channels(f)
    cb = np.asarray(c, dtype=bool)
    g = (f3 * cb) if g0 is None else (_as_channels(g0) * cb)
    g = g.astype(np.float64)
    r = f3 - B_apply(g, c)
    z = Bt_apply(r, c)
    btf = np.sqrt(np.sum(Bt_apply(f3, c) ** 2, axis=(1, 2)))
    btf = np.where(btf > 0, btf, 1.0)
    zz = np.sum(z * z, axis=(1, 2))
    p = z.copy()
    hist = {"mse": [float(np.mean(r * r))], "rel": [float(np.max(np.sqrt(zz) / btf))]}
    for _ in range(max_iter):
        if hist["rel"][-1] <= rtol:
            break
        w = B_apply(p, c)
        ww = np.sum(w * w, axis=(1, 2))
        alpha = np.where(ww > 0, zz / np.where(ww > 0, ww, 1.0), 0.0)
        g = g + alpha[:, None, None] * p
        r = r - alpha[:, None, None] * w
        z = Bt_apply(r, c)
        zz_new = np.sum(z * z, axis=(1, 2))
        beta = np.where(zz > 0, zz_new / np.where(zz > 0, zz, 1.0), 0.0)
        p = z + beta[:, None, None] * p
        zz = zz_new
        hist["mse"].append(float(np.mean(r * r)))
        hist["rel"].append(float(np.max(np.sqrt(zz) / btf)))
        if mse_gain > 0 and mse_gain_stop(hist["mse"][-2], hist["mse"][-1], mse_gain):
            break
    g = g * cb
    return (g if np.ndim(f) == 3 else g[0]), hist


def mse(u: np.ndarray, f: np.ndarray) -> float:
    """Mean squared error over all pixels and channels (Sec. 4, Sec. 6)."""
    d = np.asarray(u, np.float64) - np.asarray(f, np.float64)
    return float(np.mean(d * d))


_ = sp  # scipy.sparse is used through the split objects
