"""Discrete gradient, costs, terminal adjoint, shrinkage and dual ascent, in float64.

TEST INFRASTRUCTURE (see the package docstring): never imported by the CUDA path.

Fields: c is (H, W, C); the split variable v and the multiplier mu are (H, W, 2, C),
component 0 along x (columns), component 1 along y (rows).

Readings taken here (each also recorded in the design notes):

* The discrete Jacobian of Definition 3.1 is built as an explicit sparse matrix G from
  its central differences and the reflective index rules of Eq. reflective_boundary
  (a missing index +-1 is replaced by its mirror -+1, so G is zero on the border
  rows/columns in the normal direction).  A side of length 1 has no neighbour at all;
  G along that axis is zero.
* Section 3.1 and Eq. admm_terminal write the Laplacian and divergence terms with a
  "wide" Laplacian and div#, which equal G^T G and -G^T only two or more pixels from the
  border (the +-2 reflection is also undefined by Eq. reflective_boundary).  We use the
  exact transpose G^T of the sparse matrix, i.e. the exact derivative of the discrete
  cost, so every gradient here is what finite differences measure.
* Colour (C > 1, not in the paper): G acts per channel; |v_i| is the Frobenius norm of
  the 2 x C block (coupled vectorial TV, tv_mode 0), and the shrinkage of
  Eq. soft_threshold is the group soft-threshold on that block.  tv_mode 1 takes the
  norm per channel instead.  With C = 1 both are the paper verbatim.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

from .model import Params


@functools.lru_cache(maxsize=32)
def grad_matrix(H: int, W: int) -> sp.csr_matrix:
    """Sparse G of shape (2N, N) on row-major pixel index i = row * W + col: rows 0..N-1
    hold the x-differences, rows N..2N-1 the y-differences (Definition 3.1)."""
    hx, hy = 1.0 / W, 1.0 / H
    N = H * W

    def mirror(k, n):
        # indices k in [-1, n]: -1 -> 1 and n -> n-2 (Eq. reflective_boundary)
        k = k.copy()
        k[k < 0] = 1
        k[k >= n] = n - 2
        return k

    rr, qq = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    i = (rr * W + qq).ravel()
    rows, cols, vals = [], [], []
    if W > 1:
        right = (rr * W + mirror(qq + 1, W)).ravel()
        left = (rr * W + mirror(qq - 1, W)).ravel()
        rows += [i, i]
        cols += [right, left]
        vals += [np.full(N, 1.0 / (2 * hx)), np.full(N, -1.0 / (2 * hx))]
    if H > 1:
        up = (mirror(rr + 1, H) * W + qq).ravel()
        down = (mirror(rr - 1, H) * W + qq).ravel()
        rows += [N + i, N + i]
        cols += [up, down]
        vals += [np.full(N, 1.0 / (2 * hy)), np.full(N, -1.0 / (2 * hy))]
    if not rows:
        return sp.csr_matrix((2 * N, N))
    G = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * N, N)).tocsr()
    G.sum_duplicates()
    G.eliminate_zeros()
    return G


def grad(c: np.ndarray) -> np.ndarray:
    """(G c) per channel, shape (H, W, 2, C)."""
    H, W, C = c.shape
    G = grad_matrix(H, W)
    out = np.empty((H, W, 2, C))
    for ch in range(C):
        g = G @ c[:, :, ch].reshape(-1)
        out[:, :, 0, ch] = g[:H * W].reshape(H, W)
        out[:, :, 1, ch] = g[H * W:].reshape(H, W)
    return out


def grad_T(w: np.ndarray) -> np.ndarray:
    """(G^T w) per channel for w of shape (H, W, 2, C); result (H, W, C)."""
    H, W, two, C = w.shape
    assert two == 2
    GT = grad_matrix(H, W).T.tocsr()
    out = np.empty((H, W, C))
    for ch in range(C):
        flat = np.concatenate([w[:, :, 0, ch].reshape(-1), w[:, :, 1, ch].reshape(-1)])
        out[:, :, ch] = (GT @ flat).reshape(H, W)
    return out


def _norms(w: np.ndarray, tv_mode: int) -> np.ndarray:
    """Per-pixel TV norm of (H, W, 2, C) data: Frobenius over the 2xC block (mode 0) or
    the 2-vector norm per channel (mode 1, shape (H, W, C))."""
    if tv_mode == 0:
        return np.sqrt(np.sum(w * w, axis=(-2, -1)))
    if tv_mode == 1:
        return np.sqrt(np.sum(w * w, axis=-2))
    raise ValueError("tv_mode must be 0 or 1")


def tv_sum(w: np.ndarray, tv_mode: int) -> float:
    return float(np.sum(_norms(w, tv_mode)))


def shrink(a: np.ndarray, theta: float, tv_mode: int = 0) -> np.ndarray:
    """argmin_w theta |w| + 1/2 |w - a|^2 (Eq. soft_threshold with theta = 1/rho):
    0 where |a| <= theta, (|a| - theta) a / |a| otherwise."""
    n = _norms(a, tv_mode)
    keep = np.where(n > theta, 1.0 - theta / np.where(n > 0, n, 1.0), 0.0)
    if tv_mode == 0:
        return a * keep[..., None, None]
    return a * keep[..., None, :]


def project_ball(a: np.ndarray, radius: float, tv_mode: int = 0) -> np.ndarray:
    """Projection onto the per-pixel ball |w| <= radius (the dual ball)."""
    n = _norms(a, tv_mode)
    scale = np.where(n > radius, radius / np.where(n > 0, n, 1.0), 1.0)
    if tv_mode == 0:
        return a * scale[..., None, None]
    return a * scale[..., None, :]


def _cell(c: np.ndarray) -> float:
    H, W, _ = c.shape
    return (1.0 / W) * (1.0 / H)


def cost_J(c: np.ndarray, c0: np.ndarray, p: Params) -> float:
    """Eq. cost_functional: 1/2 dx dy sum_i [|G c_i|^2 + alpha |c_i - c0_i|^2]."""
    g = grad(c)
    return 0.5 * _cell(c) * float(np.sum(g * g) + p.alpha * np.sum((c - c0) ** 2))


def cost_K(c: np.ndarray, c0: np.ndarray, p: Params) -> float:
    """Eq. cost_TV: dx dy sum_i [|G c_i| + alpha/2 |c_i - c0_i|^2]."""
    return _cell(c) * (tv_sum(grad(c), p.tv_mode) + 0.5 * p.alpha * float(np.sum((c - c0) ** 2)))


def cost_L(c, v, mu, c0, p: Params) -> float:
    """Eq. cost_tv_regular: dx dy sum_i [|v_i| + mu_i.(v_i - G c_i)
    + rho/2 |v_i - G c_i|^2 + alpha/2 |c_i - c0_i|^2]."""
    r = v - grad(c)
    return _cell(c) * (tv_sum(v, p.tv_mode) + float(np.sum(mu * r))
                       + 0.5 * p.rho * float(np.sum(r * r))
                       + 0.5 * p.alpha * float(np.sum((c - c0) ** 2)))


def cost_Ltilde(c, v, mu, c0, p: Params) -> float:
    """Eq. complete_square: dx dy sum_i [rho/2 |v_i - G c_i + mu_i/rho|^2 + |v_i|
    + alpha/2 |c_i - c0_i|^2]."""
    q = v - grad(c) + mu / p.rho
    return _cell(c) * (0.5 * p.rho * float(np.sum(q * q)) + tv_sum(v, p.tv_mode)
                       + 0.5 * p.alpha * float(np.sum((c - c0) ** 2)))


def dLtilde_dc(c, v, mu, c0, p: Params) -> np.ndarray:
    """Gradient of L~ in c (Eq. admm_terminal in exact-transpose form):
    dx dy [G^T (rho G c - rho v - mu) + alpha (c - c0)]."""
    return _cell(c) * (grad_T(p.rho * grad(c) - p.rho * v - mu) + p.alpha * (c - c0))


def dJ_dc(c, c0, p: Params) -> np.ndarray:
    """Gradient of J in c (Section 3.1, exact-transpose form): dx dy [G^T G c + alpha (c - c0)]."""
    return _cell(c) * (grad_T(grad(c)) + p.alpha * (c - c0))


def terminal_adjoint(c, v, mu, c0, p: Params) -> np.ndarray:
    """lambda(T) = -dL~/dc at c(T) (Eq. opt_system-b terminal condition, Section 4.1)."""
    return -dLtilde_dc(c, v, mu, c0, p)


def v_step(c, mu, p: Params) -> np.ndarray:
    """v = argmin_v L(c, v, mu) = shrink(G c - mu/rho, 1/rho) (Eq. soft_threshold)."""
    return shrink(grad(c) - mu / p.rho, 1.0 / p.rho, p.tv_mode)


def dual_ascent(mu, v, c, p: Params) -> np.ndarray:
    """mu <- mu + gamma (v - G c) (Eq. dual_ascent)."""
    return mu + p.gamma * (v - grad(c))


def alm_stats(c, v, v_prev, c_prev, c0, p: Params) -> dict:
    """Residuals reported with each multiplier step:
    r = |v - G c|_2 (primal), s = rho |G^T (v - v_prev)|_2 (dual),
    gap = gamma dx dy |v - G c|^2 (increase of L across the mu-step, exact because L is
    linear in mu), rel_dc = |c - c_prev| / |c|, and the ROF energy K(c)."""
    rr = v - grad(c)
    r = float(np.sqrt(np.sum(rr * rr)))
    s = p.rho * float(np.sqrt(np.sum(grad_T(v - v_prev) ** 2)))
    gap = p.gamma * _cell(c) * float(np.sum(rr * rr))
    nc = float(np.sqrt(np.sum(c * c)))
    rel = float(np.sqrt(np.sum((c - c_prev) ** 2))) / nc if nc > 0 else 0.0
    return {"r": r, "s": s, "gap": gap, "rel_dc": rel, "K": cost_K(c, c0, p)}
