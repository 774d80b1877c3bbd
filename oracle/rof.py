"""ROF (Eq. cost_TV) solved without the agents, as pins for the TV operators.

TEST INFRASTRUCTURE (see the package docstring): never imported by the CUDA path.

Two independent loops over a free colour field c, each using the oracle's G, G^T and
the per-pixel ball projection / shrinkage:

* ``rof_chambolle_pock``: the primal-dual algorithm of Chambolle and Pock (cited by the
  paper for ROF) on  min_c sum_i |G c_i| + alpha/2 |c - c0|^2  (the cell factor dx dy
  is a constant and is dropped), with the dual ball |p_i| <= 1.
* ``rof_admm``: the splitting of Section 4.1 with an exact c-step -- c minimises
  L~(., v, mu) by solving dLtilde_dc = 0, i.e. (alpha I + rho G^T G) c = alpha c0
  + G^T (rho v + mu); then the v-step (Eq. soft_threshold) and the dual ascent
  (Eq. dual_ascent).  Its fixed point is the ROF minimiser, so it pins the terminal
  gradient, the shrinkage and the ascent signs together.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .model import Params
from .tv import grad, grad_T, grad_matrix, project_ball, v_step, dual_ascent


def rof_primal(c, c0, alpha, tv_mode=0):
    g = grad(c)
    if tv_mode == 0:
        tv = np.sum(np.sqrt(np.sum(g * g, axis=(-2, -1))))
    else:
        tv = np.sum(np.sqrt(np.sum(g * g, axis=-2)))
    return float(tv + 0.5 * alpha * np.sum((c - c0) ** 2))


def rof_dual(pdual, c0, alpha):
    """D(p) = <G^T p, c0> - |G^T p|^2 / (2 alpha), for |p_i| <= 1."""
    gtp = grad_T(pdual)
    return float(np.sum(gtp * c0) - np.sum(gtp * gtp) / (2.0 * alpha))


def rof_chambolle_pock(c0, alpha, iters, tv_mode=0):
    """Accelerated primal-dual iteration (strongly convex in c).  Returns (c, p, gaps)."""
    c0 = np.asarray(c0, dtype=np.float64)
    H, W, C = c0.shape
    L = float(np.sqrt((W ** 2) + (H ** 2)))      # |G| <= sqrt(1/dx^2 + 1/dy^2)
    tau = sigma = 0.99 / L
    c = c0.copy()
    cbar = c.copy()
    pd = np.zeros((H, W, 2, C))
    gaps = []
    for _ in range(iters):
        pd = project_ball(pd + sigma * grad(cbar), 1.0, tv_mode)
        c_new = (c - tau * grad_T(pd) + tau * alpha * c0) / (1.0 + tau * alpha)
        theta = 1.0 / np.sqrt(1.0 + 2.0 * alpha * tau)
        tau, sigma = theta * tau, sigma / theta
        cbar = c_new + theta * (c_new - c)
        c = c_new
        gaps.append(rof_primal(c, c0, alpha, tv_mode) - rof_dual(pd, c0, alpha))
    return c, pd, np.array(gaps)


def rof_admm(c0, alpha, rho, iters, tv_mode=0):
    """Exact-c-step ADMM on L~ (Section 4.1 splitting without the agents)."""
    c0 = np.asarray(c0, dtype=np.float64)
    H, W, C = c0.shape
    p = Params(alpha=alpha, rho=rho, gamma=rho, tv_mode=tv_mode)
    G = grad_matrix(H, W)
    # dLtilde_dc = cell [G^T (rho G c - rho v - mu) + alpha (c - c0)] = 0
    A = (alpha * sp.identity(H * W) + rho * (G.T @ G)).tocsc()
    solve = spla.factorized(A)
    c = c0.copy()
    mu = np.zeros((H, W, 2, C))
    v = v_step(c, mu, p)
    for _ in range(iters):
        rhs = alpha * c0 + grad_T(rho * v + mu)
        for ch in range(C):
            c[:, :, ch] = solve(rhs[:, :, ch].reshape(-1)).reshape(H, W)
        v = v_step(c, mu, p)
        mu = dual_ascent(mu, v, c, p)
    return c, v, mu
