"""Agent dynamics, explicit Euler and its exact discrete adjoint, in float64.

TEST INFRASTRUCTURE (see the package docstring): never imported by the CUDA path.

State: a colour field ``c`` of shape (H, W, C), float64.  Memory row ``k`` is the
paper's k-th row counted from the bottom (Section 2: rows ordered bottom to top, agent
index i = k * N_C + col + 1), so no index flip is ever needed.  Pixel positions are in
the unit square: x = col * dx, y = row * dy with dx = 1/N_C, dy = 1/N_R
(Definition 3.1), because Section 2 places the interaction ellipsoid in [0, 1]^3.

Readings of the paper taken here (each also recorded in the design notes):

* Kernel (Eq. kernel).  The printed polynomial (4r - 1)(1 - r)^4 is negative for
  r < 1/4 and gives phi(0) = -1, which would make close agents repel; the cited C2
  Wendland function is (1 - r)^4 (4 r + 1).  We use the Wendland function:
  phi(r) = (1 - r)^4 (4 r + 1) on [0, 1], 0 beyond; phi'(r) = -20 r (1 - r)^3.
* Window.  Eq. MAsystem sums over all N agents with weight 1/N.  Here agent i
  interacts with the in-image agents j != i whose row and column differ from i's by at
  most R (clipped at the border, no reflection), with a constant weight 1/M,
  M = (2R+1)^2 (norm_mode 0).  norm_mode 1 uses M = N; with R >= max(H, W) that is
  Eq. MAsystem verbatim.
* Colour.  The paper is grey-scale; for C channels (c_j - c_i)^2 in Eq. ellipsoid
  becomes the squared Euclidean norm over channels.  C = 1 is the paper verbatim.
* Time.  Explicit Euler with step dt (Section 3.2), the control piecewise constant on
  each step: c^{n+1} = c^n + dt F(c^n, eps^n), n = 0..T-1.
* Adjoint.  The paper integrates Eq. opt_system-b backwards without saying how.  We use
  the exact adjoint of the explicit Euler scheme, lambda^n = lambda^{n+1}
  + dt J_F(c^n, eps^n)^T lambda^{n+1}, so that dL/deps^n = -dt D^n exactly with
  D^n = sum_i lambda^{n+1}_i . dF_i/deps (c^n, eps^n) (Algorithm 1, line D).
* Jacobian diagonal.  Section 3.1 prints the diagonal entry dF_i/dc_i as a sum over all
  j including j = i; the exact derivative excludes j = i (its term is phi(0)/N
  spuriously).  We use the exact derivative.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Params:
    """Problem constants.  Defaults are the paper's (Section 3.2, Section 4.2):
    dt = 0.25, E = [2, 1100]^2, rho = gamma = 1e-2; alpha = 3000 is the fidelity weight
    of the ADMM comparison runs."""
    radius: int = 2
    nsteps: int = 20
    dt: float = 0.25
    alpha: float = 3000.0
    rho: float = 1e-2
    gamma: float = 1e-2
    eps_lo: tuple = (2.0, 2.0)
    eps_hi: tuple = (1100.0, 1100.0)
    norm_mode: int = 0          # 0: M = (2R+1)^2; 1: M = N (Eq. MAsystem's 1/N)
    tv_mode: int = 0            # 0: coupled (Frobenius over the 2xC block); 1: per channel


def phi(r):
    """C2 Wendland kernel (Eq. kernel, read as (1-r)^4 (4r+1)); zero for r > 1."""
    r = np.asarray(r, dtype=np.float64)
    t = 1.0 - r
    t2 = t * t
    return np.where(r <= 1.0, t2 * t2 * (4.0 * r + 1.0), 0.0)


def dphi(r):
    """Derivative of phi: -20 r (1-r)^3 on [0, 1], zero for r > 1."""
    r = np.asarray(r, dtype=np.float64)
    t = 1.0 - r
    return np.where(r <= 1.0, -20.0 * r * (t * t * t), 0.0)


def window_offsets(radius: int):
    """Offsets (drow, dcol) of the (2R+1)^2 - 1 window neighbours, row-major."""
    return [(oy, ox) for oy in range(-radius, radius + 1)
            for ox in range(-radius, radius + 1) if (oy, ox) != (0, 0)]


def norm_constant(H: int, W: int, p: Params) -> float:
    if p.norm_mode == 0:
        return float((2 * p.radius + 1) ** 2)
    if p.norm_mode == 1:
        return float(H * W)
    raise ValueError("norm_mode must be 0 or 1")


def _dot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-pixel inner product over the channel axis."""
    out = a[..., 0] * b[..., 0]
    for ch in range(1, a.shape[-1]):
        out = out + a[..., ch] * b[..., ch]
    return out


def _pair_slices(H: int, W: int, oy: int, ox: int):
    """Slices selecting every agent i whose neighbour j = i + (oy, ox) is in the image,
    and the matching slices of those j."""
    r0, r1 = max(0, -oy), min(H, H - oy)
    c0, c1 = max(0, -ox), min(W, W - ox)
    if r1 <= r0 or c1 <= c0:
        return None
    si = (slice(r0, r1), slice(c0, c1))
    sj = (slice(r0 + oy, r1 + oy), slice(c0 + ox, c1 + ox))
    return si, sj


def _pairs(c: np.ndarray, eps_x: float, eps_c: float, p: Params):
    """Yield (si, sj, delta, d2, s, r) over all window offsets: delta = c_j - c_i,
    d2 = |x_j - x_i|^2 + |y_j - y_i|^2, s = |delta|^2, and r_ij of Eq. ellipsoid."""
    H, W, _ = c.shape
    hx, hy = 1.0 / W, 1.0 / H
    for oy, ox in window_offsets(p.radius):
        sl = _pair_slices(H, W, oy, ox)
        if sl is None:
            continue
        si, sj = sl
        delta = c[sj] - c[si]
        d2 = (ox * hx) ** 2 + (oy * hy) ** 2
        s = _dot(delta, delta)
        r = 0.5 * eps_x * d2 + 0.5 * eps_c * s
        yield si, sj, delta, d2, s, r


def velocity(c: np.ndarray, eps_x: float, eps_c: float, p: Params) -> np.ndarray:
    """F(c, eps): F_i = (1/M) sum_{j in W(i)} phi(r_ij) (c_j - c_i)  (Eq. MAsystem)."""
    H, W, _ = c.shape
    F = np.zeros_like(c)
    for si, _sj, delta, _d2, _s, r in _pairs(c, eps_x, eps_c, p):
        F[si] += phi(r)[..., None] * delta
    return F / norm_constant(H, W, p)


def forward(c0: np.ndarray, eps: np.ndarray, p: Params):
    """Explicit Euler trajectory [c^0, ..., c^T] under control eps of shape (T, 2)."""
    eps = np.asarray(eps, dtype=np.float64)
    if eps.shape != (p.nsteps, 2):
        raise ValueError("eps must have shape (T, 2)")
    traj = [np.asarray(c0, dtype=np.float64)]
    for n in range(p.nsteps):
        c = traj[-1]
        traj.append(c + p.dt * velocity(c, eps[n, 0], eps[n, 1], p))
    return traj


def forward_final(c0: np.ndarray, eps: np.ndarray, p: Params) -> np.ndarray:
    """c^T only (no trajectory kept)."""
    eps = np.asarray(eps, dtype=np.float64)
    c = np.asarray(c0, dtype=np.float64)
    for n in range(p.nsteps):
        c = c + p.dt * velocity(c, eps[n, 0], eps[n, 1], p)
    return c


def jacobian_transpose_apply(c: np.ndarray, lam: np.ndarray, eps_x: float, eps_c: float,
                             p: Params) -> np.ndarray:
    """(dF/dc)^T lam, assembled from the Jacobian entries of Section 3.1 in scatter
    form: for every agent i and neighbour k in W(i), the block
    dF_i/dc_k = (1/M) [phi'(r_ik) eps_c (c_k - c_i)(c_k - c_i)^T + phi(r_ik) I]
    sends dF_i/dc_k^T lam_i to row k, and the diagonal block dF_i/dc_i, which is minus
    the sum of those blocks over k in W(i), sends its share to row i."""
    H, W, _ = c.shape
    out = np.zeros_like(c)
    lam = np.asarray(lam, dtype=np.float64)
    for si, sj, delta, _d2, _s, r in _pairs(c, eps_x, eps_c, p):
        lam_i = lam[si]
        proj = _dot(delta, lam_i)
        block_lam = (dphi(r) * eps_c * proj)[..., None] * delta + phi(r)[..., None] * lam_i
        out[sj] += block_lam      # k = j: off-diagonal entry
        out[si] -= block_lam      # k = i: diagonal entry
    return out / norm_constant(H, W, p)


def control_derivative(c: np.ndarray, lam: np.ndarray, eps_x: float, eps_c: float,
                       p: Params) -> np.ndarray:
    """D = sum_i lam_i . dF_i/deps at (c, eps), with (Section 3.1)
    dF_i/deps_x = 1/(2M) sum_j phi'(r_ij) |x_j - x_i|^2 (c_j - c_i),
    dF_i/deps_c = 1/(2M) sum_j phi'(r_ij) |c_j - c_i|^2 (c_j - c_i)."""
    H, W, _ = c.shape
    dx_sum = 0.0
    dc_sum = 0.0
    lam = np.asarray(lam, dtype=np.float64)
    for si, _sj, delta, d2, s, r in _pairs(c, eps_x, eps_c, p):
        g = dphi(r) * _dot(lam[si], delta)
        dx_sum += float(np.sum(g * d2))
        dc_sum += float(np.sum(g * s))
    scale = 1.0 / (2.0 * norm_constant(H, W, p))
    return np.array([dx_sum * scale, dc_sum * scale])


def adjoint_step(c_n: np.ndarray, lam_next: np.ndarray, eps_n, p: Params):
    """One step of the discrete adjoint of explicit Euler: returns (lam^n, D^n)."""
    ex, ec = float(eps_n[0]), float(eps_n[1])
    lam_n = lam_next + p.dt * jacobian_transpose_apply(c_n, lam_next, ex, ec, p)
    return lam_n, control_derivative(c_n, lam_next, ex, ec, p)


def adjoint(traj, eps: np.ndarray, lamT: np.ndarray, p: Params):
    """Backward sweep n = T-1..0 from lam^T.  Returns (lam^0, D) with D of shape (T, 2);
    the gradient of the terminal cost with respect to eps^n is -dt * D[n]."""
    eps = np.asarray(eps, dtype=np.float64)
    lam = np.asarray(lamT, dtype=np.float64)
    D = np.zeros((p.nsteps, 2))
    for n in range(p.nsteps - 1, -1, -1):
        lam, D[n] = adjoint_step(traj[n], lam, eps[n], p)
    return lam, D


def project(eps: np.ndarray, p: Params) -> np.ndarray:
    """Pi_E: componentwise clip onto the box E = [lo_x, hi_x] x [lo_c, hi_c]."""
    lo = np.asarray(p.eps_lo, dtype=np.float64)
    hi = np.asarray(p.eps_hi, dtype=np.float64)
    return np.minimum(np.maximum(np.asarray(eps, dtype=np.float64), lo), hi)


def velocity_at(c: np.ndarray, rows, cols, eps_x: float, eps_c: float, p: Params) -> np.ndarray:
    """F_i (Eq. MAsystem) at the listed pixels only, one pixel at a time: for checking
    samples of a full-size field.  Returns shape (len(rows), C)."""
    H, W, C = c.shape
    hx, hy = 1.0 / W, 1.0 / H
    M = norm_constant(H, W, p)
    out = np.zeros((len(rows), C))
    for n, (r, q) in enumerate(zip(rows, cols)):
        r0, r1 = max(0, r - p.radius), min(H, r + p.radius + 1)
        q0, q1 = max(0, q - p.radius), min(W, q + p.radius + 1)
        win = c[r0:r1, q0:q1]
        dr = (np.arange(r0, r1) - r)[:, None]
        dq = (np.arange(q0, q1) - q)[None, :]
        delta = win - c[r, q]
        d2 = (dq * hx) ** 2 + (dr * hy) ** 2
        rr = 0.5 * eps_x * d2 + 0.5 * eps_c * np.sum(delta * delta, axis=-1)
        w = phi(rr)
        w[r - r0, q - q0] = 0.0          # j != i
        out[n] = np.sum(w[..., None] * delta, axis=(0, 1)) / M
    return out


def jacobian_transpose_apply_at(c: np.ndarray, lam: np.ndarray, rows, cols, eps_x: float,
                                eps_c: float, p: Params) -> np.ndarray:
    """(dF/dc)^T lam at the listed pixels k, one pixel at a time: row k collects
    dF_i/dc_k^T lam_i from every agent i with k in W(i), plus the diagonal block
    dF_k/dc_k^T lam_k = -sum_{j in W(k)} dF_k/dc_j^T lam_k (Section 3.1)."""
    H, W, C = c.shape
    hx, hy = 1.0 / W, 1.0 / H
    M = norm_constant(H, W, p)
    out = np.zeros((len(rows), C))
    for n, (r, q) in enumerate(zip(rows, cols)):
        acc = np.zeros(C)
        for oy in range(-p.radius, p.radius + 1):
            for ox in range(-p.radius, p.radius + 1):
                ri, qi = r + oy, q + ox          # the other agent of the pair
                if (oy, ox) == (0, 0) or not (0 <= ri < H and 0 <= qi < W):
                    continue
                # k is in W(i) exactly when i is in W(k) (symmetric window)
                delta = c[r, q] - c[ri, qi]      # c_k - c_i
                rr = 0.5 * eps_x * ((ox * hx) ** 2 + (oy * hy) ** 2) + 0.5 * eps_c * np.dot(delta, delta)
                # off-diagonal: block dF_i/dc_k applied to lam_i
                acc += (dphi(rr) * eps_c * np.dot(delta, lam[ri, qi])) * delta + phi(rr) * lam[ri, qi]
                # diagonal: minus block dF_k/dc_i (same r, delta -> -delta) applied to lam_k
                acc -= (dphi(rr) * eps_c * np.dot(delta, lam[r, q])) * delta + phi(rr) * lam[r, q]
        out[n] = acc / M
    return out
