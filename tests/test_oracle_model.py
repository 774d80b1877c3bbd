"""Pins for the oracle's agent dynamics and adjoint (Section 2, Section 3.1, Eq. kernel).

Each check is fixed by the paper or by mathematics, not by re-typing the oracle: special
values of the Wendland kernel, invariants of the alignment dynamics, a brute-force
all-pairs evaluation of Eq. MAsystem, and finite differences for every derivative.
"""
import numpy as np
import pytest

from oracle import (Params, phi, dphi, velocity, forward, forward_final, velocity_at,
                    jacobian_transpose_apply_at,
                    jacobian_transpose_apply, control_derivative, adjoint, project,
                    window_offsets)
from oracle.tv import cost_Ltilde, dLtilde_dc, cost_J, dJ_dc


# ---------------------------------------------------------------- kernel (Eq. kernel)

def test_phi_special_values():
    # C2 Wendland function (1-r)^4 (4r+1): phi(0)=1, phi(1/2)=3/16, phi(1/4)=(3/4)^4*2
    assert phi(0.0) == 1.0
    assert phi(0.5) == pytest.approx(3.0 / 16.0, abs=1e-15)
    assert phi(0.25) == pytest.approx(0.6328125, abs=1e-15)
    assert phi(1.0) == 0.0 and dphi(1.0) == 0.0
    assert phi(1.5) == 0.0 and dphi(7.0) == 0.0
    # the printed (4r-1)(1-r)^4 would give phi(0) = -1 (repulsion); the reading is >= 0
    r = np.linspace(0.0, 3.0, 3001)
    assert np.all(phi(r) >= 0.0)
    # monotone non-increasing on [0, 1]
    assert np.all(np.diff(phi(np.linspace(0, 1, 1001))) <= 0.0)


def test_dphi_is_derivative_and_c2_at_support_edge():
    r = np.linspace(0.01, 1.4, 500)
    h = 1e-6
    fd = (phi(r + h) - phi(r - h)) / (2 * h)
    assert np.max(np.abs(fd - dphi(r))) < 1e-8
    # second derivative vanishes at r = 1 from the left (C2 support edge)
    h = 1e-4
    d2 = (phi(1 - 2 * h) - 2 * phi(1 - h) + phi(1.0)) / h ** 2
    assert abs(d2) < 1e-2


# ---------------------------------------------------------------- dynamics (Eq. MAsystem)

def _brute_velocity(c, ex, ec, R, norm_mode):
    """Double loop over ordered agent pairs, written from Eq. MAsystem / Eq. ellipsoid."""
    H, W, C = c.shape
    N = H * W
    M = (2 * R + 1) ** 2 if norm_mode == 0 else N
    F = np.zeros_like(c)
    for i in range(N):
        ri, qi = divmod(i, W)
        for j in range(N):
            rj, qj = divmod(j, W)
            if j == i or abs(rj - ri) > R or abs(qj - qi) > R:
                continue
            dist2 = ((qj - qi) / W) ** 2 + ((rj - ri) / H) ** 2
            col2 = sum((c[rj, qj, k] - c[ri, qi, k]) ** 2 for k in range(C))
            r = ex / 2 * dist2 + ec / 2 * col2
            w = (1 - r) ** 4 * (4 * r + 1) if r <= 1 else 0.0
            for k in range(C):
                F[ri, qi, k] += w * (c[rj, qj, k] - c[ri, qi, k]) / M
    return F


@pytest.mark.parametrize("C", [1, 3])
def test_all_pairs_special_case(C, rng):
    # With R >= max(H, W) and M = N the windowed dynamics are Eq. MAsystem verbatim.
    c = rng.uniform(0.3, 0.6, size=(5, 4, C))
    p = Params(radius=6, norm_mode=1)
    F = velocity(c, 9.0, 20.0, p)
    assert np.max(np.abs(F - _brute_velocity(c, 9.0, 20.0, 6, 1))) < 1e-15
    assert np.max(np.abs(F)) > 1e-3      # the case is not trivially zero


def test_windowed_matches_brute_force(rng):
    c = rng.uniform(0.0, 1.0, size=(7, 5, 3))
    p = Params(radius=2)
    F = velocity(c, 30.0, 4.0, p)
    assert np.max(np.abs(F - _brute_velocity(c, 30.0, 4.0, 2, 0))) < 1e-15


def test_window_offsets_count():
    for R in range(1, 6):
        off = window_offsets(R)
        assert len(off) == (2 * R + 1) ** 2 - 1 and len(set(off)) == len(off)


def test_constant_image_is_fixed_point():
    c0 = np.full((9, 11, 3), 0.37)
    p = Params(radius=3, nsteps=6)
    eps = np.full((6, 2), 5.0)
    cT = forward_final(c0, eps, p)
    assert np.array_equal(cT, c0)


def test_convex_hull_and_extrema(rng):
    # Explicit Euler with dt * sum(phi)/M <= 1 is a convex combination of the window.
    c = rng.uniform(0.0, 1.0, size=(12, 10, 3))
    p = Params(radius=2, nsteps=8)
    eps = np.column_stack([np.full(8, 2.0), np.full(8, 3.0)])
    traj = forward(c, eps, p)
    for n in range(p.nsteps):
        a, b = traj[n], traj[n + 1]
        H, W, _ = a.shape
        for r in range(H):
            for q in range(W):
                win = a[max(0, r - 2):r + 3, max(0, q - 2):q + 3].reshape(-1, 3)
                assert np.all(b[r, q] >= win.min(axis=0) - 1e-14)
                assert np.all(b[r, q] <= win.max(axis=0) + 1e-14)
        assert np.all(b.max(axis=(0, 1)) <= a.max(axis=(0, 1)) + 1e-14)
        assert np.all(b.min(axis=(0, 1)) >= a.min(axis=(0, 1)) - 1e-14)
    assert np.max(np.abs(traj[-1] - traj[0])) > 1e-3


def test_no_interaction_when_far_apart():
    # colours more than sqrt(2/eps_c) apart never interact: a two-level image is fixed
    c = np.zeros((6, 6, 1))
    c[:, 3:] = 1.0
    p = Params(radius=2, nsteps=3)
    eps = np.full((3, 2), 50.0)
    assert np.array_equal(forward_final(c, eps, p), c)


# ---------------------------------------------------------------- derivatives (Section 3.1)

def test_jacobian_transpose_by_finite_differences(rng):
    c = rng.uniform(0.2, 0.7, size=(6, 7, 3))
    lam = rng.normal(size=c.shape)
    u = rng.normal(size=c.shape)
    p = Params(radius=2)
    ex, ec = 40.0, 9.0
    h = 1e-6
    Ju = (velocity(c + h * u, ex, ec, p) - velocity(c - h * u, ex, ec, p)) / (2 * h)
    lhs = np.sum(jacobian_transpose_apply(c, lam, ex, ec, p) * u)
    rhs = np.sum(lam * Ju)
    assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs))
    assert abs(rhs) > 1e-3


def test_control_derivative_by_finite_differences(rng):
    c = rng.uniform(0.2, 0.7, size=(6, 7, 3))
    lam = rng.normal(size=c.shape)
    p = Params(radius=2)
    ex, ec = 40.0, 9.0
    h = 1e-5
    D = control_derivative(c, lam, ex, ec, p)
    fx = (np.sum(lam * velocity(c, ex + h, ec, p)) - np.sum(lam * velocity(c, ex - h, ec, p))) / (2 * h)
    fc = (np.sum(lam * velocity(c, ex, ec + h, p)) - np.sum(lam * velocity(c, ex, ec - h, p))) / (2 * h)
    assert D[0] == pytest.approx(fx, rel=1e-6, abs=1e-12)
    assert D[1] == pytest.approx(fc, rel=1e-6, abs=1e-12)


@pytest.mark.parametrize("H,W,C,R", [(9, 13, 3, 3), (5, 6, 1, 6), (7, 4, 2, 1)])
def test_control_derivative_paired_form(H, W, C, R):
    # D_x = 1/(2M) sum_i sum_j phi'(r_ij) |x_j - x_i|^2 (lam_i . delta_ij) (likewise D_c
    # with |delta_ij|^2).  phi'(r_ij) and both distances are symmetric in (i, j), delta_ij
    # is antisymmetric and the window relation is symmetric, so pairing (i, j) with
    # (j, i) gives -1/2 sum_i sum_j phi'(r_ij) |x_j - x_i|^2 (delta_ij . (lam_j - lam_i)):
    # the form the GPU adjoint accumulates.  Brute force over ordered pairs.
    rng = np.random.default_rng(H * 100 + W * 10 + C + R)
    c = rng.uniform(0.3, 0.7, size=(H, W, C))
    lam = rng.normal(size=c.shape)
    p = Params(radius=R)
    ex, ec = 37.0, 11.0
    M = (2 * R + 1) ** 2
    paired = np.zeros(2)
    for i in range(H):
        for j in range(W):
            for k in range(max(0, i - R), min(H, i + R + 1)):
                for m in range(max(0, j - R), min(W, j + R + 1)):
                    if (k, m) == (i, j):
                        continue
                    d = c[k, m] - c[i, j]
                    s = float(d @ d)
                    d2 = ((m - j) / W) ** 2 + ((k - i) / H) ** 2
                    r = 0.5 * ex * d2 + 0.5 * ec * s
                    g = float(dphi(r)) * float(d @ (lam[k, m] - lam[i, j]))
                    paired += -0.5 * g * np.array([d2, s])
    paired /= 2 * M
    D = control_derivative(c, lam, ex, ec, p)
    assert np.all(np.abs(paired) > 1e-7)
    assert np.allclose(D, paired, rtol=1e-12, atol=1e-18)


def _adjoint_case(rng, C=3, H=8, W=8, T=6):
    img = rng.uniform(0.2, 0.8, size=(H, W, C))
    p = Params(radius=2, nsteps=T, alpha=30.0, rho=0.5)
    v = rng.normal(scale=2.0, size=(H, W, 2, C))
    mu = rng.normal(scale=0.5, size=(H, W, 2, C))
    eps = rng.uniform(3.0, 60.0, size=(T, 2))
    return img, p, v, mu, eps


def test_terminal_adjoint_by_finite_differences(rng):
    img, p, v, mu, _ = _adjoint_case(rng)
    c = img + rng.normal(scale=0.05, size=img.shape)
    g = dLtilde_dc(c, v, mu, img, p)
    h = 1e-6
    # L~ and J are quadratic in c, so the central difference is exact but for the rounding
    # of the two evaluations, a few eps |L~| / h: 10 eps |L~| / h covers it.
    eps = np.finfo(float).eps
    for _ in range(6):
        u = rng.normal(size=c.shape)
        fd = (cost_Ltilde(c + h * u, v, mu, img, p) - cost_Ltilde(c - h * u, v, mu, img, p)) / (2 * h)
        tol = 10 * eps * abs(cost_Ltilde(c, v, mu, img, p)) / h
        assert np.sum(g * u) == pytest.approx(fd, rel=1e-7, abs=tol)
    gJ = dJ_dc(c, img, p)
    u = rng.normal(size=c.shape)
    fd = (cost_J(c + h * u, img, p) - cost_J(c - h * u, img, p)) / (2 * h)
    tol = 10 * eps * abs(cost_J(c, img, p)) / h
    assert np.sum(gJ * u) == pytest.approx(fd, rel=1e-7, abs=tol)


@pytest.mark.parametrize("T", [5, 12])
def test_control_gradient_by_finite_differences(T, rng):
    # dL~(c(T; eps))/deps^n = -dt D^n  (exact discrete adjoint of explicit Euler)
    img, p, v, mu, eps = _adjoint_case(rng, T=T)
    traj = forward(img, eps, p)
    lamT = -dLtilde_dc(traj[-1], v, mu, img, p)
    _, D = adjoint(traj, eps, lamT, p)
    grad = -p.dt * D

    def cost(e):
        return cost_Ltilde(forward_final(img, e, p), v, mu, img, p)

    def fd_grad(h):
        out = np.zeros_like(eps)
        for n in range(T):
            for k in range(2):
                e1, e2 = eps.copy(), eps.copy()
                e1[n, k] += h
                e2[n, k] -= h
                out[n, k] = (cost(e1) - cost(e2)) / (2 * h)
        return out

    scale = np.max(np.abs(grad))
    # Normwise error: single entries can be 1e-8 next to |L~| ~ 10, where central
    # differences lose all digits to round-off (about eps_mach |L~| / h).
    assert np.max(np.abs(fd_grad(1e-4) - grad)) <= 1e-6 * scale
    # h = 1e-6 is round-off limited: eps_mach * |L~| / h ~ 3e-9 absolute
    L = abs(cost(eps))
    assert np.max(np.abs(fd_grad(1e-6) - grad)) <= 10 * 2.2e-16 * L / 1e-6 + 1e-6 * scale
    # and along a random direction
    d = rng.normal(size=eps.shape)
    fd = (cost(eps + 1e-4 * d) - cost(eps - 1e-4 * d)) / 2e-4
    assert np.sum(grad * d) == pytest.approx(fd, rel=1e-6)


def test_control_gradient_single_channel_all_pairs(rng):
    # C = 1, M = N, window covering the image: the paper's grey-scale system verbatim
    H, W, T = 4, 5, 4
    img = rng.uniform(0.3, 0.5, size=(H, W, 1))
    p = Params(radius=8, nsteps=T, norm_mode=1, alpha=10.0, rho=1.0)
    v = np.zeros((H, W, 2, 1))
    mu = np.zeros((H, W, 2, 1))
    eps = rng.uniform(3.0, 30.0, size=(T, 2))
    traj = forward(img, eps, p)
    _, D = adjoint(traj, eps, -dLtilde_dc(traj[-1], v, mu, img, p), p)
    h = 1e-4
    grad = -p.dt * D
    fd = np.zeros_like(grad)
    for n in range(T):
        for k in range(2):
            e1, e2 = eps.copy(), eps.copy()
            e1[n, k] += h
            e2[n, k] -= h
            fd[n, k] = (cost_Ltilde(forward_final(img, e1, p), v, mu, img, p)
                        - cost_Ltilde(forward_final(img, e2, p), v, mu, img, p)) / (2 * h)
    assert np.max(np.abs(fd - grad)) <= 1e-6 * np.max(np.abs(grad))
    assert np.max(np.abs(grad)) > 0.0


def test_projection_is_box_clip():
    p = Params()
    e = np.array([[1.0, 5000.0], [57.0, -3.0], [2.0, 1100.0]])
    assert np.array_equal(project(e, p), np.array([[2.0, 1100.0], [57.0, 2.0], [2.0, 1100.0]]))


def test_pointwise_evaluations_match_field_versions(rng):
    c = rng.uniform(0.2, 0.7, size=(9, 13, 3))
    lam = rng.normal(size=c.shape)
    p = Params(radius=3)
    rows = [0, 0, 4, 8, 8, 3]
    cols = [0, 12, 6, 0, 12, 1]
    F = velocity(c, 40.0, 12.0, p)
    assert np.allclose(velocity_at(c, rows, cols, 40.0, 12.0, p), F[rows, cols], atol=1e-15)
    JT = jacobian_transpose_apply(c, lam, 40.0, 12.0, p)
    assert np.allclose(jacobian_transpose_apply_at(c, lam, rows, cols, 40.0, 12.0, p),
                       JT[rows, cols], atol=1e-14)
