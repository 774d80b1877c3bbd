"""Pins for the oracle's discrete TV operators, costs and ADMM sub-steps (Section 4).

Fixed by the paper or by mathematics: the central-difference gradient on an affine ramp
and on a hand-worked 3x4 example with the reflective rule (Definition 3.1,
Eq. reflective_boundary); G^T against a dense transpose assembled column by column;
the shrinkage against brute-force minimisation of the function whose minimiser
Eq. soft_threshold derives; the identities Eq. complete_square and the linearity of L in
mu (Section 4.1); and the ROF closed form on a two-level step, reached by two different
solvers built from these operators.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import Params
from oracle.tv import (grad, grad_T, shrink, project_ball, cost_J, cost_K, cost_L,
                       cost_Ltilde, v_step, dual_ascent, alm_stats)
from oracle.rof import rof_chambolle_pock, rof_admm


def test_grad_affine_ramp():
    H, W = 6, 9
    a, b = 0.3, -0.7
    rows, cols = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    c = (a * cols / W + b * rows / H + 0.1)[:, :, None]
    g = grad(c)
    # interior: exact slope
    assert np.allclose(g[1:-1, 1:-1, 0, 0], a, atol=1e-12)
    assert np.allclose(g[1:-1, 1:-1, 1, 0], b, atol=1e-12)
    # reflective boundary: zero normal derivative, tangential slope kept
    assert np.allclose(g[:, 0, 0, 0], 0.0) and np.allclose(g[:, -1, 0, 0], 0.0)
    assert np.allclose(g[0, :, 1, 0], 0.0) and np.allclose(g[-1, :, 1, 0], 0.0)
    assert np.allclose(g[0, 1:-1, 0, 0], a) and np.allclose(g[1:-1, 0, 1, 0], b)


def test_grad_hand_example():
    # 3 rows x 4 cols, dx = 1/4, dy = 1/3; 1/(2dx) = 2, 1/(2dy) = 1.5
    c = np.array([[0., 1., 3., 6.],
                  [2., 2., 5., 1.],
                  [4., 0., 1., 7.]])[:, :, None]
    g = grad(c)
    gx = np.array([[0., 2 * (3 - 0), 2 * (6 - 1), 0.],
                   [0., 2 * (5 - 2), 2 * (1 - 2), 0.],
                   [0., 2 * (1 - 4), 2 * (7 - 0), 0.]])
    gy = np.array([[0., 0., 0., 0.],
                   [1.5 * (4 - 0), 1.5 * (0 - 1), 1.5 * (1 - 3), 1.5 * (7 - 6)],
                   [0., 0., 0., 0.]])
    assert np.allclose(g[:, :, 0, 0], gx) and np.allclose(g[:, :, 1, 0], gy)


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (4, 1), (2, 2), (5, 7)])
def test_grad_T_is_dense_transpose(shape, rng):
    H, W = shape
    C = 2
    N = H * W
    dense = np.zeros((2 * N * C, N * C))
    for k in range(N * C):
        e = np.zeros(N * C)
        e[k] = 1.0
        dense[:, k] = grad(e.reshape(H, W, C)).reshape(-1)
    w = rng.normal(size=(H, W, 2, C))
    assert np.allclose(grad_T(w).reshape(-1), dense.T @ w.reshape(-1), atol=1e-12)
    x = rng.normal(size=(H, W, C))
    assert np.sum(grad(x) * w) == pytest.approx(np.sum(x * grad_T(w)), abs=1e-10)
    if H <= 2 and W <= 2:
        assert np.all(dense == 0.0)       # no interior: G vanishes (sides 1 or 2)


@pytest.mark.parametrize("C", [1, 3])
def test_shrink_is_prox_by_brute_force(C, rng):
    rho = 0.7
    theta = 1.0 / rho
    cases = [rng.normal(scale=2.5, size=(2, C)) for _ in range(6)]
    a_edge = rng.normal(size=(2, C))
    cases.append(a_edge / np.linalg.norm(a_edge) * theta)   # |a| = 1/rho exactly
    cases.append(np.zeros((2, C)))
    for a in cases:
        f = lambda w: 0.5 * rho * np.sum((w - a.ravel()) ** 2) + np.linalg.norm(w)
        best = min((minimize(f, x0, method="Nelder-Mead",
                             options={"xatol": 1e-12, "fatol": 1e-14, "maxiter": 40000})
                    for x0 in (a.ravel(), np.zeros(a.size) + 1e-3)), key=lambda r: r.fun)
        w = shrink(a[None, None], theta)[0, 0]
        assert f(w.ravel()) <= best.fun + 1e-10
        assert np.allclose(w.ravel(), best.x, atol=1e-5)


def test_moreau_identity(rng):
    a = rng.normal(scale=3.0, size=(5, 6, 2, 3))
    theta = 2.0
    assert np.allclose(shrink(a, theta) + project_ball(a, theta), a, atol=1e-14)
    n = np.sqrt(np.sum(project_ball(a, theta) ** 2, axis=(-2, -1)))
    assert np.all(n <= theta + 1e-12)


def test_channelwise_tv_mode(rng):
    a = rng.normal(scale=3.0, size=(4, 4, 2, 3))
    w = shrink(a, 2.0, tv_mode=1)
    for ch in range(3):
        assert np.allclose(w[..., ch:ch + 1], shrink(a[..., ch:ch + 1], 2.0, tv_mode=0))


def _fields(rng, H=6, W=5, C=3):
    c0 = rng.uniform(size=(H, W, C))
    c = c0 + rng.normal(scale=0.1, size=c0.shape)
    v = rng.normal(size=(H, W, 2, C))
    mu = rng.normal(size=(H, W, 2, C))
    return c0, c, v, mu


def test_complete_square_identity(rng):
    # Eq. complete_square: L~ = L + dx dy / (2 rho) sum |mu_i|^2
    c0, c, v, mu = _fields(rng)
    p = Params(alpha=7.0, rho=0.3)
    H, W, _ = c.shape
    lhs = cost_Ltilde(c, v, mu, c0, p)
    rhs = cost_L(c, v, mu, c0, p) + (1.0 / (W * H)) / (2 * p.rho) * np.sum(mu * mu)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_J_is_Ltilde_special_case(rng):
    c0, c, _, _ = _fields(rng)
    p = Params(alpha=7.0, rho=1.0)
    z = np.zeros(c.shape[:2] + (2, c.shape[2]))
    assert cost_J(c, c0, p) == pytest.approx(cost_Ltilde(c, z, z, c0, p), rel=1e-13)


def test_K_at_v_equal_grad(rng):
    # at v = G c the penalty and multiplier terms vanish: L = K
    c0, c, _, mu = _fields(rng)
    p = Params(alpha=7.0, rho=0.3)
    assert cost_L(c, grad(c), mu, c0, p) == pytest.approx(cost_K(c, c0, p), rel=1e-13)


def test_v_step_minimises_L():
    rng = np.random.default_rng(2024)
    c0, c, _, mu = _fields(rng)
    # choose rho so that the threshold 1/rho splits the pixels: both shrink branches occur
    a_norm = np.sqrt(np.sum((grad(c)) ** 2, axis=(-2, -1)))
    mu = mu * 0.0
    p = Params(alpha=7.0, rho=1.0 / float(np.median(a_norm)))
    v = v_step(c, mu, p)
    base = cost_L(c, v, mu, c0, p)
    for _ in range(20):
        dv = rng.normal(scale=1e-3, size=v.shape)
        assert cost_L(c, v + dv, mu, c0, p) >= base - 1e-15
    zero = np.all(v == 0.0, axis=(-2, -1))
    assert np.any(zero) and not np.all(zero)
    assert np.array_equal(zero, a_norm <= 1.0 / p.rho)


def test_dual_ascent_gap(rng):
    # L is linear in mu, so the mu-step raises L by exactly gamma dx dy |v - G c|^2
    c0, c, v, mu = _fields(rng)
    p = Params(alpha=7.0, rho=0.3, gamma=0.3)
    mu2 = dual_ascent(mu, v, c, p)
    inc = cost_L(c, v, mu2, c0, p) - cost_L(c, v, mu, c0, p)
    stats = alm_stats(c, v, v, c, c0, p)
    assert inc == pytest.approx(stats["gap"], rel=1e-10)
    assert stats["s"] == 0.0 and stats["rel_dc"] == 0.0
    assert stats["r"] == pytest.approx(np.sqrt(np.sum((v - grad(c)) ** 2)), rel=1e-14)


def _two_level_step():
    c0 = np.zeros((4, 64, 1))
    c0[:, :32] = 0.2
    c0[:, 32:] = 0.8
    return c0


def test_rof_two_level_step_admm():
    # ROF on a step a | b over half the width each: p = a + 1/(alpha s), q = b - 1/(alpha s)
    # with s = 1/2, alpha = 50: 0.24 | 0.76
    c, v, mu = rof_admm(_two_level_step(), alpha=50.0, rho=1.0, iters=2000)
    assert np.max(np.abs(c[:, :32] - 0.24)) < 1e-6
    assert np.max(np.abs(c[:, 32:] - 0.76)) < 1e-6


def test_rof_two_level_step_chambolle_pock():
    c0 = _two_level_step()
    c, pd, gaps = rof_chambolle_pock(c0, alpha=50.0, iters=20000)
    assert np.max(np.abs(c[:, :32] - 0.24)) < 1e-5
    assert np.max(np.abs(c[:, 32:] - 0.76)) < 1e-5
    # the primal-dual gap falls by six orders of magnitude, running minimum monotone
    assert np.all(gaps >= -1e-9)
    assert gaps[-1] <= 1e-6 * gaps[0]
    run = np.minimum.accumulate(gaps)
    assert np.all(np.diff(run) <= 0.0)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_alm_stats_hand_example(axis):
    # three pixels along one axis, C = 1, spacing h = 1/3: 1/(2h) = 1.5.  Only the middle
    # pixel has a central difference; (G c)_mid = 1.5 (c_2 - c_0) and G^T w sends the
    # middle pixel's w to (-1.5 w, 0, +1.5 w).
    shape = (1, 3, 1) if axis == "x" else (3, 1, 1)
    comp = 0 if axis == "x" else 1
    c = np.array([1.0, 2.0, 2.0]).reshape(shape)
    c_prev = np.array([1.0, 2.0, 0.0]).reshape(shape)
    c0 = np.zeros(shape)
    v = np.zeros(shape[:2] + (2, 1))
    v_prev = np.zeros_like(v)
    mid = (0, 1) if axis == "x" else (1, 0)
    v[mid + (comp, 0)] = 5.0
    v_prev[mid + (comp, 0)] = 3.0
    p = Params(alpha=4.0, rho=0.37, gamma=0.21)
    st = alm_stats(c, v, v_prev, c_prev, c0, p)
    # v - G c = 5 - 1.5 = 3.5 at the middle pixel, 0 elsewhere
    assert st["r"] == pytest.approx(3.5, rel=1e-15)
    assert st["gap"] == pytest.approx(0.21 * (1.0 / 3.0) * 3.5 ** 2, rel=1e-14)
    # G^T (v - v_prev) = (-3, 0, 3): s = rho * 3 sqrt(2)
    assert st["s"] == pytest.approx(0.37 * 3.0 * np.sqrt(2.0), rel=1e-14)
    # |c - c_prev| = 2, |c| = 3
    assert st["rel_dc"] == pytest.approx(2.0 / 3.0, rel=1e-15)
    # K = dx dy [|G c| + alpha/2 |c - c0|^2] = (1/3)(1.5 + 2 * 9)
    assert st["K"] == pytest.approx((1.0 / 3.0) * (1.5 + 2.0 * 9.0), rel=1e-14)


def test_alm_stats_dual_residual_against_dense_transpose(rng):
    # s = rho |G^T (v - v_prev)| with G^T the transpose of a dense G assembled column by
    # column from unit images; rel_dc from its definition on random fields
    H, W, C = 4, 5, 2
    N = H * W
    dense = np.zeros((2 * N * C, N * C))
    for k in range(N * C):
        e = np.zeros(N * C)
        e[k] = 1.0
        dense[:, k] = grad(e.reshape(H, W, C)).reshape(-1)
    c0, c, v, _ = _fields(rng, H, W, C)
    c_prev = c + rng.normal(scale=0.05, size=c.shape)
    v_prev = v + rng.normal(scale=0.5, size=v.shape)
    p = Params(alpha=7.0, rho=0.37, gamma=0.21)
    st = alm_stats(c, v, v_prev, c_prev, c0, p)
    s_dense = 0.37 * np.linalg.norm(dense.T @ (v - v_prev).reshape(-1))
    assert st["s"] == pytest.approx(s_dense, rel=1e-12)
    rel = np.sqrt(np.sum((c - c_prev) ** 2)) / np.sqrt(np.sum(c * c))
    assert st["rel_dc"] == pytest.approx(rel, rel=1e-13)
    r_dense = np.linalg.norm(v.reshape(-1) - dense @ c.reshape(-1))
    assert st["r"] == pytest.approx(r_dense, rel=1e-13)
