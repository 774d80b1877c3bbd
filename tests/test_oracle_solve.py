"""Pins for the oracle's Algorithm 1 (DAL + projected two-way Armijo) and Algorithm 2
(ADMM).  The end-to-end values have no printed counterpart in the paper (parity
unpinned beyond these); what is fixed is: the exact trial sequence, accepted step and
carried sigma of the two-way loop on a cost whose values along the search path are known
in closed form (shrink and grow branches, trial cap, stall, stationarity, the projected
direction norm); the Armijo sufficient-decrease inequality, the control staying in E,
the directional derivative along D being -|D|^2, the stall on a constant image, the
extreme regimes of Section 3 (large alpha keeps the image, small alpha drives toward
consensus), the order of the v-step and the multiplier ascent inside a multiplier step
(closed form on a constant image), and the multiplier-step bookkeeping."""
import numpy as np
import pytest

from oracle import Params, SolveOpts, forward, forward_final, adjoint, project
from oracle.solve import (dal_iteration, LtildeObjective, JObjective, admm_solve,
                          dal_solve, initial_control)
from oracle.tv import cost_Ltilde, dLtilde_dc, grad, v_step
from synth import ImageSpec, make_image

SMALL = ImageSpec(16, 16, 3, regions=3, sigma=0.05)


def test_direction_is_descent_with_slope_minus_norm():
    c0 = make_image(SMALL, 3)
    p = Params(radius=2, nsteps=5, alpha=300.0)
    mu = np.zeros((16, 16, 2, 3))
    v = v_step(c0, mu, p)
    eps = initial_control(p)
    traj = forward(c0, eps, p)
    _, D = adjoint(traj, eps, -dLtilde_dc(traj[-1], v, mu, c0, p), p)
    gnorm2 = p.dt * np.sum(D * D)
    h = 1e-3 / np.sqrt(np.sum(D * D))
    f = lambda t: cost_Ltilde(forward_final(c0, eps + t * D, p), v, mu, c0, p)
    slope = (f(h) - f(-h)) / (2 * h)
    assert slope == pytest.approx(-gnorm2, rel=1e-6)
    assert gnorm2 > 0


def test_dal_iterations_decrease_and_stay_in_box():
    c0 = make_image(SMALL, 4)
    p = Params(radius=2, nsteps=5, alpha=300.0)
    o = SolveOpts()
    mu = np.zeros((16, 16, 2, 3))
    obj = LtildeObjective(c0, v_step(c0, mu, p), mu, p)
    eps, sigma = initial_control(p), o.sigma0
    last = None
    for _ in range(6):
        eps, sigma, info = dal_iteration(c0, eps, sigma, obj, p, o)
        assert np.all(eps >= 2.0) and np.all(eps <= 1100.0)
        if info.gnorm2 == 0.0:
            # at eps = 1100 on a 16x16 grid the spatial term alone exceeds 1 for every
            # neighbour: no pair interacts, D = 0 and the iteration stalls without trials
            assert info.stalled and info.trials == 0
            assert np.all(eps == 1100.0)
        else:
            assert 1 <= info.trials <= o.max_ls
        if not info.stalled:
            assert info.L <= info.L0 - o.ls_c * info.tau * info.gnorm2
            assert info.L == pytest.approx(obj.value(forward_final(c0, eps, p)), rel=1e-14)
        if last is not None:
            assert info.L0 == pytest.approx(last, rel=1e-14)
        last = info.L


def test_constant_image_stalls():
    c0 = np.full((8, 8, 3), 0.4)
    p = Params(radius=2, nsteps=4)
    o = SolveOpts(k_out=2, k_in=3)
    res = admm_solve(c0, p, o)
    assert np.array_equal(res["c"], c0)
    assert np.array_equal(res["eps"], initial_control(p))
    assert all(i.stalled and i.trials == 0 for i in res["inner"])
    assert np.all(res["mu"] == 0.0)


def test_large_alpha_keeps_the_image():
    c0 = make_image(SMALL, 5)
    p = Params(radius=2, nsteps=5, alpha=1e8)
    o = SolveOpts()
    z = np.zeros((16, 16, 2, 3))
    obj = LtildeObjective(c0, z, z, p)
    eps, sigma = initial_control(p), o.sigma0
    d0 = np.abs(forward_final(c0, eps, p) - c0).max()
    for _ in range(4):
        eps, sigma, info = dal_iteration(c0, eps, sigma, obj, p, o)
    d1 = np.abs(forward_final(c0, eps, p) - c0).max()
    assert d1 < 0.5 * d0
    assert np.mean(eps) > 57.0          # interactions shrink: the ellipsoid gets smaller


def test_small_alpha_drives_toward_consensus():
    c0 = make_image(SMALL, 6)
    p = Params(radius=2, nsteps=5, alpha=1e-3, rho=1.0)
    o = SolveOpts()
    obj = JObjective(c0, p)
    eps, sigma = initial_control(p), o.sigma0
    g0 = np.sum(grad(forward_final(c0, eps, p)) ** 2)
    for _ in range(4):
        eps, sigma, info = dal_iteration(c0, eps, sigma, obj, p, o)
    g1 = np.sum(grad(forward_final(c0, eps, p)) ** 2)
    assert g1 < g0
    assert np.mean(eps) < 57.0          # interactions grow


def test_admm_small_run_bookkeeping():
    c0 = make_image(ImageSpec(20, 24, 3, regions=3, sigma=0.05), 7)
    p = Params(radius=2, nsteps=4)
    o = SolveOpts(k_out=4, k_in=3)
    res = admm_solve(c0, p, o)
    assert res["outer_done"] == 4 and len(res["outer"]) == 4
    assert np.all(res["eps"] >= 2.0) and np.all(res["eps"] <= 1100.0)
    for s in res["outer"]:
        assert s["gap"] == pytest.approx(p.gamma * s["r"] ** 2 / (20 * 24), rel=1e-12)
    # the returned state is consistent: c = c(T; eps), v = shrink(G c - mu_prev/rho)
    assert np.allclose(res["c"], forward_final(c0, res["eps"], p), atol=0, rtol=0)


def test_admm_tolerance_stops_early():
    # a constant image is a fixed point with G c = v = mu = 0: res_1 = 0 < tol
    c0 = np.full((8, 8, 3), 0.4)
    p = Params(radius=2, nsteps=3)
    res = admm_solve(c0, p, SolveOpts(k_out=6, k_in=2, tol=1e-4))
    assert res["outer_done"] == 1 and res["outer"][0]["res"] == 0.0
    res = admm_solve(c0, p, SolveOpts(k_out=3, k_in=2, tol=0.0))
    assert res["outer_done"] == 3


def test_dal_solve_with_J_decreases_cost():
    c0 = make_image(SMALL, 8)
    p = Params(radius=2, nsteps=5, alpha=50.0, rho=1.0)
    res = dal_solve(c0, p, SolveOpts(), max_iter=5)
    Ls = [i.L for i in res["log"]]
    assert all(b <= a for a, b in zip(Ls, Ls[1:]))
    assert res["log"][-1].L < res["log"][0].L0


# ---------------------------------------------------------------------------------------
# Algorithm 1's two-way Armijo loop on an objective whose trial values are known in
# closed form.  The forward sweep, the adjoint and the terminal cost are replaced by a
# quadratic f(eps) = 1/2 |eps - e*|^2 of the control itself, with the adjoint returning
# D = lambda^T / dt so that df/deps = -dt D, the convention of the real sweep.  Along
# eps + tau D the cost is f0 (1 - tau/dt)^2 and |P D|^2 = dt |D|^2 = 2 f0 / dt, so the
# sufficient-decrease test f(tau) <= f0 - c tau |PD|^2 holds exactly for
# 0 < tau <= 2 (1 - c) dt: with dt = 1/4, c = 1e-4 that is tau <= 0.49995, and the trial
# sequence of every case below follows by hand.
# ---------------------------------------------------------------------------------------

class _QuadraticControlCost:
    """f(e) = 1/2 sum (e - target)^2; records every control it is evaluated at."""

    def __init__(self, target):
        self.target = np.asarray(target, dtype=np.float64)
        self.calls = []

    def value(self, e):
        self.calls.append(np.array(e, dtype=np.float64))
        return 0.5 * float(np.sum((e - self.target) ** 2))

    def gradient(self, e):
        return np.asarray(e, dtype=np.float64) - self.target


@pytest.fixture
def control_only_sweeps(monkeypatch):
    """The state is the control: c(T; eps) = eps, and the adjoint hands back D = lambda^T/dt."""
    import oracle.solve as solve_mod
    monkeypatch.setattr(solve_mod, "forward", lambda c0, eps, p: [np.array(eps, dtype=np.float64)])
    monkeypatch.setattr(solve_mod, "forward_final", lambda c0, eps, p: np.array(eps, dtype=np.float64))
    monkeypatch.setattr(solve_mod, "adjoint", lambda traj, eps, lamT, p: (None, np.asarray(lamT) / p.dt))
    return solve_mod


def _trial_steps(obj, eps, D):
    """The step tau of every trial control the loop evaluated (the first call is L0)."""
    taus = []
    for e in obj.calls[1:]:
        moved = D != 0.0
        taus.append(float(np.mean((e[moved] - eps[moved]) / D[moved])))
    return taus


def _armijo_case(solve_mod, sigma, max_ls=30, ls_c=1e-4, eps=None, target=None, p=None):
    p = p or Params(radius=1, nsteps=2)
    eps = np.full((2, 2), 500.0) if eps is None else np.asarray(eps, dtype=np.float64)
    target = np.full((2, 2), 600.0) if target is None else np.asarray(target, dtype=np.float64)
    obj = _QuadraticControlCost(target)
    o = SolveOpts(max_ls=max_ls, ls_c=ls_c)
    D = -(eps - target) / p.dt
    eps_new, sigma_new, info = solve_mod.dal_iteration(None, eps, sigma, obj, p, o)
    return eps_new, sigma_new, info, _trial_steps(obj, eps, D), D, obj


def test_armijo_shrink_branch_trace(control_only_sweeps):
    # sigma = 1 fails, 1/2 fails (0.5 > 0.49995: only the c-term rejects it), 1/4 passes
    eps_new, sigma_new, info, taus, D, obj = _armijo_case(control_only_sweeps, sigma=1.0)
    assert taus == [1.0, 0.5, 0.25]
    assert info.trials == 3 and info.tau == 0.25 and sigma_new == 0.25
    assert not info.stalled and not info.stationary
    f0 = 0.5 * 4 * 100.0 ** 2
    assert info.L0 == f0 and info.gnorm2 == pytest.approx(2 * f0 / 0.25, rel=1e-15)
    assert info.L == pytest.approx(f0 * (1 - 0.25 / 0.25) ** 2, abs=1e-9)
    assert np.allclose(eps_new, 500.0 + 0.25 * D, rtol=0, atol=0)


def test_armijo_grow_branch_accepts_last_passing_step(control_only_sweeps):
    # sigma = 1/64 passes, the loop doubles while the test passes: 1/32 .. 1/4 pass,
    # 1/2 fails, and the LAST PASSING step 1/4 is accepted and carried as sigma
    eps_new, sigma_new, info, taus, D, obj = _armijo_case(control_only_sweeps, sigma=1.0 / 64)
    assert taus == [1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2]
    assert info.trials == 6 and info.tau == 0.25 and sigma_new == 0.25
    assert np.allclose(eps_new, 500.0 + 0.25 * D, rtol=0, atol=0)


def test_armijo_grow_branch_stops_at_trial_cap(control_only_sweeps):
    eps_new, sigma_new, info, taus, D, obj = _armijo_case(control_only_sweeps, sigma=1.0 / 64,
                                                          max_ls=3)
    assert taus == [1 / 64, 1 / 32, 1 / 16]
    assert info.trials == 3 and info.tau == 1 / 16 and sigma_new == 1 / 16
    assert np.allclose(eps_new, 500.0 + D / 16, rtol=0, atol=0)


def test_armijo_stall_keeps_control_and_sigma(control_only_sweeps):
    # tau = 4 and 2 both increase the cost (eps moves 80 tau towards a target 20 away,
    # staying inside E); with two trials allowed nothing passes
    eps = np.full((2, 2), 300.0)
    eps_new, sigma_new, info, taus, D, obj = _armijo_case(
        control_only_sweeps, sigma=4.0, max_ls=2, eps=eps, target=np.full((2, 2), 320.0))
    assert taus == [4.0, 2.0]
    assert info.stalled and not info.stationary and info.tau == 0.0 and info.trials == 2
    assert sigma_new == 4.0 and np.array_equal(eps_new, eps)
    assert info.L == info.L0


def test_armijo_projected_direction_norm(control_only_sweeps):
    # eps^0_x sits on the upper bound 1100 and D pushes it outward: that component is
    # blocked, |P D|^2 = dt * (three free components of 400^2) = 120000, not 160000.
    # Along the projected path f = 5000 + 15000 (1 - 4 tau)^2 and the test with c = 0.4
    # passes for tau <= (1 - c)/2 = 0.3 (with the unprojected |D|^2 it would need
    # tau <= 0.2333), so sigma = 1/4 passes, 1/2 fails and 1/4 is accepted.
    eps = np.array([[1100.0, 500.0], [500.0, 500.0]])
    target = np.array([[1200.0, 600.0], [600.0, 600.0]])
    eps_new, sigma_new, info, taus, D, obj = _armijo_case(
        control_only_sweeps, sigma=0.25, ls_c=0.4, eps=eps, target=target)
    assert info.gnorm2 == pytest.approx(0.25 * 3 * 400.0 ** 2, rel=1e-15)
    assert info.trials == 2 and info.tau == 0.25 and sigma_new == 0.25
    assert eps_new[0, 0] == 1100.0                       # clipped by Pi_E
    assert np.allclose(eps_new[[0, 1, 1], [1, 0, 1]], 600.0, rtol=0, atol=0)
    assert info.L == pytest.approx(5000.0, abs=1e-9)


def test_armijo_stationary_control_takes_no_trial(control_only_sweeps):
    # every component on the upper bound with D pointing outward: the variational
    # inequality holds, no trial is evaluated
    eps = np.full((2, 2), 1100.0)
    eps_new, sigma_new, info, taus, D, obj = _armijo_case(
        control_only_sweeps, sigma=1.0, eps=eps, target=np.full((2, 2), 1300.0))
    assert info.stationary and info.stalled and info.trials == 0 and taus == []
    assert np.array_equal(eps_new, eps) and sigma_new == 1.0 and info.gnorm2 == 0.0


# ---------------------------------------------------------------------------------------
# Algorithm 2's order inside a multiplier step: v^j = shrink(G c^j - mu^(j-1)/rho, 1/rho)
# FIRST, then mu^j = mu^(j-1) + gamma (v^j - G c^j).  On a constant image G c = 0 and the
# control cannot move (D = 0), so from a multiplier mu^0 the first step gives in closed
# form v^1 = -(mu^0/rho) (1 - 1/|mu^0_i|)_+ and, with gamma = rho, mu^1 = the projection
# of mu^0 onto the unit ball of each pixel's 2xC block.  Doing the ascent first would
# leave v^1 = 0 wherever |mu^0_i| > 1.
# ---------------------------------------------------------------------------------------

def test_admm_v_step_uses_previous_multiplier():
    H, W, C = 6, 5, 3
    c0 = np.full((H, W, C), 0.4)
    p = Params(radius=2, nsteps=3)                      # rho = gamma = 1e-2
    rng = np.random.default_rng(77)
    mu0 = rng.normal(scale=0.9, size=(H, W, 2, C))
    n = np.sqrt(np.sum(mu0 * mu0, axis=(-2, -1)))
    assert np.any(n > 1.0) and np.any(n < 1.0)          # both shrink branches occur
    res = admm_solve(c0, p, SolveOpts(k_out=1, k_in=2), mu0=mu0)
    keep = np.maximum(1.0 - 1.0 / n, 0.0)[..., None, None]
    v1 = -(mu0 / p.rho) * keep
    mu1 = mu0 * np.minimum(1.0, 1.0 / n)[..., None, None]
    assert np.array_equal(res["c"], c0)
    assert np.allclose(res["v"], v1, rtol=1e-13, atol=1e-13)
    assert np.allclose(res["mu"], mu1, rtol=1e-13, atol=1e-15)
    # second step: |mu^1| <= 1 everywhere, so v^2 = 0 and mu^2 = mu^1
    res2 = admm_solve(c0, p, SolveOpts(k_out=2, k_in=2), mu0=mu0)
    assert np.all(np.abs(res2["v"]) <= 1e-12)
    assert np.allclose(res2["mu"], mu1, rtol=1e-13, atol=1e-15)
