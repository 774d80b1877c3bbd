"""Algorithm 1 (DAL with projected two-way Armijo) and Algorithm 2 (ADMM), in float64.

TEST INFRASTRUCTURE (see the package docstring): never imported by the CUDA path.

Readings taken here (each also recorded in the design notes):

* Search direction.  Algorithm 1 tests the trial control eps - tau D but then updates
  eps + sigma D.  With lambda(T) = -grad (Eq. opt_system-b), D^n is minus the gradient
  divided by dt, i.e. a descent direction, so the trial and the update both use
  eps + tau D.
* Stationarity.  A component of D is active-blocked when the control sits on a bound of
  E and D pushes it outward; the projection leaves it unchanged.  When every nonzero
  component is blocked, the variational inequality of the Remark on convergence criteria
  holds exactly (D . (e - eps) <= 0 for all e in E): the control is stationary and the
  epsilon-step ends without trials.
* Sufficient decrease.  The test is L(Pi_E(eps + tau D)) < L(eps) and
  L(Pi_E(eps + tau D)) <= L(eps) - c tau |P D|^2, with |P D|^2 = dt sum_n |P D^n|^2
  (rectangular quadrature, Section 3.2) and P D the direction with blocked components
  zeroed.  Without active bounds P D = D, the printed test; with them, |P D|^2 is minus
  the slope of L along the projected path, whereas the printed |D|^2 would demand a
  decrease the projection cannot deliver and reject every step.  The strict inequality
  is implied by the printed one in exact arithmetic; it stops the rounding of
  L(eps) - c tau |P D|^2 from accepting a step that does not lower L.
* Two-way loop.  Start at tau = sigma.  If the test fails, halve (tau <- b tau) until it
  passes; if it passes, double (tau <- tau / b) while it keeps passing and accept the
  last tau that passed (the printed loop would return the first failing tau).  At most
  max_ls trials per iteration.  If no trial passes the iteration is a stall: eps and
  sigma are unchanged and the current epsilon-step ends (repeating it would repeat the
  same trials).  sigma carries the accepted tau to the next iteration.
* Algorithm 2.  mu^(0) = 0 and eps^(0) = 57 (Section 3.2) unless given; the
  epsilon-argmin of its control step is approximated by k_in DAL iterations at fixed
  (v^(j-1), mu^(j-1)); gamma = rho (Section 4.2).
* Stopping.  The "gap" of Section 4.1 is reported as gamma dx dy |v - G c|^2; the
  optional tolerance test is res_j = max(|c^j - c^(j-1)| / |c^j|,
  |L~_j - L~_(j-1)| / |L~_(j-1)|) < tol, with L~_j = L~(c^j, v^j, mu^j).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .model import Params, forward, forward_final, adjoint, project
from .tv import (cost_Ltilde, dLtilde_dc, cost_J, dJ_dc, grad, v_step, dual_ascent,
                 alm_stats)


@dataclass(frozen=True)
class SolveOpts:
    """Algorithm 1/2 options; Armijo defaults sigma0 = 1, b = 1/2, c = 1e-4 (Section 3.2)."""
    k_out: int = 10
    k_in: int = 30
    max_ls: int = 30
    sigma0: float = 1.0
    ls_b: float = 0.5
    ls_c: float = 1e-4
    tol: float = 0.0            # 0: run all k_out multiplier steps


class LtildeObjective:
    """Terminal cost L~(c(T), v, mu) of Eq. complete_square and its c-gradient."""

    def __init__(self, c0, v, mu, p: Params):
        self.c0, self.v, self.mu, self.p = c0, v, mu, p

    def value(self, cT):
        return cost_Ltilde(cT, self.v, self.mu, self.c0, self.p)

    def gradient(self, cT):
        return dLtilde_dc(cT, self.v, self.mu, self.c0, self.p)


class JObjective:
    """Terminal cost J(c(T)) of Eq. cost_functional and its c-gradient."""

    def __init__(self, c0, p: Params):
        self.c0, self.p = c0, p

    def value(self, cT):
        return cost_J(cT, self.c0, self.p)

    def gradient(self, cT):
        return dJ_dc(cT, self.c0, self.p)


@dataclass
class DalInfo:
    L0: float
    L: float
    gnorm2: float
    tau: float
    trials: int
    stalled: bool            # the epsilon-step ends here (stationary or no admissible step)
    stationary: bool = False


def free_components(eps, D, p: Params) -> np.ndarray:
    """Mask of the components of D that the projection onto E does not block."""
    lo = np.asarray(p.eps_lo, dtype=np.float64)
    hi = np.asarray(p.eps_hi, dtype=np.float64)
    return (D != 0.0) & ((eps < hi) | (D < 0.0)) & ((eps > lo) | (D > 0.0))


def dal_iteration(c0, eps, sigma, obj, p: Params, o: SolveOpts):
    """One pass of Algorithm 1's loop body.  Returns (eps_new, sigma_new, DalInfo)."""
    traj = forward(c0, eps, p)
    L0 = obj.value(traj[-1])
    _, D = adjoint(traj, eps, -obj.gradient(traj[-1]), p)
    free = free_components(eps, D, p)
    gnorm2 = p.dt * float(np.sum(np.where(free, D, 0.0) ** 2))
    if not np.any(free):
        return eps, sigma, DalInfo(L0, L0, 0.0, 0.0, 0, True, True)

    def trial(tau):
        e = project(eps + tau * D, p)
        L = obj.value(forward_final(c0, e, p))
        return (L < L0) and (L <= L0 - o.ls_c * tau * gnorm2), L, e

    tau = sigma
    ok, L, e = trial(tau)
    trials = 1
    if ok:
        best = (tau, L, e)
        while trials < o.max_ls:
            tau = tau / o.ls_b
            ok, L, e = trial(tau)
            trials += 1
            if not ok:
                break
            best = (tau, L, e)
    else:
        best = None
        while trials < o.max_ls:
            tau = tau * o.ls_b
            ok, L, e = trial(tau)
            trials += 1
            if ok:
                best = (tau, L, e)
                break
    if best is None:
        return eps, sigma, DalInfo(L0, L0, gnorm2, 0.0, trials, True)
    tau, L, e = best
    return e, tau, DalInfo(L0, L, gnorm2, tau, trials, False)


def initial_control(p: Params, value: float = 57.0) -> np.ndarray:
    """eps^(0) = (57, 57) at every step (Section 3.2)."""
    return np.full((p.nsteps, 2), value)


def admm_solve(c0, p: Params, o: SolveOpts, eps0=None, mu0=None):
    """Algorithm 2.  Returns a dict with eps, c, v, mu, the per-multiplier-step log and
    the per-DAL-iteration log."""
    c0 = np.asarray(c0, dtype=np.float64)
    H, W, C = c0.shape
    eps = initial_control(p) if eps0 is None else np.array(eps0, dtype=np.float64)
    mu = np.zeros((H, W, 2, C)) if mu0 is None else np.array(mu0, dtype=np.float64)
    sigma = o.sigma0
    c = forward_final(c0, eps, p)
    v = v_step(c, mu, p)
    L_prev = cost_Ltilde(c, v, mu, c0, p)
    outer_log, inner_log = [], []
    done = 0
    for j in range(1, o.k_out + 1):
        obj = LtildeObjective(c0, v, mu, p)
        for _ in range(o.k_in):
            eps, sigma, info = dal_iteration(c0, eps, sigma, obj, p, o)
            inner_log.append(info)
            if info.stalled:
                break
        c_new = forward_final(c0, eps, p)
        v_new = v_step(c_new, mu, p)
        mu_new = dual_ascent(mu, v_new, c_new, p)
        stats = alm_stats(c_new, v_new, v, c, c0, p)
        L_new = cost_Ltilde(c_new, v_new, mu_new, c0, p)
        res = max(stats["rel_dc"], abs(L_new - L_prev) / abs(L_prev) if L_prev != 0 else 0.0)
        stats.update({"Ltilde": L_new, "res": res, "sigma": sigma})
        outer_log.append(stats)
        c, v, mu, L_prev = c_new, v_new, mu_new, L_new
        done = j
        if o.tol > 0.0 and res < o.tol:
            break
    return {"eps": eps, "c": c, "v": v, "mu": mu, "outer": outer_log, "inner": inner_log,
            "outer_done": done}


def dal_solve(c0, p: Params, o: SolveOpts, max_iter: int = 100, eta: float = 1e-10,
              eps0=None):
    """Algorithm 1 with the quadratic cost J (Section 3), stopping on the relative change
    of the cost below eta (Remark on convergence criteria) or after max_iter iterations."""
    c0 = np.asarray(c0, dtype=np.float64)
    eps = initial_control(p) if eps0 is None else np.array(eps0, dtype=np.float64)
    sigma = o.sigma0
    obj = JObjective(c0, p)
    log = []
    for _ in range(max_iter):
        eps, sigma, info = dal_iteration(c0, eps, sigma, obj, p, o)
        log.append(info)
        if info.stalled or (info.L0 != 0 and abs(info.L - info.L0) / abs(info.L0) < eta):
            break
    return {"eps": eps, "c": forward_final(c0, eps, p), "log": log}
