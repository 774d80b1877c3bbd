"""GPU parity of the TV kernels (shrinkage v-step, float64 multiplier update with its
residuals, objective L~ and terminal adjoint) against the FP64 oracle, through the C ABI.

Inputs are float32; the oracle receives the same float32 values promoted to float64.
Tolerances follow from float32 arithmetic on O(1) colours and O(W) gradients: fields
within 1e-5 of their largest entry, float64-reduced scalars within 1e-5 relative, the
float64 multiplier update within one float32 rounding of the oracle's exact value.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, f32, zeros_dev, torch
import oracle
from oracle.tv import v_step, dual_ascent, alm_stats, cost_Ltilde, terminal_adjoint, grad
from paper_2510_16154_gb300 import lib

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 3), (1, 9, 3), (9, 1, 1), (2, 2, 3), (3, 4, 1), (37, 150, 3), (129, 67, 1),
          (40, 70, 5), (256, 300, 3)]


def _inputs(rng, H, W, C):
    c0 = f32(rng.uniform(0, 1, size=(H, W, C)))
    c = f32(np.clip(c0 + rng.normal(scale=0.1, size=c0.shape), 0, 1))
    g = grad(c)
    scale = max(float(np.median(np.abs(g))), 1.0)
    v = f32(rng.normal(scale=scale, size=(H, W, 2, C)))
    mu = f32(rng.normal(scale=0.3 * scale, size=(H, W, 2, C)))
    return c0, c, v, mu, scale


def _rho_for(c, mu, scale):
    # threshold 1/rho near the median |G c - mu/rho| so both shrink branches occur
    a = np.sqrt(np.sum(grad(c) ** 2, axis=(-2, -1)))
    med = float(np.median(a))
    return 1.0 / med if med > 0 else 1.0 / scale


@pytest.mark.parametrize("tv_mode", [0, 1])
@pytest.mark.parametrize("H,W,C", SHAPES)
def test_pd_tv_step(H, W, C, tv_mode):
    ensure_lib()
    rng = np.random.default_rng(H * 31 + W + C)
    c0, c, _, mu, scale = _inputs(rng, H, W, C)
    rho = _rho_for(c, mu * 0, scale)
    mu = f32(mu * 0.2 * rho)       # keeps mu/rho comparable to G c
    p, op = params(H, W, C, 2, 1, rho=rho, gamma=rho, tv_mode=tv_mode)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        v = zeros_dev(H, W, 2, C)
        lib.pd_tv_step(ctx.handle, dev(c, np.float32), dev(mu, np.float32), v)
        got = host(v).astype(np.float64)
    want = v_step(c, mu, op)
    a = grad(c) - mu / rho
    tol = 1e-5 * max(np.max(np.abs(a)), 1e-30)
    assert np.max(np.abs(got - want)) <= tol
    if H > 2 and W > 2:
        assert np.any(want == 0) and np.any(want != 0)


def _assert_correctly_rounded(got, mu, v, c, op, rng, samples=3000):
    """On sampled entries the update is the float32 value nearest to the exact
    mu + gamma (v - G c) (gamma the float64 nearest its value), computed in rational
    arithmetic from the oracle's gradient (exact here: float32 colours times W/2, H/2),
    except where the exact value lies within 1e-6 ulp of a float32 midpoint: there the
    float64 rounding of the update decides (gamma near 1/20 makes such near-ties common,
    and the oracle's own float64 evaluation falls on either side of them too); the result
    is then one of the two neighbours."""
    from fractions import Fraction
    g = grad(c)
    n = got.size
    idx = rng.choice(n, size=min(samples, n), replace=False)
    gf, mf, vf, gr = (x.reshape(-1) for x in (got, mu, v, g))
    gam = Fraction(op.gamma)
    ties = 0
    for i in idx:
        exact = Fraction(mf[i]) + gam * (Fraction(vf[i]) - Fraction(gr[i]))
        y = np.float32(float(exact))
        cands = [y, np.nextafter(y, np.float32(np.inf)), np.nextafter(y, np.float32(-np.inf))]
        dist = [abs(Fraction(float(z)) - exact) for z in cands]
        best = cands[int(np.argmin(dist))]
        if np.float32(gf[i]) == best:
            continue
        ulp = Fraction(float(np.spacing(np.abs(best))))
        d_got = abs(Fraction(float(np.float32(gf[i]))) - exact)
        assert d_got <= ulp, f"entry {i}: more than one ulp off"
        assert abs(d_got / ulp - Fraction(1, 2)) < Fraction(1, 10**6), f"entry {i}: not a near-tie"
        ties += 1


@pytest.mark.parametrize("H,W,C", SHAPES)
def test_alm_update(H, W, C):
    ensure_lib()
    rng = np.random.default_rng(H * 17 + W + C)
    c0, c, v, mu, scale = _inputs(rng, H, W, C)
    c_prev = f32(np.clip(c + rng.normal(scale=0.01, size=c.shape), 0, 1))
    v_prev = f32(v + rng.normal(scale=0.1 * scale, size=v.shape))
    p, op = params(H, W, C, 2, 1, alpha=50.0, rho=0.05, gamma=0.05)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        m = dev(mu, np.float32)
        stats = np.zeros(5)
        lib.alm_update(ctx.handle, dev(c, np.float32), dev(c_prev, np.float32),
                       dev(v, np.float32), dev(v_prev, np.float32), m, stats)
        got = host(m).astype(np.float64)
    want = dual_ascent(mu, v, c, op)
    # float64 update rounded once to float32: within one float32 ulp of the exact value
    ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got - want) <= ulp)
    _assert_correctly_rounded(got, mu, v, c, op, rng)
    ws = alm_stats(c, v, v_prev, c_prev, c0, op)
    for k, name in enumerate(["r", "s", "gap", "rel_dc", "K"]):
        assert stats[k] == pytest.approx(ws[name], rel=1e-5, abs=1e-12), name


def test_alm_update_null_prev_and_device_stats():
    ensure_lib()
    rng = np.random.default_rng(4)
    c0, c, v, mu, _ = _inputs(rng, 20, 33, 3)
    p, op = params(20, 33, 3, 2, 1)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        st = torch.zeros(5, dtype=torch.float64, device="cuda")
        lib.alm_update(ctx.handle, dev(c, np.float32), None, dev(v, np.float32), None,
                       dev(mu, np.float32), st)
        st = host(st)
    assert st[1] == 0.0 and st[3] == 0.0
    ws = alm_stats(c, v, v, c, c0, op)
    assert st[0] == pytest.approx(ws["r"], rel=1e-5) and st[4] == pytest.approx(ws["K"], rel=1e-5)


@pytest.mark.parametrize("tv_mode", [0, 1])
@pytest.mark.parametrize("H,W,C", SHAPES)
def test_objective_and_terminal_adjoint(H, W, C, tv_mode):
    ensure_lib()
    rng = np.random.default_rng(H * 7 + W + C)
    c0, c, v, mu, _ = _inputs(rng, H, W, C)
    p, op = params(H, W, C, 2, 1, alpha=300.0, rho=0.2, tv_mode=tv_mode)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        lam = zeros_dev(H, W, C)
        obj = np.zeros(1)
        lib.agents_objective(ctx.handle, dev(c, np.float32), dev(v, np.float32),
                             dev(mu, np.float32), obj, lam)
        got = host(lam).astype(np.float64)
    assert obj[0] == pytest.approx(cost_Ltilde(c, v, mu, c0, op), rel=1e-6)
    want = terminal_adjoint(c, v, mu, c0, op)
    assert np.max(np.abs(got - want)) <= 1e-5 * max(np.max(np.abs(want)), 1e-30)


@pytest.mark.parametrize("tv_mode", [0, 1])
@pytest.mark.parametrize("H,W,C", SHAPES + [(517, 391, 3), (300, 1030, 1)])
def test_terminal_objective_equals_trial_objective_bitwise(H, W, C, tv_mode):
    # Algorithm 1 compares the L~ that comes with the terminal adjoint against the L~ of
    # each Armijo trial (objective only): for the same fields they must be the same
    # float64 number, or rounding alone could accept or reject a trial.
    ensure_lib()
    rng = np.random.default_rng(H * 11 + W + 3 * C)
    c0, c, v, mu, _ = _inputs(rng, H, W, C)
    p, _ = params(H, W, C, 2, 1, alpha=300.0, rho=0.2, tv_mode=tv_mode)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        cd, vd, md = dev(c, np.float32), dev(v, np.float32), dev(mu, np.float32)
        with_lam, without = np.zeros(1), np.zeros(1)
        lib.agents_objective(ctx.handle, cd, vd, md, with_lam, zeros_dev(H, W, C))
        lib.agents_objective(ctx.handle, cd, vd, md, without, None)
    assert with_lam[0] == without[0]


def test_full_size_tv_kernels():
    # the 1024 x 1024 x 3 fields of the throughput benchmark
    ensure_lib()
    from synth import ImageSpec, make_image
    rng = np.random.default_rng(9)
    c0 = f32(make_image(ImageSpec(1024, 1024, 3, regions=12, ramp=0.1, sigma=0.08), 2))
    c = f32(np.clip(c0 + rng.normal(scale=0.01, size=c0.shape), 0, 1))
    mu = f32(rng.normal(scale=0.5, size=(1024, 1024, 2, 3)))
    p, op = params(1024, 1024, 3, 5, 1)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        cd, md = dev(c, np.float32), dev(mu, np.float32)
        v = zeros_dev(1024, 1024, 2, 3)
        lib.pd_tv_step(ctx.handle, cd, md, v)
        vh = host(v).astype(np.float64)
        obj = np.zeros(1)
        lam = zeros_dev(1024, 1024, 3)
        lib.agents_objective(ctx.handle, cd, v, md, obj, lam)
        stats = np.zeros(5)
        lib.alm_update(ctx.handle, cd, dev(c0, np.float32), v, None, md, stats)
        muh = host(md).astype(np.float64)
        lamh = host(lam).astype(np.float64)
    want_v = v_step(c, mu, op)
    a = grad(c) - mu / op.rho
    assert np.max(np.abs(vh - want_v)) <= 1e-5 * np.max(np.abs(a))
    assert np.count_nonzero(want_v) > 1000
    assert obj[0] == pytest.approx(cost_Ltilde(c, vh, mu, c0, op), rel=1e-6)
    want_lam = terminal_adjoint(c, vh, mu, c0, op)
    assert np.max(np.abs(lamh - want_lam)) <= 1e-5 * np.max(np.abs(want_lam))
    want_mu = dual_ascent(mu, vh, c, op)
    ulp = np.spacing(np.abs(want_mu).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(muh - want_mu) <= ulp)
    _assert_correctly_rounded(muh, mu, vh, c, op, rng)
    ws = alm_stats(c, vh, vh, c0, c0, op)
    assert stats[0] == pytest.approx(ws["r"], rel=1e-5)
    assert stats[2] == pytest.approx(ws["gap"], rel=1e-5)
    assert stats[4] == pytest.approx(ws["K"], rel=1e-5)
