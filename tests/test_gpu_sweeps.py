"""GPU parity of the agent sweeps (forward Euler step, adjoint step, control derivative)
against the FP64 oracle, through the C ABI.

Tolerances: one forward step <= 1e-6 max-abs on colours in [0, 1]; a 20-step sweep
<= 1e-5; adjoint state <= 1e-5 relative to its largest entry; the control derivative
<= 1e-5 relative per component: D_x against its own largest entry and D_c against its
own (a component is checked against the largest entry of D only where it is below 1e-6
of the other, which none of these cases reaches).  Shapes span
several 64 x 8 / 64 x 4 tiles with ragged tails, the border-only case of images smaller
than one window, the generic kernel (C = 5, R = 9), the wide-channel kernel (C = 31,
R = 2..7, 32 x 4 tiles), and the full 1024 x 1024 x 3, R = 5
launch the benchmark times (checked on sampled pixels and on one full adjoint step).
"""
import numpy as np
import pytest

from gpuutil import (ensure_lib, dev, host, params, f32, zeros_dev, torch,
                     assert_control_derivative)
import oracle
from paper_2510_16154_gb300 import lib
from synth import ImageSpec, make_image

pytestmark = pytest.mark.gpu


def _field(rng, H, W, C):
    # colours close enough that most window pairs interact (|delta| well inside support;
    # narrower for many channels, whose |delta|^2 sums C terms)
    half = 0.15 if C <= 8 else 0.05
    return f32(rng.uniform(0.5 - half, 0.5 + half, size=(H, W, C)))


SHAPES = [(1, 1, 3, 2), (3, 2, 3, 1), (7, 5, 3, 2), (64, 64, 3, 2), (37, 150, 3, 5),
          (100, 150, 1, 3), (9, 130, 3, 8), (33, 70, 5, 2), (20, 30, 3, 9), (150, 200, 3, 7),
          (37, 70, 31, 3), (9, 40, 31, 7), (5, 3, 31, 2), (36, 64, 31, 5)]


@pytest.mark.parametrize("H,W,C,R", SHAPES)
def test_forward_one_step(H, W, C, R):
    ensure_lib()
    rng = np.random.default_rng(H * 1000 + W * 10 + C + R)
    c0 = _field(rng, H, W, C)
    p, op = params(H, W, C, R, 1)
    eps = np.array([[rng.uniform(2, 60), rng.uniform(2, 60)]])
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        out = zeros_dev(H, W, C)
        lib.agents_forward(ctx.handle, eps, out, store=False)
        got = host(out).astype(np.float64)
    want = oracle.forward_final(c0, eps, op)
    assert np.max(np.abs(got - want)) <= 1e-6
    # non-trivial except on images whose only neighbours sit beyond the support (the
    # spatial term alone exceeds 1 on a 3 x 2 grid at these controls)
    assert np.max(np.abs(want - c0)) > 0 or H * W <= 6


@pytest.mark.parametrize("ec", [0.0, 1e-6, 1100.0])
def test_forward_step_colour_weight_extremes(ec):
    # eps_c = 0 (spatial interaction only), a tiny one and the top of E, on the tiled
    # kernels (C = 1, 3) and the wide one (C = 31)
    ensure_lib()
    for H, W, C, R in [(40, 70, 3, 5), (23, 67, 1, 2), (20, 40, 31, 3)]:
        rng = np.random.default_rng(H + W + C)
        c0 = _field(rng, H, W, C)
        p, op = params(H, W, C, R, 1, eps_lo=(0.0, 0.0))
        eps = np.array([[30.0, ec]])
        with lib.Context(p, dev(c0, np.float32)) as ctx:
            out = zeros_dev(H, W, C)
            lib.agents_forward(ctx.handle, eps, out, store=False)
            got = host(out).astype(np.float64)
        want = oracle.forward_final(c0, eps, op)
        assert np.max(np.abs(got - want)) <= 1e-6
        assert np.max(np.abs(want - c0)) > 0 or ec > 100   # large eps_c: colours apart


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_forward_sweep_20_steps(norm_mode):
    ensure_lib()
    c0 = f32(make_image(ImageSpec(64, 64, 3, regions=4, sigma=0.05), 11))
    T = 20
    p, op = params(64, 64, 3, 2, T, norm_mode=norm_mode)
    rng = np.random.default_rng(5)
    eps = np.column_stack([rng.uniform(2, 200, T), rng.uniform(2, 200, T)])
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        out = zeros_dev(64, 64, 3)
        lib.agents_forward(ctx.handle, eps, out, store=True)
        got = host(out).astype(np.float64)
    want = oracle.forward_final(c0, eps, op)
    assert np.max(np.abs(got - want)) <= 1e-5
    assert np.max(np.abs(want - c0)) > (1e-3 if norm_mode == 0 else 1e-4)   # 1/N: slow


def test_all_pairs_window_is_paper_system():
    # R >= max(H, W) and weight 1/N: Eq. MAsystem verbatim (grey-scale), tiled kernel R=8
    ensure_lib()
    rng = np.random.default_rng(3)
    c0 = f32(rng.uniform(0.3, 0.6, size=(6, 8, 1)))
    p, op = params(6, 8, 1, 8, 3, norm_mode=1)
    eps = np.full((3, 2), 4.0)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        out = zeros_dev(6, 8, 1)
        lib.agents_forward(ctx.handle, eps, out, store=False)
        got = host(out).astype(np.float64)
    assert np.max(np.abs(got - oracle.forward_final(c0, eps, op))) <= 1e-6


def test_constant_image_is_bitwise_fixed_point():
    ensure_lib()
    c0 = np.full((70, 90, 3), 0.3711, dtype=np.float32)
    p, _ = params(70, 90, 3, 5, 6)
    with lib.Context(p, dev(c0)) as ctx:
        out = zeros_dev(70, 90, 3)
        lib.agents_forward(ctx.handle, np.full((6, 2), 9.0), out, store=False)
        assert np.array_equal(host(out), c0)


def test_forward_convex_hull_at_full_size():
    # any size: each step is a convex combination of the window (weights >= 0, dt <= 1)
    ensure_lib()
    c0 = make_image(ImageSpec(1024, 1024, 3, regions=12, ramp=0.1, sigma=0.08), 0).astype(np.float32)
    p, _ = params(1024, 1024, 3, 5, 1)
    x = dev(c0)
    with lib.Context(p, x) as ctx:
        out = zeros_dev(1024, 1024, 3)
        lib.agents_forward(ctx.handle, np.array([[57.0, 57.0]]), out, store=False)
        pool = torch.nn.functional.max_pool2d
        xm = x.permute(2, 0, 1)[None]
        hi = pool(xm, 11, stride=1, padding=5)[0].permute(1, 2, 0)
        lo = -pool(-xm, 11, stride=1, padding=5)[0].permute(1, 2, 0)
        assert bool(((out <= hi + 1e-6) & (out >= lo - 1e-6)).all())


def _adjoint_inputs(rng, H, W, C, T):
    c0 = _field(rng, H, W, C)
    v = f32(rng.normal(scale=3.0, size=(H, W, 2, C)))
    mu = f32(rng.normal(scale=0.05, size=(H, W, 2, C)))
    eps = np.column_stack([rng.uniform(2, 80, T), rng.uniform(2, 80, T)])
    return c0, v, mu, eps


def _run_adjoint(p, c0, v, mu, eps):
    H, W, C = c0.shape
    T = eps.shape[0]
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        lib.agents_forward(ctx.handle, eps, None, store=True)
        D = np.zeros((T, 2))
        obj = np.zeros(1)
        lam0 = zeros_dev(H, W, C)
        lib.agents_adjoint(ctx.handle, eps, dev(v, np.float32), dev(mu, np.float32), D, obj, lam0)
        return D, obj[0], host(lam0).astype(np.float64)


def _oracle_adjoint(op, c0, v, mu, eps):
    traj = oracle.forward(c0, eps, op)
    lamT = oracle.terminal_adjoint(traj[-1], v, mu, c0, op)
    lam0, D = oracle.adjoint(traj, eps, lamT, op)
    return D, oracle.cost_Ltilde(traj[-1], v, mu, c0, op), lam0


@pytest.mark.parametrize("H,W,C,R,T", [(24, 70, 3, 2, 5), (9, 130, 1, 3, 4), (40, 66, 3, 5, 3),
                                       (13, 11, 5, 2, 3), (6, 5, 3, 9, 2), (20, 45, 31, 3, 3),
                                       (7, 9, 31, 7, 2)])
def test_adjoint_sweep(H, W, C, R, T):
    ensure_lib()
    rng = np.random.default_rng(H + W + C + R + T)
    c0, v, mu, eps = _adjoint_inputs(rng, H, W, C, T)
    p, op = params(H, W, C, R, T, alpha=40.0, rho=0.5, gamma=0.5)
    D, obj, lam0 = _run_adjoint(p, c0, v, mu, eps)
    Dw, objw, lamw = _oracle_adjoint(op, c0, v, mu, eps)
    print(f"max|D_x| {np.max(np.abs(Dw[:, 0])):.3e} max|D_c| {np.max(np.abs(Dw[:, 1])):.3e} "
          f"rel err D_x {np.max(np.abs(D[:, 0] - Dw[:, 0])) / np.max(np.abs(Dw[:, 0])):.2e} "
          f"D_c {np.max(np.abs(D[:, 1] - Dw[:, 1])) / np.max(np.abs(Dw[:, 1])):.2e}")
    assert_control_derivative(D, Dw)
    assert obj == pytest.approx(objw, rel=1e-6)
    assert np.max(np.abs(lam0 - lamw)) <= 1e-5 * np.max(np.abs(lamw))
    assert np.max(np.abs(Dw)) > 0


def test_checkpointed_adjoint_is_bitwise_equal():
    ensure_lib()
    rng = np.random.default_rng(77)
    H, W, C, R, T = 30, 80, 3, 3, 9
    c0, v, mu, eps = _adjoint_inputs(rng, H, W, C, T)
    outs = []
    for mode in (0, 1, 2, 4, 8, 9):
        p, _ = params(H, W, C, R, T, alpha=40.0, rho=0.5, traj_mode=mode)
        outs.append(_run_adjoint(p, c0, v, mu, eps))
    for D, obj, lam in outs[1:]:
        assert np.array_equal(D, outs[0][0]) and obj == outs[0][1]
        assert np.array_equal(lam, outs[0][2])


def test_full_size_forward_step_sampled():
    # the 1024 x 1024 x 3, R = 5 launch of the throughput benchmark, sampled pixels
    ensure_lib()
    img = make_image(ImageSpec(1024, 1024, 3, regions=12, ramp=0.1, sigma=0.08), 0)
    c0 = f32(img)
    p, op = params(1024, 1024, 3, 5, 1)
    eps = np.array([[57.0, 57.0]])
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        out = zeros_dev(1024, 1024, 3)
        lib.agents_forward(ctx.handle, eps, out, store=False)
        got = host(out).astype(np.float64)
    rng = np.random.default_rng(0)
    rows = list(rng.integers(0, 1024, 300)) + [0, 0, 1023, 1023, 511, 4, 1019]
    cols = list(rng.integers(0, 1024, 300)) + [0, 1023, 0, 1023, 3, 1020, 512]
    F = oracle.velocity_at(c0, rows, cols, 57.0, 57.0, op)
    want = c0[rows, cols] + op.dt * F
    assert np.max(np.abs(got[rows, cols] - want)) <= 1e-6
    assert np.max(np.abs(F)) > 1e-4


def test_full_size_adjoint_step():
    # one adjoint step at 1024 x 1024 x 3, R = 5: lambda^0 sampled, D^0 exact
    ensure_lib()
    img = make_image(ImageSpec(1024, 1024, 3, regions=12, ramp=0.1, sigma=0.08), 1)
    c0 = f32(img)
    rng = np.random.default_rng(1)
    v = f32(rng.normal(scale=50.0, size=(1024, 1024, 2, 3)))
    mu = f32(rng.normal(scale=0.1, size=(1024, 1024, 2, 3)))
    eps = np.array([[57.0, 57.0]])
    p, op = params(1024, 1024, 3, 5, 1)
    D, obj, lam0 = _run_adjoint(p, c0, v, mu, eps)
    c1 = oracle.forward_final(c0, eps, op)
    lamT = oracle.terminal_adjoint(c1, v, mu, c0, op)
    Dw = oracle.control_derivative(c0, lamT, 57.0, 57.0, op)
    print(f"D {D[0]} oracle {Dw}")
    assert_control_derivative(D[0], Dw)
    rows = list(rng.integers(0, 1024, 200)) + [0, 1023, 0, 1023]
    cols = list(rng.integers(0, 1024, 200)) + [0, 1023, 1023, 0]
    want = lamT[rows, cols] + op.dt * oracle.jacobian_transpose_apply_at(c0, lamT, rows, cols,
                                                                          57.0, 57.0, op)
    assert np.max(np.abs(lam0[rows, cols] - want)) <= 1e-5 * np.max(np.abs(lamT))
    assert obj == pytest.approx(oracle.cost_Ltilde(c1, v, mu, c0, op), rel=1e-6)


@pytest.mark.parametrize("ec", [0.0, 1e-6, 1100.0])
def test_adjoint_step_colour_weight_extremes(ec):
    # the adjoint tile stages colours scaled by sqrt(eps_c / 2) (floored at 1e-8): eps_c = 0,
    # a tiny one and the top of E, on the tiled kernels (C = 1, 3) and the wide one (C = 31)
    ensure_lib()
    for H, W, C, R in [(40, 70, 3, 5), (23, 67, 1, 2), (20, 40, 31, 3)]:
        rng = np.random.default_rng(H + W + C + 1)
        c0, v, mu, _ = _adjoint_inputs(rng, H, W, C, 2)
        eps = np.array([[30.0, ec], [20.0, ec]])
        p, op = params(H, W, C, R, 2, alpha=40.0, rho=0.5, gamma=0.5, eps_lo=(0.0, 0.0))
        D, obj, lam0 = _run_adjoint(p, c0, v, mu, eps)
        Dw, objw, lamw = _oracle_adjoint(op, c0, v, mu, eps)
        assert np.max(np.abs(lam0 - lamw)) <= 1e-5 * np.max(np.abs(lamw))
        assert obj == pytest.approx(objw, rel=1e-6)
        if np.max(np.abs(Dw)) == 0.0:
            # eps_c = 1100: every colour pair lies outside the support, nothing interacts
            assert np.max(np.abs(D)) == 0.0 and ec > 100
        else:
            assert_control_derivative(D, Dw)
