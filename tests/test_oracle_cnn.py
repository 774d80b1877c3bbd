"""Pins of the warm-start network oracle (oracle/cnn.py) against independent facts:
torch's bfloat16 conversion and hand-worked ties, SciPy's 2-D correlation, finite
differences, adjointness of pooling and upsampling, and a planted mistake."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn
from synth import init_net_params


def test_bf16_round_worked_values():
    one = 1.0
    assert cnn.bf16_round([one + 2.0 ** -8])[0] == 1.0                 # tie -> even (down)
    assert cnn.bf16_round([one + 3 * 2.0 ** -8])[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert cnn.bf16_round([one + 2.0 ** -8 + 2.0 ** -20])[0] == 1.0 + 2.0 ** -7
    assert cnn.bf16_round([-2.5])[0] == -2.5
    assert np.isnan(cnn.bf16_round([np.nan])[0])


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(scale=10.0, size=5000).astype(np.float32),
                        (1.0 + np.arange(256) * 2.0 ** -15).astype(np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16_round(x), want)


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 7, 9, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cnn.conv3x3(x, w, b, bf16=False)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, i], w[o, :, :, i], mode="same",
                                         boundary="fill") for i in range(3))
            assert np.allclose(y[n, :, :, o], ref, rtol=0, atol=1e-12)
    assert np.array_equal(cnn.conv3x3(x, w, b, relu=True, bf16=False), np.maximum(y, 0))


def test_conv3x3_backward_finite_differences_and_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 5, 6, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    dy = rng.normal(size=(1, 5, 6, 2))
    dx, dw, db = cnn.conv3x3_backward(x, w, dy, bf16=False)
    f = lambda xx, ww, bb: float(np.sum(dy * cnn.conv3x3(xx, ww, bb, bf16=False)))
    # linear in each argument: one central difference is exact up to round-off
    u = rng.normal(size=x.shape)
    assert np.sum(dx * u) == pytest.approx((f(x + u, w, b) - f(x - u, w, b)) / 2, rel=1e-12)
    v = rng.normal(size=w.shape)
    assert np.sum(dw * v) == pytest.approx((f(x, w + v, b) - f(x, w - v, b)) / 2, rel=1e-12)
    assert np.allclose(db, dy.sum(axis=(0, 1, 2)))
    # <conv(x), dy> = <x, conv^T(dy)> with b = 0
    assert np.sum(cnn.conv3x3(x, w, 0 * b, bf16=False) * dy) == pytest.approx(np.sum(x * dx),
                                                                              rel=1e-12)


def test_pool_and_upsample_are_adjoint_pairs():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 8, 6, 3))
    y = rng.normal(size=(2, 4, 3, 3))
    assert np.sum(cnn.avgpool2(x) * y) == pytest.approx(np.sum(x * cnn.avgpool2_backward(y)))
    assert np.sum(cnn.upsample2(y) * x) == pytest.approx(np.sum(y * cnn.upsample2_backward(x)))
    assert np.allclose(cnn.avgpool2(np.full((1, 4, 4, 2), 0.3)), 0.3)
    assert np.array_equal(cnn.upsample2(y)[:, ::2, 1::2], y)


def _tiny():
    cfg = cnn.NetConfig(in_ch=3, out_ch=6, base=3, levels=3, nsteps=2)
    theta = init_net_params(cnn.param_shapes(cfg), 7).astype(np.float64)
    rng = np.random.default_rng(4)
    x = rng.uniform(size=(2, 8, 8, 3))
    mu_t = rng.normal(scale=0.5, size=(2, 8, 8, 6))
    le_t = np.log(rng.uniform(2, 1100, size=(2, 4)))
    return cfg, theta, x, mu_t, le_t


def test_param_layout_counts():
    cfg = cnn.NetConfig()
    names = [n for n, _, _ in cnn.conv_list(cfg)]
    assert len(names) == 15 and names[0] == "enc1a" and names[-1] == "head"
    assert cnn.num_params(cfg) == sum(9 * i * o + o for _, i, o in cnn.conv_list(cfg)) + 40 * 256 + 40


def test_network_gradient_finite_differences():
    cfg, theta, x, mu_t, le_t = _tiny()
    loss, g = cnn.net_loss_backward(cfg, theta, x, mu_t, le_t, 0.3, bf16=False)
    rng = np.random.default_rng(5)
    for _ in range(3):
        u = rng.normal(size=theta.shape)
        h = 1e-6
        lp = cnn.loss_value(*cnn.net_forward(cfg, theta + h * u, x, bf16=False)[:2], mu_t, le_t, 0.3)
        lm = cnn.loss_value(*cnn.net_forward(cfg, theta - h * u, x, bf16=False)[:2], mu_t, le_t, 0.3)
        assert np.sum(g * u) == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
    # per-block checks: every parameter group receives a non-zero gradient
    parts = cnn.unflatten(cfg, g)
    assert all(np.any(v != 0) for v in parts.values())


def test_network_gradient_catches_a_dropped_skip():
    """A planted mistake: losing the skip-connection gradient must fail the FD check."""
    cfg, theta, x, mu_t, le_t = _tiny()
    orig = cnn.avgpool2_backward
    try:
        cnn.avgpool2_backward = lambda dy: 0.0 * orig(dy)       # drop the pooled path
        _, g_bad = cnn.net_loss_backward(cfg, theta, x, mu_t, le_t, 0.3, bf16=False)
    finally:
        cnn.avgpool2_backward = orig
    _, g = cnn.net_loss_backward(cfg, theta, x, mu_t, le_t, 0.3, bf16=False)
    assert np.linalg.norm(g_bad - g) > 1e-3 * np.linalg.norm(g)


def test_bf16_network_close_to_exact():
    cfg, theta, x, mu_t, le_t = _tiny()
    l1, g1 = cnn.net_loss_backward(cfg, theta, x, mu_t, le_t, 0.3, bf16=True)
    l0, g0 = cnn.net_loss_backward(cfg, theta, x, mu_t, le_t, 0.3, bf16=False)
    assert l1 == pytest.approx(l0, rel=2e-2)
    assert np.linalg.norm(g1 - g0) <= 3e-2 * np.linalg.norm(g0)
