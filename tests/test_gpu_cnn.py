"""GPU checks of the warm-start network's kernels against the FP64 oracle (oracle/cnn.py).

Single convolutions: operands are generated as exact bfloat16 values, so the GPU and the
oracle multiply identical numbers; the only difference is float32 accumulation, bounded
elementwise by K u sum|terms| (K terms, u = 2^-24), with a factor 2 of slack.
Whole network: the loss and its gradient against the oracle with the same bfloat16
rounding points.  A float32 intermediate that lands on the other side of a bfloat16
rounding boundary than its float64 counterpart moves that operand by one bfloat16 ulp
(2^-8 relative), and the move propagates through the later layers.  Injecting
float32-sized relative noise (sqrt(K) 2^-24) before every rounding in the oracle moves mu
by 1.0e-3 (3 levels, base 8) and 2.9e-3 (4 levels, base 16) normwise, the gradient by
3.5e-4 and 5.8e-3 (worst parameter block 1.6e-3 and 1.2e-2), the loss by 2e-6 and
3.3e-4; the tolerances below are about three times those figures.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, torch
from oracle import cnn
from paper_2510_16154_gb300 import lib
from synth import init_net_params

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _bf(rng, *shape, scale=1.0):
    return cnn.bf16_round(rng.normal(scale=scale, size=shape))


def _w16(w):
    Cout, _, _, Cin = w.shape
    wd = dev(w, np.float32)
    w16 = torch.empty(w.size, dtype=torch.int16, device="cuda")
    wt16 = torch.empty(w.size, dtype=torch.int16, device="cuda")
    lib.ws_transpose_weights(wd, w16, wt16, Cin, Cout)
    return w16, wt16


def _bound(ref_abs, K):
    return 2.0 * K * U * ref_abs + 1e-30


CONV_CASES = [  # N, H, W, Cin, Cout, up
    (2, 13, 11, 3, 6, 0), (2, 9, 20, 16, 40, 0), (1, 16, 12, 24, 32, 1), (3, 8, 8, 64, 8, 0),
    (1, 6, 34, 8, 72, 1),
    # width >= 128, channel counts multiples of 16: the tcgen05 kernel (ragged last
    # segment, 2x upsampled input, two 128-channel output tiles, 16 K groups, N = 16)
    (1, 3, 200, 16, 32, 0), (2, 4, 128, 32, 64, 1), (1, 2, 300, 48, 256, 0),
    (1, 3, 130, 128, 16, 0),
    # enough CTAs for four output rows per CTA (the last row block holds two)
    (1, 610, 256, 16, 32, 0),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_forward(case):
    ensure_lib()
    N, H, W, Cin, Cout, up = case
    rng = np.random.default_rng(sum(case))
    xs = (N, H // 2, W // 2, Cin) if up else (N, H, W, Cin)
    x = _bf(rng, *xs)
    w = _bf(rng, Cout, 3, 3, Cin, scale=0.3)
    b = rng.normal(size=Cout).astype(np.float32).astype(np.float64)
    add = rng.normal(size=(N, H, W, Cout)).astype(np.float32).astype(np.float64)
    w16, _ = _w16(w)
    y = torch.empty(N, H, W, Cout, device="cuda")
    y2 = torch.empty_like(y)
    lib.ws_conv3x3_forward(dev(x, np.float32), w16, dev(b, np.float32), y, N, H, W, Cin, Cout,
                           relu=True, up=bool(up), add=dev(add, np.float32), y2=y2)
    xf = cnn.upsample2(x) if up else x
    ref = cnn.conv3x3(xf, w, b, relu=True)
    ref_abs = cnn.conv3x3(np.abs(xf), np.abs(w), np.abs(b), bf16=False)
    got = host(y).astype(np.float64)
    assert np.all(np.abs(got - ref) <= _bound(ref_abs, 9 * Cin + 1))
    assert np.all(np.abs(host(y2) - (got + add)) <= 1e-6 * (np.abs(got) + np.abs(add)))
    assert not lib.ws_tensor_core_fault_take()


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_backward_data_and_weight(case):
    ensure_lib()
    N, H, W, Cin, Cout, up = case
    rng = np.random.default_rng(100 + sum(case))
    xs = (N, H // 2, W // 2, Cin) if up else (N, H, W, Cin)
    x = _bf(rng, *xs)
    w = _bf(rng, Cout, 3, 3, Cin, scale=0.3)
    dy = _bf(rng, N, H, W, Cout)
    _, wt16 = _w16(w)
    xf = cnn.upsample2(x) if up else x
    dx_ref, dw_ref, db_ref = cnn.conv3x3_backward(xf, w, dy)
    dxa, dwa, _ = cnn.conv3x3_backward(np.abs(xf), np.abs(w), np.abs(dy), bf16=False)

    dx = torch.empty(N, H, W, Cin, device="cuda")
    lib.ws_conv3x3_backward_data(dev(dy, np.float32), wt16, dx, N, H, W, Cin, Cout)
    assert np.all(np.abs(host(dx) - dx_ref) <= _bound(dxa, 9 * Cout))
    assert not lib.ws_tensor_core_fault_take()

    ws = torch.empty(lib.ws_conv3x3_backward_weight_workspace(N, H, W, Cin, Cout) // 4 + 1,
                     device="cuda")
    dw = torch.empty(Cout, 3, 3, Cin, device="cuda")
    db = torch.empty(Cout, device="cuda")
    lib.ws_conv3x3_backward_weight(dev(x, np.float32), dev(dy, np.float32), dw, db, N, H, W,
                                   Cin, Cout, ws, up=bool(up))
    assert np.all(np.abs(host(dw) - dw_ref) <= _bound(dwa, N * H * W))
    assert np.all(np.abs(host(db) - db_ref) <= _bound(np.abs(dy).sum(axis=(0, 1, 2)), N * H * W))
    # bitwise reproducible (fixed-order split-K)
    dw2 = torch.empty_like(dw)
    lib.ws_conv3x3_backward_weight(dev(x, np.float32), dev(dy, np.float32), dw2, None, N, H, W,
                                   Cin, Cout, ws, up=bool(up))
    assert torch.equal(dw, dw2)


def _net_case(levels=3, base=8, T=4, N=2, H=16, W=24, seed=0):
    from paper_2510_16154_gb300.warmstart import NetSpec, WarmStartNet
    cfg = cnn.NetConfig(in_ch=3, out_ch=6, base=base, levels=levels, nsteps=T)
    spec = NetSpec(in_ch=3, out_ch=6, base=base, levels=levels, nsteps=T)
    theta = init_net_params(cnn.param_shapes(cfg), seed)
    rng = np.random.default_rng(seed + 1)
    x = rng.uniform(size=(N, H, W, 3)).astype(np.float32)
    mu_t = rng.normal(scale=0.4, size=(N, H, W, 6)).astype(np.float32)
    le_t = np.log(rng.uniform(2, 1100, size=(N, 2 * T))).astype(np.float32)
    net = WarmStartNet(spec)
    net.set_params(theta)
    return cfg, net, theta.astype(np.float64), x, mu_t, le_t


def test_network_layout_matches_oracle():
    ensure_lib()
    cfg, net, theta, *_ = _net_case()
    assert net.num_params == cnn.num_params(cfg)
    assert [s for _, s in net.spec.param_shapes()] == [s for _, s in cnn.param_shapes(cfg)]
    assert np.array_equal(net.get_params(), theta.astype(np.float32))
    net.close()


# (levels, base, N, H, W) and the (mu, z, loss, gradient, worst block) tolerances.  The
# third case is 128 pixels wide, so its level-1 convolutions other than the first and the
# head run on the tcgen05 kernel (forward and backward-data); the same noise injection
# gives 2.7e-3 (mu), 6e-7 (z), 3.2e-5 (loss), 7.8e-4 (gradient), 1.7e-3 (worst block).
NET_TOL = [(3, 8, 2, 16, 24, 3e-3, 1e-4, 1e-4, 2e-3, 1e-2),
           (4, 16, 2, 16, 24, 1e-2, 1e-3, 2e-3, 2e-2, 5e-2),
           (2, 16, 1, 8, 128, 1e-2, 1e-4, 1e-4, 3e-3, 6e-3)]


@pytest.mark.parametrize("levels,base,N,H,W,t_mu,t_z,t_loss,t_g,t_block", NET_TOL)
def test_network_forward_and_gradient_against_oracle(levels, base, N, H, W, t_mu, t_z, t_loss,
                                                     t_g, t_block):
    ensure_lib()
    cfg, net, theta, x, mu_t, le_t = _net_case(levels=levels, base=base, N=N, H=H, W=W)
    mu, z = net.raw(dev(x, np.float32))
    mu_ref, z_ref, _ = cnn.net_forward(cfg, theta, x)
    err_mu = np.linalg.norm(host(mu) - mu_ref) / np.linalg.norm(mu_ref)
    print(f"levels={levels} base={base}: mu normwise rel error {err_mu:.2e}")
    assert err_mu <= t_mu
    assert np.max(np.abs(host(z) - z_ref)) <= t_z * np.max(np.abs(z_ref))
    g = torch.empty(net.num_params, device="cuda")
    loss = net.loss_grad(dev(x, np.float32), dev(mu_t, np.float32), dev(le_t, np.float32),
                         0.3, grad_out=g)
    loss_ref, g_ref = cnn.net_loss_backward(cfg, theta, x, mu_t, le_t, 0.3)
    assert loss == pytest.approx(loss_ref, rel=t_loss)
    gg = host(g).astype(np.float64)
    rel = np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref)
    print(f"levels={levels} base={base}: gradient normwise rel error {rel:.2e}")
    assert rel <= t_g
    # every parameter block, normwise
    off = 0
    for name, shape in cnn.param_shapes(cfg):
        n = int(np.prod(shape))
        a, b = gg[off:off + n], g_ref[off:off + n]
        assert np.linalg.norm(a - b) <= t_block * np.linalg.norm(b) + 1e-9, name
        off += n
    assert not lib.ws_tensor_core_fault_take()
    net.close()


def test_forward_pads_crops_and_projects():
    ensure_lib()
    cfg, net, theta, _, _, _ = _net_case(levels=3, base=8, T=4)
    rng = np.random.default_rng(9)
    x = rng.uniform(size=(1, 13, 19, 3)).astype(np.float32)
    mu, eps = net.predict(dev(x, np.float32), project=1)
    xp = np.pad(x, ((0, 0), (0, 3), (0, 1), (0, 0)), mode="edge")
    mu_ref, z_ref, _ = cnn.net_forward(cfg, theta, xp)
    mu_ref = mu_ref[:, :13, :19]
    nrm = np.linalg.norm(mu_ref, axis=-1, keepdims=True)
    mu_ref = mu_ref / np.maximum(nrm, 1.0)
    got = host(mu)
    assert np.all(np.linalg.norm(got, axis=-1) <= 1.0 + 1e-6)
    assert np.linalg.norm(got - mu_ref) <= 3e-3 * np.linalg.norm(mu_ref)
    eps_ref = np.clip(np.exp(z_ref), 2.0, 1100.0).reshape(1, 4, 2)
    assert np.allclose(host(eps), eps_ref, rtol=1e-4)
    net.close()


def test_training_reduces_the_loss():
    ensure_lib()
    cfg, net, theta, x, mu_t, le_t = _net_case(levels=3, base=8, T=4, N=4, H=16, W=16)
    xd, md, ld = dev(x, np.float32), dev(mu_t, np.float32), dev(le_t, np.float32)
    hist = net.fit(xd, md, ld, epochs=60, batch=4, lr=3e-3)
    print(f"training loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    assert hist[-1] < 0.5 * hist[0]
    net.close()
