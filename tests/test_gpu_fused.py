"""Whole-sweep launches against one launch per step.

For the tiled (R, C) a sweep can run all its Euler (or adjoint) steps in one persistent
launch whose blocks take (step, tile) jobs in order and wait for the 3 x 3 neighbouring
tiles of the previous step (mode 2 of the test hook forces it for every sweep; the default
uses it only where it measured faster).  A tile's arithmetic is the one-step kernels' own, so every
result must be BITWISE equal to the one-launch-per-step path: forward sweeps with and
without storage, sweeps longer than one launch's step table, the adjoint (lambda^0, D,
L~), the checkpointed adjoint (whose segment recomputations are whole-sweep launches),
and a short solve.  Shapes include ragged tiles, one tile, a 1 x 1 image, and R = 8 (the
largest halo, equal to the tile height).  The time limit of the waits is exercised by a
test hook that makes one launch wait for flag values no tile writes: the call returns
AGENTS_ETIMEOUT without a fault or a hang, and the context then works as before.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, zeros_dev, torch
from paper_2510_16154_gb300 import lib
from synth import ImageSpec, make_image

pytestmark = pytest.mark.gpu

# (H, W, C, R, T)
SHAPES = [
    (37, 150, 3, 5, 6),    # ragged in both directions, 3 x 5 tiles
    (64, 64, 3, 5, 4),     # whole tiles
    (9, 130, 1, 3, 5),     # one tile row plus a ragged one
    (24, 200, 3, 8, 3),    # R = 8: the halo reaches the next tile row exactly
    (1, 1, 3, 1, 3),       # one pixel
    (130, 70, 1, 2, 4),
]


def _case(H, W, C, R, T, seed=0):
    img = make_image(ImageSpec(H, W, C, regions=4, sigma=0.05), seed).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    eps = np.stack([rng.uniform(20.0, 400.0, T), rng.uniform(20.0, 400.0, T)], axis=1)
    return img, eps


def _fused(on: bool):
    lib.agents_debug_set_fused(2 if on else 0, 0, 0)


@pytest.fixture(autouse=True)
def _restore_default():
    ensure_lib()
    yield
    lib.agents_debug_set_fused(1, 0, 0)


def _forward(img, eps, p, store, on):
    _fused(on)
    H, W, C = img.shape
    cT = zeros_dev(H, W, C)
    with lib.Context(p, dev(img)) as ctx:
        lib.agents_forward(ctx.handle, eps, cT, store=store)
    return host(cT)


@pytest.mark.parametrize("H,W,C,R,T", SHAPES)
@pytest.mark.parametrize("store", [True, False])
def test_forward_sweep_bitwise(H, W, C, R, T, store):
    img, eps = _case(H, W, C, R, T)
    p, _ = params(H, W, C, R, T)
    a = _forward(img, eps, p, store, True)
    b = _forward(img, eps, p, store, False)
    assert np.array_equal(a, b)
    if H * W > 1:
        assert not np.array_equal(a, img)     # the flow moved the image


def _adjoint(img, eps, p, on, traj_mode=0):
    H, W, C = img.shape
    T = eps.shape[0]
    p.traj_mode = traj_mode
    rng = np.random.default_rng(5)
    mu = dev(rng.normal(0.0, 0.5, (H, W, 2, C)).astype(np.float32))
    v = dev(rng.normal(0.0, 0.2, (H, W, 2, C)).astype(np.float32))
    D = np.zeros((T, 2))
    obj = np.zeros(1)
    lam0 = zeros_dev(H, W, C)
    _fused(on)
    with lib.Context(p, dev(img)) as ctx:
        lib.agents_forward(ctx.handle, eps, None, store=True)
        lib.agents_adjoint(ctx.handle, eps, v, mu, D, obj, lam0)
    return D, obj, host(lam0)


@pytest.mark.parametrize("H,W,C,R,T", SHAPES)
def test_adjoint_sweep_bitwise(H, W, C, R, T):
    img, eps = _case(H, W, C, R, T, seed=3)
    p, _ = params(H, W, C, R, T)
    Da, oa, la = _adjoint(img, eps, p, True)
    Db, ob, lb = _adjoint(img, eps, p, False)
    assert np.array_equal(Da, Db) and np.array_equal(oa, ob) and np.array_equal(la, lb)
    if H * W > 1:
        assert np.any(Da != 0.0)


def test_checkpointed_adjoint_bitwise():
    # checkpoint every 4 states: each segment's recomputation is a whole-sweep launch
    H, W, C, R, T = 45, 140, 3, 4, 11
    img, eps = _case(H, W, C, R, T, seed=7)
    p, _ = params(H, W, C, R, T)
    Da, oa, la = _adjoint(img, eps, p, True, traj_mode=4)
    Db, ob, lb = _adjoint(img, eps, p, False, traj_mode=4)
    assert np.array_equal(Da, Db) and np.array_equal(oa, ob) and np.array_equal(la, lb)
    # and equal to the full store
    p2, _ = params(H, W, C, R, T)
    Dc, oc, lc = _adjoint(img, eps, p2, True, traj_mode=0)
    assert np.array_equal(Da, Dc) and np.array_equal(la, lc)


def test_sweeps_longer_than_one_launch():
    # 300 Euler steps: three forward launches of at most 128 steps; one adjoint launch
    H, W, C, R, T = 40, 70, 3, 3, 300
    img, eps = _case(H, W, C, R, T, seed=11)
    eps *= 0.1
    p, _ = params(H, W, C, R, T)
    for store in (True, False):
        a = _forward(img, eps, p, store, True)
        b = _forward(img, eps, p, store, False)
        assert np.array_equal(a, b)
    Da, oa, la = _adjoint(img, eps, p, True)
    Db, ob, lb = _adjoint(img, eps, p, False)
    assert np.array_equal(Da, Db) and np.array_equal(la, lb)


def test_solve_bitwise():
    H, W, C, R, T = 48, 80, 3, 5, 5
    img = make_image(ImageSpec(H, W, C, regions=4, sigma=0.05), 21).astype(np.float32)
    p, _ = params(H, W, C, R, T)
    out = []
    for on in (True, False):
        _fused(on)
        o = lib.agents_default_solve_opts()
        o.k_out, o.k_in = 2, 3
        eps = np.full((T, 2), 57.0)
        mu = np.zeros((H, W, 2, C), dtype=np.float32)
        c = np.zeros((H, W, C), dtype=np.float32)
        with lib.Context(p, dev(img)) as ctx:
            info = lib.solve(ctx.handle, o, eps, mu, None, c, None)
        out.append((eps, mu, c, info.forward_steps, info.adjoint_steps))
    a, b = out
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert a[3:] == b[3:]


def test_wait_time_limit_reports_etimeout_and_recovers():
    H, W, C, R, T = 40, 150, 3, 5, 6
    img, eps = _case(H, W, C, R, T, seed=13)
    p, _ = params(H, W, C, R, T)
    want = _forward(img, eps, p, True, False)
    Dw, ow, lw = _adjoint(img, eps, p, False)
    rng = np.random.default_rng(5)
    mu = dev(rng.normal(0.0, 0.5, (H, W, 2, C)).astype(np.float32))
    v = dev(rng.normal(0.0, 0.2, (H, W, 2, C)).astype(np.float32))
    cT = zeros_dev(H, W, C)
    with lib.Context(p, dev(img)) as ctx:
        # forward: the launch waits 1 ms for flags no tile writes, then winds down
        lib.agents_debug_set_fused(2, 1_000_000, 1 << 20)
        with pytest.raises(lib.AgentsError) as e:
            lib.agents_forward(ctx.handle, eps, cT, store=True)
        assert e.value.code == lib.AGENTS_ETIMEOUT and "time limit" in str(e.value)
        lib.agents_debug_set_fused(1, 0, 0)
        lib.agents_forward(ctx.handle, eps, cT, store=True)
        assert np.array_equal(host(cT), want)
        # adjoint: the same on the reverse sweep
        D = np.zeros((T, 2))
        obj = np.zeros(1)
        lam0 = zeros_dev(H, W, C)
        lib.agents_debug_set_fused(2, 1_000_000, 1 << 20)
        with pytest.raises(lib.AgentsError) as e:
            lib.agents_adjoint(ctx.handle, eps, v, mu, D, obj, lam0)
        assert e.value.code == lib.AGENTS_ETIMEOUT
        lib.agents_debug_set_fused(1, 0, 0)
        lib.agents_adjoint(ctx.handle, eps, v, mu, D, obj, lam0)
        assert np.array_equal(D, Dw) and np.array_equal(obj, ow)
        assert np.array_equal(host(lam0), lw)
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_debug_set_fused(2, -1, 0)
    assert e.value.code == lib.AGENTS_EINVAL
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_debug_set_fused(3, 0, 0)
    assert e.value.code == lib.AGENTS_EINVAL


def test_repeated_runs_are_bitwise_stable():
    # a race between jobs (a tile staged before its neighbours' stores are visible) would
    # show up as run-to-run differences
    H, W, C, R, T = 256, 640, 3, 5, 8
    img, eps = _case(H, W, C, R, T, seed=17)
    p, _ = params(H, W, C, R, T)
    want = _adjoint(img, eps, p, False)
    for _ in range(10):
        got = _adjoint(img, eps, p, True)
        for a, b in zip(got, want):
            assert np.array_equal(a, b)


def test_other_stream_occupying_the_gpu():
    # Kernels of another stream hold SMs while a whole-sweep launch runs, so not all of its
    # persistent blocks are resident at once: jobs are still taken in order and every wait
    # ends (a stuck wait would give up after its time limit and fail the call, not hang).
    H, W, C, R, T = 512, 768, 3, 5, 12
    img, eps = _case(H, W, C, R, T, seed=19)
    p, _ = params(H, W, C, R, T)
    want = _forward(img, eps, p, True, False)
    Dw, ow, lw = _adjoint(img, eps, p, False)
    busy = torch.cuda.Stream()
    mine = torch.cuda.Stream()
    a = torch.randn(4096, 4096, device="cuda")
    rng = np.random.default_rng(5)
    mu = dev(rng.normal(0.0, 0.5, (H, W, 2, C)).astype(np.float32))
    v = dev(rng.normal(0.0, 0.2, (H, W, 2, C)).astype(np.float32))
    torch.cuda.synchronize()
    _fused(True)
    cT = zeros_dev(H, W, C)
    lam0 = zeros_dev(H, W, C)
    D = np.zeros((T, 2))
    obj = np.zeros(1)
    with lib.Context(p, dev(img), mine) as ctx:
        torch.cuda.synchronize()
        for _ in range(3):
            with torch.cuda.stream(busy):
                for _ in range(4):
                    a = torch.tanh(a @ a * 1e-4)
            lib.agents_forward(ctx.handle, eps, cT, store=True)
            lib.agents_adjoint(ctx.handle, eps, v, mu, D, obj, lam0)
            torch.cuda.synchronize()
            assert np.array_equal(host(cT), want)
            assert np.array_equal(D, Dw) and np.array_equal(obj, ow)
            assert np.array_equal(host(lam0), lw)


def test_benchmark_size_default_mode_is_bitwise_the_per_step_path():
    # at 1024^2 x 3, R = 5 the default mode runs the adjoint sweep as one launch
    H, W, C, R, T = 1024, 1024, 3, 5, 6
    img, eps = _case(H, W, C, R, T, seed=23)
    p, _ = params(H, W, C, R, T)
    ref = _adjoint(img, eps, p, False)
    lib.agents_debug_set_fused(1, 0, 0)
    rng = np.random.default_rng(5)
    mu = dev(rng.normal(0.0, 0.5, (H, W, 2, C)).astype(np.float32))
    v = dev(rng.normal(0.0, 0.2, (H, W, 2, C)).astype(np.float32))
    D = np.zeros((T, 2))
    obj = np.zeros(1)
    lam0 = zeros_dev(H, W, C)
    with lib.Context(p, dev(img)) as ctx:
        lib.agents_forward(ctx.handle, eps, None, store=True)
        lib.agents_adjoint(ctx.handle, eps, v, mu, D, obj, lam0)
    assert np.array_equal(D, ref[0]) and np.array_equal(obj, ref[1])
    assert np.array_equal(host(lam0), ref[2])
    assert np.array_equal(_forward(img, eps, p, True, True), _forward(img, eps, p, True, False))
