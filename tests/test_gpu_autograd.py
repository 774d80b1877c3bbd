"""GPU checks of the differentiable forward sweep (torch.autograd.Function over the C ABI).

* Gradients of L = sum(w * c(T)) with respect to the control and to the input image
  against the FP64 oracle's discrete adjoint (checkpointed context, 1e-5 of the largest
  entry, as for the adjoint sweep tests).
* For the method's own terminal cost L~, the autograd gradient equals agents_adjoint's
  control derivative bit for bit (same kernels, same lambda(T)).
* Gradient workload: a 16 x 16 crop of the 2048 x 2048 RGB image (24 regions, ramp,
  sigma 0.1), R = 5, T = 200, checkpoints every 14 steps; the float32 gradient against
  the FP64 oracle adjoint and against an FP64 central difference (h = 1e-6) along a
  random direction.  Tolerance 1e-4 relative: 200 float32 Euler and adjoint steps.
* Full 2048 x 2048 x 3, T = 200: checkpointing every 14 steps gives bitwise the same
  gradient as storing the whole trajectory, in under a fifth of the memory.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, f32, torch
import oracle
from oracle.tv import cost_Ltilde, terminal_adjoint
from paper_2510_16154_gb300 import lib
from synth import ImageSpec, make_image, GRADIENT_2048_RGB

pytestmark = pytest.mark.gpu


def _autograd(p, c0, eps, grad_cT_fn):
    from paper_2510_16154_gb300.autograd import FlowContext, flow
    fc = FlowContext(p, dev(c0, np.float32))
    try:
        e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
        x = dev(c0, np.float32).requires_grad_()
        cT = flow(fc, e, x)
        cT.backward(gradient=grad_cT_fn(fc, cT.detach()))
        return host(e.grad), host(x.grad).astype(np.float64), host(cT).astype(np.float64)
    finally:
        fc.close()


def test_autograd_matches_oracle_adjoint():
    ensure_lib()
    rng = np.random.default_rng(5)
    H, W, C, R, T = 24, 40, 3, 2, 12
    c0 = f32(make_image(ImageSpec(H, W, C, regions=3, sigma=0.05), 4))
    w = f32(rng.normal(size=(H, W, C)))
    eps = np.column_stack([rng.uniform(2, 80, T), rng.uniform(2, 80, T)])
    p, op = params(H, W, C, R, T, traj_mode=4)
    g_eps, g_c0, cT = _autograd(p, c0, eps, lambda fc, cT: dev(w, np.float32))
    traj = oracle.forward(c0, eps, op)
    lam0, D = oracle.adjoint(traj, eps, -w, op)
    want_eps, want_c0 = -op.dt * D, -lam0
    assert np.max(np.abs(cT - traj[-1])) <= 1e-5
    assert np.max(np.abs(g_eps - want_eps)) <= 1e-5 * np.max(np.abs(want_eps))
    assert np.max(np.abs(g_c0 - want_c0)) <= 1e-5 * np.max(np.abs(want_c0))


def test_autograd_equals_library_adjoint_for_Ltilde():
    ensure_lib()
    rng = np.random.default_rng(6)
    H, W, C, R, T = 30, 70, 3, 3, 9
    c0 = f32(make_image(ImageSpec(H, W, C, regions=4, sigma=0.05), 2))
    v = dev(rng.normal(scale=3.0, size=(H, W, 2, C)), np.float32)
    mu = dev(rng.normal(scale=0.05, size=(H, W, 2, C)), np.float32)
    eps = np.column_stack([rng.uniform(2, 80, T), rng.uniform(2, 80, T)])
    p, _ = params(H, W, C, R, T, alpha=40.0, rho=0.5)

    def grad_Ltilde(fc, cT):
        lam = torch.empty_like(cT)
        lib.agents_objective(fc.handle, cT, v, mu, None, lam)     # lam = -dL~/dc
        return -lam

    g_eps, _, _ = _autograd(p, c0, eps, grad_Ltilde)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        lib.agents_forward(ctx.handle, eps, None, store=True)
        D = np.zeros((T, 2))
        lib.agents_adjoint(ctx.handle, eps, v, mu, D)
    assert np.array_equal(g_eps, -p.dt * D)


def _crop_case():
    img = make_image(GRADIENT_2048_RGB, 0)
    c0 = f32(img[1000:1016, 1000:1016])
    rng = np.random.default_rng(8)
    T = 200
    v = f32(rng.normal(scale=2.0, size=(16, 16, 2, 3)))
    mu = f32(rng.normal(scale=0.05, size=(16, 16, 2, 3)))
    eps = np.column_stack([rng.uniform(2, 60, T), rng.uniform(2, 60, T)])
    return c0, v, mu, eps


def test_gradient_workload_crop_against_fp64_oracle_and_fd():
    ensure_lib()
    c0, v, mu, eps = _crop_case()
    T = eps.shape[0]
    p, op = params(16, 16, 3, 5, T, alpha=40.0, rho=0.5, traj_mode=14)
    vd, mud = dev(v, np.float32), dev(mu, np.float32)

    def grad_Ltilde(fc, cT):
        lam = torch.empty_like(cT)
        lib.agents_objective(fc.handle, cT, vd, mud, None, lam)
        return -lam

    g_eps, _, _ = _autograd(p, c0, eps, grad_Ltilde)
    traj = oracle.forward(c0, eps, op)
    _, D = oracle.adjoint(traj, eps, terminal_adjoint(traj[-1], v, mu, c0, op), op)
    want = -op.dt * D
    rel = np.max(np.abs(g_eps - want)) / np.max(np.abs(want))
    print(f"crop T=200: max rel err vs FP64 adjoint {rel:.2e}")
    assert rel <= 1e-4

    def cost(e):
        return cost_Ltilde(oracle.forward_final(c0, e, op), v, mu, c0, op)

    u = np.random.default_rng(9).normal(size=eps.shape)
    h = 1e-6
    fd = (cost(eps + h * u) - cost(eps - h * u)) / (2 * h)
    assert np.sum(want * u) == pytest.approx(fd, rel=1e-5)          # oracle vs FD (FP64)
    assert np.sum(g_eps * u) == pytest.approx(fd, rel=1e-4)         # GPU vs FD


def test_full_size_checkpointing_bitwise_and_memory():
    ensure_lib()
    img = f32(make_image(GRADIENT_2048_RGB, 0))
    H, W, C, R, T = 2048, 2048, 3, 5, 200
    rng = np.random.default_rng(10)
    eps = np.column_stack([rng.uniform(2, 80, T), rng.uniform(2, 80, T)])
    w = dev(rng.normal(size=(H, W, C)), np.float32)
    grads, footprint = [], []
    for mode in (14, 0):
        p, _ = params(H, W, C, R, T, traj_mode=mode)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        from paper_2510_16154_gb300.autograd import FlowContext, flow
        fc = FlowContext(p, dev(img, np.float32))
        footprint.append(free0 - torch.cuda.mem_get_info()[0])
        e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
        cT = flow(fc, e, dev(img, np.float32))
        cT.backward(gradient=w)
        grads.append(host(e.grad))
        fc.close()
    field = H * W * C * 4
    print(f"context footprint: checkpointed {footprint[0] / 1e9:.2f} GB, "
          f"full store {footprint[1] / 1e9:.2f} GB")
    assert np.array_equal(grads[0], grads[1])
    assert np.all(np.isfinite(grads[0])) and np.max(np.abs(grads[0])) > 0
    assert footprint[0] < 0.2 * footprint[1]
    assert footprint[1] >= (T - 1) * field
