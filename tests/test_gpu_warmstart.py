"""GPU checks of the learned warm start with the committed weights
(paper_2510_16154_gb300/weights/warmstart_rgb_T20_R5.npz, trained by train_warmstart on
4000 method-generated solves of 256 x 256 images).

* On unseen images of the training generator, the batched solve started from the
  network's mu needs fewer multiplier steps to the relative residual 1e-4 than the cold
  start, and ends at an objective no worse than the cold start's (within 1e-3 relative).
* The fallback: a warm start that diverges (here a NaN dual field) is replaced by the
  cold solve, whose result is bitwise the plain solve's.
"""
import os

import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, torch
from paper_2510_16154_gb300 import lib

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2510_16154_gb300", "weights", "warmstart_rgb_T20_R5.npz")
R, T = 5, 20


def _images(n, size, seed):
    from paper_2510_16154_gb300.train_warmstart import make_images
    return make_images(n, size, seed, torch.device("cuda"))


def test_warm_start_cuts_multiplier_steps():
    ensure_lib()
    from paper_2510_16154_gb300.warmstart import WarmStartNet
    net = WarmStartNet.load(WEIGHTS)
    n, S = 12, 256
    imgs = _images(n, S, 4242)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in, o.tol = 40, 10, 1e-4
    ctxs = [lib.Context(lib.agents_default_params(S, S, 3, R, T), imgs[i].contiguous())
            for i in range(n)]
    res = {}
    try:
        for mode in ("cold", "warm"):
            eps = [torch.full((T, 2), 57.0, dtype=torch.float64, device="cuda") for _ in range(n)]
            if mode == "cold":
                mus = [torch.zeros(S, S, 2, 3, device="cuda") for _ in range(n)]
            else:
                mu_p, _ = net.predict(imgs)
                mus = [mu_p[i].reshape(S, S, 2, 3).contiguous() for i in range(n)]
            infos = lib.agents_solve_batch([c.handle for c in ctxs], o, eps, mus, None,
                                           autotune=False, use_graph=True)
            res[mode] = infos
    finally:
        for c in ctxs:
            c.close()
        net.close()
    cold = [i.outer_done for i in res["cold"]]
    warm = [i.outer_done for i in res["warm"]]
    obj_c = np.mean([i.final_obj for i in res["cold"]])
    obj_w = np.mean([i.final_obj for i in res["warm"]])
    print(f"multiplier steps cold {cold} (sum {sum(cold)}) warm {warm} (sum {sum(warm)}); "
          f"mean final L~ cold {obj_c:.4f} warm {obj_w:.4f}")
    assert sum(warm) < sum(cold)
    assert obj_w <= obj_c * (1 + 1e-3)


class _NaNNet:
    """Stands in for a network whose prediction makes the solve diverge."""

    def __init__(self, nsteps):
        from paper_2510_16154_gb300.warmstart import NetSpec
        self.spec = NetSpec(nsteps=nsteps)

    def predict(self, img, lift=1):
        H, W, C = img.shape
        mu = torch.full((H, W, 2 * C), float("nan"), device=img.device)
        return mu, torch.full((self.spec.nsteps, 2), 57.0, dtype=torch.float64, device=img.device)


def test_divergent_warm_start_falls_back_to_the_cold_solve():
    ensure_lib()
    from paper_2510_16154_gb300.warmstart import warm_solve
    img = _images(1, 64, 77)[0].contiguous()
    p = lib.agents_default_params(64, 64, 3, 2, 6)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = 2, 3
    c_warm = torch.empty(64, 64, 3, device="cuda")
    c_cold = torch.empty(64, 64, 3, device="cuda")
    with lib.Context(p, img) as ctx:
        info, eps, mu, fb = warm_solve(ctx.handle, _NaNNet(6), img, o, c_out=c_warm)
        eps0 = torch.full((6, 2), 57.0, dtype=torch.float64, device="cuda")
        mu0 = torch.zeros(64, 64, 2, 3, device="cuda")
        lib.solve(ctx.handle, o, eps0, mu0, None, c_cold)
    assert fb
    assert torch.equal(c_warm, c_cold) and torch.equal(eps, eps0) and torch.equal(mu, mu0)


# ------------------------------------------------------------------ against the oracle

def test_warm_started_solve_matches_oracle_from_the_same_start():
    """The warm start changes only the starting point (eps(0), mu(0)) of Algorithm 2.  From
    the network's prediction for an unseen 48 x 48 image, the GPU solve and the FP64
    oracle's admm_solve take the same steps: colours within 1e-4 max-abs, control within
    1e-3 relative, multiplier within 1e-4 (the plain solve's parity bar).  The oracle's
    own cold-started run of the same image is printed beside it: the two starts can end
    at different stationary points of the non-convex problem."""
    ensure_lib()
    import oracle
    from paper_2510_16154_gb300.warmstart import WarmStartNet
    S, k_out, k_in = 48, 2, 3
    img_t = _images(1, S, 5151)[0].contiguous()
    img = host(img_t).astype(np.float64)
    net = WarmStartNet.load(WEIGHTS)
    try:
        mu_p, eps_p = net.predict(img_t)
    finally:
        net.close()
    mu0 = mu_p.reshape(S, S, 2, 3).contiguous()
    eps0 = eps_p.contiguous()
    mu0_h, eps0_h = host(mu0).astype(np.float64), host(eps0)
    p = lib.agents_default_params(S, S, 3, R, T)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = k_out, k_in
    eps, mu = eps0.clone(), mu0.clone()
    c = torch.empty(S, S, 3, device="cuda")
    with lib.Context(p, img_t) as ctx:
        info = lib.solve(ctx.handle, o, eps, mu, None, c)
    op = oracle.Params(radius=R, nsteps=T)
    ref = oracle.admm_solve(img, op, oracle.SolveOpts(k_out=k_out, k_in=k_in),
                            eps0=eps0_h, mu0=mu0_h)
    err = np.max(np.abs(host(c) - ref["c"]))
    cold = oracle.admm_solve(img, op, oracle.SolveOpts(k_out=k_out, k_in=k_in))
    print(f"warm GPU vs warm oracle: max|dc| {err:.2e}; warm vs cold (oracle): "
          f"max|dc| {np.max(np.abs(ref['c'] - cold['c'])):.2e}, "
          f"L~ {ref['outer'][-1]['Ltilde']:.4f} vs {cold['outer'][-1]['Ltilde']:.4f}")
    assert info.trials == sum(i.trials for i in ref["inner"])
    assert err <= 1e-4
    assert np.max(np.abs(host(eps) - ref["eps"])) <= 1e-3 * np.max(np.abs(ref["eps"]))
    assert np.max(np.abs(host(mu) - ref["mu"])) <= 1e-4 * max(1.0, np.max(np.abs(ref["mu"])))


def test_warm_started_2048_result_on_a_crop_against_oracle():
    """A 2048 x 2048 image (the evaluation size of the warm start): the colours the
    warm-started GPU solve returns are c(T; eps*) for its final control eps*; the FP64
    oracle integrates the same control on a crop whose centre 32 x 32 pixels lie T R = 100
    pixels inside it (the dynamics move information at most R pixels per step, so the
    crop's cut edges cannot reach the centre).  The crop is square and cut from a square
    image, so the spatial spacing of the full image is kept by scaling eps_x by
    (crop side / image side)^2.  Tolerance 1e-4 max-abs (the parity bar)."""
    ensure_lib()
    import oracle
    from paper_2510_16154_gb300.warmstart import WarmStartNet, warm_solve
    N, k_out, k_in = 2048, 2, 3
    img_t = _images(1, N, 6161)[0].contiguous()
    net = WarmStartNet.load(WEIGHTS)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = k_out, k_in
    c = torch.empty(N, N, 3, device="cuda")
    try:
        with lib.Context(lib.agents_default_params(N, N, 3, R, T), img_t) as ctx:
            info, eps, mu, fb = warm_solve(ctx.handle, net, img_t, o, c_out=c)
    finally:
        net.close()
    assert not fb and info.outer_done == k_out
    margin, core = T * R, 32
    side = core + 2 * margin
    r0, q0 = 900, 1300
    crop = host(img_t[r0:r0 + side, q0:q0 + side]).astype(np.float64)
    eps_crop = host(eps).copy()
    eps_crop[:, 0] *= (side / N) ** 2
    op = oracle.Params(radius=R, nsteps=T)
    want = oracle.forward_final(crop, eps_crop, op)[margin:margin + core, margin:margin + core]
    got = host(c[r0 + margin:r0 + margin + core, q0 + margin:q0 + margin + core])
    err = np.max(np.abs(got - want))
    print(f"2048^2 warm result, crop of {core}x{core}: max|c - oracle| {err:.2e}, "
          f"moved {np.max(np.abs(want - crop[margin:margin + core, margin:margin + core])):.2e}")
    assert err <= 1e-4


def test_lifted_prediction_is_the_coarse_prediction_upsampled():
    """ws_net_forward_lifted: the prediction for a 1024 x 1024 image made at 256 x 256 (the
    4 x 4 block means) and upsampled by nearest neighbour is bitwise the prediction for the
    block-mean image itself, repeated 4 x 4 (the block means formed here in the kernel's
    order: float32 sums over the block's rows, then its columns, times 1/16); the control
    is the coarse image's."""
    ensure_lib()
    from paper_2510_16154_gb300.warmstart import WarmStartNet, lift_factor
    net = WarmStartNet.load(WEIGHTS)
    try:
        img = _images(1, 1024, 8181)[0].contiguous()
        assert lift_factor(1024, 1024) == 4 and lift_factor(256, 256) == 1
        mu_l, eps_l = net.predict(img, lift=4)
        blocks = img.reshape(256, 4, 256, 4, 3)
        acc = torch.zeros(256, 256, 3, device="cuda")
        for u in range(4):
            for v in range(4):
                acc = acc + blocks[:, u, :, v]
        small = (acc * (1.0 / 16.0)).contiguous()
        mu_s, eps_s = net.predict(small)
    finally:
        net.close()
    up = mu_s.repeat_interleave(4, dim=0).repeat_interleave(4, dim=1)
    print(f"lifted vs coarse prediction: max |dmu| {(mu_l - up).abs().max().item():.2e}")
    assert torch.equal(mu_l, up)
    assert torch.equal(eps_l, eps_s)
    # exactly piecewise constant on 4 x 4 blocks
    assert torch.equal(mu_l[0::4, 0::4], mu_l[3::4, 3::4])
