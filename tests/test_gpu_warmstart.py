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

    def predict(self, img):
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
