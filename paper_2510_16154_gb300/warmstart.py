"""Learned warm start for solve(): a small U-Net that predicts the initial dual field mu(0)
and control eps(0) of Algorithm 2 from the image (include/warmstart.h).

Marshalling only: the network's convolutions, pooling, heads, loss gradient and Adam
updates all run in ``libagents.so`` (BF16 tensor-core convolutions with float32
accumulation).  PyTorch holds the device buffers.

The solve still decides the answer: ``warm_solve`` starts solve() from the
prediction and, if that solve diverges or ends without reaching the tolerance, runs the
plain cold-started solve instead (the fallback).
"""
from __future__ import annotations

import ctypes
import json
import math
import os
from dataclasses import dataclass, asdict

import numpy as np
import torch

from . import _lib as lib

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")


@dataclass(frozen=True)
class NetSpec:
    in_ch: int = 3
    out_ch: int = 6
    base: int = 32
    levels: int = 4
    nsteps: int = 20
    eps_lo: tuple = (2.0, 2.0)
    eps_hi: tuple = (1100.0, 1100.0)

    def width(self, l: int) -> int:
        return self.base * 2 ** (l - 1)

    def param_shapes(self):
        """(name, shape) of the flat parameter vector, in the library's order."""
        convs, cin = [], self.in_ch
        for l in range(1, self.levels + 1):
            convs += [(f"enc{l}a", cin, self.width(l)), (f"enc{l}b", self.width(l), self.width(l))]
            cin = self.width(l)
        for l in range(self.levels - 1, 0, -1):
            convs += [(f"dec{l}a", self.width(l + 1), self.width(l)),
                      (f"dec{l}b", self.width(l), self.width(l))]
        convs.append(("head", self.width(1), self.out_ch))
        shapes = []
        for name, ci, co in convs:
            shapes += [(name + ".W", (co, 3, 3, ci)), (name + ".b", (co,))]
        shapes += [("eps.A", (2 * self.nsteps, self.width(self.levels))),
                   ("eps.c", (2 * self.nsteps,))]
        return shapes


class WarmStartNet:
    """The network on one CUDA device, bound to a torch stream."""

    def __init__(self, spec: NetSpec = NetSpec(), device=None, stream=None):
        self.spec = spec
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        cfg = lib.ws_net_config()
        cfg.in_ch, cfg.out_ch, cfg.base = spec.in_ch, spec.out_ch, spec.base
        cfg.levels, cfg.nsteps = spec.levels, spec.nsteps
        cfg.eps_lo[0], cfg.eps_lo[1] = spec.eps_lo
        cfg.eps_hi[0], cfg.eps_hi[1] = spec.eps_hi
        h = ctypes.c_void_p()
        lib._ws_check(lib.load().ws_net_create(ctypes.byref(cfg), lib._stream(self.stream),
                                               ctypes.byref(h)), "ws_net_create")
        self.handle = h
        self.num_params = int(lib.load().ws_net_num_params(h))

    def close(self):
        if self.handle:
            lib.load().ws_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters
    def init_params(self, seed: int) -> None:
        """He-normal convolution weights, zero biases, control head at log 57 (the seeded
        initial values of ``synth.params.init_net_params``)."""
        from synth.params import init_net_params
        self.set_params(init_net_params(self.spec.param_shapes(), seed))

    def set_params(self, theta) -> None:
        if isinstance(theta, np.ndarray):
            theta = np.ascontiguousarray(theta, dtype=np.float32)
            n = theta.size
        else:
            theta = theta.contiguous()
            n = theta.numel()
        if n != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {n}")
        lib._ws_check(lib.load().ws_net_set_params(self.handle, lib._ptr(theta, "float32")),
                      "ws_net_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        lib._ws_check(lib.load().ws_net_get_params(self.handle, out.ctypes.data),
                      "ws_net_get_params")
        return out

    def save(self, path: str) -> None:
        np.savez_compressed(path, theta=self.get_params(),
                            spec=json.dumps(asdict(self.spec)))

    @classmethod
    def load(cls, path: str, device=None, stream=None) -> "WarmStartNet":
        z = np.load(path)
        d = json.loads(str(z["spec"]))
        d["eps_lo"], d["eps_hi"] = tuple(d["eps_lo"]), tuple(d["eps_hi"])
        net = cls(NetSpec(**d), device, stream)
        net.set_params(z["theta"])
        return net

    # -- use
    def predict(self, img: torch.Tensor, project: int = 1, lift: int = 1):
        """img [N,H,W,in_ch] or [H,W,in_ch] float32 CUDA -> (mu [..,H,W,out_ch] float32,
        eps [..,T,2] float64), both CUDA tensors.  lift = f > 1 predicts from the f x f
        block means of the image and upsamples mu back (ws_net_forward_lifted): for
        images f times the training resolution."""
        single = img.dim() == 3
        x = img.unsqueeze(0) if single else img
        x = x.contiguous()
        N, H, W, _ = x.shape
        mu = torch.empty(N, H, W, self.spec.out_ch, dtype=torch.float32, device=x.device)
        eps = torch.empty(N, self.spec.nsteps, 2, dtype=torch.float64, device=x.device)
        if lift > 1:
            lib._ws_check(lib.load().ws_net_forward_lifted(
                self.handle, lib._ptr(x, "float32"), N, H, W, int(lift), int(project),
                lib._ptr(mu, "float32"), lib._ptr(eps, "float64")), "ws_net_forward_lifted")
        else:
            lib._ws_check(lib.load().ws_net_forward(self.handle, lib._ptr(x, "float32"), N, H, W,
                                                    int(project), lib._ptr(mu, "float32"),
                                                    lib._ptr(eps, "float64"), None),
                          "ws_net_forward")
        return (mu[0], eps[0]) if single else (mu, eps)

    def raw(self, img: torch.Tensor):
        """Unprojected mu and the log-control z [N, 2T] (float32) for [N,H,W,in_ch]."""
        N, H, W, _ = img.shape
        mu = torch.empty(N, H, W, self.spec.out_ch, dtype=torch.float32, device=img.device)
        z = torch.empty(N, 2 * self.spec.nsteps, dtype=torch.float32, device=img.device)
        lib._ws_check(lib.load().ws_net_forward(self.handle, lib._ptr(img.contiguous(), "float32"),
                                                N, H, W, 0, lib._ptr(mu, "float32"), None,
                                                lib._ptr(z, "float32")), "ws_net_forward")
        return mu, z

    # -- training
    def loss_grad(self, img, mu_t, log_eps_t, lam_eps: float = 0.1, grad_out=None) -> float:
        N, H, W, _ = img.shape
        loss = ctypes.c_double()
        lib._ws_check(lib.load().ws_net_loss_grad(
            self.handle, lib._ptr(img, "float32"), lib._ptr(mu_t, "float32"),
            lib._ptr(log_eps_t, "float32"), N, H, W, float(lam_eps), ctypes.byref(loss),
            lib._ptr(grad_out, "float32")), "ws_net_loss_grad")
        return loss.value

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  adam_eps: float = 1e-8, weight_decay: float = 0.0) -> None:
        lib._ws_check(lib.load().ws_net_adam_step(self.handle, lr, beta1, beta2, adam_eps,
                                                  weight_decay), "ws_net_adam_step")

    def fit(self, imgs: torch.Tensor, mu_t: torch.Tensor, log_eps_t: torch.Tensor, epochs: int,
            batch: int = 16, lr: float = 1e-3, lam_eps: float = 0.1, seed: int = 0,
            lr_final: float | None = None, log=None):
        """Adam over shuffled mini-batches; cosine decay from lr to lr_final.  Returns the
        mean loss of every epoch."""
        n = imgs.shape[0]
        rng = np.random.default_rng(seed)
        steps = epochs * max(1, n // batch)
        lr_final = lr * 0.05 if lr_final is None else lr_final
        k, history = 0, []
        for ep in range(epochs):
            order = rng.permutation(n)
            tot, cnt = 0.0, 0
            for b in range(0, n - batch + 1, batch):
                idx = torch.from_numpy(order[b:b + batch]).to(imgs.device)
                x = imgs.index_select(0, idx).contiguous()
                m = mu_t.index_select(0, idx).contiguous()
                le = log_eps_t.index_select(0, idx).contiguous()
                tot += self.loss_grad(x, m, le, lam_eps)
                cnt += 1
                a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max(1, steps)))
                self.adam_step(a)
                k += 1
            history.append(tot / max(1, cnt))
            if log:
                log(f"epoch {ep + 1}/{epochs}: loss {history[-1]:.5f}")
        return history


TRAIN_SIZE = 256      # side of the images the committed weights were trained on


def lift_factor(H: int, W: int, train_size: int = TRAIN_SIZE) -> int:
    """The largest power of two f with H / f, W / f >= train_size dividing both sides (1 if
    none): the factor at which the network sees an image at its training resolution."""
    f = 1
    while H % (2 * f) == 0 and W % (2 * f) == 0 and min(H, W) // (2 * f) >= train_size:
        f *= 2
    return f


def warm_solve(ctx_handle, net: WarmStartNet, img: torch.Tensor, opts, use_eps: bool = True,
               c_out=None, fallback_on_miss: bool = False, lift: int | None = None):
    """solve() started from the network's mu(0) and eps(0) (mu only without use_eps); falls back
    to the cold start (mu = 0, eps = 57) when the warm solve diverges (AGENTS_EDIVERGED),
    and with fallback_on_miss also when it ends without reaching opts.tol.  The prediction is
    made at the training resolution (lift_factor) unless `lift` is given.
    Returns (info, eps, mu, used_fallback)."""
    T = net.spec.nsteps
    f = lift_factor(img.shape[0], img.shape[1]) if lift is None else lift
    mu0, eps0 = net.predict(img, lift=f)
    eps = eps0.contiguous() if use_eps else torch.full((T, 2), 57.0, dtype=torch.float64,
                                                       device=img.device)
    mu = mu0.reshape(img.shape[0], img.shape[1], 2, -1).contiguous()
    try:
        info = lib.solve(ctx_handle, opts, eps, mu, None, c_out)
        ok = not fallback_on_miss or opts.tol <= 0 or info.final_res < opts.tol
    except lib.AgentsError as e:
        if e.code != lib.AGENTS_EDIVERGED:
            raise
        ok, info = False, None
    if ok:
        return info, eps, mu, False
    eps = torch.full((T, 2), 57.0, dtype=torch.float64, device=img.device)
    mu = torch.zeros_like(mu)
    info = lib.solve(ctx_handle, opts, eps, mu, None, c_out)
    return info, eps, mu, True
