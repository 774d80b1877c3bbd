"""FP64 oracle of the warm-start network: a small convolutional U-Net that maps an image
to the initial dual field mu(0) and the initial control eps(0) of Algorithm 2.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT (see the package docstring).

The paper has no network; it starts every solve from mu(0) = 0 and eps(0) = 57.  This
module states, in float64 NumPy, what the CUDA warm-start network computes, so that its
kernels and its training gradients can be checked element by element:

* conv3x3: y[n, h, w, o] = b[o] + sum_{ky, kx, i} x[n, h + ky - 1, w + kx - 1, i] W[o, ky, kx, i]
  with zero padding (a 3 x 3 cross-correlation, 'same' size), optionally followed by
  ReLU; and its exact backward (dx, dW, db).
* avgpool2 / upsample2: 2 x 2 mean pooling and nearest-neighbour 2x upsampling and
  their adjoints.
* the network (levels L, base width B; widths B 2^(l-1) for l = 1..L):
  encoder level l: two conv3x3 + ReLU, then avgpool2 before the next level;
  decoder level l = L-1..1: upsample2, conv3x3 + ReLU to width B 2^(l-1), add the
  encoder output of level l, conv3x3 + ReLU;
  mu head: conv3x3 to out_ch channels (no activation);
  eps head: global mean of the level-L output, then a linear map to 2T values z; the
  control is eps = clip(exp(z), E) (z is a log-control, trained against log eps*).
* the loss  mean((mu - mu*)^2) + lam_eps mean((z - log eps*)^2)  and its gradient with
  respect to the flat parameter vector.

Mixed precision: the tensor-core convolutions take bfloat16 operands and accumulate in
float32.  With ``bf16=True`` the oracle rounds exactly the operands the GPU rounds (the
weights, each convolution's input and, in the backward pass, each convolution's output
gradient after the ReLU mask) to the nearest bfloat16 (ties to even, from float32) and
then computes in float64.  Everything else (bias, ReLU, pooling, sums, the eps head,
the loss) is unrounded.

Flat parameter layout (shared by contract with the CUDA network, stated in its header):
for every convolution in the order enc(1)a, enc(1)b, ..., enc(L)a, enc(L)b,
dec(L-1)a, dec(L-1)b, ..., dec(1)a, dec(1)b, head: W[Cout][3][3][Cin] then b[Cout];
then the eps head A[2T][B 2^(L-1)] and c[2T].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# ---------------------------------------------------------------- bfloat16 rounding
def bf16_round(a) -> np.ndarray:
    """Round to float32, then to the nearest bfloat16 (ties to even); returned as float64.

    bfloat16 keeps the upper 16 bits of the IEEE float32 pattern.  Round-to-nearest-even
    adds 0x7FFF plus the lowest kept bit to the pattern and truncates the lower 16 bits.
    """
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def _rb(a, on: bool):
    return bf16_round(a) if on else np.asarray(a, dtype=np.float64)


# ---------------------------------------------------------------- layers
def conv3x3(x, w, b, relu: bool = False, bf16: bool = True):
    """3 x 3 'same' cross-correlation with zero padding; x [N,H,W,Cin], w [Cout,3,3,Cin]."""
    x = _rb(x, bf16)
    w = _rb(w, bf16)
    N, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(np.asarray(b, dtype=np.float64), (N, H, W, w.shape[0])).copy()
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nhwi,oi->nhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return np.maximum(y, 0.0) if relu else y


def conv3x3_backward(x, w, dy, bf16: bool = True):
    """Gradients of sum(dy * conv3x3(x, w, b)) with respect to x, w and b.

    With bf16, dy, x and w are rounded as the GPU rounds them (dy after the ReLU mask,
    which the caller applies)."""
    dyr = _rb(dy, bf16)
    x = _rb(x, bf16)
    w = _rb(w, bf16)
    N, H, W, Cin = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("nhwo,oi->nhwi", dyr, w[:, ky, kx, :])
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwi->oi", dyr, xp[:, ky:ky + H, kx:kx + W, :])
    db = np.asarray(dy, dtype=np.float64).sum(axis=(0, 1, 2))
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, db


def avgpool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


# ---------------------------------------------------------------- network
@dataclass(frozen=True)
class NetConfig:
    in_ch: int = 3
    out_ch: int = 6
    base: int = 32
    levels: int = 4
    nsteps: int = 20

    def width(self, l: int) -> int:          # l = 1..levels
        return self.base * 2 ** (l - 1)


def conv_list(cfg: NetConfig):
    """(name, Cin, Cout) of every convolution in flat-parameter order."""
    out = []
    cin = cfg.in_ch
    for l in range(1, cfg.levels + 1):
        out.append((f"enc{l}a", cin, cfg.width(l)))
        out.append((f"enc{l}b", cfg.width(l), cfg.width(l)))
        cin = cfg.width(l)
    for l in range(cfg.levels - 1, 0, -1):
        out.append((f"dec{l}a", cfg.width(l + 1), cfg.width(l)))
        out.append((f"dec{l}b", cfg.width(l), cfg.width(l)))
    out.append(("head", cfg.width(1), cfg.out_ch))
    return out


def param_shapes(cfg: NetConfig):
    shapes = []
    for name, cin, cout in conv_list(cfg):
        shapes.append((name + ".W", (cout, 3, 3, cin)))
        shapes.append((name + ".b", (cout,)))
    shapes.append(("eps.A", (2 * cfg.nsteps, cfg.width(cfg.levels))))
    shapes.append(("eps.c", (2 * cfg.nsteps,)))
    return shapes


def num_params(cfg: NetConfig) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(cfg)))


def unflatten(cfg: NetConfig, theta) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shape in param_shapes(cfg):
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    if k != theta.size:
        raise ValueError(f"expected {k} parameters, got {theta.size}")
    return out


def flatten(cfg: NetConfig, grads: dict) -> np.ndarray:
    return np.concatenate([np.asarray(grads[name], dtype=np.float64).ravel()
                           for name, _ in param_shapes(cfg)])


def net_forward(cfg: NetConfig, theta, x, bf16: bool = True):
    """mu [N,H,W,out_ch] and z [N,2T] (log-control) for images x [N,H,W,in_ch]; H and W
    must be multiples of 2^(levels-1).  Returns (mu, z, cache)."""
    P = unflatten(cfg, theta)
    x = np.asarray(x, dtype=np.float64)
    cache = {"x": x}
    h = x
    enc = {}
    for l in range(1, cfg.levels + 1):
        if l > 1:
            h = avgpool2(enc[l - 1])
        cache[f"in_enc{l}a"] = h
        a = conv3x3(h, P[f"enc{l}a.W"], P[f"enc{l}a.b"], relu=True, bf16=bf16)
        cache[f"enc{l}a"] = a
        enc[l] = conv3x3(a, P[f"enc{l}b.W"], P[f"enc{l}b.b"], relu=True, bf16=bf16)
        cache[f"enc{l}b"] = enc[l]
    d = enc[cfg.levels]
    for l in range(cfg.levels - 1, 0, -1):
        u = upsample2(d)
        cache[f"in_dec{l}a"] = u
        a = conv3x3(u, P[f"dec{l}a.W"], P[f"dec{l}a.b"], relu=True, bf16=bf16)
        cache[f"dec{l}a"] = a
        s = a + enc[l]
        cache[f"in_dec{l}b"] = s
        d = conv3x3(s, P[f"dec{l}b.W"], P[f"dec{l}b.b"], relu=True, bf16=bf16)
        cache[f"dec{l}b"] = d
    cache["in_head"] = d
    mu = conv3x3(d, P["head.W"], P["head.b"], relu=False, bf16=bf16)
    g = enc[cfg.levels].mean(axis=(1, 2))
    cache["gap"] = g
    z = g @ P["eps.A"].T + P["eps.c"]
    return mu, z, cache


def loss_value(mu, z, mu_t, log_eps_t, lam_eps: float) -> float:
    return float(np.mean((mu - mu_t) ** 2) + lam_eps * np.mean((z - log_eps_t) ** 2))


def net_loss_backward(cfg: NetConfig, theta, x, mu_t, log_eps_t, lam_eps: float,
                      bf16: bool = True):
    """Loss and its gradient with respect to the flat parameters (same layout)."""
    P = unflatten(cfg, theta)
    mu, z, cache = net_forward(cfg, theta, x, bf16=bf16)
    mu_t = np.asarray(mu_t, dtype=np.float64)
    log_eps_t = np.asarray(log_eps_t, dtype=np.float64)
    loss = loss_value(mu, z, mu_t, log_eps_t, lam_eps)
    G = {}
    dmu = 2.0 * (mu - mu_t) / mu.size
    dz = 2.0 * lam_eps * (z - log_eps_t) / z.size

    def conv_back(name, inp, out, dout, relu):
        dpre = dout * (out > 0.0) if relu else dout
        dx, dw, db = conv3x3_backward(inp, P[name + ".W"], dpre, bf16=bf16)
        G[name + ".W"], G[name + ".b"] = dw, db
        return dx

    # eps head
    G["eps.A"] = dz.T @ cache["gap"]
    G["eps.c"] = dz.sum(axis=0)
    dg = dz @ P["eps.A"]
    L = cfg.levels
    eL = cache[f"enc{L}b"]
    d_enc = {L: np.broadcast_to(dg[:, None, None, :] / (eL.shape[1] * eL.shape[2]),
                                eL.shape).copy()}
    # mu head
    dd = conv_back("head", cache["in_head"], mu, dmu, relu=False)
    # decoder, level 1 up to L-1
    for l in range(1, L):
        ds = conv_back(f"dec{l}b", cache[f"in_dec{l}b"], cache[f"dec{l}b"], dd, relu=True)
        d_enc[l] = ds.copy()                       # skip connection
        du = conv_back(f"dec{l}a", cache[f"in_dec{l}a"], cache[f"dec{l}a"], ds, relu=True)
        dd = upsample2_backward(du)
    d_enc[L] = d_enc[L] + dd
    # encoder, level L down to 1
    for l in range(L, 0, -1):
        da = conv_back(f"enc{l}b", cache[f"enc{l}a"], cache[f"enc{l}b"], d_enc[l], relu=True)
        dh = conv_back(f"enc{l}a", cache[f"in_enc{l}a"], cache[f"enc{l}a"], da, relu=True)
        if l > 1:
            d_enc[l - 1] = d_enc[l - 1] + avgpool2_backward(dh)
    return loss, flatten(cfg, G)
