"""Seeded initial parameters of the warm-start network (random inputs, no network logic).

``shapes`` is the list of (name, shape) of the flat parameter vector, in order; names
end in ".W" (convolution weights [Cout, 3, 3, Cin]), ".b" (biases), "eps.A" (the control
head's matrix) or "eps.c" (its bias).
"""
from __future__ import annotations

import numpy as np


def init_net_params(shapes, seed: int, log_eps0: float = float(np.log(57.0))) -> np.ndarray:
    """He-normal convolution weights, zero biases, a small control-head matrix and a
    control-head bias of log 57 (the solve's default eps(0)).  float32 values."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in shapes:
        if name.endswith(".W"):
            fan_in = int(np.prod(shape[1:]))
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shape).ravel())
        elif name == "eps.A":
            parts.append(rng.normal(0.0, 0.01, size=shape).ravel())
        elif name == "eps.c":
            parts.append(np.full(shape, log_eps0).ravel())
        else:
            parts.append(np.zeros(shape).ravel())
    return np.concatenate(parts).astype(np.float32)
