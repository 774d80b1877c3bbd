"""GPU checks of the high-resolution control transfer (Section 4.3).

* The transfer is the forward sweep with the window radius scaled by the resolution
  factor: parity with the FP64 oracle's forward sweep at the scaled radius (1e-5, the
  20-step sweep tolerance).
* On a 128 x 128 scene and its 2 x 2 mean-pooled 64 x 64 version, the control solved on
  the small image, applied to the large one, yields a result whose pooled version stays
  close to the small image's result (0.02 mean-abs) and whose total variation falls by
  at least the fraction the small image's own solve removes, less 0.1.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, f32, torch
import oracle
from oracle.tv import grad
from paper_2510_16154_gb300 import lib
from paper_2510_16154_gb300.hires import apply_control, transfer_radius
from synth import ImageSpec, make_image

pytestmark = pytest.mark.gpu


def test_transfer_is_scaled_window_forward_sweep():
    ensure_lib()
    rng = np.random.default_rng(3)
    img = f32(make_image(ImageSpec(40, 36, 3, regions=4, sigma=0.05), 2))
    eps = np.column_stack([rng.uniform(2, 60, 6), rng.uniform(2, 60, 6)])
    out = apply_control(eps, dev(img, np.float32), 2, 2.0)
    assert transfer_radius(2, 2.0) == 4
    _, op = params(40, 36, 3, 4, 6)
    want = oracle.forward_final(img, eps, op)
    assert np.max(np.abs(host(out) - want)) <= 1e-5


def _tv(c):
    g = np.stack([np.gradient(c[..., k]) for k in range(c.shape[-1])])
    return float(np.sum(np.sqrt(np.sum(g ** 2, axis=(0, 1)))))


def test_control_from_low_resolution_segments_high_resolution():
    ensure_lib()
    hi = f32(make_image(ImageSpec(128, 128, 3, regions=6, ramp=0.05, sigma=0.06), 11))
    lo = f32(hi.reshape(64, 2, 64, 2, 3).mean(axis=(1, 3)))
    R, T = 2, 20
    p, _ = params(64, 64, 3, R, T)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = 6, 10
    eps = np.full((T, 2), 57.0)
    mu = np.zeros((64, 64, 2, 3), dtype=np.float32)
    c_lo = np.zeros((64, 64, 3), dtype=np.float32)
    with lib.Context(p, dev(lo, np.float32)) as ctx:
        lib.solve(ctx.handle, o, eps, mu, None, c_lo)
    c_hi = host(apply_control(eps, dev(hi, np.float32), R, 2.0)).astype(np.float64)
    pooled = c_hi.reshape(64, 2, 64, 2, 3).mean(axis=(1, 3))
    diff = np.mean(np.abs(pooled - c_lo))
    r_lo, r_hi = _tv(c_lo.astype(np.float64)) / _tv(lo), _tv(c_hi) / _tv(hi)
    print(f"mean |pool(c_hi) - c_lo| = {diff:.4f}; TV ratio low-res solve {r_lo:.3f}, "
          f"transferred {r_hi:.3f}")
    assert diff <= 0.02
    assert r_hi < 1.0 and r_hi <= r_lo + 0.1
