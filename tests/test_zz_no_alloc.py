"""The allocation-free objective entry point, checked against the context-based one.

agents_objective_noalloc exists for callers that may not allocate device memory: hosts
that reserve the whole device budget themselves and hand a library only pre-allocated
buffers, and latency-critical loops that must not call cudaMalloc because it can
synchronise the device.  It keeps its reduction scratch in a static device array inside
the library.  Through the C ABI, this test checks that two calls in a row return the
objective and the terminal adjoint of agents_objective within the tolerances of the
other TV tests (the array keeps the previous call's partial sums, which must not leak
into the next result), that a smaller image in between changes nothing, and that an
image too large for the static array is refused.  This file is collected last so that a
run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, f32, zeros_dev, torch
from paper_2510_16154_gb300 import lib

pytestmark = pytest.mark.gpu


def _case(rng, H, W, C):
    c0 = f32(rng.uniform(size=(H, W, C)))
    c = f32(np.clip(c0 + rng.normal(scale=0.1, size=c0.shape), 0, 1))
    v = f32(rng.normal(scale=20.0, size=(H, W, 2, C)))
    mu = f32(rng.normal(scale=5.0, size=(H, W, 2, C)))
    return c0, c, v, mu


def _reference(c0, c, v, mu, alpha, rho):
    """agents_objective through a context (which allocates its own workspaces)."""
    H, W, C = c.shape
    p, _ = params(H, W, C, 2, 1, alpha=alpha, rho=rho)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        obj = np.zeros(1)
        lam = zeros_dev(H, W, C)
        lib.agents_objective(ctx.handle, dev(c, np.float32), dev(v, np.float32),
                             dev(mu, np.float32), obj, lam)
        return obj[0], host(lam).astype(np.float64)


def _noalloc(c0, c, v, mu, alpha, rho):
    H, W, C = c.shape
    obj = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    lam = torch.full((H, W, C), float("nan"), device="cuda")
    lib.agents_objective_noalloc(H, W, C, alpha, rho, 0, dev(c, np.float32),
                                 dev(c0, np.float32), dev(v, np.float32), dev(mu, np.float32),
                                 obj, lam)
    return host(obj)[0], host(lam).astype(np.float64)


def test_noalloc_objective_matches_context_entry_point():
    ensure_lib()
    rng = np.random.default_rng(31)
    alpha, rho = 300.0, 0.2
    big = _case(rng, 300, 517, 3)
    small = _case(rng, 37, 41, 3)
    obj_ref, lam_ref = _reference(*big, alpha, rho)
    for _ in range(2):                                # two calls in a row
        obj, lam = _noalloc(*big, alpha, rho)
        assert obj == pytest.approx(obj_ref, rel=1e-6)
        assert np.max(np.abs(lam - lam_ref)) <= 1e-5 * np.max(np.abs(lam_ref))
    obj_s_ref, lam_s_ref = _reference(*small, alpha, rho)
    obj_s, lam_s = _noalloc(*small, alpha, rho)       # fewer blocks than the call before
    assert obj_s == pytest.approx(obj_s_ref, rel=1e-6)
    assert np.max(np.abs(lam_s - lam_s_ref)) <= 1e-5 * np.max(np.abs(lam_s_ref))


def test_noalloc_rejects_images_beyond_the_static_scratch():
    ensure_lib()
    x = torch.zeros(64, device="cuda")
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.AgentsError) as e:         # 8192 x 8192 needs 65536 blocks
        lib.agents_objective_noalloc(8192, 8192, 3, 300.0, 0.2, 0, x, x, x, x, obj, None)
    assert e.value.code == lib.AGENTS_EINVAL
    assert "static scratch" in str(e.value)
