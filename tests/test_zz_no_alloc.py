"""The allocation-free objective entry point, checked against the context-based one.

agents_objective_noalloc exists for callers that may not allocate device memory: hosts
that reserve the whole device budget themselves and hand a library only pre-allocated
buffers, and latency-critical loops that must not call cudaMalloc because it can
synchronise the device.  It keeps its reduction scratch in a static device array inside
the library.  Through the C ABI, this test checks that two calls in a row return the
objective and the terminal adjoint of agents_objective within the tolerances of the
other TV tests (the array keeps the previous call's partial sums, which must not leak
into the next result), for both TV norms, for 3 and 31 channels (the generic objective
kernel), on the default stream and on a side stream; that a smaller image in between
changes nothing; and that an image too large for the static array, or a host buffer, is
refused.  This file is collected last so that a run stopping at its first failure has
already run every other test.
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


def _reference(c0, c, v, mu, alpha, rho, tv_mode):
    """agents_objective through a context (which allocates its own workspaces)."""
    H, W, C = c.shape
    p, _ = params(H, W, C, 2, 1, alpha=alpha, rho=rho, tv_mode=tv_mode)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        obj = np.zeros(1)
        lam = zeros_dev(H, W, C)
        lib.agents_objective(ctx.handle, dev(c, np.float32), dev(v, np.float32),
                             dev(mu, np.float32), obj, lam)
        return obj[0], host(lam).astype(np.float64)


def _noalloc(c0, c, v, mu, alpha, rho, tv_mode, stream=None):
    H, W, C = c.shape
    fields = [dev(x, np.float32) for x in (c, c0, v, mu)]
    obj = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    lam = torch.full((H, W, C), float("nan"), device="cuda")
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())   # inputs are ready on it
        with torch.cuda.stream(stream):
            lib.agents_objective_noalloc(H, W, C, alpha, rho, tv_mode, *fields, obj, lam,
                                         stream=stream)
        stream.synchronize()
    else:
        lib.agents_objective_noalloc(H, W, C, alpha, rho, tv_mode, *fields, obj, lam)
    return host(obj)[0], host(lam).astype(np.float64)


def _close(got, want):
    obj, lam = got
    obj_ref, lam_ref = want
    assert obj == pytest.approx(obj_ref, rel=1e-6)
    assert np.max(np.abs(lam - lam_ref)) <= 1e-5 * np.max(np.abs(lam_ref))


@pytest.mark.parametrize("C", [3, 31])
@pytest.mark.parametrize("tv_mode", [0, 1])
def test_noalloc_objective_matches_context_entry_point(tv_mode, C):
    ensure_lib()
    rng = np.random.default_rng(31 + C + tv_mode)
    alpha, rho = 300.0, 0.2
    big = _case(rng, 300, 517, C) if C <= 3 else _case(rng, 90, 260, C)
    small = _case(rng, 37, 41, C)
    ref = _reference(*big, alpha, rho, tv_mode)
    for _ in range(2):                                # two calls in a row
        _close(_noalloc(*big, alpha, rho, tv_mode), ref)
    _close(_noalloc(*small, alpha, rho, tv_mode),     # fewer blocks than the call before
           _reference(*small, alpha, rho, tv_mode))
    side = torch.cuda.Stream()
    _close(_noalloc(*big, alpha, rho, tv_mode, stream=side), ref)


def test_noalloc_rejects_images_beyond_the_static_scratch():
    ensure_lib()
    raw = lib.load().agents_objective_noalloc
    x = torch.zeros(64, device="cuda")
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 8192 x 8192 needs 65536 reduction blocks; the library refuses before any launch
    st = raw(8192, 8192, 3, 300.0, 0.2, 0, x.data_ptr(), x.data_ptr(), x.data_ptr(),
             x.data_ptr(), obj.data_ptr(), None, None)
    assert st == lib.AGENTS_EINVAL
    assert "static scratch" in lib.agents_last_error()
    # the Python binding refuses buffers smaller than the fields before calling
    with pytest.raises(ValueError):
        lib.agents_objective_noalloc(64, 64, 3, 300.0, 0.2, 0, x, x, x, x, obj, None)
    # a host buffer is refused by the library
    buf = np.zeros(4 * 4 * 2 * 3 + 4, dtype=np.float32)
    off = (-buf.ctypes.data % 16) // 4                 # a 16-byte aligned host view
    h = buf[off:off + 4 * 4 * 2 * 3]
    d = torch.zeros(4 * 4 * 2 * 3, device="cuda")
    st = raw(4, 4, 3, 300.0, 0.2, 0, h.ctypes.data, d.data_ptr(), d.data_ptr(), d.data_ptr(),
             obj.data_ptr(), None, None)
    assert st == lib.AGENTS_EINVAL
    assert "device memory" in lib.agents_last_error()
