"""Failure paths of the C ABI, made on the host or by a loop bound, never by a GPU fault.

* AGENTS_ETIMEOUT: the union-find loops of the labels are bounded; a test hook lowers the
  bound to one iteration, so the loops give up (they exit; every index they follow is a
  label value inside the image) and agents_labels and solve() report the give-up.  The
  context stays usable and, with the default bound restored, labels are the oracle's.
* AGENTS_ENOMEM: a process-wide cap on the memory the library's contexts hold makes
  agents_init fail (and releases everything the half-built context had taken), and makes
  the first solve on a context fail when its solve buffers no longer fit; the optional
  trajectory-reuse buffers are skipped under the cap and the solve stays bitwise the same.
* AGENTS_EDIVERGED in a batch: one image's multiplier holds a NaN, so its objective is
  NaN from the start; that image stops while every other image finishes bitwise equal to
  its own solve(), and every output is written.
"""
import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, f32, zeros_dev, torch
from oracle.labels import cluster_labels
from paper_2510_16154_gb300 import lib
from synth import ImageSpec, make_image

pytestmark = pytest.mark.gpu


def _snake(H, W):
    """One component winding through the whole image: deep union-find trees."""
    c = np.zeros((H, W, 1), dtype=np.float32)
    for r in range(H):
        if r % 2 == 1:
            c[r, :, 0] = 0.9
            c[r, W - 1 if (r // 2) % 2 == 0 else 0, 0] = 0.0
    return c


def test_label_loop_bound_reports_etimeout():
    ensure_lib()
    c = _snake(61, 47)
    p, _ = params(61, 47, 1, 2, 2)
    with lib.Context(p, dev(c)) as ctx:
        lab = np.zeros((61, 47), dtype=np.int32)
        lib.agents_debug_set_label_loop_cap(1)
        try:
            with pytest.raises(lib.AgentsError) as e:
                lib.agents_labels(ctx.handle, dev(c), 0.02, lab)
            assert e.value.code == lib.AGENTS_ETIMEOUT and "loop bound" in str(e.value)
            # solve() writes its outputs, then reports the labels' give-up
            o = lib.agents_default_solve_opts()
            o.k_out, o.k_in = 1, 1
            with pytest.raises(lib.AgentsError) as e:
                lib.solve(ctx.handle, o, np.full((2, 2), 57.0),
                          np.zeros((61, 47, 2, 1), np.float32), None, None, lab)
            assert e.value.code == lib.AGENTS_ETIMEOUT
        finally:
            lib.agents_debug_set_label_loop_cap(0)
        n = lib.agents_labels(ctx.handle, dev(c), 0.02, lab)
    want, count = cluster_labels(c)
    assert n == count and np.array_equal(lab, want)
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_debug_set_label_loop_cap(-1)
    assert e.value.code == lib.AGENTS_EINVAL


def _solve(ctx, T, H, W, C):
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = 2, 3
    eps = np.full((T, 2), 57.0)
    mu = np.zeros((H, W, 2, C), dtype=np.float32)
    c = np.zeros((H, W, C), dtype=np.float32)
    info = lib.solve(ctx.handle, o, eps, mu, None, c, None)
    return eps, mu, c, info


def test_memory_limit_reports_enomem():
    ensure_lib()
    H, W, C, T = 40, 48, 3, 5
    img = f32(make_image(ImageSpec(H, W, C, regions=4, sigma=0.05), 21))
    p, _ = params(H, W, C, 2, T)
    torch.cuda.synchronize()
    held0 = lib.agents_memory_held()
    lib.agents_set_memory_limit(held0 + 4096)         # far below one context
    try:
        with pytest.raises(lib.AgentsError) as e:
            lib.Context(p, dev(img, np.float32))
        assert e.value.code == lib.AGENTS_ENOMEM and "memory limit" in str(e.value)
        assert lib.agents_memory_held() == held0     # the half-built context gave it back
    finally:
        lib.agents_set_memory_limit(0)
    # a context that fits, but whose solve buffers do not
    ctx = lib.Context(p, dev(img, np.float32))
    try:
        held1 = lib.agents_memory_held()
        assert held1 > held0
        lib.agents_set_memory_limit(held1 + 1024)
        try:
            with pytest.raises(lib.AgentsError) as e:
                _solve(ctx, T, H, W, C)
            assert e.value.code == lib.AGENTS_ENOMEM
        finally:
            lib.agents_set_memory_limit(0)
        # with the cap lifted the solve runs; its reuse buffers were skipped under the
        # cap, and the result is bitwise that of a context that had them
        got = _solve(ctx, T, H, W, C)
    finally:
        ctx.close()
    assert lib.agents_memory_held() == held0
    with lib.Context(p, dev(img, np.float32)) as ctx2:
        want = _solve(ctx2, T, H, W, C)
    for a, b in zip(got[:3], want[:3]):
        assert np.array_equal(a, b)
    assert got[3].trials == want[3].trials
    assert got[3].forward_steps > want[3].forward_steps    # recomputed without reuse


def test_batch_reports_a_diverging_image_and_finishes_the_rest():
    ensure_lib()
    T = 5
    cases = [(30, 40, 3, 2, 4, 31), (26, 33, 3, 3, 3, 32), (20, 28, 1, 2, 3, 33)]
    imgs = [f32(make_image(ImageSpec(H, W, C, regions=K, sigma=0.05), s))
            for H, W, C, R, K, s in cases]
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = 2, 3
    bad = 1
    ctxs, eps, mus, cs = [], [], [], []
    try:
        for k, ((H, W, C, R, K, s), img) in enumerate(zip(cases, imgs)):
            p, _ = params(H, W, C, R, T)
            ctxs.append(lib.Context(p, dev(img, np.float32)))
            eps.append(np.full((T, 2), 57.0))
            mu = np.zeros((H, W, 2, C), dtype=np.float32)
            if k == bad:
                mu[3, 4, 0, 0] = np.nan
            mus.append(mu)
            cs.append(np.full((H, W, C), -1.0, dtype=np.float32))
        with pytest.raises(lib.AgentsError) as e:
            lib.agents_solve_batch([c.handle for c in ctxs], o, eps, mus, cs,
                                   autotune=False, use_graph=True)
        assert e.value.code == lib.AGENTS_EDIVERGED
        infos = e.value.infos
    finally:
        for c in ctxs:
            c.close()
    assert infos is not None and infos[bad].outer_done < o.k_out
    assert np.all(cs[bad] != -1.0)                       # its output was written
    for k, ((H, W, C, R, K, s), img) in enumerate(zip(cases, imgs)):
        if k == bad:
            continue
        p, _ = params(H, W, C, R, T)
        with lib.Context(p, dev(img, np.float32)) as ctx:
            e1, m1, c1, i1 = _solve_opts(ctx, o, T, H, W, C)
        assert np.array_equal(eps[k], e1) and np.array_equal(mus[k], m1)
        assert np.array_equal(cs[k], c1)
        assert infos[k].outer_done == o.k_out == i1.outer_done


def _solve_opts(ctx, o, T, H, W, C):
    eps = np.full((T, 2), 57.0)
    mu = np.zeros((H, W, 2, C), dtype=np.float32)
    c = np.zeros((H, W, C), dtype=np.float32)
    info = lib.solve(ctx.handle, o, eps, mu, None, c, None)
    return eps, mu, c, info
