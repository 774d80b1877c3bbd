"""GPU parity of the cluster labels (bit-exact: an index computation, decided in float32
on both sides) and of the full solve (Algorithm 2 with Algorithm 1 inside) against the
FP64 oracle, plus the error contract of the C ABI on the device path."""
import os

import numpy as np
import pytest

from gpuutil import ensure_lib, dev, host, params, f32, zeros_dev, torch
import oracle
from oracle.labels import cluster_labels, label_agreement
from paper_2510_16154_gb300 import lib
from synth import ImageSpec, make_image, PARITY_64_RGB

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- labels

def _snake(H, W):
    """One component winding through the whole image (worst case for union-find depth)."""
    c = np.zeros((H, W, 1), dtype=np.float32)
    for r in range(H):
        if r % 2 == 1:
            c[r, :, 0] = 0.9
            c[r, W - 1 if (r // 2) % 2 == 0 else 0, 0] = 0.0
    return c


@pytest.mark.parametrize("H,W,C,levels", [(1, 1, 3, 4), (1, 37, 3, 4), (37, 1, 1, 3), (50, 70, 3, 6),
                                          (256, 256, 1, 3), (300, 517, 3, 40)])
def test_labels_bit_exact(H, W, C, levels):
    ensure_lib()
    rng = np.random.default_rng(H + W + C)
    c = (np.round(rng.uniform(size=(H, W, C)) * levels) / levels * 0.05).astype(np.float32)
    p, _ = params(H, W, C, 2, 1)
    with lib.Context(p, dev(c)) as ctx:
        lab = torch.zeros(H, W, dtype=torch.int32, device="cuda")
        n = lib.agents_labels(ctx.handle, dev(c), 0.02, lab)
        got = host(lab)
    want, count = cluster_labels(c)
    assert n == count and np.array_equal(got, want)


def test_labels_snake_and_threshold_edge():
    ensure_lib()
    c = _snake(101, 77)
    p, _ = params(101, 77, 1, 2, 1)
    with lib.Context(p, dev(c)) as ctx:
        lab = np.zeros((101, 77), dtype=np.int32)       # host output
        n = lib.agents_labels(ctx.handle, dev(c), 0.02, lab)
    want, count = cluster_labels(c)
    assert n == count and np.array_equal(lab, want)
    # exact float32 threshold: a difference of exactly fl32(0.02) joins
    a = np.float32(0.25)
    b = np.float32(a + np.float32(0.02))
    c2 = np.array([[[a], [b], [np.float32(b + np.float32(0.03))]]], dtype=np.float32)
    p, _ = params(1, 3, 1, 1, 1)
    with lib.Context(p, dev(c2)) as ctx:
        lab = np.zeros((1, 3), dtype=np.int32)
        n = lib.agents_labels(ctx.handle, dev(c2), 0.02, lab)
    want, count = cluster_labels(c2)
    assert n == count and np.array_equal(lab, want)


# ---------------------------------------------------------------- solve

def _solve_gpu(c0, R, T, k_out, k_in, device_buffers=True, **kw):
    H, W, C = c0.shape
    p, op = params(H, W, C, R, T, **kw)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = k_out, k_in
    eps = np.full((T, 2), 57.0)
    mu = np.zeros((H, W, 2, C), dtype=np.float32)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        if device_buffers:
            eps_d, mu_d = dev(eps), dev(mu)
            c_d, v_d = zeros_dev(H, W, C), zeros_dev(H, W, 2, C)
            lab_d = torch.zeros(H, W, dtype=torch.int32, device="cuda")
            info = lib.solve(ctx.handle, o, eps_d, mu_d, v_d, c_d, lab_d)
            out = dict(eps=host(eps_d), mu=host(mu_d), v=host(v_d), c=host(c_d), labels=host(lab_d))
        else:
            c_h = np.zeros((H, W, C), dtype=np.float32)
            v_h = np.zeros((H, W, 2, C), dtype=np.float32)
            lab_h = np.zeros((H, W), dtype=np.int32)
            info = lib.solve(ctx.handle, o, eps, mu, v_h, c_h, lab_h)
            out = dict(eps=eps, mu=mu, v=v_h, c=c_h, labels=lab_h)
    return out, info, op


def test_small_solve_matches_oracle():
    ensure_lib()
    c0 = f32(make_image(ImageSpec(20, 24, 3, regions=3, sigma=0.05), 7))
    out, info, op = _solve_gpu(c0, 2, 4, 3, 3)
    ref = oracle.admm_solve(c0, op, oracle.SolveOpts(k_out=3, k_in=3))
    assert info.outer_done == 3
    assert info.trials == sum(i.trials for i in ref["inner"])
    assert np.max(np.abs(out["c"] - ref["c"])) <= 1e-4
    assert np.max(np.abs(out["eps"] - ref["eps"])) <= 1e-3 * np.max(np.abs(ref["eps"]))
    assert np.max(np.abs(out["mu"] - ref["mu"])) <= 1e-4 * max(1.0, np.max(np.abs(ref["mu"])))


def test_host_and_device_buffers_agree():
    ensure_lib()
    c0 = f32(make_image(ImageSpec(33, 40, 3, regions=4, sigma=0.05), 3))
    a, ia, _ = _solve_gpu(c0, 2, 5, 2, 3, device_buffers=True)
    b, ib, _ = _solve_gpu(c0, 2, 5, 2, 3, device_buffers=False)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert ia.as_dict() == ib.as_dict()


def test_constant_image_solve_stalls():
    ensure_lib()
    c0 = np.full((16, 16, 3), 0.4, dtype=np.float32)
    out, info, _ = _solve_gpu(c0, 2, 4, 2, 3)
    assert np.array_equal(out["c"], c0)
    assert np.all(out["eps"] == 57.0) and info.trials == 0
    assert info.stationary == 2 and info.stalls == 0   # D = 0: nothing can move
    assert np.all(out["labels"] == 0)


def _differing_join_decisions(c_gpu, c_ref, thr=0.02):
    """Max-channel colour differences (reference side) of every 4-neighbour pair that is
    joined on one side and not on the other."""
    g = np.asarray(c_gpu, dtype=np.float32)
    r = np.asarray(c_ref).astype(np.float32)
    t = np.float32(thr)
    out = []
    for sl_a, sl_b in (((slice(None), slice(1, None)), (slice(None), slice(None, -1))),
                       ((slice(1, None), slice(None)), (slice(None, -1), slice(None)))):
        dg = np.max(np.abs(g[sl_a] - g[sl_b]), axis=-1)
        dr = np.max(np.abs(r[sl_a] - r[sl_b]), axis=-1)
        differ = (dg <= t) != (dr <= t)
        out.extend(dr[differ].astype(np.float64).tolist())
    return np.array(out)


# The one declared deviation from "equal cluster count": at alpha = 3000 the 64 x 64 seed-0
# workload ends with ~3900 near-singleton clusters, and a neighbour pair whose largest
# channel difference lies within the colour tolerance of the 0.02 threshold may be joined
# on one side only.  Accepted there alone, for at most this many such pairs, each within
# twice the measured max|c - c_oracle| of the threshold.
TIE_SEED, TIE_ALPHA, MAX_TIE_PAIRS = 0, 3000.0, 4


@pytest.mark.parametrize("alpha", [3000.0, 100.0])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_parity_64_rgb_full_solve(seed, alpha):
    """64x64x3, 4 Voronoi regions, sigma 0.05; R = 2, T = 20, 30 DAL iterations per
    multiplier step, 10 multiplier steps, against the stored FP64 oracle run (written by
    tests/golden/make_oracle_parity.py).  Colours within 1e-4 max-abs; cluster labels
    agree on >= 99.9% of pixels with equal count, except in the one declared case
    (seed 0 at alpha = 3000, ~3900 near-singleton clusters): there a count difference is
    accepted only for at most MAX_TIE_PAIRS neighbour pairs decided differently, each a
    threshold tie within twice the colour error.

    Late Armijo tests can sit within float32 rounding of the state (relative differences
    of L~ near 1e-8, mostly at alpha = 3000), so the two decision traces may part; such
    steps move c by ~1e-7.  The fraction of DAL iterations with the same trial count is
    printed, not asserted."""
    ensure_lib()
    path = os.path.join(GOLDEN, f"oracle_parity64_a{int(alpha)}_seed{seed}.npz")
    if not os.path.exists(path):
        pytest.fail(f"missing {path}: run tests/golden/make_oracle_parity.py")
    ref = np.load(path)
    c0 = f32(make_image(PARITY_64_RGB, seed))
    H, W, C = c0.shape
    p, _ = params(H, W, C, 2, 20, alpha=alpha)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = 10, 30
    eps = np.full((20, 2), 57.0)
    mu = np.zeros((H, W, 2, C), dtype=np.float32)
    c = np.zeros((H, W, C), dtype=np.float32)
    labels = np.zeros((H, W), dtype=np.int32)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        info = lib.solve(ctx.handle, o, eps, mu, None, c, labels)
        log = lib.agents_solve_log(ctx.handle)
    err = np.max(np.abs(c - ref["c"]))
    agree = label_agreement(labels, ref["labels"])
    n_gpu = len(np.unique(labels))
    trials = np.array([r["trials"] for r in log])
    n = min(len(trials), len(ref["trials"]))
    same = float(np.mean(trials[:n] == ref["trials"][:n])) if n else 1.0
    print(f"alpha {alpha} seed {seed}: max|dc| {err:.3e} agree {agree:.5f} "
          f"count {n_gpu}/{int(ref['count'])} trials {trials.sum()}/{int(ref['trials'].sum())} "
          f"same-trace {same:.3f}")
    assert err <= 1e-4
    assert agree >= 0.999
    ties = _differing_join_decisions(c, ref["c"])
    print(f"  pairs decided differently: {len(ties)} "
          f"(max |diff - 0.02| {np.max(np.abs(ties - 0.02)) if len(ties) else 0.0:.2e})")
    if n_gpu != int(ref["count"]):
        # only the declared deviation: seed 0 at alpha = 3000, a bounded number of
        # threshold ties
        assert (seed, alpha) == (TIE_SEED, TIE_ALPHA)
        assert 0 < len(ties) <= MAX_TIE_PAIRS
        assert np.all(np.abs(ties - 0.02) <= 2.0 * err)
    assert info.outer_done == 10
    # the primal-dual gap of the last multiplier step is below that of the first
    assert info.final_gap < ref["gap"][0]


# ---------------------------------------------------------------- error contract

def test_abi_errors_on_device():
    ensure_lib()
    c0 = np.full((8, 8, 3), 0.5, dtype=np.float32)
    p, _ = params(8, 8, 3, 2, 3)
    with lib.Context(p, dev(c0)) as ctx:
        v = zeros_dev(8, 8, 2, 3)
        D = np.zeros((3, 2))
        eps = np.full((3, 2), 57.0)
        with pytest.raises(lib.AgentsError) as e:          # adjoint before any stored forward
            lib.agents_adjoint(ctx.handle, eps, v, v, D)
        assert e.value.code == lib.AGENTS_ESTATE
        lib.agents_forward(ctx.handle, eps, None, store=True)
        with pytest.raises(lib.AgentsError) as e:          # different control
            lib.agents_adjoint(ctx.handle, eps + 1.0, v, v, D)
        assert e.value.code == lib.AGENTS_ESTATE
        lib.agents_adjoint(ctx.handle, eps, v, v, D)       # same control: fine
        big = torch.zeros(8 * 8 * 3 + 1, device="cuda")
        with pytest.raises(lib.AgentsError) as e:          # misaligned field pointer
            lib.pd_tv_step(ctx.handle, big.data_ptr() + 4, v, v)
        assert e.value.code == lib.AGENTS_EINVAL
        with pytest.raises(lib.AgentsError) as e:          # NaN control
            lib.agents_forward(ctx.handle, np.full((3, 2), np.nan), None, store=False)
        assert e.value.code == lib.AGENTS_EINVAL
        with pytest.raises(lib.AgentsError) as e:          # negative semi-axis
            lib.agents_forward(ctx.handle, np.full((3, 2), -1.0), None, store=False)
        assert e.value.code == lib.AGENTS_EINVAL
        o = lib.agents_default_solve_opts()
        o.ls_b = 1.5
        with pytest.raises(lib.AgentsError) as e:
            lib.solve(ctx.handle, o, eps.copy(), np.zeros((8, 8, 2, 3), np.float32))
        assert e.value.code == lib.AGENTS_EINVAL
    # the context stays usable after errors
    with lib.Context(p, dev(c0)) as ctx:
        out = zeros_dev(8, 8, 3)
        lib.agents_forward(ctx.handle, np.full((3, 2), 57.0), out, store=False)
        assert np.array_equal(host(out), c0)


# ---------------------------------------------------------------- Algorithm 1 with J

@pytest.mark.parametrize("alpha", [50.0, 2000.0])
def test_dal_solve_with_J_matches_oracle(alpha):
    """Algorithm 1 as published (quadratic cost J = L~ with rho = 1, v = mu = 0), stopping
    on the relative cost change eta = 1e-10 or after 8 iterations, against the oracle."""
    ensure_lib()
    c0 = f32(make_image(ImageSpec(32, 40, 3, regions=4, sigma=0.05), 12))
    T = 8
    p, op = params(32, 40, 3, 2, T, alpha=alpha, rho=1.0, gamma=1.0)
    o = lib.agents_default_solve_opts()
    o.k_in, o.tol = 8, 1e-10
    eps = np.full((T, 2), 57.0)
    c = np.zeros((32, 40, 3), dtype=np.float32)
    with lib.Context(p, dev(c0, np.float32)) as ctx:
        info = lib.dal_solve(ctx.handle, o, eps, c)
        log = lib.agents_solve_log(ctx.handle)
    ref = oracle.dal_solve(c0, op, oracle.SolveOpts(), max_iter=8, eta=1e-10)
    assert np.max(np.abs(c - ref["c"])) <= 1e-4
    assert info.final_obj == pytest.approx(ref["log"][-1].L, rel=1e-5)
    Ls = [r["L"] for r in log if r["status"] == 0]
    assert all(b <= a for a, b in zip(Ls, Ls[1:]))          # J decreases
    assert oracle.cost_J(c.astype(np.float64), c0, op) == pytest.approx(info.final_obj, rel=1e-5)


def test_trajectory_reuse_changes_nothing():
    """Full-store mode reuses accepted trial trajectories (fewer Euler steps); the
    checkpointed mode recomputes them.  Both must give bitwise the same solve."""
    ensure_lib()
    img = f32(make_image(ImageSpec(40, 52, 3, regions=5, ramp=0.05, sigma=0.06), 4))
    outs = []
    for mode in (0, 3):
        p, _ = params(40, 52, 3, 3, 9, traj_mode=mode)
        o = lib.agents_default_solve_opts()
        o.k_out, o.k_in = 3, 6
        eps = np.full((9, 2), 57.0)
        mu = np.zeros((40, 52, 2, 3), dtype=np.float32)
        c = np.zeros((40, 52, 3), dtype=np.float32)
        with lib.Context(p, dev(img, np.float32)) as ctx:
            info = lib.solve(ctx.handle, o, eps, mu, None, c)
            eps2 = eps.copy()
            dinfo = lib.dal_solve(ctx.handle, o, eps2, c2 := np.zeros_like(c))
        outs.append((eps, mu, c, info, eps2, c2, dinfo))
    (e0, m0, c0, i0, f0, d0, j0), (e1, m1, c1, i1, f1, d1, j1) = outs
    assert np.array_equal(e0, e1) and np.array_equal(m0, m1) and np.array_equal(c0, c1)
    assert np.array_equal(f0, f1) and np.array_equal(d0, d1)
    assert i0.trials == i1.trials and i0.outer_done == i1.outer_done
    # mode 0 skips the recomputations; mode 3 also recomputes checkpoint segments
    assert i0.forward_steps < i1.forward_steps
    assert j0.forward_steps < j1.forward_steps


def test_solve_logs(tmp_path):
    """Per-multiplier-step records agree with solve_info and the DAL records."""
    ensure_lib()
    img = f32(make_image(ImageSpec(30, 34, 3, regions=4, sigma=0.05), 8))
    p, _ = params(30, 34, 3, 2, 6)
    o = lib.agents_default_solve_opts()
    o.k_out, o.k_in = 4, 5
    eps = np.full((6, 2), 57.0)
    mu = np.zeros((30, 34, 2, 3), dtype=np.float32)
    with lib.Context(p, dev(img, np.float32)) as ctx:
        info = lib.solve(ctx.handle, o, eps, mu)
        outer = lib.agents_solve_outer_log(ctx.handle)
        dal = lib.agents_solve_log(ctx.handle)
        path = tmp_path / "log.jsonl"
        lib.write_solve_log_jsonl(ctx.handle, str(path), info)
    assert [r["outer"] for r in outer] == list(range(1, info.outer_done + 1))
    assert sum(r["inner_done"] for r in outer) == info.inner_done == len(dal)
    last = outer[-1]
    assert last["L"] == info.final_obj and last["res"] == info.final_res
    assert last["gap"] == info.final_gap and last["sigma"] == info.final_sigma
    assert all(r["r"] >= 0 and r["K"] > 0 and np.isfinite(r["s"]) for r in outer)
    lines = path.read_text().splitlines()
    assert len(lines) == len(dal) + len(outer) + 1
