"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas only: every rank solves
its own image, the only collective is the whole-job timing).  The slowest rank's time
and the sum of all ranks' pixel-steps give the aggregate; ranks get distinct images; the
reference arm runs on rank 0 only.  Also the rule by which a timed region's clock record
disqualifies it (measured once more), and the pair count behind the roofline's
algorithmic flops against a brute-force enumeration."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, ps = bench.reduce_over_ranks(torch, dist, elapsed=1.5 + rank, pixel_steps=1000 * (rank + 1),
                                        device="cpu")
        out[rank] = (t, ps, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0][:2] == res[1][:2] == (2.5, 3000.0)       # max time, summed work
    assert res[0][2] != res[1][2]                            # independent images


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(torch, None, 2.0, 7, "cpu") == (2.0, 7.0)


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        warmup, steps = 1, 1
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda: called.append(1) or (1, 1.0))
    assert bench.run_reference(A, rank=1, world=2) == 0
    assert called == [] and capsys.readouterr().out == ""


@pytest.mark.parametrize("clk,rejected", [
    (None, False),
    ({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, False),
    ({"sm_mhz": 1900.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]}, False),
    ({"sm_mhz": 1400.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]}, False),
    ({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown"]}, True),
    ({"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_thermal_slowdown"]}, True),
    ({"sm_mhz": 1200.0, "sm_max_mhz": 2070.0, "reasons": []}, True),   # a leftover lock
])
def test_clock_record_rejection(clk, rejected):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.clocks_rejected(clk) is rejected


@pytest.mark.parametrize("h,w,r", [(1, 1, 1), (3, 5, 1), (7, 4, 2), (9, 9, 5), (6, 13, 3)])
def test_roofline_pair_count_is_the_brute_force_count(h, w, r):
    # The roofline numerator counts each unordered in-window pair of distinct in-image
    # pixels once (window: |drow|, |dcol| <= r).  Enumerate the pairs directly.
    sys.path.insert(0, ROOT)
    import bench
    pairs = 0
    for i in range(h * w):
        for j in range(i + 1, h * w):
            (ri, ci), (rj, cj) = divmod(i, w), divmod(j, w)
            if abs(ri - rj) <= r and abs(ci - cj) <= r:
                pairs += 1
    for c in (1, 3, 31):
        assert bench.forward_flops_per_launch(h, w, c, r) == pairs * (7 * c + 9)
        assert bench.adjoint_flops_per_launch(h, w, c, r) == pairs * (11 * c + 18)
