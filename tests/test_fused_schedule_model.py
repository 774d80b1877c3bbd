"""A model, on the CPU, of the job protocol of the whole-sweep launches.

A persistent grid takes (step k, tile t) jobs in step-major order from one counter; a job
of step k > 0 waits until the 3 x 3 tiles around t have finished step k - 1, then reads
their step-(k - 1) outputs and writes tile t of step k's output.  With two ping-pong
buffers, step k + 1 writes the buffer that step k reads.  The kernel relies on two
arguments, which this discrete-event model checks under random job durations, fewer
blocks than jobs, and blocks that become resident late (another kernel holding SMs):

* no schedule deadlocks: every job a block waits for has a smaller index and has been
  taken by a running block;
* every read sees the previous step's version, and no job overwrites a tile while a job
  that reads it is still running, because the neighbourhood is symmetric: the jobs that
  read tile n of a buffer are exactly the ones job (k + 1, n) waits for.

A planted mistake (waiting for the tile itself only) must break the second argument.
"""
import heapq

import numpy as np
import pytest


def neighbours(t, tx_n, ty_n):
    """The 3 x 3 tiles around tile t (row-major tile index), clipped to the grid."""
    tx, ty = t % tx_n, t // tx_n
    return [(ty + dy) * tx_n + tx + dx for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if 0 <= tx + dx < tx_n and 0 <= ty + dy < ty_n]


def simulate(tx_n, ty_n, nsteps, nblocks, rng, late_blocks=0, wait_set=neighbours, lag=0):
    """Run the protocol; returns (finished without deadlock, steps completed per tile).
    Raises AssertionError when a read sees a wrong version or a write hits a tile that is
    being read.  Step k reads buffer k % 2 and writes the other one; the input is buffer 0.
    lag > 0 plants an impossible wait (for steps not yet taken)."""
    ntiles = tx_n * ty_n
    njobs = ntiles * nsteps
    flags = np.zeros(ntiles, dtype=int)
    version = np.full((2, ntiles), -2, dtype=int)   # step whose output a buffer holds
    version[0, :] = -1                              # the input
    readers = np.zeros((2, ntiles), dtype=int)      # running jobs reading a tile
    events, waiting = [], {}
    seq = nxt = 0
    for b in range(nblocks):
        t0 = rng.uniform(5.0, 50.0) if b >= nblocks - late_blocks else 0.0
        heapq.heappush(events, (t0, seq, "grab", b, -1))
        seq += 1
    now = 0.0

    def ready(job):
        k, t = divmod(job, ntiles)
        return k == 0 or all(flags[n] >= k + lag for n in wait_set(t, tx_n, ty_n))

    def start(b, job):
        nonlocal seq
        k, t = divmod(job, ntiles)
        rb, wb = k % 2, 1 - k % 2
        for n in neighbours(t, tx_n, ty_n):        # the halo always spans the 3 x 3 tiles
            assert version[rb, n] == k - 1, "a read saw the wrong version"
            readers[rb, n] += 1
        assert readers[wb, t] == 0, "a tile was overwritten while being read"
        heapq.heappush(events, (now + rng.exponential(1.0) + 0.2, seq, "done", b, job))
        seq += 1

    while events:
        now, _, kind, b, job = heapq.heappop(events)
        if kind == "grab":
            if nxt < njobs:
                job, nxt = nxt, nxt + 1
                if ready(job):
                    start(b, job)
                else:
                    waiting[b] = job
            continue
        k, t = divmod(job, ntiles)
        rb, wb = k % 2, 1 - k % 2
        for n in neighbours(t, tx_n, ty_n):
            readers[rb, n] -= 1
        version[wb, t] = k
        flags[t] = k + 1
        heapq.heappush(events, (now, seq, "grab", b, -1))
        seq += 1
        for wb_, wjob in list(waiting.items()):
            if ready(wjob):
                del waiting[wb_]
                start(wb_, wjob)
    return not waiting and nxt == njobs, flags


@pytest.mark.parametrize("tx_n,ty_n,nsteps,nblocks,late", [
    (4, 6, 7, 5, 0),
    (5, 3, 9, 16, 0),
    (7, 9, 5, 13, 6),
    (1, 1, 12, 3, 1),
    (3, 40, 6, 20, 10),
    (16, 16, 4, 60, 30),
])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_protocol_never_deadlocks_and_never_overwrites_a_tile_being_read(
        tx_n, ty_n, nsteps, nblocks, late, seed):
    ok, flags = simulate(tx_n, ty_n, nsteps, nblocks, np.random.default_rng(seed),
                         late_blocks=late)
    assert ok
    assert np.all(flags == nsteps)


def test_a_narrower_wait_is_caught():
    def self_only(t, tx_n, ty_n):
        return [t]
    caught = 0
    for seed in range(5):
        try:
            simulate(6, 6, 8, 12, np.random.default_rng(seed), wait_set=self_only)
        except AssertionError:
            caught += 1
    assert caught == 5


def test_the_model_detects_a_deadlock():
    # a wait for the job's own completion can never be met: the model must report it
    # (blocks left waiting with no event pending), not loop
    ok, flags = simulate(3, 3, 4, 4, np.random.default_rng(0), wait_set=neighbours, lag=1)
    assert not ok and np.all(flags <= 1)
