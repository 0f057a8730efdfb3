"""Round schedules of the warp-per-cell squaring chain (paper_2509_25347_gb300/sched.py).

The kernels trust these tables for correctness: every dependency between the
off-diagonal products and the row-sum restorations of consecutive squarings
must hold, every task must appear exactly once, and no round may exceed 32
lanes. Checked here for every matrix size the warp-per-cell kernels accept.
"""
import os

import pytest

from paper_2509_25347_gb300 import sched


@pytest.mark.parametrize("restore_first", [False, True])
@pytest.mark.parametrize("n", list(range(2, 33)))
def test_schedule_dependencies(n, restore_first):
    rounds, end = sched.schedule(n, restore_first=restore_first)
    sched.check(n, rounds)
    assert len(end) == sched.H + 1
    assert all(end[h] <= end[h + 1] for h in range(sched.H))
    assert end[sched.H] == len(rounds)
    ntasks = sum(len(r) for r in rounds)
    assert ntasks == n + sched.H * (n * (n - 1) // 2 + n)
    for h in range(sched.H + 1):           # rounds past end[h] hold no task with t <= h
        for rnd in rounds[end[h]:]:
            assert all(t > h for (t, _, _) in rnd)


def test_pipelining_saves_rounds():
    """Phase by phase a squaring costs ceil(n(n-1)/2/32) + ceil(n/32) rounds;
    the pipelined schedule the library uses needs fewer on average, at n = 17
    within 1 % of the lane count's bound of (n(n-1)/2 + n) / 32."""
    for n, expect in ((13, 3.5), (17, 4.8), (24, 9.6)):
        rounds, end = sched.best_schedule(n)
        sched.check(n, rounds)
        per = (end[32] - end[16]) / 16
        phased = -(-(n * (n - 1) // 2) // 32) + -(-n // 32)
        assert per <= expect < phased
    rounds, end = sched.best_schedule(17)
    assert len(rounds) <= 1.01 * (17 + 32 * (17 * 16 // 2 + 17)) / 32


def test_best_schedule_is_the_shorter_order():
    """Per n the library takes the order with fewer rounds summed over every
    chunk length, never more than the products-first order."""
    for n in range(2, 33):
        a = sched.schedule(n)[1]
        b = sched.schedule(n, restore_first=True)[1]
        best = sched.best_schedule(n)[1]
        assert sum(best) == min(sum(a), sum(b)) and sum(best) <= sum(a)


def test_packing_and_header(tmp_path):
    assert sched.pack(32, 5, 17) == 5 | (17 << 5) | (32 << 10)      # (t, i, j)
    path = os.path.join(tmp_path, "t.inc")
    sched.write_header(str(path))
    text = open(path).read()
    assert "dx_sched_task" in text and "dx_sched_end" in text and "dx_sched_off" in text
