"""Round schedules for the warp-per-cell squaring chain (build-time generator).

One squaring of the symmetric form E <- E^2 consists of n(n-1)/2 off-diagonal
dot products ("O" tasks, n FMAs each) and n row-sum restorations ("R" tasks,
E_ii = 1 - sigma_i^-1 sum_{k != i} E_ik sigma_k: n-1 FMAs + 1). A warp runs 32
tasks per round, one per lane, so a squaring done phase by phase needs
ceil(n(n-1)/2 / 32) + ceil(n / 32) rounds and leaves lanes idle in its last
rounds. Dependencies are finer than phases:

* R(t, i) needs every O(t, i, .) of squaring t;
* O(t+1, i, j) needs rows i and j of E_t complete, i.e. R(t, i) and R(t, j)
  (which also ends every read of rows i and j of E_{t-1}, the buffer it
  overwrites).

A greedy list schedule that fills each round with the ready tasks of the
oldest squaring first overlaps the restorations of squaring t with the first
products of squaring t+1; for n = 17 it needs 5.0 rounds per squaring instead
of 6. Within a squaring it can take the ready restorations before or after
the ready products; taking them first lets the next squaring start sooner for
some sizes (n = 17: 155 rounds for 32 squarings instead of 162, against an
ideal of 153.5) and costs a round for others, so each n gets the order with
fewer rounds summed over the chunk lengths h = 0..32. Schedules cover a
chunk: the restoration of the starting matrix (t = 0) and up to H = 32
squarings (t = 1..32). A task is packed in 16 bits:
i | j << 5 | t << 10 (i == j for R tasks), 0xFFFF for an idle lane. END[n][h]
is the number of rounds that completes every task with t <= h.

``write_header`` emits the tables as C++ source for the CUDA library.
"""
from __future__ import annotations

H = 32
LANES = 32
NMAX = 32
IDLE = 0xFFFF


def schedule(n: int, horizon: int = H, lanes: int = LANES, restore_first: bool = False):
    """Returns (rounds, end): rounds is a list of lists of (t, i, j); end[h] for h = 0..horizon.
    restore_first: within a squaring, the ready restorations are taken before the ready products."""
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    # per squaring t: pending O tasks (row-major order) and pending R rows
    pend_o = {t: list(pairs) for t in range(1, horizon + 1)}
    pend_r = {t: list(range(n)) for t in range(0, horizon + 1)}
    left = {t: [n - 1] * n for t in range(1, horizon + 1)}     # O tasks of squaring t left on row r
    rdone = {t: [False] * n for t in range(0, horizon + 1)}
    rounds = []
    lo = 0                                                        # oldest squaring with pending work
    while lo <= horizon:
        pick = []
        for t in range(lo, min(lo + 3, horizon + 1)):
            ready_r = [i for i in pend_r[t] if t == 0 or left[t][i] == 0]
            ready_o = [(i, j) for (i, j) in pend_o.get(t, []) if rdone[t - 1][i] and rdone[t - 1][j]]
            tasks = [(t, i, i) for i in ready_r] + [(t, i, j) for (i, j) in ready_o] if restore_first else \
                [(t, i, j) for (i, j) in ready_o] + [(t, i, i) for i in ready_r]
            pick.extend(tasks[:lanes - len(pick)])
            if len(pick) == lanes:
                break
        if not pick:
            raise RuntimeError(f"schedule deadlock at n={n}")
        # commit the round (a task only depends on earlier rounds)
        for (t, i, j) in pick:
            if i == j:
                pend_r[t].remove(i)
                rdone[t][i] = True
            else:
                pend_o[t].remove((i, j))
                left[t][i] -= 1
                left[t][j] -= 1
        rounds.append(pick)
        while lo <= horizon and not pend_r[lo] and (lo == 0 or not pend_o[lo]):
            lo += 1
    end = []
    for h in range(horizon + 1):
        last = max(r for r, rnd in enumerate(rounds) if any(t <= h for (t, _, _) in rnd))
        end.append(last + 1)
    return rounds, end


def best_schedule(n: int, horizon: int = H, lanes: int = LANES):
    """The schedule of the two task orders with fewer rounds summed over the
    chunk lengths h = 0..horizon (ties: products first). Returns (rounds, end)."""
    a = schedule(n, horizon, lanes, restore_first=False)
    b = schedule(n, horizon, lanes, restore_first=True)
    return b if sum(b[1]) < sum(a[1]) else a


def check(n: int, rounds, horizon: int = H) -> None:
    """Re-verify every dependency of a schedule (used by the tests)."""
    when = {}
    for r, rnd in enumerate(rounds):
        assert len(rnd) <= LANES
        for task in rnd:
            assert task not in when
            when[task] = r
    for t in range(0, horizon + 1):
        for i in range(n):
            assert (t, i, i) in when
            if t >= 1:
                for k in range(n):
                    if k != i:
                        a, b = min(i, k), max(i, k)
                        assert when[(t, a, b)] < when[(t, i, i)]
        if t >= 1:
            for i in range(n):
                for j in range(i + 1, n):
                    assert when[(t - 1, i, i)] < when[(t, i, j)]
                    assert when[(t - 1, j, j)] < when[(t, i, j)]


def pack(t: int, i: int, j: int) -> int:
    return i | (j << 5) | (t << 10)


def write_header(path: str) -> None:
    codes, offs, ends = [], [0] * (NMAX + 2), []
    total = 0
    for n in range(0, NMAX + 1):
        offs[n] = total
        if n < 2:
            ends.append([0] * (H + 1))
            continue
        rounds, end = best_schedule(n)
        for rnd in rounds:
            row = [pack(*tk) for tk in rnd] + [IDLE] * (LANES - len(rnd))
            codes.extend(row)
        total += len(rounds)
        ends.append(end)
    offs[NMAX + 1] = total
    with open(path, "w") as f:
        f.write("// Generated by paper_2509_25347_gb300/sched.py (build step); do not edit.\n")
        f.write(f"#define DX_SCHED_H {H}\n#define DX_SCHED_ROUNDS {total}\n")
        f.write("__device__ const int dx_sched_off[%d] = {%s};\n" % (NMAX + 2, ",".join(map(str, offs))))
        flat = [e for row in ends for e in row]
        f.write("__device__ const unsigned short dx_sched_end[%d] = {%s};\n" % (len(flat), ",".join(map(str, flat))))
        f.write("__device__ const unsigned short dx_sched_task[%d] = {\n" % (len(codes)))
        for k in range(0, len(codes), 32):
            f.write(",".join(str(c) for c in codes[k:k + 32]) + ",\n")
        f.write("};\n")


if __name__ == "__main__":
    import sys
    write_header(sys.argv[1])
