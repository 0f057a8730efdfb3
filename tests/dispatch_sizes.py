"""Sizes at which drag_expm_apply / drag_expm_backward switch from one
tile-sorted launch to the binned pipeline (6 launches), read from the
library's own launch-count queries (host-only, no GPU needed)."""

INT32_MAX = 2**31 - 1


def binned_threshold(dx, N, adjoint=False):
    """Smallest cell count that the forward (adjoint) runs binned for N
    species, or None if no size up to 2^31 - 1 is binned. The launch count
    is 1 below it and 6 from it on (checked by tests/test_dispatch_cpu.py)."""
    q = dx.backward_launches if adjoint else dx.apply_launches
    if q(INT32_MAX, N) != 6:
        return None
    lo, hi = 1, INT32_MAX
    if q(lo, N) == 6:
        return lo
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if q(mid, N) == 6:
            hi = mid
        else:
            lo = mid
    return hi
