"""Host-side dispatch of the lane-per-cell sizes (no GPU): from which cell count
the forward and the adjoint bin the whole input by (k*, s*) before running it,
as the library's launch-count queries report it."""
import pytest

import paper_2509_25347_gb300 as dx
from paper_2509_25347_gb300 import build as dxbuild
from tests.dispatch_sizes import INT32_MAX, binned_threshold


@pytest.fixture(scope="module")
def lib():
    dxbuild.build()
    return dx.load_library()


def test_binned_thresholds_per_size(lib):
    fwd = {N: binned_threshold(dx, N) for N in range(1, 12)}
    bwd = {N: binned_threshold(dx, N, adjoint=True) for N in range(1, 12)}
    # N = 1 runs the forward in the velocity form, a few dozen FP64 operations a
    # cell: one launch at every size (binning measured slower up to 2,097,152 cells)
    assert fwd[1] is None
    for C in (1, 10**5, 10**6, INT32_MAX, INT32_MAX + 1):
        assert dx.apply_launches(C, 1) == 1
    # the lane-per-cell adjoint stops at N = 8 (n = 9); the binned forward reaches N = 11 (n = 12)
    for N in (9, 10, 11):
        assert bwd[N] is None and fwd[N] is not None
    for N in range(1, 12):
        for q, thr in ((dx.apply_launches, fwd[N]), (dx.backward_launches, bwd[N])):
            if (q is dx.apply_launches and N == 1) or (q is dx.backward_launches and N >= 9):
                continue
            assert thr is not None and thr > 1
            # one launch below the threshold, six from it on, up to the int32 cell limit
            for C in (1, thr // 2, thr - 1):
                assert q(C, N) == 1
            for C in (thr, thr + 1, 2 * thr, INT32_MAX):
                assert q(C, N) == 6
            assert q(INT32_MAX + 1, N) == 1
        # the adjoint's squarings cost ~5x the forward's: binning pays no later there
        assert N == 1 or N >= 9 or bwd[N] <= fwd[N]
    # larger matrices vary more in per-warp work with (k*, s*): binning pays earlier
    assert all(fwd[N + 1] <= fwd[N] for N in range(2, 11))
    assert all(bwd[N + 1] <= bwd[N] for N in range(1, 8))
    # warp-per-cell sizes never bin
    for N in (12, 16, 31):
        assert binned_threshold(dx, N) is None and binned_threshold(dx, N, adjoint=True) is None
        assert dx.apply_launches(10**6, N) == 1 and dx.backward_launches(10**6, N) == 1


def test_host_pipeline_chunk_follows_binning(lib):
    """drag_expm_apply_host's default chunk is 262,144 cells where the forward
    bins that many cells, else 131,072: the two device slabs of a chunk hold
    rho_g, rho_d, t_s and v (1 + 2N + 3(N+1) doubles per cell)."""
    for N in (1, 2, 4, 8, 9, 16):
        chunk = 262144 if dx.apply_launches(262144, N) == 6 else 131072
        want = 2 * 8 * chunk * (1 + 2 * N + 3 * (N + 1))
        assert lib.drag_expm_host_workspace_bytes(N, 0) == want
    assert dx.apply_launches(262144, 1) == 1 and dx.apply_launches(262144, 2) == 6
