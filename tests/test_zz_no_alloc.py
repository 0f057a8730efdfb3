"""drag_expm_apply_batched_noalloc: the batched update for callers that cannot
allocate device scratch (a host code whose device memory is all owned by its
own pool, or one that must not call cudaMalloc inside a time step because it
synchronises the device). It runs on a fixed scratch array inside the library.

The test calls it through the C ABI twice in a row on different batches. Both
entry points run the same kernels with the same arithmetic on the same inputs,
so each result must equal drag_expm_apply_batched's (the entry point that
takes a caller workspace) bit for bit: stale scratch contents left by the
first call would show up in the second, however small. One call is also
checked against the oracle's batched update at the forward tolerance of the
other tests. This file is collected last; it also runs on its own in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    from paper_2509_25347_gb300 import build
    build.build()
    import paper_2509_25347_gb300 as m
    m.load_library()
    m.get_status()
    return m


def _batch(seed, nblocks, block_cells):
    rng = np.random.default_rng(seed)
    blocks = []
    for b in range(nblocks):
        N = int(rng.choice([1, 3, 4, 8, 12, 16]))
        C = int(rng.integers(0, block_cells + 1))
        dt = 2.0 ** -int(rng.integers(0, 7))
        blocks.append((N, dt, W.mrn(C, N, seed=seed * 7919 + b, stiff_lo=-4.0, stiff_hi=8.0, dt=dt, t_ref=1.0)))
    return W.Batch(blocks)


def _noalloc(dx, desc_dev, nblocks, nmax, rg, rd, ts, v, out):
    import torch
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    rc = dx.load_library().drag_expm_apply_batched_noalloc(
        nblocks, p(desc_dev), rg.numel(), rd.numel(), v.numel(), nmax, p(rg), p(rd), p(ts), p(v), p(out),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc


def test_noalloc_matches_workspace_entry_point_two_calls(dx):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for call, (seed, nblocks, bc) in enumerate(((11, 200, 300), (12, 97, 515))):
        desc, rg, rd, ts, v = _batch(seed, nblocks, bc).pack()
        assert rg.size <= 262144
        nmax = int(desc["nspecies"].max())
        # both outputs start from the same sentinel, so unwritten entries compare too
        ref = dx.apply_batched(desc, t(rg), t(rd), t(ts), t(v), t(np.full_like(v, 7.0))).cpu().numpy()
        out = t(np.full_like(v, 7.0))
        desc_dev = torch.from_numpy(desc.view(np.uint8).copy()).cuda()
        rc = _noalloc(dx, desc_dev, len(desc), nmax, t(rg), t(rd), t(ts), t(v), out)
        assert rc == 0
        got = out.cpu().numpy()
        assert np.array_equal(got, ref, equal_nan=True), (call, int(np.sum(got != ref)))
        assert np.all(np.isfinite(got))
        if call == 0:
            orc, st = oracle.drag_apply_batched(desc, rg, rd, ts, v)
            assert st == 0
            for b in range(len(desc)):
                N, C, vo = int(desc[b]["nspecies"]), int(desc[b]["ncells"]), int(desc[b]["vel_offset"])
                if C == 0:
                    continue
                sl = slice(vo, vo + 3 * (N + 1) * C)
                sc = np.abs(v[sl].reshape(3, N + 1, C)).max(axis=1, keepdims=True)
                err = np.max(np.abs(got[sl] - orc[sl]).reshape(3, N + 1, C) / sc)
                assert err <= TOL, (b, N, err)
    assert dx.get_status() == 0


def test_noalloc_rejects_batches_beyond_its_scratch(dx):
    import torch
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    blocks = torch.zeros(40, dtype=torch.uint8, device="cuda")
    lib = dx.load_library()
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.drag_expm_apply_batched_noalloc(16385, p(blocks), 8, 8, 8, 4, p(z), p(z), p(z), p(z), p(z), s) == -7
    assert lib.drag_expm_apply_batched_noalloc(1, p(blocks), 262145, 8, 8, 4, p(z), p(z), p(z), p(z), p(z), s) == -7
    assert b"fixed scratch" in lib.drag_expm_strerror(-7)
