"""Seeded random cases across the dispatch boundaries of drag_expm_apply and the
adjoint tape: sizes below, at and above the forward's and the adjoint's binning
sizes (per N, as the library reports them),
species counts on every kernel family (lane per cell in registers, hybrid, warp
per cell), ragged cell counts, random stiffness ranges and time steps. The
forward is checked against the oracle on sampled cells at 1e-13 of the velocity
scale; the taped adjoint against the recomputing adjoint at the adjoint
tolerances of tests/test_backward_gpu.py. The lower accuracy targets and the
host-array pipeline are run above the threshold too."""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W
from tests.dispatch_sizes import binned_threshold
from tests.test_backward_gpu import assert_adjoint_parity

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


def t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def cases():
    rng = np.random.default_rng(2024)
    out = []
    for k in range(16):
        N = int(rng.choice([1, 3, 5, 6, 7, 8, 11, 12, 16, 20]))
        C = str(rng.choice(["1", "31", "4097", "below", "at", "above", "adj_below", "adj_at", "300007"]))
        lo = float(rng.uniform(-6.0, 0.0))
        hi = float(rng.uniform(lo + 4.5, 9.0))
        dt = float(2.0 ** -int(rng.integers(0, 5)))
        out.append((k, N, C, lo, hi, dt))
    return out


def resolve_size(dx, N, label):
    """A size label of cases() as a cell count: a number, or one relative to
    the forward's ("below", "at", "above") or the adjoint's ("adj_below",
    "adj_at") binning size; 262,144 stands in for sizes that never bin."""
    if label.isdigit():
        return int(label)
    adj = label.startswith("adj_")
    thr = binned_threshold(dx, N, adjoint=adj) or 262144
    return thr + {"below": -1, "at": 0, "above": 1}[label.split("_")[-1]]


@pytest.mark.parametrize("k,N,C,lo,hi,dt", cases())
def test_dispatch_fuzz(dx, k, N, C, lo, hi, dt):
    import torch
    C = resolve_size(dx, N, C)
    cells = W.mrn(C, N, seed=5000 + k, stiff_lo=lo, stiff_hi=hi, dt=dt, t_ref=1.0)
    rg, rd, ts, v = t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v)
    out = dx.apply(rg, rd, ts, dt, v)
    idx = np.unique(np.concatenate([np.random.default_rng(k).integers(0, C, 96), [0, C - 1]]))
    sub = cells.subset(idx)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v)
    got = out[:, :, torch.from_numpy(idx).cuda()].cpu().numpy()
    sc = np.abs(sub.v).max(axis=1, keepdims=True)
    assert np.max(np.abs(got - ref) / sc) <= TOL
    # taped forward and adjoint against the plain ones
    out2, tape = dx.apply_taped(rg, rd, ts, dt, v)
    assert torch.equal(out, out2)
    g_np = np.random.default_rng(k + 100).standard_normal(cells.v.shape)
    g = t(g_np)
    taped = [x.cpu().numpy()[..., idx] for x in dx.backward(rg, rd, ts, dt, v, g, tape=tape)]
    plain = [x.cpu().numpy()[..., idx] for x in dx.backward(rg, rd, ts, dt, v, g)]
    assert_adjoint_parity(sub, g_np[:, :, idx], taped, plain)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N,ubits", [(4, 24), (8, 11), (16, 24)])
def test_targets_above_binning_threshold(dx, N, ubits):
    """The lower accuracy targets on 300,001 cells (the binned path carries the
    target's theta table for N <= 8): sampled cells against the oracle at the
    same target, and (k*, s*) bit-exact."""
    import torch
    C = 300001
    cells = W.mrn(C, N, seed=80 + N, stiff_lo=-4.0, stiff_hi=8.0)
    rg, rd, ts, v = t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v)
    out = dx.apply(rg, rd, ts, cells.dt, v, ubits=ubits)
    idx = np.unique(np.concatenate([np.random.default_rng(N).integers(0, C, 96), [0, C - 1]]))
    sub = cells.subset(idx)
    u = 2.0 ** -ubits
    ref, k, s, st = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, return_ks=True, u=u)
    got = out[:, :, torch.from_numpy(idx).cuda()].cpu().numpy()
    sc = np.abs(sub.v).max(axis=1, keepdims=True)
    assert st == 0 and np.max(np.abs(got - ref) / sc) <= TOL
    kg, sg = dx.select(rg, rd, ts, cells.dt, ubits=ubits)
    assert np.array_equal(kg.cpu().numpy()[idx], k) and np.array_equal(sg.cpu().numpy()[idx], s)
    assert dx.get_status() == 0


@pytest.mark.parametrize("N,C,chunk", [(4, 600011, 0), (8, 524300, 0), (16, 300001, 65536), (3, 270000, 100000)])
def test_host_pipeline_large(dx, N, C, chunk):
    """drag_expm_apply_host over several chunks, binned ones included (default
    chunk 262,144 for N = 2..8): bit-identical to drag_expm_apply on the device."""
    import torch
    cells = W.mrn(C, N, seed=90 + N, stiff_lo=-4.0, stiff_hi=8.0)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    out = dx.apply_host(pin(cells.rho_g), pin(cells.rho_d), pin(cells.t_s), cells.dt, pin(cells.v),
                        chunk_cells=chunk)
    torch.cuda.synchronize()
    dev_out = dx.apply(t(cells.rho_g), t(cells.rho_d), t(cells.t_s), cells.dt, t(cells.v)).cpu()
    if chunk == 0 and N + 1 <= 9:
        assert torch.equal(out, dev_out)     # same binned kernel chunk by chunk
    else:
        sc = np.abs(cells.v).max(axis=1, keepdims=True)
        assert np.max(np.abs(out.numpy() - dev_out.numpy()) / sc) <= TOL
    assert dx.get_status() == 0
