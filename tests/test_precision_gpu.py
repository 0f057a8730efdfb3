"""GPU parity of the lower accuracy targets (Eq. B8 with u = 2^-24, 2^-11).

drag_expm_apply_target runs Algorithm 2 on the theta table of u = 2^-ubits
and then the same FP64 arithmetic as drag_expm_apply. Against the oracle run
with the same target (same (k*, s*), FP64 arithmetic): (k*, s*) bit-exact and
|v_gpu - v_oracle| <= 1e-13 max_f |v_in[d, f]|, the forward tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2509_25347_gb300 import workloads as W
from tests.test_forward_gpu import assert_parity, dev

pytestmark = pytest.mark.gpu
TARGETS = (24, 11)


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    from paper_2509_25347_gb300 import build
    build.build()
    import paper_2509_25347_gb300 as m
    m.load_library()
    m.get_status()
    return m


def nonstiff(C, N, seed):
    rng = np.random.default_rng(seed)
    return W.Cells(np.ones(C), rng.uniform(0.1, 1.0, (N, C)), 10.0 ** rng.uniform(-0.7, 0.7, (N, C)),
                   rng.standard_normal((3, N + 1, C)), 1.0)


CASES = [("dustybox_n1_32k", 2001), ("mrn_n4_128cube", 1025), ("mrn_n8_128cube_adjoint", 513),
         ("mrn_n16_128cube", 257)]


@pytest.mark.parametrize("ubits", TARGETS)
@pytest.mark.parametrize("name,C", CASES)
def test_target_select_and_apply_parity(dx, ubits, name, C):
    cells = W.workload(name, ncells=C)
    rg, rd, ts, v = dev(cells)
    k, s = dx.select(rg, rd, ts, cells.dt, ubits=ubits)
    ref, ko, so, _ = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, return_ks=True,
                                       u=2.0 ** -ubits)
    assert np.array_equal(k.cpu().numpy(), ko)
    assert np.array_equal(s.cpu().numpy(), so)
    out = dx.apply(rg, rd, ts, cells.dt, v, ubits=ubits).cpu().numpy()
    assert_parity(out, ref, cells.v)
    assert dx.get_status() == 0


@pytest.mark.parametrize("ubits", TARGETS)
@pytest.mark.parametrize("N", [1, 2, 3, 5, 6, 7, 9, 10, 12, 13, 16, 17, 24, 31])
def test_target_every_family(dx, ubits, N):
    """Lane-per-cell (registers, shared memory) and warp-per-cell sizes,
    stiff and non-stiff cells, ragged counts."""
    for cells in (W.mrn(67 + N, N, seed=300 + N, stiff_lo=-4.0, stiff_hi=8.0), nonstiff(45 + N, N, 400 + N)):
        rg, rd, ts, v = dev(cells)
        out = dx.apply(rg, rd, ts, cells.dt, v, ubits=ubits).cpu().numpy()
        ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -ubits)
        assert_parity(out, ref, cells.v)


def test_target_53_is_the_default(dx):
    cells = W.workload("mrn_n16_128cube", ncells=129)
    rg, rd, ts, v = dev(cells)
    a = dx.apply(rg, rd, ts, cells.dt, v).cpu().numpy()
    b = dx.apply(rg, rd, ts, cells.dt, v, ubits=53).cpu().numpy()
    assert np.array_equal(a, b)


def test_target_in_place_and_dt_zero(dx):
    cells = W.workload("mrn_n8_128cube_adjoint", ncells=200)
    rg, rd, ts, v = dev(cells)
    ref = oracle.drag_apply(cells.rho_g, cells.rho_d, cells.t_s, cells.dt, cells.v, u=2.0 ** -24)
    dx.apply(rg, rd, ts, cells.dt, v, v, ubits=24)
    assert_parity(v.cpu().numpy(), ref, cells.v)
    _, _, _, v0 = dev(cells)
    out = dx.apply(rg, rd, ts, 0.0, v0, ubits=11).cpu().numpy()
    assert np.array_equal(out, cells.v)


def test_target_invalid_ubits(dx):
    cells = W.workload("mrn_n4_128cube", ncells=8)
    rg, rd, ts, v = dev(cells)
    with pytest.raises(dx.DragExpmError):
        dx.apply(rg, rd, ts, cells.dt, v, ubits=16)


@pytest.mark.parametrize("ubits", TARGETS)
def test_target_full_size_sampled(dx, ubits):
    """Headline launch shape (2,097,152 N = 16 cells): 400 sampled cells
    against the oracle one by one, and the total cost k* + s* below the
    u = 2^-53 run."""
    import torch
    cells = W.workload("mrn_n16_128cube")
    rg, rd, ts, v = dev(cells)
    out = dx.apply(rg, rd, ts, cells.dt, v, ubits=ubits)
    k1, s1 = dx.select(rg, rd, ts, cells.dt, ubits=ubits)
    k0, s0 = dx.select(rg, rd, ts, cells.dt)
    cost1 = int(k1.to(torch.int64).sum() + s1.to(torch.int64).sum())
    cost0 = int(k0.to(torch.int64).sum() + s0.to(torch.int64).sum())
    assert cost1 < cost0
    idx = np.random.default_rng(ubits).choice(cells.ncells, 400, replace=False)
    sub = cells.subset(idx)
    ref = oracle.drag_apply(sub.rho_g, sub.rho_d, sub.t_s, sub.dt, sub.v, u=2.0 ** -ubits)
    got = out[:, :, torch.from_numpy(idx).cuda()].cpu().numpy()
    assert_parity(got, ref, sub.v)
    assert dx.get_status() == 0
