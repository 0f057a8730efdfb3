"""drag_expm_apply_host: the forward update on host arrays through the
chunked two-stream pipeline must give exactly what drag_expm_apply gives on
device copies of the same arrays (same kernels, same per-cell arithmetic;
only the cells' grouping into launches differs, and no cell depends on
another), for ragged chunkings, pinned and pageable memory, in place."""
import numpy as np
import pytest

from paper_2509_25347_gb300 import workloads as W
from tests.test_forward_gpu import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    from paper_2509_25347_gb300 import build
    build.build()
    import paper_2509_25347_gb300 as m
    m.load_library()
    m.get_status()
    return m


def host(cells, pin):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    out = [t(cells.rho_g), t(cells.rho_d), t(cells.t_s), t(cells.v)]
    return [x.pin_memory() for x in out] if pin else out


@pytest.mark.parametrize("name,C,chunk", [("mrn_n16_128cube", 30001, 4096), ("mrn_n16_128cube", 2000, 0),
                                          ("mrn_n4_128cube", 100003, 16384), ("dustybox_n1_32k", 32768, 5000),
                                          ("mrn_n8_128cube_adjoint", 9999, 9999)])
@pytest.mark.parametrize("pin", [True, False])
def test_host_pipeline_matches_device(dx, name, C, chunk, pin):
    import torch
    cells = W.workload(name, ncells=C)
    rg, rd, ts, v = dev(cells)
    ref = dx.apply(rg, rd, ts, cells.dt, v).cpu().numpy()
    hrg, hrd, hts, hv = host(cells, pin)
    out = dx.apply_host(hrg, hrd, hts, cells.dt, hv, chunk_cells=chunk)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(out.numpy(), ref)
    # in place on the host
    dx.apply_host(hrg, hrd, hts, cells.dt, hv, hv, chunk_cells=chunk)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(hv.numpy(), ref)
    assert dx.get_status() == 0


def test_host_pipeline_errors(dx):
    import torch
    cells = W.workload("mrn_n4_128cube", ncells=1000)
    hrg, hrd, hts, hv = host(cells, True)
    import ctypes
    lib = dx.load_library()
    ptrs = [ctypes.c_void_p(x.data_ptr()) for x in (hrg, hrd, hts)]
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    rc = lib.drag_expm_apply_host(1000, 4, *ptrs, cells.dt, ctypes.c_void_p(hv.data_ptr()),
                                  ctypes.c_void_p(hv.data_ptr()), 512, ctypes.c_void_p(small.data_ptr()), 1024,
                                  ctypes.c_void_p(0))
    assert rc == -5                                         # workspace too small
    ws = torch.empty(dx.host_workspace_bytes(4, 512) + 256, dtype=torch.uint8, device="cuda")
    rc = lib.drag_expm_apply_host(1000, 4, ctypes.c_void_p(hrg.data_ptr()), ctypes.c_void_p(hrd.data_ptr()),
                                  ctypes.c_void_p(hts.data_ptr()), cells.dt, ctypes.c_void_p(hv.data_ptr()),
                                  ctypes.c_void_p(hv.data_ptr()), 512, ctypes.c_void_p(ws.data_ptr() + 8),
                                  dx.host_workspace_bytes(4, 512), ctypes.c_void_p(0))
    assert rc == -3                                         # misaligned workspace
    assert dx.host_workspace_bytes(0, 512) == 0 and dx.host_workspace_bytes(4, -1) == 0


def test_binding_rejects_misplaced_scratch(dx):
    """The binding hands the library device pointers only: a host tensor or an
    undersized tensor as the pipeline's workspace is refused before any call."""
    import torch
    cells = W.workload("mrn_n4_128cube", ncells=1000)
    hrg, hrd, hts, hv = host(cells, True)
    need = dx.host_workspace_bytes(4, 512)
    with pytest.raises(dx.DragExpmError, match="CUDA tensor"):
        dx.apply_host(hrg, hrd, hts, cells.dt, hv, chunk_cells=512, workspace=torch.empty(need, dtype=torch.uint8))
    with pytest.raises(dx.DragExpmError, match="needs"):
        dx.apply_host(hrg, hrd, hts, cells.dt, hv, chunk_cells=512,
                      workspace=torch.empty(need - 1, dtype=torch.uint8, device="cuda"))
    # a float64 workspace counts in bytes
    out = dx.apply_host(hrg, hrd, hts, cells.dt, hv, chunk_cells=512,
                        workspace=torch.empty((need + 7) // 8, dtype=torch.float64, device="cuda"))
    torch.cuda.current_stream().synchronize()
    rg, rd, ts, v = dev(cells)
    assert np.array_equal(out.numpy(), dx.apply(rg, rd, ts, cells.dt, v).cpu().numpy())
    assert dx.get_status() == 0
