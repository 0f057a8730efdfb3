"""GB300-native exponential drag solver for a gas plus N dust species (FP64, sm_103a).

Thin binding over the C ABI of ``libdragexpm.so`` (declared in
``include/drag_expm.h``): argument checks and marshalling only. Every step of
the drag update runs in the library's CUDA kernels; there is no CPU path. If
the library is missing or fails to load, every call raises.

Tensors are torch float64 CUDA tensors in the library's SoA layout:
``rho_g (C,)``, ``rho_d (N, C)``, ``t_s (N, C)``, ``v (3, N+1, C)``.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "load_library", "apply", "apply_heat", "backward", "rk1_apply", "apply_batched", "batched_workspace_bytes",
    "select", "get_status", "theta", "DragExpm", "DragExpmError", "apply_opts", "pade_theta", "apply_host",
    "host_workspace_bytes", "apply_launches", "backward_launches", "apply_taped", "Tape", "tape_bytes", "tape_levels", "tape_levels_needed",
    "DragExpmTaped", "probe_fp64_rate", "probe_square", "NMAX", "STATUS_BAD_CELL", "STATUS_BAD_BLOCK", "STATUS_QUEUE_GUARD"
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdragexpm.so")
NMAX = 31
STATUS_BAD_CELL = 0x1
STATUS_BAD_BLOCK = 0x2
STATUS_QUEUE_GUARD = 0x4

_lib = None


class DragExpmError(RuntimeError):
    pass


def load_library(path: str | None = None):
    """Load libdragexpm.so (built by ``paper_2509_25347_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise DragExpmError(f"{p} not found: build it with `python -m paper_2509_25347_gb300.build` "
                            "(the drag update has no CPU fallback)")
    lib = ctypes.CDLL(p)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.drag_expm_apply.restype = ctypes.c_int
    lib.drag_expm_apply.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, vp]
    lib.drag_expm_backward.restype = ctypes.c_int
    lib.drag_expm_backward.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, vp, vp, vp, vp, vp]
    lib.drag_expm_batched_workspace_bytes.restype = ctypes.c_size_t
    lib.drag_expm_batched_workspace_bytes.argtypes = [i64, i64]
    lib.drag_expm_apply_batched.restype = ctypes.c_int
    lib.drag_expm_apply_batched.argtypes = [i64, vp, i64, i64, i64, i32, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.drag_expm_apply_batched_noalloc.restype = ctypes.c_int
    lib.drag_expm_apply_batched_noalloc.argtypes = [i64, vp, i64, i64, i64, i32, vp, vp, vp, vp, vp, vp]
    lib.drag_expm_set_mode.restype = ctypes.c_int
    lib.drag_expm_set_mode.argtypes = [i32, i32]
    lib.drag_expm_get_mode.restype = ctypes.c_int
    lib.drag_expm_get_mode.argtypes = [i32, ctypes.POINTER(ctypes.c_int32)]
    lib.drag_expm_autotune.restype = ctypes.c_int
    lib.drag_expm_autotune.argtypes = [i32, ctypes.c_char_p, vp]
    lib.drag_expm_apply_heat.restype = ctypes.c_int
    lib.drag_expm_apply_heat.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, vp, vp]
    lib.drag_rk1_apply.restype = ctypes.c_int
    lib.drag_rk1_apply.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, vp]
    lib.drag_expm_select.restype = ctypes.c_int
    lib.drag_expm_select.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, vp]
    lib.drag_expm_get_status.restype = ctypes.c_int
    lib.drag_expm_get_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    lib.drag_expm_theta.restype = ctypes.c_int
    lib.drag_expm_theta.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
    lib.drag_expm_theta_target.restype = ctypes.c_int
    lib.drag_expm_theta_target.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double)]
    lib.drag_expm_apply_target.restype = ctypes.c_int
    lib.drag_expm_apply_target.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, i32, vp]
    lib.drag_expm_host_workspace_bytes.restype = ctypes.c_size_t
    lib.drag_expm_host_workspace_bytes.argtypes = [i32, i64]
    lib.drag_expm_apply_host.restype = ctypes.c_int
    lib.drag_expm_apply_host.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, i64, vp, ctypes.c_size_t, vp]
    lib.drag_expm_apply_opts.restype = ctypes.c_int
    lib.drag_expm_apply_opts.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, ctypes.POINTER(DragOptions), vp, vp, vp]
    lib.drag_expm_pade_theta.restype = ctypes.c_int
    lib.drag_expm_pade_theta.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double)]
    lib.drag_expm_select_target.restype = ctypes.c_int
    lib.drag_expm_select_target.argtypes = [i64, i32, vp, vp, vp, dbl, i32, vp, vp, vp]
    lib.drag_expm_tape_bytes.restype = ctypes.c_size_t
    lib.drag_expm_tape_bytes.argtypes = [i64, i32, i32]
    lib.drag_expm_tape_levels.restype = ctypes.c_int32
    lib.drag_expm_tape_levels.argtypes = [i32]
    lib.drag_expm_apply_taped.restype = ctypes.c_int
    lib.drag_expm_apply_taped.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, i32, vp, ctypes.c_size_t, vp]
    lib.drag_expm_backward_taped.restype = ctypes.c_int
    lib.drag_expm_backward_taped.argtypes = [i64, i32, vp, vp, vp, dbl, vp, vp, vp, vp, vp, vp, i32, vp,
                                             ctypes.c_size_t, vp]
    lib.drag_expm_apply_launches.restype = ctypes.c_int32
    lib.drag_expm_apply_launches.argtypes = [i64, i32]
    lib.drag_expm_backward_launches.restype = ctypes.c_int32
    lib.drag_expm_backward_launches.argtypes = [i64, i32]
    lib.drag_expm_probe_fp64_rate.restype = ctypes.c_int
    lib.drag_expm_probe_fp64_rate.argtypes = [i32, i64, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.drag_expm_probe_square.restype = ctypes.c_int
    lib.drag_expm_probe_square.argtypes = [i32, i32, i64, i32, vp, vp, vp, vp]
    lib.drag_expm_strerror.restype = ctypes.c_char_p
    lib.drag_expm_strerror.argtypes = [ctypes.c_int]
    lib.drag_expm_version.restype = ctypes.c_int
    lib.drag_expm_version.argtypes = []
    if path is None:
        _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        msg = load_library().drag_expm_strerror(rc).decode()
        raise DragExpmError(f"libdragexpm error {rc}: {msg}")


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    if s.device.index != torch.cuda.current_device():
        raise DragExpmError(f"stream is on {s.device}, the library launches on the current device "
                            f"cuda:{torch.cuda.current_device()}")
    return ctypes.c_void_p(s.cuda_stream)


def _on_current_device(name, t):
    """The library launches on the current CUDA device; every buffer it is given must live there."""
    import torch
    if t.device.index != torch.cuda.current_device():
        raise DragExpmError(f"{name} is on {t.device}, not on the current device cuda:{torch.cuda.current_device()}")


def _bytes_cuda(name, t):
    """(pointer, size in bytes) of a contiguous CUDA scratch tensor (workspace, tape) on the current device."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise DragExpmError(f"{name} must be a contiguous CUDA tensor")
    _on_current_device(name, t)
    return ctypes.c_void_p(t.data_ptr()), t.numel() * t.element_size()


def _f64_cuda(name, t, shape):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise DragExpmError(f"{name} must be a float64 CUDA tensor")
    _on_current_device(name, t)
    if tuple(t.shape) != tuple(shape):
        raise DragExpmError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise DragExpmError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _shapes(rho_g, rho_d):
    C = int(rho_g.shape[0])
    N = int(rho_d.shape[0])
    return C, N


UBITS_TARGETS = (53, 24, 11)
METHOD_TAYLOR = 0
METHOD_PADE = 1


class DragOptions(ctypes.Structure):
    """drag_expm_options_t of include/drag_expm.h."""
    _fields_ = [("ubits", ctypes.c_int32), ("method", ctypes.c_int32), ("bound_test", ctypes.c_int32),
                ("arith", ctypes.c_int32)]


def apply(rho_g, rho_d, t_s, dt: float, v_in, v_out=None, stream=None, ubits: int = 53):
    """v_out = exp(dt Omega_v) v_in per cell (forward drag update). Returns v_out.

    ``v_out`` may be ``v_in`` (in place) or None (a new tensor is allocated).
    ``ubits`` selects the accuracy target u = 2^-ubits whose theta table
    Algorithm 2 uses (53, 24 or 11; the arithmetic is FP64 in every case).
    """
    import torch
    C, N = _shapes(rho_g, rho_d)
    if v_out is None:
        v_out = torch.empty_like(v_in)
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    vi = _f64_cuda("v_in", v_in, (3, N + 1, C))
    vo = _f64_cuda("v_out", v_out, (3, N + 1, C))
    if ubits == 53:
        _check(load_library().drag_expm_apply(C, N, *args, float(dt), vi, vo, _stream_handle(stream)))
    else:
        _check(load_library().drag_expm_apply_target(C, N, *args, float(dt), vi, vo, int(ubits),
                                                     _stream_handle(stream)))
    return v_out


def _f64_host(name, t, shape):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.is_cuda:
        raise DragExpmError(f"{name} must be a float64 CPU tensor")
    if tuple(t.shape) != tuple(shape):
        raise DragExpmError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise DragExpmError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def apply_launches(ncells: int, nspecies: int) -> int:
    """Kernels :func:`apply` launches for this size (the binned path launches 6)."""
    return int(load_library().drag_expm_apply_launches(int(ncells), int(nspecies)))


def backward_launches(ncells: int, nspecies: int) -> int:
    """Kernels drag_expm_backward launches for this size (0: bad size)."""
    return int(load_library().drag_expm_backward_launches(int(ncells), int(nspecies)))


def host_workspace_bytes(nspecies: int, chunk_cells: int = 0) -> int:
    return int(load_library().drag_expm_host_workspace_bytes(int(nspecies), int(chunk_cells)))


def apply_host(rho_g, rho_d, t_s, dt: float, v_in, v_out=None, chunk_cells: int = 0, workspace=None, stream=None):
    """Forward update on host (CPU, ideally pinned) float64 tensors, pipelined
    through the GPU in chunks (drag_expm_apply_host). Returns v_out (host)."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    if v_out is None:
        v_out = torch.empty_like(v_in)
    args = [_f64_host("rho_g", rho_g, (C,)), _f64_host("rho_d", rho_d, (N, C)), _f64_host("t_s", t_s, (N, C))]
    vi = _f64_host("v_in", v_in, (3, N + 1, C))
    vo = _f64_host("v_out", v_out, (3, N + 1, C))
    nbytes = host_workspace_bytes(N, chunk_cells)
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    wp, wbytes = _bytes_cuda("workspace", workspace)
    if wbytes < nbytes:
        raise DragExpmError(f"workspace holds {wbytes} bytes, drag_expm_apply_host needs {nbytes}")
    _check(load_library().drag_expm_apply_host(C, N, *args, float(dt), vi, vo, int(chunk_cells), wp, nbytes,
                                               _stream_handle(stream)))
    return v_out


def apply_opts(rho_g, rho_d, t_s, dt: float, v_in, v_out=None, ubits: int = 53, method: str = "taylor",
               bound_test: bool = False, arith: str = "fp64", return_ms: bool = False, stream=None):
    """Forward update with the paper's variants (drag_expm_apply_opts): method
    'taylor' (bound_test adds the second modification) or 'pade'; arith 'fp32'
    is the mixed-precision path (Taylor at ubits 24 or 11). With return_ms,
    also returns the degree evaluated (int8) and s* (int16) per cell."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    if v_out is None:
        v_out = torch.empty_like(v_in)
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    vi = _f64_cuda("v_in", v_in, (3, N + 1, C))
    vo = _f64_cuda("v_out", v_out, (3, N + 1, C))
    opts = DragOptions(int(ubits), {"taylor": METHOD_TAYLOR, "pade": METHOD_PADE}[method], int(bool(bound_test)),
                       {"fp64": 0, "fp32": 1}[arith])
    m = s = None
    mp = sp = ctypes.c_void_p(0)
    if return_ms:
        m = torch.empty(C, dtype=torch.int8, device=v_in.device)
        s = torch.empty(C, dtype=torch.int16, device=v_in.device)
        mp, sp = ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(s.data_ptr())
    _check(load_library().drag_expm_apply_opts(C, N, *args, float(dt), vi, vo, ctypes.byref(opts), mp, sp,
                                               _stream_handle(stream)))
    return (v_out, m, s) if return_ms else v_out


def pade_theta(m: int, ubits: int = 53) -> float:
    """theta_m of the Pade variant as used by the library (m in 3, 5, 7, 9, 13)."""
    out = ctypes.c_double(0.0)
    _check(load_library().drag_expm_pade_theta(int(m), int(ubits), ctypes.byref(out)))
    return out.value


def apply_heat(rho_g, rho_d, t_s, dt: float, v_in, v_out=None, heat_out=None, stream=None):
    """Forward update plus the dissipated kinetic energy per cell. Returns (v_out, heat)."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    if v_out is None:
        v_out = torch.empty_like(v_in)
    if heat_out is None:
        heat_out = torch.empty((C,), dtype=torch.float64, device=v_in.device)
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    vi = _f64_cuda("v_in", v_in, (3, N + 1, C))
    vo = _f64_cuda("v_out", v_out, (3, N + 1, C))
    ho = _f64_cuda("heat_out", heat_out, (C,))
    _check(load_library().drag_expm_apply_heat(C, N, *args, float(dt), vi, vo, ho, _stream_handle(stream)))
    return v_out, heat_out


def rk1_apply(rho_g, rho_d, t_s, dt: float, v_in, v_out=None, stream=None):
    """Analytic implicit RK1 drag step (App. A.2): v_out = (I - dt Omega_v)^-1 v_in."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    if v_out is None:
        v_out = torch.empty_like(v_in)
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    vi = _f64_cuda("v_in", v_in, (3, N + 1, C))
    vo = _f64_cuda("v_out", v_out, (3, N + 1, C))
    _check(load_library().drag_rk1_apply(C, N, *args, float(dt), vi, vo, _stream_handle(stream)))
    return v_out


def _opt_ptr(name, t, shape):
    if t is None:
        return ctypes.c_void_p(0)
    return _f64_cuda(name, t, shape)


class Tape:
    """Adjoint tape written by :func:`apply_taped` (a uint8 CUDA tensor of
    drag_expm_tape_bytes bytes) with the geometry it was written for."""

    __slots__ = ("buf", "ncells", "nspecies", "levels")

    def __init__(self, buf, ncells: int, nspecies: int, levels: int):
        self.buf, self.ncells, self.nspecies, self.levels = buf, int(ncells), int(nspecies), int(levels)

    @property
    def nbytes(self) -> int:
        return int(self.buf.numel() * self.buf.element_size())


def tape_bytes(ncells: int, nspecies: int, levels: int) -> int:
    """Bytes of an adjoint tape (0 for bad arguments)."""
    return int(load_library().drag_expm_tape_bytes(int(ncells), int(nspecies), int(levels)))


def tape_levels(sstar: int) -> int:
    """Tape levels a cell with s* = sstar needs, max(s* - 1, 1)."""
    return int(load_library().drag_expm_tape_levels(int(sstar)))


def tape_levels_needed(rho_g, rho_d, t_s, dt: float, stream=None) -> int:
    """The capacity that records every cell: tape_levels(max s*) over the cells
    (runs drag_expm_select; synchronises with the device)."""
    C, _ = _shapes(rho_g, rho_d)
    if C == 0:
        return 1
    _, s = select(rho_g, rho_d, t_s, dt, stream=stream)
    return max(tape_levels(int(s.max().item())), 1)


def apply_taped(rho_g, rho_d, t_s, dt: float, v_in, v_out=None, levels: int | None = None, tape=None,
                stream=None):
    """:func:`apply` (bit-identical v_out) that also records
    the adjoint tape; returns (v_out, Tape). ``levels`` is the tape capacity per
    cell (default: :func:`tape_levels_needed`); ``tape`` may pass a Tape to reuse
    (its buffer must be large enough)."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    if levels is None:
        levels = tape_levels_needed(rho_g, rho_d, t_s, dt, stream=stream)
    nbytes = tape_bytes(C, N, levels)
    if C > 0 and nbytes == 0:
        raise DragExpmError(f"bad tape geometry: ncells={C} nspecies={N} levels={levels}")
    if tape is None or tape.nbytes < nbytes:
        tape = Tape(torch.empty((max(nbytes, 1),), dtype=torch.uint8, device=rho_g.device), C, N, levels)
    else:
        tape = Tape(tape.buf, C, N, levels)
    tp, tbytes = _bytes_cuda("tape", tape.buf)
    if v_out is None:
        v_out = torch.empty_like(v_in)
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    _check(load_library().drag_expm_apply_taped(C, N, *args, float(dt), _f64_cuda("v_in", v_in, (3, N + 1, C)),
                                                _f64_cuda("v_out", v_out, (3, N + 1, C)), int(levels), tp, tbytes,
                                                _stream_handle(stream)))
    return v_out, tape


def backward(rho_g, rho_d, t_s, dt: float, v_in, grad_v_out, need_v_in=True, need_rho_g=True, need_rho_d=True,
             need_t_s=True, out=None, stream=None, tape=None):
    """Adjoint of :func:`apply`: returns (grad_v_in, grad_rho_g, grad_rho_d, grad_t_s),
    None for the ones not requested. ``out`` may pass preallocated output tensors
    (a 4-tuple, None entries are not computed). ``tape``: a Tape from
    :func:`apply_taped` on these inputs (drag_expm_backward_taped; same gradients,
    less FP64 work)."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    dev = rho_g.device
    if out is not None:
        gvi, grg, grd, gts = out
    else:
        gvi = torch.empty((3, N + 1, C), dtype=torch.float64, device=dev) if need_v_in else None
        grg = torch.empty((C,), dtype=torch.float64, device=dev) if need_rho_g else None
        grd = torch.empty((N, C), dtype=torch.float64, device=dev) if need_rho_d else None
        gts = torch.empty((N, C), dtype=torch.float64, device=dev) if need_t_s else None
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    vi = _f64_cuda("v_in", v_in, (3, N + 1, C))
    go = _f64_cuda("grad_v_out", grad_v_out, (3, N + 1, C))
    outs = [_opt_ptr("grad_v_in", gvi, (3, N + 1, C)), _opt_ptr("grad_rho_g", grg, (C,)),
            _opt_ptr("grad_rho_d", grd, (N, C)), _opt_ptr("grad_t_s", gts, (N, C))]
    if tape is None:
        _check(load_library().drag_expm_backward(C, N, *args, float(dt), vi, go, *outs, _stream_handle(stream)))
    else:
        if (tape.ncells, tape.nspecies) != (C, N):
            raise DragExpmError(f"tape written for ncells={tape.ncells} nspecies={tape.nspecies}, "
                                f"called with ncells={C} nspecies={N}")
        tp, tbytes = _bytes_cuda("tape", tape.buf)
        _check(load_library().drag_expm_backward_taped(C, N, *args, float(dt), vi, go, *outs, tape.levels, tp,
                                                       tbytes, _stream_handle(stream)))
    return gvi, grg, grd, gts


def _autograd_function():
    import torch

    class _DragExpm(torch.autograd.Function):
        """v_out = exp(dt Omega_v) v_in with a hand-written adjoint kernel.

        forward(rho_g, rho_d, t_s, dt, v_in) -> v_out; backward returns gradients
        for rho_g, rho_d, t_s and v_in (None for dt)."""

        @staticmethod
        def forward(ctx, rho_g, rho_d, t_s, dt, v_in):
            v_out = apply(rho_g.contiguous(), rho_d.contiguous(), t_s.contiguous(), float(dt), v_in.contiguous())
            ctx.save_for_backward(rho_g, rho_d, t_s, v_in)
            ctx.dt = float(dt)
            return v_out

        @staticmethod
        def backward(ctx, grad_out):
            rho_g, rho_d, t_s, v_in = ctx.saved_tensors
            need = ctx.needs_input_grad
            gvi, grg, grd, gts = backward(rho_g.contiguous(), rho_d.contiguous(), t_s.contiguous(), ctx.dt,
                                          v_in.contiguous(), grad_out.contiguous(), need_v_in=need[4],
                                          need_rho_g=need[0], need_rho_d=need[1], need_t_s=need[2])
            return grg, grd, gts, None, gvi

    class _DragExpmTaped(torch.autograd.Function):
        """DragExpm whose forward records the adjoint tape (apply_taped) and whose
        backward reads it: identical values; gradients identical for N <= 5 and from
        N = 12 on under the default modes (to rounding for 6 <= N <= 11, where the
        lane-per-cell forward writes a tape the warp-per-cell adjoint reads); less FP64
        work in the backward for a tape of about ncells * levels * 4 (N+1)(N+2) bytes.

        forward(rho_g, rho_d, t_s, dt, v_in, levels=None)."""

        @staticmethod
        def forward(ctx, rho_g, rho_d, t_s, dt, v_in, levels=None):
            rg, rd, ts = rho_g.contiguous(), rho_d.contiguous(), t_s.contiguous()
            v_out, tape = apply_taped(rg, rd, ts, float(dt), v_in.contiguous(), levels=levels)
            ctx.save_for_backward(rho_g, rho_d, t_s, v_in)
            ctx.dt = float(dt)
            ctx.tape = tape
            return v_out

        @staticmethod
        def backward(ctx, grad_out):
            rho_g, rho_d, t_s, v_in = ctx.saved_tensors
            need = ctx.needs_input_grad
            gvi, grg, grd, gts = backward(rho_g.contiguous(), rho_d.contiguous(), t_s.contiguous(), ctx.dt,
                                          v_in.contiguous(), grad_out.contiguous(), need_v_in=need[4],
                                          need_rho_g=need[0], need_rho_d=need[1], need_t_s=need[2], tape=ctx.tape)
            ctx.tape = None
            return grg, grd, gts, None, gvi, None

    return _DragExpm, _DragExpmTaped


class _LazyFunction:
    _fns = None

    def __init__(self, which: int):
        self._which = which

    def apply(self, *args):
        if _LazyFunction._fns is None:
            _LazyFunction._fns = _autograd_function()
        return _LazyFunction._fns[self._which].apply(*args)


DragExpm = _LazyFunction(0)
DragExpmTaped = _LazyFunction(1)


BLOCK_BYTES = 40   # sizeof(drag_block_t)


def batched_workspace_bytes(nblocks: int, total_cells: int) -> int:
    """Scratch bytes :func:`apply_batched` needs."""
    return int(load_library().drag_expm_batched_workspace_bytes(int(nblocks), int(total_cells)))


def _flat_f64(name, t):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise DragExpmError(f"{name} must be a contiguous float64 CUDA tensor")
    _on_current_device(name, t)
    return ctypes.c_void_p(t.data_ptr()), t.numel()


def apply_batched(blocks, rho_g, rho_d, t_s, v_in, v_out=None, nspecies_max=None, workspace=None, stream=None):
    """Batched forward update over block slabs (drag_expm_apply_batched).

    ``blocks``: a CUDA uint8 tensor of nblocks*40 bytes holding drag_block_t
    records (with ``nspecies_max`` given), or a host numpy array of the
    ``workloads.BLOCK_DTYPE`` record type (uploaded here). The arrays are flat
    float64 CUDA tensors. ``workspace`` (uint8 CUDA tensor) is allocated if
    not given. Returns v_out.
    """
    import numpy as np
    import torch
    if isinstance(blocks, np.ndarray):
        if nspecies_max is None:
            nspecies_max = int(blocks["nspecies"].max()) if len(blocks) else 1
        blocks = torch.from_numpy(np.ascontiguousarray(blocks).view(np.uint8).copy()).to(rho_g.device)
    if nspecies_max is None:
        raise DragExpmError("nspecies_max is required when blocks are already on the device")
    if not isinstance(blocks, torch.Tensor) or blocks.dtype != torch.uint8 or not blocks.is_cuda or \
            not blocks.is_contiguous() or blocks.numel() % BLOCK_BYTES:
        raise DragExpmError("blocks must be a contiguous CUDA uint8 tensor of drag_block_t records")
    _on_current_device("blocks", blocks)
    nblocks = blocks.numel() // BLOCK_BYTES
    if v_out is None:
        v_out = torch.empty_like(v_in)
    prg, C = _flat_f64("rho_g", rho_g)
    prd, nd = _flat_f64("rho_d", rho_d)
    pts, nt = _flat_f64("t_s", t_s)
    pvi, nv = _flat_f64("v_in", v_in)
    pvo, nvo = _flat_f64("v_out", v_out)
    if nt != nd or nvo != nv:
        raise DragExpmError("t_s must match rho_d and v_out must match v_in in length")
    need = batched_workspace_bytes(nblocks, C)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=rho_g.device)
    wp, wbytes = _bytes_cuda("workspace", workspace)
    _check(load_library().drag_expm_apply_batched(nblocks, ctypes.c_void_p(blocks.data_ptr()), C, nd, nv,
                                                  int(nspecies_max), prg, prd, pts, pvi, pvo, wp, wbytes,
                                                  _stream_handle(stream)))
    return v_out


def select(rho_g, rho_d, t_s, dt: float, stream=None, ubits: int = 53):
    """(k*, s*) per cell as chosen by Algorithm 2 (theta table of u = 2^-ubits):
    int8 and int16 CUDA tensors."""
    import torch
    C, N = _shapes(rho_g, rho_d)
    k = torch.empty(C, dtype=torch.int8, device=rho_g.device)
    s = torch.empty(C, dtype=torch.int16, device=rho_g.device)
    args = [_f64_cuda("rho_g", rho_g, (C,)), _f64_cuda("rho_d", rho_d, (N, C)), _f64_cuda("t_s", t_s, (N, C))]
    _check(load_library().drag_expm_select_target(C, N, *args, float(dt), int(ubits), ctypes.c_void_p(k.data_ptr()),
                                                  ctypes.c_void_p(s.data_ptr()), _stream_handle(stream)))
    return k, s


MODE_WARP_PER_CELL = 0
MODE_LANE_REGISTERS = 1
MODE_LANE_SHARED = 2
MODE_LANE_HYBRID = 3


def set_mode(nspecies: int, mode: int) -> None:
    """Force the kernel family used for ``nspecies`` on the current device."""
    _check(load_library().drag_expm_set_mode(int(nspecies), int(mode)))


def get_mode(nspecies: int) -> int:
    out = ctypes.c_int32(0)
    _check(load_library().drag_expm_get_mode(int(nspecies), ctypes.byref(out)))
    return int(out.value)


def autotune(nspecies_max: int, cache_path: str | None = None, stream=None) -> dict:
    """Measure the fastest mode per N (1..nspecies_max); returns {N: mode}."""
    p = cache_path.encode() if cache_path else None
    _check(load_library().drag_expm_autotune(int(nspecies_max), p, _stream_handle(stream)))
    return {N: get_mode(N) for N in range(1, int(nspecies_max) + 1)}


def probe_fp64_rate(kind: str = "dfma", iters: int = 20000, sink=None, stream=None) -> float:
    """Launch the FP64 throughput probe (kind "dfma": the FP64 pipe; "dmma":
    the FP64 tensor cores) on the stream; returns the launch's FP64 FLOPs.
    Time it with CUDA events around the call."""
    import torch
    if sink is None:
        sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    _on_current_device("sink", sink)
    flop = ctypes.c_double(0.0)
    _check(load_library().drag_expm_probe_fp64_rate({"dfma": 0, "dmma": 1}[kind], int(iters),
                                                    ctypes.c_void_p(sink.data_ptr()), ctypes.byref(flop),
                                                    _stream_handle(stream)))
    return flop.value


def probe_square(E, sig, reps: int, kind: str = "dfma", out=None, stream=None):
    """`reps` restored squarings of each symmetric matrix E[m] (float64 CUDA,
    (nmat, n, n)) with sigma sig[m] ((nmat, n)): kind "dfma" is the forward
    kernels' routine, "dmma" the FP64 tensor-core tiles. Returns the result."""
    import torch
    if E.dim() != 3 or E.shape[1] != E.shape[2] or sig.shape != E.shape[:2]:
        raise DragExpmError("E must be (nmat, n, n) and sig (nmat, n)")
    for nm, x in (("E", E), ("sig", sig)):
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise DragExpmError(f"{nm} must be a contiguous float64 CUDA tensor")
        _on_current_device(nm, x)
    if out is None:
        out = torch.empty_like(E)
    _check(load_library().drag_expm_probe_square({"dfma": 0, "dmma": 1}[kind], E.shape[1], E.shape[0], int(reps),
                                                 ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(sig.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def get_status(stream=None) -> int:
    """Read and clear the device's sticky status bits (STATUS_*)."""
    st = ctypes.c_uint32(0)
    _check(load_library().drag_expm_get_status(_stream_handle(stream), ctypes.byref(st)))
    return int(st.value)


def theta(k: int, ubits: int = 53) -> float:
    """theta_{m_k} (Eq. B8, u = 2^-ubits) as used by the library, k = 1..9."""
    out = ctypes.c_double(0.0)
    _check(load_library().drag_expm_theta_target(int(k), int(ubits), ctypes.byref(out)))
    return out.value
