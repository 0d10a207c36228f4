"""GB300 (sm_103a) local-inertial shallow-water flood model behind a C ABI.

Python binding of ``include/flood.h``: argument marshalling only.  Every step
of the method (Eq. 3-6 of Pierce et al., the CFL rule, the ledgers, the
adjoint) runs in the CUDA kernels of ``libflood_gb300.so``; PyTorch provides
the device memory allocator and streams.  Importing this package loads the
library and fails loudly if it is missing or cannot be built; there is no CPU
fallback.

The functions ``flood_create``, ``flood_step``, ``flood_read``, ... mirror the
C entry points one to one; :class:`Sim` wraps a handle for NumPy / torch users.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_CFL, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
F32, F64 = 0, 1
XMIN, XMAX, YMIN, YMAX = 0, 1, 2, 3
INFLOW, OUTFLOW = 0, 1
KERNEL_AUTO, KERNEL_REFERENCE, KERNEL_ROWS, KERNEL_TILED, KERNEL_STREAM, KERNEL_TMA = 0, 1, 2, 3, 4, 5
FIELD_H, FIELD_QX, FIELD_QY, FIELD_Z, FIELD_N, FIELD_LEDGER = 0, 1, 2, 3, 4, 5
LEDGER_KEYS = ("t", "dt", "V_in", "V_out", "V_clip", "volume", "h_max", "step", "cfl_exceed")


class FloodError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"flood status {status}: {msg}")
        self.status = status


class flood_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("precision", C.c_int32)]


class flood_bc_section(C.Structure):
    _fields_ = [("side", C.c_int32), ("kind", C.c_int32), ("frac_start", C.c_double),
                ("frac_end", C.c_double), ("slope", C.c_double),
                ("t_s", C.POINTER(C.c_double)), ("q_m3s", C.POINTER(C.c_double)), ("n_pts", C.c_int32)]


class flood_opts(C.Structure):
    _fields_ = [("g", C.c_double), ("h_dry", C.c_double), ("cfl_alpha", C.c_double), ("dt_cap", C.c_double),
                ("dt_const", C.c_double), ("dt_mode", C.c_int32), ("epoch_steps", C.c_int32),
                ("bc_form", C.c_int32), ("kernel", C.c_int32), ("steps_per_launch", C.c_int32),
                ("tile_x", C.c_int32), ("tile_y", C.c_int32), ("use_graph", C.c_int32),
                ("stream", C.c_void_p), ("theta", C.c_double),
                ("friction", C.c_int32)]


class flood_halo_copy(C.Structure):
    _fields_ = [("field", C.c_int32), ("src_part", C.c_int32), ("src_row", C.c_int32), ("dst_part", C.c_int32),
                ("dst_row", C.c_int32), ("rows", C.c_int32)]


_lib = None
LIB_PATH = None


def _load():
    global _lib, LIB_PATH
    if _lib is not None:
        return _lib
    import torch  # loads c10 / c10_cuda / cudart before the library
    if torch.cuda.is_available():
        torch.cuda.init()        # the caching allocator must be initialised before the library allocates
    path = _build.build()
    L = C.CDLL(path, mode=C.RTLD_GLOBAL)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    H = C.c_void_p
    L.flood_check_bounded_wait.argtypes = [C.c_double]
    L.flood_check_bounded_wait.restype = C.c_int
    L.flood_default_opts.argtypes = [C.POINTER(flood_opts)]
    L.flood_default_opts.restype = None
    L.flood_create.argtypes = [C.POINTER(flood_grid), vp, vp, C.POINTER(flood_bc_section), i32,
                               C.POINTER(flood_opts), C.POINTER(H)]
    L.flood_step.argtypes = [H, i64]
    L.flood_advance.argtypes = [vp, C.c_double, C.POINTER(i64)]
    L.flood_sync.argtypes = [H]
    L.flood_read.argtypes = [H, i32, vp, C.c_size_t, i32]
    L.flood_write_state.argtypes = [H, vp, vp, vp, i32]
    L.flood_set_clock.argtypes = [H, dbl, i64, dbl, dbl, dbl, dbl]
    L.flood_set_manning.argtypes = [H, vp, i32]
    L.flood_run_gauges.argtypes = [H, i64, C.POINTER(C.c_int64), i32, vp, i32]
    L.flood_adjoint.argtypes = [H, i64, C.POINTER(C.c_int64), i32, C.POINTER(C.c_double), i32, vp, vp, i32]
    L.flood_adjoint_forward_steps.argtypes = [H]
    L.flood_adjoint_forward_steps.restype = i64
    L.flood_revolve_plan.argtypes = [i64, i32, i32, i64, i32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int32)]
    L.flood_destroy.argtypes = [H]
    L.flood_last_error.argtypes = [H]
    L.flood_last_error.restype = C.c_char_p
    L.flood_version.restype = C.c_char_p
    L.flood_adjoint_profile.argtypes = [H, i32]
    L.flood_adjoint_profile.restype = C.c_int
    L.flood_adjoint_times.argtypes = [H, C.POINTER(dbl), C.POINTER(i64), C.POINTER(dbl), C.POINTER(i64)]
    L.flood_adjoint_times.restype = C.c_int
    L.flood_volume_noalloc.argtypes = [vp, i32, i32, i64, i32, dbl, vp, vp]
    L.flood_coarsen.argtypes = [i32, vp, i32, i32, i32, vp, i32, vp]
    L.flood_coarsen.restype = C.c_int
    L.flood_volume_noalloc.restype = C.c_int
    L.flood_ensemble_create.argtypes = [i32, C.POINTER(flood_grid), C.POINTER(vp), C.POINTER(vp),
                                        C.POINTER(C.POINTER(flood_bc_section)), C.POINTER(i32),
                                        C.POINTER(flood_opts), C.POINTER(vp)]
    L.flood_ensemble_set_launch.argtypes = [vp, i32, i32, i32, i32]
    L.flood_ensemble_set_kernel.argtypes = [vp, i32, i32]
    L.flood_ensemble_step.argtypes = [vp, i64]
    L.flood_ensemble_member.argtypes = [vp, i32]
    L.flood_ensemble_member.restype = vp
    L.flood_ensemble_destroy.argtypes = [vp]
    L.flood_ensemble_last_error.argtypes = [vp]
    L.flood_ensemble_last_error.restype = C.c_char_p
    L.flood_decomp_plan.argtypes = [i32, i32, i32, C.POINTER(i32), C.POINTER(flood_halo_copy), C.POINTER(i32)]
    L.flood_decomp_combine_ledgers.argtypes = [i32, C.POINTER(dbl), C.POINTER(dbl)]
    L.flood_decomp_create.argtypes = [C.POINTER(flood_grid), vp, vp, C.POINTER(flood_bc_section), i32,
                                      C.POINTER(flood_opts), i32, i32, C.POINTER(vp)]
    L.flood_decomp_step.argtypes = [vp, i64]
    L.flood_decomp_read.argtypes = [vp, i32, vp, C.c_size_t, i32]
    L.flood_decomp_write_state.argtypes = [vp, vp, vp, vp, i32]
    L.flood_decomp_sync.argtypes = [vp]
    L.flood_decomp_part.argtypes = [vp, i32]
    L.flood_decomp_part.restype = vp
    L.flood_decomp_destroy.argtypes = [vp]
    L.flood_decomp_last_error.argtypes = [vp]
    L.flood_decomp_last_error.restype = C.c_char_p
    L.flood_debug_fail_alloc_after.argtypes = [i64]
    L.flood_debug_fail_alloc_after.restype = None
    L.flood_debug_alloc_count.argtypes = []
    L.flood_debug_alloc_count.restype = i64
    L.flood_debug_padding.argtypes = [H, i32, C.POINTER(i64)]
    L.flood_debug_padding.restype = C.c_int
    L.flood_debug_tiled_split.argtypes = [i32, i32, i32, i32, i32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32)]
    for name in ("flood_decomp_plan", "flood_decomp_combine_ledgers", "flood_decomp_create", "flood_decomp_step",
                 "flood_decomp_read", "flood_decomp_write_state", "flood_decomp_sync", "flood_decomp_destroy"):
        getattr(L, name).restype = C.c_int
    for name in ("flood_ensemble_create", "flood_ensemble_set_launch", "flood_ensemble_set_kernel",
                 "flood_ensemble_step", "flood_ensemble_destroy"):
        getattr(L, name).restype = C.c_int
    for name in ("flood_create", "flood_step", "flood_advance", "flood_sync", "flood_read", "flood_write_state",
                 "flood_set_clock", "flood_set_manning", "flood_run_gauges", "flood_adjoint", "flood_destroy"):
        getattr(L, name).restype = C.c_int
    _lib = L
    LIB_PATH = path
    return L


def lib():
    return _load()


def _check(st: int, handle=None):
    if st != OK:
        msg = lib().flood_last_error(handle).decode(errors="replace")
        raise FloodError(st, msg)


def default_opts() -> flood_opts:
    o = flood_opts()
    lib().flood_default_opts(C.byref(o))
    return o


# ------------------------------------------------------------------ C-ABI mirrors
def flood_create(grid: flood_grid, dem, manning, sections, n_sections: int, opts: Optional[flood_opts]):
    h = C.c_void_p()
    st = lib().flood_create(C.byref(grid), dem, manning, sections, n_sections,
                            None if opts is None else C.byref(opts), C.byref(h))
    _check(st, None)
    return h


def flood_step(h, n_steps: int):
    _check(lib().flood_step(h, int(n_steps)), h)


def flood_advance(h, t_end: float) -> int:
    k = C.c_int64(0)
    _check(lib().flood_advance(h, float(t_end), C.byref(k)), h)
    return int(k.value)


def flood_sync(h):
    return lib().flood_sync(h)


def flood_read(h, field: int, dst_ptr, nbytes: int, dst_on_device: int):
    _check(lib().flood_read(h, int(field), dst_ptr, int(nbytes), int(dst_on_device)), h)


def flood_write_state(h, depth, qx, qy, src_on_device: int):
    _check(lib().flood_write_state(h, depth, qx, qy, int(src_on_device)), h)


def flood_set_clock(h, t, step, dt, v_in, v_out, v_clip):
    _check(lib().flood_set_clock(h, float(t), int(step), float(dt), float(v_in), float(v_out), float(v_clip)), h)


def flood_set_manning(h, manning, src_on_device: int):
    _check(lib().flood_set_manning(h, manning, int(src_on_device)), h)


def flood_run_gauges(h, n_steps, gauge_cells, n_gauges, out, out_on_device):
    _check(lib().flood_run_gauges(h, int(n_steps), gauge_cells, int(n_gauges), out, int(out_on_device)), h)


def flood_adjoint(h, n_steps, gauge_cells, n_gauges, dLdh, n_checkpoints, dLdn_out, dLdh0_out, out_on_device):
    _check(lib().flood_adjoint(h, int(n_steps), gauge_cells, int(n_gauges), dLdh, int(n_checkpoints), dLdn_out,
                               dLdh0_out, int(out_on_device)), h)


def flood_destroy(h):
    lib().flood_destroy(h)


def flood_last_error(h=None) -> str:
    return lib().flood_last_error(h).decode(errors="replace")


def flood_version() -> str:
    return lib().flood_version().decode()


def flood_volume_noalloc(depth_ptr, nx: int, ny: int, row_pitch: int, precision: int, dx: float, out_ptr,
                         stream_ptr=None):
    """Stored volume of a device depth array without any allocation (see include/flood.h)."""
    _check(lib().flood_volume_noalloc(depth_ptr, int(nx), int(ny), int(row_pitch), int(precision), float(dx),
                                      out_ptr, stream_ptr), None)


def revolve_plan(n_steps: int, n_checkpoints: int, epoch_steps: int = 16, start_step: int = 0,
                 steps_per_replay: int = 1) -> dict:
    """flood_revolve_plan: the adjoint's checkpoint schedule run on the host alone
    (see include/flood.h): steps replayed, replay launches, reversal in order."""
    f, n, ok = C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib().flood_revolve_plan(int(n_steps), int(n_checkpoints), int(epoch_steps), int(start_step),
                                    int(steps_per_replay), C.byref(f), C.byref(n), C.byref(ok)), None)
    return {"forward_steps": f.value, "replay_launches": n.value, "in_order": bool(ok.value)}


def flood_debug_fail_alloc_after(n: int) -> None:
    """Make the library's device allocation after n more successful ones fail (n < 0: off)."""
    lib().flood_debug_fail_alloc_after(int(n))


def flood_debug_tiled_split(nx: int, ny: int, k_steps: int = 4, mode: int = 0, resident: int = 912) -> dict:
    """The temporal-blocking kernel's work items for an nx x ny grid (host only)."""
    rows, blocks, items = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().flood_debug_tiled_split(int(nx), int(ny), int(k_steps), int(mode), int(resident), C.byref(rows),
                                         C.byref(blocks), C.byref(items)), None)
    return {"chunk_rows": rows.value, "blocks": blocks.value, "items": items.value}


def flood_debug_alloc_count() -> int:
    return int(lib().flood_debug_alloc_count())


def flood_debug_padding(h, fill: bool) -> int:
    """Poison the pitch padding of a handle's planes (fill), or count padding elements that changed."""
    bad = C.c_int64(0)
    _check(lib().flood_debug_padding(h, int(fill), C.byref(bad)), h)
    return int(bad.value)


# ------------------------------------------------------------------ convenience wrapper
def coarsen(field, factor: int):
    """Block mean of a (ny, nx) float32/float64 field (NumPy array or CUDA tensor)
    over factor x factor cells, the coarsening of the paper's 1 m DEM; returns the
    (ceil(ny/f), ceil(nx/f)) field of the same kind and device."""
    ny, nx = field.shape
    my, mx = -(-ny // factor), -(-nx // factor)
    if isinstance(field, np.ndarray):
        src = np.ascontiguousarray(field)
        out = np.empty((my, mx), src.dtype)
        prec = F32 if src.dtype == np.float32 else F64
    else:
        import torch
        src = field.contiguous()
        out = src.new_empty((my, mx))
        prec = F32 if src.dtype == torch.float32 else F64
    ps, dev = _ptr(src)
    pd, _ = _ptr(out)
    _check(lib().flood_coarsen(prec, ps, nx, ny, int(factor), pd, dev, None), None)
    return out


def _ptr(a):
    """(pointer, on_device) of a contiguous NumPy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return C.c_void_p(a.ctypes.data), 0
    import torch
    if isinstance(a, torch.Tensor):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    raise TypeError(type(a))


def _opts_for(problem, kernel=KERNEL_AUTO, steps_per_launch=0, tile=(0, 0), use_graph=False, stream=None):
    po = problem.opts
    o = default_opts()
    o.g, o.h_dry, o.cfl_alpha, o.dt_cap, o.dt_const = po.g, po.h_dry, po.cfl_alpha, po.dt_cap, po.dt_const
    o.dt_mode, o.epoch_steps, o.bc_form = po.dt_mode, po.epoch_steps, po.bc_form
    o.theta = getattr(po, "theta", 1.0)
    o.friction = getattr(po, "friction", 0)
    o.kernel, o.steps_per_launch = kernel, steps_per_launch
    o.tile_x, o.tile_y = tile
    o.use_graph = int(use_graph)
    o.stream = None if stream is None else C.c_void_p(stream.cuda_stream)
    return o


def _sections_for(problem, keep: list):
    """ctypes array of the problem's sections (tables appended to keep)."""
    secs = (flood_bc_section * max(1, len(problem.sections)))()
    for k, s in enumerate(problem.sections):
        t = np.ascontiguousarray(s.t_s if s.t_s is not None else np.zeros(1), np.float64)
        q = np.ascontiguousarray(s.q_m3s if s.q_m3s is not None else np.zeros(1), np.float64)
        keep += [t, q]
        secs[k] = flood_bc_section(s.side, s.kind, s.frac_start, s.frac_end, s.slope,
                                   t.ctypes.data_as(C.POINTER(C.c_double)),
                                   q.ctypes.data_as(C.POINTER(C.c_double)),
                                   t.size if s.kind == INFLOW else 0)
    return secs


class Sim:
    """One simulation handle.  ``problem`` is an ``inputs.Problem``-like object
    (nx, ny, dx, z, n, sections, opts, h0/qx0/qy0)."""

    def __init__(self, problem, precision: int = F32, kernel: int = KERNEL_AUTO, steps_per_launch: int = 0,
                 tile=(0, 0), use_graph: bool = False, stream=None):
        self.prob = problem
        self.precision = precision
        self.dtype = np.float32 if precision == F32 else np.float64
        self.nx, self.ny = problem.nx, problem.ny
        o = _opts_for(problem, kernel, steps_per_launch, tile, use_graph, stream)
        self.opts = o
        self._keep = []
        secs = _sections_for(problem, self._keep)
        z = np.ascontiguousarray(problem.z, self.dtype)
        n = np.ascontiguousarray(problem.n, self.dtype)
        self.grid = flood_grid(self.nx, self.ny, float(problem.dx), precision)
        self.h = flood_create(self.grid, C.c_void_p(z.ctypes.data), C.c_void_p(n.ctypes.data), secs,
                              len(problem.sections), o)
        if problem.h0 is not None or problem.qx0 is not None or problem.qy0 is not None:
            h0, qx0, qy0 = problem.initial_state(self.dtype)
            self.write_state(h0, qx0, qy0)

    # -- state
    def write_state(self, h, qx=None, qy=None):
        arrs = [None if a is None else (np.ascontiguousarray(a, self.dtype) if isinstance(a, np.ndarray) else a)
                for a in (h, qx, qy)]
        ptrs = [_ptr(a) for a in arrs]
        dev = max(p[1] for p in ptrs if p[0] is not None)
        flood_write_state(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], dev)

    def read(self, field: int):
        shape = {FIELD_H: (self.ny, self.nx), FIELD_QX: (self.ny, self.nx + 1), FIELD_QY: (self.ny + 1, self.nx),
                 FIELD_Z: (self.ny, self.nx), FIELD_N: (self.ny, self.nx)}[field]
        out = np.empty(shape, self.dtype)
        flood_read(self.h, field, C.c_void_p(out.ctypes.data), out.nbytes, 0)
        return out

    def state(self):
        return self.read(FIELD_H), self.read(FIELD_QX), self.read(FIELD_QY)

    def ledger(self):
        out = np.zeros(len(LEDGER_KEYS), np.float64)
        flood_read(self.h, FIELD_LEDGER, C.c_void_p(out.ctypes.data), out.nbytes, 0)
        return dict(zip(LEDGER_KEYS, out.tolist()))

    def set_clock(self, t, step, dt, v_in=0.0, v_out=0.0, v_clip=0.0):
        flood_set_clock(self.h, t, step, dt, v_in, v_out, v_clip)

    def set_manning(self, n):
        a = np.ascontiguousarray(n, self.dtype) if isinstance(n, np.ndarray) else n
        p, dev = _ptr(a)
        flood_set_manning(self.h, p, dev)

    # -- stepping
    def step(self, n_steps: int = 1, check: bool = False):
        flood_step(self.h, n_steps)
        if check:
            self.sync()

    def advance(self, t_end: float) -> int:
        """Advance to simulated time t_end, the last step shortened to land on it;
        returns the number of steps."""
        return flood_advance(self.h, t_end)

    def sync(self):
        st = flood_sync(self.h)
        _check(st, self.h)

    def run_gauges(self, n_steps: int, gauges: np.ndarray, out=None):
        cells = np.ascontiguousarray(gauges[:, 1].astype(np.int64) * self.nx + gauges[:, 0], np.int64)
        if out is None:
            out = np.zeros((n_steps, cells.size), np.float64)
        p, dev = _ptr(out)
        flood_run_gauges(self.h, n_steps, cells.ctypes.data_as(C.POINTER(C.c_int64)), cells.size, p, dev)
        return out

    def adjoint(self, n_steps: int, gauges: np.ndarray, dLdh: np.ndarray, n_checkpoints: int = 40,
                want_dh0: bool = False):
        cells = np.ascontiguousarray(gauges[:, 1].astype(np.int64) * self.nx + gauges[:, 0], np.int64)
        seed = np.ascontiguousarray(dLdh, np.float64)
        assert seed.shape == (n_steps, cells.size)
        gn = np.zeros((self.ny, self.nx), self.dtype)
        gh = np.zeros((self.ny, self.nx), self.dtype) if want_dh0 else None
        flood_adjoint(self.h, n_steps, cells.ctypes.data_as(C.POINTER(C.c_int64)), cells.size,
                      seed.ctypes.data_as(C.POINTER(C.c_double)), n_checkpoints, C.c_void_p(gn.ctypes.data),
                      None if gh is None else C.c_void_p(gh.ctypes.data), 0)
        return (gn, gh) if want_dh0 else gn

    def adjoint_forward_steps(self) -> int:
        return int(lib().flood_adjoint_forward_steps(self.h))

    def adjoint_profile(self, enable: bool = True) -> None:
        _check(lib().flood_adjoint_profile(self.h, int(enable)), self.h)

    def adjoint_times(self) -> dict:
        """Device time (ms) of the last profiled flood_adjoint call's reverse steps and forward replays."""
        rm, fm = C.c_double(), C.c_double()
        rn, fn = C.c_int64(), C.c_int64()
        _check(lib().flood_adjoint_times(self.h, C.byref(rm), C.byref(rn), C.byref(fm), C.byref(fn)), self.h)
        return {"reverse_ms": rm.value, "reverse_steps": rn.value, "forward_ms": fm.value, "forward_steps": fn.value}

    def close(self):
        if getattr(self, "h", None) is not None:
            flood_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ ensembles
def _ens_check(st: int, ens=None):
    if st != OK:
        raise FloodError(st, lib().flood_ensemble_last_error(ens).decode(errors="replace"))


def flood_ensemble_create(n, grids, dems, mannings, sections, n_sections, opts):
    e = C.c_void_p()
    _ens_check(lib().flood_ensemble_create(n, grids, dems, mannings, sections, n_sections, C.byref(opts),
                                           C.byref(e)))
    return e


def flood_ensemble_set_launch(e, warps, rows, steps_per_graph, use_graph):
    _ens_check(lib().flood_ensemble_set_launch(e, int(warps), int(rows), int(steps_per_graph), int(use_graph)), e)


def flood_ensemble_set_kernel(e, kernel, steps_per_launch):
    _ens_check(lib().flood_ensemble_set_kernel(e, int(kernel), int(steps_per_launch)), e)


def flood_ensemble_step(e, n_steps):
    _ens_check(lib().flood_ensemble_step(e, int(n_steps)), e)


def flood_ensemble_member(e, k):
    return C.c_void_p(lib().flood_ensemble_member(e, int(k)))


def flood_ensemble_destroy(e):
    lib().flood_ensemble_destroy(e)


class _Member(Sim):
    """View of one ensemble scenario's handle (owned by the ensemble)."""

    def __init__(self, handle, problem):
        self.prob = problem
        self.precision = F32
        self.dtype = np.float32
        self.nx, self.ny = problem.nx, problem.ny
        self.h = handle

    def close(self):
        self.h = None


class Ensemble:
    """FP32 scenarios of different sizes stepped together (see include/flood.h)."""

    def __init__(self, problems, stream=None):
        self.problems = list(problems)
        n = len(self.problems)
        po = self.problems[0].opts
        o = default_opts()
        o.g, o.h_dry, o.cfl_alpha, o.dt_cap, o.dt_const = po.g, po.h_dry, po.cfl_alpha, po.dt_cap, po.dt_const
        o.dt_mode, o.epoch_steps, o.bc_form = po.dt_mode, po.epoch_steps, po.bc_form
        o.theta = getattr(po, "theta", 1.0)
        o.friction = getattr(po, "friction", 0)
        o.stream = None if stream is None else C.c_void_p(stream.cuda_stream)
        import torch
        # the stream every launch of the ensemble goes to (the current one at creation if none is given)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = []
        grids = (flood_grid * n)()
        dems = (C.c_void_p * n)()
        mans = (C.c_void_p * n)()
        secs = (C.POINTER(flood_bc_section) * n)()
        nsec = (C.c_int32 * n)()
        for k, p in enumerate(self.problems):
            grids[k] = flood_grid(p.nx, p.ny, float(p.dx), F32)
            z = np.ascontiguousarray(p.z, np.float32)
            m = np.ascontiguousarray(p.n, np.float32)
            self._keep += [z, m]
            dems[k] = z.ctypes.data
            mans[k] = m.ctypes.data
            arr = (flood_bc_section * max(1, len(p.sections)))()
            for i, s in enumerate(p.sections):
                t = np.ascontiguousarray(s.t_s if s.t_s is not None else np.zeros(1), np.float64)
                q = np.ascontiguousarray(s.q_m3s if s.q_m3s is not None else np.zeros(1), np.float64)
                self._keep += [t, q]
                arr[i] = flood_bc_section(s.side, s.kind, s.frac_start, s.frac_end, s.slope,
                                          t.ctypes.data_as(C.POINTER(C.c_double)),
                                          q.ctypes.data_as(C.POINTER(C.c_double)),
                                          t.size if s.kind == INFLOW else 0)
            self._keep.append(arr)
            secs[k] = C.cast(arr, C.POINTER(flood_bc_section))
            nsec[k] = len(p.sections)
        self.e = flood_ensemble_create(n, grids, dems, mans, secs, nsec, o)
        self.members = [_Member(flood_ensemble_member(self.e, k), p) for k, p in enumerate(self.problems)]
        for mb, p in zip(self.members, self.problems):
            if p.h0 is not None or p.qx0 is not None or p.qy0 is not None:
                mb.write_state(*p.initial_state(np.float32))
        self.cells = sum(p.nx * p.ny for p in self.problems)

    def set_launch(self, warps=4, rows=64, steps_per_graph=None, use_graph=True):
        E = self.problems[0].opts.epoch_steps
        flood_ensemble_set_launch(self.e, warps, rows, steps_per_graph or E, int(use_graph))

    def set_kernel(self, kernel=KERNEL_STREAM, steps_per_launch=0):
        """KERNEL_STREAM (one step per launch) or KERNEL_TILED with K steps per launch."""
        flood_ensemble_set_kernel(self.e, kernel, steps_per_launch)

    def step(self, n_steps: int):
        flood_ensemble_step(self.e, n_steps)

    def close(self):
        if getattr(self, "e", None) is not None:
            flood_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ domain decomposition
def _dec_check(st: int, d=None):
    if st != OK:
        raise FloodError(st, lib().flood_decomp_last_error(d).decode(errors="replace"))


def flood_decomp_plan(ny: int, n_parts: int, halo: int):
    """Row split and halo copies of a decomposition: (rows (n_parts, 4) int32 array
    of y0, y1, a, b; list of (field, src_part, src_row, dst_part, dst_row, rows))."""
    rows = np.zeros((max(n_parts, 1), 4), np.int32)
    n = C.c_int32(0)
    rp = rows.ctypes.data_as(C.POINTER(C.c_int32))
    _dec_check(lib().flood_decomp_plan(int(ny), int(n_parts), int(halo), rp, None, C.byref(n)))
    arr = (flood_halo_copy * max(n.value, 1))()
    _dec_check(lib().flood_decomp_plan(int(ny), int(n_parts), int(halo), rp, arr, C.byref(n)))
    copies = [(c.field, c.src_part, c.src_row, c.dst_part, c.dst_row, c.rows) for c in arr[:n.value]]
    return rows, copies


def flood_decomp_combine_ledgers(part_ledgers: np.ndarray) -> np.ndarray:
    """Whole-grid ledger (FLOOD_LEDGER_LEN doubles) from the parts' ledgers (n_parts rows)."""
    L = np.ascontiguousarray(part_ledgers, np.float64)
    out = np.zeros(len(LEDGER_KEYS), np.float64)
    _dec_check(lib().flood_decomp_combine_ledgers(L.shape[0], L.ctypes.data_as(C.POINTER(C.c_double)),
                                                   out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


class Decomp:
    """A grid split into n_parts row strips with `halo` rows of overlap, advanced
    together with a halo exchange every `halo` steps (see include/flood.h).
    Holds a flood_decomp (not a flood_handle): only flood_decomp_* calls take it."""

    def __init__(self, problem, n_parts: int, halo: int, precision: int = F32, kernel: int = KERNEL_AUTO,
                 steps_per_launch: int = 0, tile=(0, 0), stream=None):
        self.prob = problem
        self.precision = precision
        self.dtype = np.float32 if precision == F32 else np.float64
        self.nx, self.ny = problem.nx, problem.ny
        self.n_parts, self.halo = n_parts, halo
        o = _opts_for(problem, kernel, steps_per_launch, tile, False, stream)
        self.opts = o
        self._keep = []
        secs = _sections_for(problem, self._keep)
        z = np.ascontiguousarray(problem.z, self.dtype)
        n = np.ascontiguousarray(problem.n, self.dtype)
        self.grid = flood_grid(self.nx, self.ny, float(problem.dx), precision)
        d = C.c_void_p()
        _dec_check(lib().flood_decomp_create(C.byref(self.grid), C.c_void_p(z.ctypes.data),
                                             C.c_void_p(n.ctypes.data), secs, len(problem.sections), C.byref(o),
                                             int(n_parts), int(halo), C.byref(d)))
        self.h = d
        if problem.h0 is not None or problem.qx0 is not None or problem.qy0 is not None:
            self.write_state(*problem.initial_state(self.dtype))

    def write_state(self, h, qx=None, qy=None):
        arrs = [None if a is None else (np.ascontiguousarray(a, self.dtype) if isinstance(a, np.ndarray) else a)
                for a in (h, qx, qy)]
        ptrs = [_ptr(a) for a in arrs]
        dev = max(p[1] for p in ptrs if p[0] is not None)
        _dec_check(lib().flood_decomp_write_state(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], dev), self.h)

    def read(self, field: int):
        shape = {FIELD_H: (self.ny, self.nx), FIELD_QX: (self.ny, self.nx + 1), FIELD_QY: (self.ny + 1, self.nx),
                 FIELD_Z: (self.ny, self.nx), FIELD_N: (self.ny, self.nx)}[field]
        out = np.empty(shape, self.dtype)
        _dec_check(lib().flood_decomp_read(self.h, field, C.c_void_p(out.ctypes.data), out.nbytes, 0), self.h)
        return out

    def ledger(self):
        out = np.zeros(len(LEDGER_KEYS), np.float64)
        _dec_check(lib().flood_decomp_read(self.h, FIELD_LEDGER, C.c_void_p(out.ctypes.data), out.nbytes, 0),
                   self.h)
        return dict(zip(LEDGER_KEYS, out.tolist()))

    def state(self):
        return self.read(FIELD_H), self.read(FIELD_QX), self.read(FIELD_QY)

    def part_ledger(self, k: int):
        """Part k's own ledger terms (FLOOD_LEDGER_LEN doubles)."""
        out = np.zeros(len(LEDGER_KEYS), np.float64)
        flood_read(lib().flood_decomp_part(self.h, int(k)), FIELD_LEDGER, C.c_void_p(out.ctypes.data), out.nbytes, 0)
        return out

    def step(self, n_steps: int = 1, check: bool = False):
        _dec_check(lib().flood_decomp_step(self.h, int(n_steps)), self.h)
        if check:
            self.sync()

    def sync(self):
        _dec_check(lib().flood_decomp_sync(self.h), self.h)

    def part_handle(self, k: int):
        return C.c_void_p(lib().flood_decomp_part(self.h, int(k)))

    def part_view(self, k: int) -> "_PartView":
        """Part k's stored rows (its own rows and its halo rows) as a read-only Sim."""
        rows, _ = flood_decomp_plan(self.ny, self.n_parts, self.halo)
        return _PartView(self.part_handle(k), self.nx, int(rows[k, 3] - rows[k, 2]), self.precision)

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().flood_decomp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _PartView(Sim):
    """View of one part's handle (owned by its decomposition; stepping it is refused)."""

    def __init__(self, handle, nx: int, ny: int, precision: int):
        self.h = handle
        self.nx, self.ny = nx, ny
        self.precision = precision
        self.dtype = np.float32 if precision == F32 else np.float64

    def close(self):
        self.h = None
