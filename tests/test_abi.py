"""C-ABI library checks that need no GPU: it builds for sm_103a, loads, exports
every entry point that include/flood.h declares, and rejects bad arguments in
host code before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "flood.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(
        r"^\s*(?:flood_status|void|int64_t|const\s+char\s*\*)\s*\**\s*(flood_\w+)\s*\(", src, flags=re.M)))


def test_header_lists_the_boundary():
    names = header_functions()
    for n in ("flood_create", "flood_step", "flood_read", "flood_adjoint", "flood_destroy", "flood_last_error",
              "flood_write_state"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2204_10323_gb300 as F
    L = F.lib()
    missing = [n for n in header_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert "sm_103a" in F.flood_version()


def test_objects_are_built_for_sm_103a_only():
    """Every CUDA translation unit is compiled with exactly one target,
    -gencode arch=compute_103a,code=sm_103a (the build's compilation database)."""
    import json
    import paper_2204_10323_gb300 as F
    F.lib()
    with open(os.path.join(F._build.BUILD, "compile_commands.json")) as f:
        db = json.load(f)
    cu = [e for e in db if e["file"].endswith(".cu")]
    srcs = [f for f in os.listdir(F._build.CSRC) if f.endswith(".cu")]
    assert sorted(os.path.basename(e["file"]) for e in cu) == sorted(srcs)
    for e in cu:
        args = e["arguments"]
        targets = [args[i + 1] for i, a in enumerate(args) if a == "-gencode"]
        assert targets == ["arch=compute_103a,code=sm_103a"], (e["file"], targets)
        assert not any(a.startswith(("-arch", "--gpu-architecture", "--generate-code")) for a in args)


def _grid(nx, ny, dx=1.0, prec=0):
    import paper_2204_10323_gb300 as F
    return F.flood_grid(nx, ny, dx, prec)


def _create(grid, dem, secs=None, opts=None):
    import paper_2204_10323_gb300 as F
    h = C.c_void_p()
    ns = 0 if secs is None else len(secs)
    arr = None
    if secs:
        arr = (F.flood_bc_section * ns)(*secs)
    st = F.lib().flood_create(C.byref(grid), C.c_void_p(dem.ctypes.data), None, arr, ns,
                              None if opts is None else C.byref(opts), C.byref(h))
    return st, h


@pytest.mark.parametrize("nx,ny,dx", [(0, 4, 1.0), (4, 0, 1.0), (4, 4, 0.0), (4, 4, -1.0), (4, 4, float("nan"))])
def test_create_rejects_bad_grid(nx, ny, dx):
    import paper_2204_10323_gb300 as F
    st, h = _create(_grid(nx, ny, dx), np.zeros(16, np.float32))
    assert st == F.ERR_ARG and not h.value
    assert F.flood_last_error(None)


def test_create_rejects_overlapping_sections():
    import paper_2204_10323_gb300 as F
    t = np.array([0.0, 1.0])
    q = np.array([1.0, 1.0])
    tp, qp = t.ctypes.data_as(C.POINTER(C.c_double)), q.ctypes.data_as(C.POINTER(C.c_double))
    a = F.flood_bc_section(F.XMIN, F.INFLOW, 0.0, 0.5, 1e-3, tp, qp, 2)
    b = F.flood_bc_section(F.XMIN, F.OUTFLOW, 0.25, 1.0, 1e-3, None, None, 0)
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), [a, b])
    assert st == F.ERR_ARG and "overlap" in F.flood_last_error(None)


@pytest.mark.parametrize("field,value", [("slope", 0.0), ("side", 7), ("kind", 3), ("frac_end", 1.5)])
def test_create_rejects_bad_section(field, value):
    import paper_2204_10323_gb300 as F
    s = F.flood_bc_section(F.XMAX, F.OUTFLOW, 0.0, 1.0, 1e-3, None, None, 0)
    setattr(s, field, value)
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), [s])
    assert st == F.ERR_ARG


def test_create_rejects_descending_hydrograph_and_nan_dem():
    import paper_2204_10323_gb300 as F
    t = np.array([0.0, 2.0, 1.0])
    q = np.array([1.0, 1.0, 1.0])
    s = F.flood_bc_section(F.XMIN, F.INFLOW, 0.0, 1.0, 1e-3, t.ctypes.data_as(C.POINTER(C.c_double)),
                           q.ctypes.data_as(C.POINTER(C.c_double)), 3)
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), [s])
    assert st == F.ERR_ARG
    dem = np.zeros(64, np.float32)
    dem[5] = np.nan
    st, _ = _create(_grid(8, 8), dem)
    assert st == F.ERR_ARG and "NaN" in F.flood_last_error(None)


def test_create_rejects_bad_options():
    import paper_2204_10323_gb300 as F
    o = F.default_opts()
    o.epoch_steps = 0
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
    assert st == F.ERR_ARG
    o = F.default_opts()
    o.kernel = F.KERNEL_TILED
    o.epoch_steps = 16
    o.steps_per_launch = 3        # must divide E
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
    assert st == F.ERR_ARG
    o.steps_per_launch = 5        # 1..4 or 8
    o.epoch_steps = 20
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
    assert st == F.ERR_ARG and "steps_per_launch" in F.flood_last_error(None)
    o = F.default_opts()
    o.kernel = 6                  # no such kernel family
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
    assert st == F.ERR_ARG and "kernel" in F.flood_last_error(None)
    o = F.default_opts()
    o.tile_y = -1
    st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
    assert st == F.ERR_ARG and "tile" in F.flood_last_error(None)


def test_default_opts_values():
    import paper_2204_10323_gb300 as F
    o = F.default_opts()
    assert (o.g, o.h_dry, o.cfl_alpha, o.epoch_steps, o.dt_const) == (9.81, 1e-3, 0.7, 16, 0.1)


def test_null_handle_calls_fail_cleanly():
    import paper_2204_10323_gb300 as F
    L = F.lib()
    assert L.flood_step(None, 1) == F.ERR_ARG
    assert L.flood_sync(None) == F.ERR_ARG
    assert L.flood_destroy(None) == F.OK


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2204_10323_gb300 as F
    st, h = _create(_grid(8, 8), np.zeros(64, np.float32))
    assert st == F.ERR_CUDA and not h.value


def test_coarsen_rejects_bad_arguments():
    import paper_2204_10323_gb300 as F
    L = F.lib()
    a = np.zeros((4, 4), np.float32)
    b = np.zeros((2, 2), np.float32)
    pa, pb = C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data)
    assert L.flood_coarsen(F.F32, pa, 4, 4, 0, pb, 0, None) == F.ERR_ARG      # factor 0
    assert L.flood_coarsen(F.F32, pa, 0, 4, 2, pb, 0, None) == F.ERR_ARG      # empty grid
    assert L.flood_coarsen(7, pa, 4, 4, 2, pb, 0, None) == F.ERR_ARG          # precision
    assert L.flood_coarsen(F.F32, None, 4, 4, 2, pb, 0, None) == F.ERR_ARG    # NULL source
    assert "NULL" in F.flood_last_error(None)


def test_bounded_wait_check_rejects_budgets_out_of_range():
    import paper_2204_10323_gb300 as F
    for bad in (0.0, -1.0, 11.0, float("nan")):
        assert F.lib().flood_check_bounded_wait(bad) == F.ERR_ARG
        assert "budget" in F.flood_last_error(None)


def test_create_rejects_bad_friction_and_unsupported_kernels():
    import paper_2204_10323_gb300 as F
    for bad in (-1, 2, 7):
        o = F.default_opts()
        o.friction = bad
        st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
        assert st == F.ERR_ARG and "friction" in F.flood_last_error(None)
    for kernel in (F.KERNEL_ROWS,):
        o = F.default_opts()
        o.friction = 1
        o.kernel = kernel
        st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
        assert st == F.ERR_UNSUPPORTED and "friction" in F.flood_last_error(None)


def test_create_rejects_theta_out_of_range_and_unsupported_kernels():
    import paper_2204_10323_gb300 as F
    for bad in (0.0, -0.5, 1.5, float("nan")):
        o = F.default_opts()
        o.theta = bad
        st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
        assert st == F.ERR_ARG and "theta" in F.flood_last_error(None)
    for kernel in (F.KERNEL_ROWS,):
        o = F.default_opts()
        o.theta = 0.8
        o.kernel = kernel
        st, _ = _create(_grid(8, 8), np.zeros(64, np.float32), opts=o)
        assert st == F.ERR_UNSUPPORTED and "theta" in F.flood_last_error(None)


def test_header_is_plain_c(tmp_path):
    """include/flood.h compiles as ISO C99 with warnings as errors (no C++ or
    torch types in the boundary), and as C++17."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    for compiler, std, name in (("gcc", "-std=c99", "t.c"), ("g++", "-std=c++17", "t.cpp")):
        src = tmp_path / name
        src.write_text('#include "flood.h"\nint main(void) { return (int)sizeof(flood_opts) > 0 ? 0 : 1; }\n')
        r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-I",
                            os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    """A C program (no Python, no torch headers) links libflood_gb300.so and calls
    entry points that need no device: the version string, the default options
    and the adjoint's checkpoint plan (2000 steps, 40 snapshots: 5097 replays)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    import paper_2204_10323_gb300 as F
    so = F.lib()._name
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include "flood.h"
int main(void)
{
    flood_opts o;
    int64_t fwd = 0, launches = 0;
    int32_t in_order = 0;
    flood_default_opts(&o);
    if (flood_revolve_plan(2000, 40, o.epoch_steps, 0, 4, &fwd, &launches, &in_order) != FLOOD_OK) return 1;
    printf("%s|%d|%lld|%d\n", flood_version(), o.epoch_steps, (long long)fwd, (int)in_order);
    return 0;
}
''')
    exe = tmp_path / "use"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), so,
                        "-Wl,-rpath," + os.path.dirname(so), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    version, E, fwd, in_order = r.stdout.strip().split("|")
    assert "sm_103a" in version and E == "16" and fwd == "5097" and in_order == "1"
