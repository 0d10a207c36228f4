"""FP64 CPU oracle of the local-inertial shallow-water step (Eq. 3-6).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The GPU library never imports it.

``flood_oracle.c`` holds the arithmetic; this module compiles it with gcc
(``-O2 -ffp-contract=off``, OpenMP when available) into ``oracle/_build/`` and
marshals NumPy arrays to it through ctypes.  Arrays follow the layout of the
``inputs`` package: h, z, n are (ny, nx); qx is (ny, nx + 1); qy is (ny + 1, nx).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "flood_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libflood_oracle.so")


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("g", C.c_double),
                ("h_dry", C.c_double), ("cfl_alpha", C.c_double), ("dt_cap", C.c_double),
                ("dt_const", C.c_double), ("dt_mode", C.c_int32), ("epoch_steps", C.c_int32),
                ("bc_form", C.c_int32), ("theta", C.c_double), ("friction", C.c_int32)]


class SectionC(C.Structure):
    _fields_ = [("side", C.c_int32), ("kind", C.c_int32), ("frac_start", C.c_double),
                ("frac_end", C.c_double), ("slope", C.c_double),
                ("t_s", C.POINTER(C.c_double)), ("q_m3s", C.POINTER(C.c_double)),
                ("n_pts", C.c_int32)]


class Ledger(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("V_in", C.c_double),
                ("V_out", C.c_double), ("V_clip", C.c_double), ("step", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP contraction off); OpenMP if the compiler has it."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        L.orc_step.argtypes = [C.POINTER(Params), C.POINTER(SectionC), C.c_int32, dp, dp, dp, dp, dp,
                               C.c_double, C.c_double, C.POINTER(Ledger)]
        L.orc_step.restype = C.c_int
        L.orc_run.argtypes = [C.POINTER(Params), C.POINTER(SectionC), C.c_int32, dp, dp, dp, dp, dp,
                              C.c_int64, C.POINTER(Ledger), C.POINTER(C.c_int64), C.c_int32, dp, dp]
        L.orc_run.restype = C.c_int
        L.orc_advance.argtypes = [C.POINTER(Params), C.POINTER(SectionC), C.c_int32, dp, dp, dp, dp, dp,
                                  C.c_double, C.POINTER(Ledger), C.POINTER(C.c_int64)]
        L.orc_advance.restype = C.c_int
        L.orc_dt.argtypes = [C.POINTER(Params), dp]
        L.orc_dt.restype = C.c_double
        L.orc_volume.argtypes = [C.POINTER(Params), dp]
        L.orc_volume.restype = C.c_double
        L.orc_hydrograph.argtypes = [C.POINTER(SectionC), C.c_double]
        L.orc_hydrograph.restype = C.c_double
        L.orc_inflow_faces.argtypes = [C.POINTER(Params), C.POINTER(SectionC), dp, dp, C.c_double, dp]
        L.orc_inflow_faces.restype = C.c_double
        L.orc_section_range.argtypes = [C.POINTER(Params), C.POINTER(SectionC),
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_adjoint.argtypes = [C.POINTER(Params), C.POINTER(SectionC), C.c_int32, dp, dp, dp, dp, dp,
                                  C.POINTER(Ledger), C.c_int64, C.POINTER(C.c_int64), C.c_int32, dp,
                                  dp, dp, dp, dp]
        L.orc_adjoint.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


class Oracle:
    """FP64 state of one problem advanced by the C oracle."""

    def __init__(self, prob, h=None, qx=None, qy=None):
        self.prob = prob
        o = prob.opts
        self.params = Params(prob.nx, prob.ny, prob.dx, o.g, o.h_dry, o.cfl_alpha, o.dt_cap,
                             o.dt_const, o.dt_mode, o.epoch_steps, o.bc_form, getattr(o, "theta", 1.0),
                             getattr(o, "friction", 0))
        self.z = np.ascontiguousarray(prob.z, np.float64)
        self.n = np.ascontiguousarray(prob.n, np.float64)
        h0, qx0, qy0 = prob.initial_state(np.float64)
        self.h = np.ascontiguousarray(h0 if h is None else h, np.float64).copy()
        self.qx = np.ascontiguousarray(qx0 if qx is None else qx, np.float64).copy()
        self.qy = np.ascontiguousarray(qy0 if qy is None else qy, np.float64).copy()
        self._keep = []
        secs = (SectionC * max(1, len(prob.sections)))()
        for k, s in enumerate(prob.sections):
            t = np.ascontiguousarray(s.t_s if s.t_s is not None else np.zeros(0), np.float64)
            q = np.ascontiguousarray(s.q_m3s if s.q_m3s is not None else np.zeros(0), np.float64)
            self._keep += [t, q]
            secs[k] = SectionC(s.side, s.kind, s.frac_start, s.frac_end, s.slope, _dp(t), _dp(q), t.size)
        self.secs = secs
        self.nsec = len(prob.sections)
        self.ledger = Ledger(0.0, 0.0, 0.0, 0.0, 0.0, 0)

    # ------------------------------------------------------------------ forward
    def run(self, n_steps: int, gauges: Optional[np.ndarray] = None, dt_log: bool = False):
        """Advance n_steps; returns (gauge series (n_steps, G) or None, dt per step or None)."""
        L = lib()
        cells = None
        out = None
        G = 0
        if gauges is not None and len(gauges):
            cells = np.ascontiguousarray(gauges[:, 1].astype(np.int64) * self.prob.nx + gauges[:, 0], np.int64)
            G = cells.size
            out = np.zeros((n_steps, G), np.float64)
        dts = np.zeros(n_steps, np.float64) if dt_log else None
        rc = L.orc_run(C.byref(self.params), self.secs, self.nsec, _dp(self.z), _dp(self.n), _dp(self.h),
                       _dp(self.qx), _dp(self.qy), int(n_steps), C.byref(self.ledger),
                       None if cells is None else cells.ctypes.data_as(C.POINTER(C.c_int64)), G,
                       _dp(out), _dp(dts))
        if rc != 0:
            raise MemoryError("oracle work arrays")
        return out, dts

    def advance(self, t_end: float) -> int:
        """Advance to time t_end, the last step shortened to land on it (the run
        loop's final-step truncation); returns the number of steps."""
        k = C.c_int64(0)
        rc = lib().orc_advance(C.byref(self.params), self.secs, self.nsec, _dp(self.z), _dp(self.n),
                               _dp(self.h), _dp(self.qx), _dp(self.qy), float(t_end), C.byref(self.ledger),
                               C.byref(k))
        if rc == -2:
            raise ValueError("t_end is before the current time")
        if rc != 0:
            raise MemoryError("oracle work arrays")
        return int(k.value)

    def step_dt(self, dt: float) -> None:
        """One step with a given dt at the current time (does not touch the epoch counter)."""
        rc = lib().orc_step(C.byref(self.params), self.secs, self.nsec, _dp(self.z), _dp(self.n),
                            _dp(self.h), _dp(self.qx), _dp(self.qy), float(dt), self.ledger.t,
                            C.byref(self.ledger))
        if rc != 0:
            raise MemoryError("oracle work arrays")
        self.ledger.t += dt

    def dt(self) -> float:
        return lib().orc_dt(C.byref(self.params), _dp(self.h))

    def volume(self) -> float:
        return lib().orc_volume(C.byref(self.params), _dp(self.h))

    def section_range(self, k: int):
        a, b = C.c_int32(), C.c_int32()
        lib().orc_section_range(C.byref(self.params), C.byref(self.secs[k]), C.byref(a), C.byref(b))
        return a.value, b.value

    def hydrograph(self, k: int, t: float) -> float:
        return lib().orc_hydrograph(C.byref(self.secs[k]), float(t))

    def inflow_faces(self, k: int, Q: float):
        a, b = self.section_range(k)
        out = np.zeros(max(b - a, 1), np.float64)
        W = lib().orc_inflow_faces(C.byref(self.params), C.byref(self.secs[k]), _dp(self.z), _dp(self.n),
                                   float(Q), _dp(out))
        return W, out[: b - a]

    def ledger_dict(self):
        L = self.ledger
        return dict(t=L.t, dt=L.dt, V_in=L.V_in, V_out=L.V_out, V_clip=L.V_clip, step=L.step)

    # ------------------------------------------------------------------ adjoint
    def adjoint(self, n_steps: int, gauges: np.ndarray, dLdh: np.ndarray, n: Optional[np.ndarray] = None,
                want_state: bool = False):
        """dL/dn (and optionally dL/d(h0, qx0, qy0)) of sum_k,g dLdh[k,g] * h_g(after step k).

        Starts from the current state and ledger; the state is not modified."""
        nn = self.n if n is None else np.ascontiguousarray(n, np.float64)
        cells = np.ascontiguousarray(gauges[:, 1].astype(np.int64) * self.prob.nx + gauges[:, 0], np.int64)
        seed = np.ascontiguousarray(dLdh, np.float64)
        assert seed.shape == (n_steps, cells.size)
        gn = np.zeros_like(self.h)
        lh = np.zeros_like(self.h) if want_state else None
        lqx = np.zeros_like(self.qx) if want_state else None
        lqy = np.zeros_like(self.qy) if want_state else None
        rc = lib().orc_adjoint(C.byref(self.params), self.secs, self.nsec, _dp(self.z), _dp(nn),
                               _dp(self.h), _dp(self.qx), _dp(self.qy), C.byref(self.ledger), int(n_steps),
                               cells.ctypes.data_as(C.POINTER(C.c_int64)), cells.size, _dp(seed), _dp(gn),
                               _dp(lh), _dp(lqx), _dp(lqy))
        if rc != 0:
            raise MemoryError("oracle adjoint store")
        return (gn, lh, lqx, lqy) if want_state else gn

    def copy(self) -> "Oracle":
        o = Oracle(self.prob, self.h, self.qx, self.qy)
        o.ledger = Ledger(*[getattr(self.ledger, f) for f, _ in Ledger._fields_])
        return o
