"""Seeded synthetic inputs for the inundation-model workloads.

This package builds terrain (DEM) grids, Manning roughness fields, inflow
hydrograph tables, boundary-section descriptions and initial states.  It is the
one module shared by the CPU oracle's tests and the GPU library's tests and
benchmark, so it holds none of the method's arithmetic: no face-discharge
update, no depth update, no Manning boundary solve, no time-step rule.

The Arkansas River 3DEP DEM used by the paper (Methods, "Data") is not
available, so every workload is synthetic: fractal terrain with a carved,
monotone-bed meandering channel stands in for the river valley, with grid
sizes spanning the paper's 8 m (15.5 M cells) to 2 m (248 M cells) runs
(Table 1).  Seeds are ``SEED_BASE + workload id (+ scenario index)`` with
NumPy's PCG64 generator.

Layout convention (shared by the oracle and the library): row-major, x
fastest; cell (i, j) is ``a[j, i]`` with i in [0, nx), j in [0, ny); the x-face
array ``qx`` has shape (ny, nx + 1) with ``qx[j, i]`` the west face of cell i;
the y-face array ``qy`` has shape (ny + 1, nx) with ``qy[j, i]`` the south face
of cell (i, j).  Units are SI; face fluxes are per unit width (m^2/s).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 2204_10323

XMIN, XMAX, YMIN, YMAX = 0, 1, 2, 3          # BoundarySide (Appendix, "Inputs")
SIDE_NAMES = {"xmin": XMIN, "xmax": XMAX, "ymin": YMIN, "ymax": YMAX}
INFLOW, OUTFLOW = 0, 1


@dataclasses.dataclass
class Section:
    """One boundary section: a contiguous run of cells along one side.

    ``frac_start``/``frac_end`` follow the paper's fraction_start/fraction_end
    inputs (Appendix, "Inputs"); the covered cells along a side of L cells are
    ``[floor(frac_start*L + 0.5), floor(frac_end*L + 0.5))``.  ``kind`` is
    INFLOW (hydrograph ``t_s``/``q_m3s`` in m^3/s, slope S_in) or OUTFLOW
    (slope S_out).
    """
    side: int
    frac_start: float
    frac_end: float
    kind: int
    slope: float
    t_s: Optional[np.ndarray] = None
    q_m3s: Optional[np.ndarray] = None

    @staticmethod
    def cells(side: int, i0: int, i1: int, kind: int, slope: float, nx: int, ny: int,
              t_s=None, q_m3s=None) -> "Section":
        L = ny if side in (XMIN, XMAX) else nx
        return Section(side, i0 / L, i1 / L, kind, slope,
                       None if t_s is None else np.asarray(t_s, np.float64),
                       None if q_m3s is None else np.asarray(q_m3s, np.float64))


@dataclasses.dataclass
class Options:
    g: float = 9.81
    h_dry: float = 1e-3
    cfl_alpha: float = 0.7
    dt_cap: float = 2.0
    dt_const: float = 0.1
    dt_mode: int = 0          # 0: CFL epochs, 1: constant dt
    epoch_steps: int = 16
    bc_form: int = 0          # 0: cross-section Manning, 1: literal A = dx^2
    theta: float = 1.0        # flux weighting: 1 = Eq. 3 as printed, < 1 de Almeida's theta scheme
    friction: int = 0         # |q| in friction: 0 the face's component, 1 vector norm with the orthogonal mean


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    dx: float
    z: np.ndarray             # (ny, nx) float64
    n: np.ndarray             # (ny, nx) float64
    sections: List[Section]
    opts: Options
    h0: Optional[np.ndarray] = None
    qx0: Optional[np.ndarray] = None
    qy0: Optional[np.ndarray] = None
    steps: int = 0
    gauges: Optional[np.ndarray] = None   # (G, 2) int: (i, j)

    def initial_state(self, dtype=np.float64):
        h = np.zeros((self.ny, self.nx), dtype) if self.h0 is None else self.h0.astype(dtype)
        qx = np.zeros((self.ny, self.nx + 1), dtype) if self.qx0 is None else self.qx0.astype(dtype)
        qy = np.zeros((self.ny + 1, self.nx), dtype) if self.qy0 is None else self.qy0.astype(dtype)
        return h, qx, qy


def rng_for(config_id: int, scenario: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + config_id + 1000 * scenario)


# --------------------------------------------------------------------------- terrain
def diamond_square(k: int, roughness: float, rng: np.random.Generator) -> np.ndarray:
    """Midpoint-displacement fractal on a (2^k+1)^2 grid.

    Corner seeds are U(0, 1); the displacement amplitude starts at 1 and is
    multiplied by ``roughness`` at every level (diamond then square step).
    """
    N = (1 << k) + 1
    a = np.zeros((N, N), np.float64)
    a[0, 0], a[0, -1], a[-1, 0], a[-1, -1] = rng.uniform(0.0, 1.0, 4)
    step, scale = N - 1, 1.0
    while step > 1:
        half = step // 2
        c = (a[0:-1:step, 0:-1:step] + a[0:-1:step, step::step]
             + a[step::step, 0:-1:step] + a[step::step, step::step]) * 0.25
        a[half::step, half::step] = c + scale * rng.uniform(-1.0, 1.0, c.shape)
        # square step, points on odd rows of the half lattice (rows half::step, cols 0::step)
        for r0, c0 in ((half, 0), (0, half)):
            rows = np.arange(r0, N, step)
            cols = np.arange(c0, N, step)
            s = np.zeros((rows.size, cols.size))
            cnt = np.zeros_like(s)
            for dr, dc in ((-half, 0), (half, 0), (0, -half), (0, half)):
                rr, cc = rows + dr, cols + dc
                okr, okc = (rr >= 0) & (rr < N), (cc >= 0) & (cc < N)
                blk = a[np.ix_(np.clip(rr, 0, N - 1), np.clip(cc, 0, N - 1))]
                m = okr[:, None] & okc[None, :]
                s += np.where(m, blk, 0.0)
                cnt += m
            a[np.ix_(rows, cols)] = s / cnt + scale * rng.uniform(-1.0, 1.0, s.shape)
        scale *= roughness
        step = half
    return a


def fractal_terrain(nx: int, ny: int, relief: float, rng, roughness: float = 0.6) -> np.ndarray:
    k = max(1, math.ceil(math.log2(max(nx, ny) - 1))) if max(nx, ny) > 2 else 1
    while (1 << k) + 1 < max(nx, ny):
        k += 1
    a = diamond_square(k, roughness, rng)[:ny, :nx]
    lo, hi = a.min(), a.max()
    return (a - lo) / (hi - lo) * relief


def meander_centre(nx: int, ny: int, amp1: float, amp2: float) -> np.ndarray:
    """Channel centreline y_c(i) in cells for each column i (cell centres)."""
    x = (np.arange(nx) + 0.5) / nx
    return ny / 2 + amp1 * ny * np.sin(2 * np.pi * x / 0.5) + amp2 * ny * np.sin(2 * np.pi * x / 0.17)


def carve_channel_x(z: np.ndarray, yc: np.ndarray, width: float, depth: float):
    """Cut a channel along x: bed = running minimum of (terrain at centre - depth).

    Returns (z_carved, channel_mask, bed_profile)."""
    ny, nx = z.shape
    jc = np.clip(np.floor(yc).astype(int), 0, ny - 1)
    bed = np.minimum.accumulate(z[jc, np.arange(nx)] - depth)
    jj = np.arange(ny)[:, None] + 0.5
    mask = np.abs(jj - yc[None, :]) < width / 2
    zc = np.where(mask, np.minimum(z, bed[None, :]), z)
    return zc, mask, bed


def carve_channel_y(z: np.ndarray, xc: np.ndarray, width: float, depth: float, j_end: np.ndarray):
    """Cut a tributary along +y for rows j < j_end[i-range] (running-minimum bed)."""
    ny, nx = z.shape
    ic = np.clip(np.floor(xc).astype(int), 0, nx - 1)
    bed = np.minimum.accumulate(z[np.arange(ny), ic] - depth)
    ii = np.arange(nx)[None, :] + 0.5
    mask = (np.abs(ii - xc[:, None]) < width / 2) & (np.arange(ny)[:, None] < j_end)
    zc = np.where(mask, np.minimum(z, bed[:, None]), z)
    return zc, mask


def gaussian_random_field(nx: int, ny: int, sigma_cells: float, rng) -> np.ndarray:
    """Unit-variance smooth field: white noise convolved with a Gaussian (periodic)."""
    from scipy.ndimage import gaussian_filter
    w = rng.standard_normal((ny, nx))
    f = gaussian_filter(w, sigma_cells, mode="wrap")
    f -= f.mean()
    return f / f.std()


def triangle_hydrograph(peak: float, T: float):
    return np.array([0.0, T / 3.0, T]), np.array([0.0, peak, 0.0])


def bed_slope(bed: np.ndarray, dx: float, first: bool, span: int = 64) -> float:
    span = min(span, bed.size - 1)
    seg = bed[:span + 1] if first else bed[-span - 1:]
    return max(float(seg[0] - seg[-1]) / (span * dx), 1e-4)


def wet_start(z: np.ndarray, dx: float, wet_fraction: float, tilt: float = 1e-4):
    """Initial depth with a gently tilted water surface wetting ``wet_fraction`` of cells."""
    ny, nx = z.shape
    xm = (np.arange(nx) + 0.5) * dx
    key = z + tilt * xm[None, :]
    c = np.quantile(key[:: max(1, ny // 512), :: max(1, nx // 512)], wet_fraction)
    return np.maximum(c - tilt * xm[None, :] - z, 0.0)


# --------------------------------------------------------------------------- workloads
def c1_tilted_channel(steps: int = 1000) -> Problem:
    """128^2, 10 m cells: tilted plane, sinusoidal 3 m channel, +-0.1 m noise, 50 m^3/s."""
    nx = ny = 128
    dx = 10.0
    rng = rng_for(1)
    xm = (np.arange(nx) + 0.5) * dx
    z = np.broadcast_to(100.0 - 1e-3 * xm, (ny, nx)).copy()
    yc = 64 + 16 * np.sin(2 * np.pi * xm / 1280.0)
    jj = np.arange(ny)[:, None] + 0.5
    chan = np.abs(jj - yc[None, :]) < 4
    z = z - 3.0 * chan + rng.uniform(-0.1, 0.1, (ny, nx))
    n = np.full((ny, nx), 0.03)
    rows = np.nonzero(chan[:, 0])[0]
    j0, j1 = int(rows.min()) - 2, int(rows.max()) + 3
    T = steps * 2.0
    secs = [Section.cells(XMIN, j0, j1, INFLOW, 1e-3, nx, ny, [0.0, T], [50.0, 50.0]),
            Section.cells(XMAX, 0, ny, OUTFLOW, 1e-3, nx, ny)]
    return Problem("c1_tilted_channel_128", nx, ny, dx, z, n, secs,
                   Options(dt_cap=2.0, epoch_steps=16), steps=steps)


def _fractal_channel(nx, ny, dx, rng, relief=40.0, width_m=120.0, depth=4.0):
    z = fractal_terrain(nx, ny, relief, rng)
    yc = meander_centre(nx, ny, 200.0 / 2048.0, 80.0 / 2048.0)
    z, mask, bed = carve_channel_x(z, yc, width_m / dx, depth)
    return z, mask, bed, yc


def c2_fractal(nx: int = 2048, ny: int = 2048, dx: float = 5.0, steps: int = 20000,
               config_id: int = 2, peak: float = 800.0, dt_cap: float = 0.5) -> Problem:
    """Fractal terrain (roughness 0.6, 40 m relief) + carved 4 m meandering channel."""
    rng = rng_for(config_id)
    z, mask, bed, yc = _fractal_channel(nx, ny, dx, rng)
    n = np.where(mask, 0.035, 0.06)
    T = steps * dt_cap
    t, q = triangle_hydrograph(peak, T)
    rows = np.nonzero(mask[:, 0])[0]
    j0, j1 = max(int(rows.min()) - 4, 0), min(int(rows.max()) + 5, ny)
    secs = [Section.cells(XMIN, j0, j1, INFLOW, bed_slope(bed, dx, True), nx, ny, t, q),
            Section.cells(XMAX, 0, ny, OUTFLOW, bed_slope(bed, dx, False), nx, ny)]
    return Problem(f"c2_fractal_{nx}x{ny}", nx, ny, dx, z, n, secs,
                   Options(dt_cap=dt_cap, epoch_steps=16), steps=steps)


def c3_large(nx: int = 16384, ny: int = 16384, dx: float = 1.0, steps: int = 5000,
             wet_fraction: float = 0.3) -> Problem:
    """Large fractal grid with main channel at xmin and a tributary at ymin (two inflows)."""
    rng = rng_for(3)
    z, mask, bed, yc = _fractal_channel(nx, ny, dx, rng)
    xt = nx / 3 + 0.05 * nx * np.sin(2 * np.pi * (np.arange(ny) + 0.5) / ny * 3)
    it = int(np.clip(xt[0], 0, nx - 1))
    j_end = int(np.clip(yc[it], 1, ny))
    z, tmask = carve_channel_y(z, xt, 120.0 / dx, 4.0, j_end)
    n = np.where(mask | tmask, 0.035, 0.06)
    T = steps * 0.1
    t, q = triangle_hydrograph(400.0, T)
    rows = np.nonzero(mask[:, 0])[0]
    j0, j1 = max(int(rows.min()) - 4, 0), min(int(rows.max()) + 5, ny)
    cols = np.nonzero(tmask[0, :])[0]
    i0, i1 = max(int(cols.min()) - 4, 0), min(int(cols.max()) + 5, nx)
    s_trib = max(float(z[0, it] - z[min(63, ny - 1), it]) / (63 * dx), 1e-4)
    secs = [Section.cells(XMIN, j0, j1, INFLOW, bed_slope(bed, dx, True), nx, ny, t, q),
            Section.cells(YMIN, i0, i1, INFLOW, s_trib, nx, ny, t, q),
            Section.cells(XMAX, 0, ny, OUTFLOW, bed_slope(bed, dx, False), nx, ny)]
    h0 = wet_start(z, dx, wet_fraction) if wet_fraction > 0 else None
    return Problem(f"c3_fractal_{nx}x{ny}", nx, ny, dx, z, n, secs,
                   Options(dt_cap=0.1, epoch_steps=16), h0=h0, steps=steps)


ENSEMBLE_SHAPES = [(256, 256), (512, 512), (1024, 1024), (1536, 1024), (2048, 2048)]


def c4_scenario(s: int, steps: int = 5000, shapes=None) -> Problem:
    """Ensemble scenario s: uneven grid, own fractal seed, scalar n, own hydrograph peak."""
    shapes = shapes or ENSEMBLE_SHAPES
    pick = rng_for(4, 0)
    idx = pick.integers(0, len(shapes), 4096)[s]
    nx, ny = shapes[idx]
    rng = rng_for(4, s + 1)
    dx = 5.0
    z, mask, bed, yc = _fractal_channel(nx, ny, dx, rng)
    nval = float(rng.uniform(0.02, 0.08))
    peak = float(rng.uniform(100.0, 1000.0))
    n = np.full((ny, nx), nval)
    T = steps * 0.5
    t, q = triangle_hydrograph(peak, T)
    rows = np.nonzero(mask[:, 0])[0]
    j0, j1 = max(int(rows.min()) - 4, 0), min(int(rows.max()) + 5, ny)
    secs = [Section.cells(XMIN, j0, j1, INFLOW, bed_slope(bed, dx, True), nx, ny, t, q),
            Section.cells(XMAX, 0, ny, OUTFLOW, bed_slope(bed, dx, False), nx, ny)]
    return Problem(f"c4_scenario_{s}_{nx}x{ny}", nx, ny, dx, z, n, secs,
                   Options(dt_cap=0.5, epoch_steps=16), steps=steps)


def c5_calibration(nx: int = 1024, ny: int = 1024, truth: bool = False, steps: int = 2000,
                   n_gauges: int = 16) -> Problem:
    """1024^2 fractal + channel with a smooth per-cell Manning field and 16 in-channel gauges."""
    rng = rng_for(5)
    dx = 5.0
    z, mask, bed, yc = _fractal_channel(nx, ny, dx, rng)
    grf_rng = rng_for(5, 1 if truth else 2)
    n = np.maximum(0.04 + 0.015 * gaussian_random_field(nx, ny, 24.0 * nx / 1024, grf_rng), 0.01)
    T = steps * 0.5
    t, q = triangle_hydrograph(600.0, T)
    rows = np.nonzero(mask[:, 0])[0]
    j0, j1 = max(int(rows.min()) - 4, 0), min(int(rows.max()) + 5, ny)
    secs = [Section.cells(XMIN, j0, j1, INFLOW, bed_slope(bed, dx, True), nx, ny, t, q),
            Section.cells(XMAX, 0, ny, OUTFLOW, bed_slope(bed, dx, False), nx, ny)]
    gi = np.round(np.linspace(2, min(nx - 3, 2 + steps // 8), n_gauges)).astype(int)
    gj = np.clip(np.floor(yc[gi]).astype(int), 0, ny - 1)
    # a fixed step: the gradient holds the time-step schedule fixed, so finite
    # differences of the loss are comparable only without the CFL rule
    return Problem(f"c5_calibration_{nx}x{ny}", nx, ny, dx, z, n, secs,
                   Options(dt_cap=0.5, dt_mode=1, dt_const=0.25, epoch_steps=16), steps=steps,
                   gauges=np.stack([gi, gj], 1))


# --------------------------------------------------------------------------- special cases
def lake_at_rest(nx: int, ny: int, seed: int = 7, eta0: float = 2.0) -> Problem:
    """Dyadic terrain (multiples of 2^-10 m, |z| < 64) and a flat dyadic water level."""
    rng = np.random.default_rng(SEED_BASE + seed)
    z = np.round(rng.uniform(0.0, 4.0, (ny, nx)) * 1024.0) / 1024.0
    h0 = np.maximum(eta0 - z, 0.0)
    return Problem(f"lake_{nx}x{ny}", nx, ny, 1.0, z, np.full((ny, nx), 0.03), [],
                   Options(dt_mode=1, dt_const=0.05), h0=h0)


def normal_depth_channel(nx: int = 96, ny: int = 8, dx: float = 10.0, S0: float = 1e-3,
                         n: float = 0.03, h_n: float = 1.0) -> Problem:
    """Straight channel with bed slope S0, walls on both sides, Manning inflow/outflow.

    The inflow discharge is chosen so that the Manning normal depth is ``h_n``:
    Q = W * dx * h_n^(5/3) * sqrt(S0) / n with W = ny cells.
    """
    xm = (np.arange(nx) + 0.5) * dx
    z = np.broadcast_to(10.0 - S0 * xm, (ny, nx)).copy()
    Q = ny * dx * h_n ** (5.0 / 3.0) * math.sqrt(S0) / n
    secs = [Section.cells(XMIN, 0, ny, INFLOW, S0, nx, ny, [0.0, 1e9], [Q, Q]),
            Section.cells(XMAX, 0, ny, OUTFLOW, S0, nx, ny)]
    return Problem(f"normal_depth_{nx}x{ny}", nx, ny, dx, z, np.full((ny, nx), n), secs,
                   Options(dt_mode=1, dt_const=1.0), h0=np.full((ny, nx), h_n))


def standing_wave(nx: int, ny: int, mx: int, my: int, H: float = 2.0, eps: float = 1e-7, dx: float = 1.5,
                  dt: float = 0.05, theta: float = 1.0, n: float = 0.0) -> Problem:
    """Closed basin, flat bed, Manning n (0: no friction), at rest: depth
    H + eps cos(kx x) cos(ky y) at the cell centres, kx = pi mx / (nx dx),
    ky = pi my / (ny dx) (the cosine modes that the walls admit), constant time
    step dt."""
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    mode = np.outer(np.cos(np.pi * my / (ny * dx) * yc), np.cos(np.pi * mx / (nx * dx) * xc))
    return Problem(f"standing_wave_{nx}x{ny}_{mx}_{my}", nx, ny, dx, np.zeros((ny, nx)), np.full((ny, nx), n), [],
                   Options(dt_mode=1, dt_const=dt, theta=theta), h0=H + eps * mode,
                   qx0=np.zeros((ny, nx + 1)), qy0=np.zeros((ny + 1, nx)))


def random_small(nx: int, ny: int, seed: int, wet: float = 0.5, inflow: float = 5.0,
                 bc_form: int = 0, dt_mode: int = 0) -> Problem:
    """Small seeded case with rough terrain, partial wetting and every boundary kind.

    Kept in the well-conditioned regime of the scheme (no depth clipping, a
    1e-15 perturbation stays below 1e-14 after 120 steps) so that it compares
    arithmetic, not the amplification of rounding by an unstable run.
    """
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    dx = 2.0
    xm = (np.arange(nx) + 0.5) * dx
    z = 5.0 - 0.01 * xm[None, :] + rng.uniform(-0.05, 0.05, (ny, nx))
    h0 = np.maximum(wet_start(z, dx, wet, 1e-3) * rng.uniform(0.5, 1.0, (ny, nx)), 0.0)
    n = rng.uniform(0.02, 0.06, (ny, nx))
    qx0 = rng.uniform(-0.01, 0.01, (ny, nx + 1))
    qy0 = rng.uniform(-0.01, 0.01, (ny + 1, nx))
    qx0[:, 0] = qx0[:, -1] = 0.0
    qy0[0, :] = qy0[-1, :] = 0.0
    a, b = ny // 4, max(ny // 4 + 1, 3 * ny // 4)
    c, d = nx // 3, max(nx // 3 + 1, 2 * nx // 3)
    secs = [Section.cells(XMIN, a, b, INFLOW, 2e-3, nx, ny, [0.0, 50.0, 200.0], [0.0, inflow, 0.5 * inflow]),
            Section.cells(YMAX, c, d, INFLOW, 1e-3, nx, ny, [0.0, 1e4], [0.3 * inflow, 0.3 * inflow]),
            Section.cells(XMAX, 0, ny, OUTFLOW, 2e-3, nx, ny),
            Section.cells(YMIN, 0, max(1, nx // 2), OUTFLOW, 1e-3, nx, ny)]
    return Problem(f"random_{nx}x{ny}_{seed}", nx, ny, dx, z, n, secs,
                   Options(dt_cap=0.2, epoch_steps=4, bc_form=bc_form, dt_mode=dt_mode, dt_const=0.1),
                   h0=h0, qx0=qx0, qy0=qy0)
