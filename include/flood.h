/*
 * flood.h -- C ABI of the GB300 (sm_103a) local-inertial shallow-water
 * flood model of Pierce et al., "Accelerating Physics Simulations with TPUs:
 * An Inundation Modeling Example" (Methods, "Shallow Water Equations").
 *
 * One time step (Eq. 3-4 with the boundary conditions of Eq. 5-6):
 *   1. boundary faces: inflow sections get the Eq. 6 distribution of the
 *      hydrograph discharge Q_in(t), outflow sections the Eq. 5 discharge of
 *      each boundary cell, every other border face is a closed wall (q = 0);
 *   2. every interior face: q' = (q - g dt h_f (eta_R - eta_L)/dx)
 *                                / (1 + g dt n_f^2 |q| h_f^(-7/3))          (Eq. 3)
 *      with eta = h + z, h_f = max(eta_L, eta_R) - max(z_L, z_R),
 *      n_f = (n_L + n_R)/2, and q' = 0 when h_f <= h_dry;
 *   3. every cell: h' = h + dt ((qx_W - qx_E) + (qy_S - qy_N)) / dx       (Eq. 4)
 *      and h' < 0 is set to 0 with the removed volume booked as V_clip.
 * The time step is constant, or chosen every E steps by the CFL rule
 * dt = min(dt_cap, alpha dx / sqrt(g h_max)).
 *
 * Layout (device and host arrays alike): row-major, x fastest; cell (i, j)
 * at j*nx + i (host) for i < nx, j < ny.  Depth h, bed z and roughness n are
 * ny x nx; the x-face array qx is ny x (nx+1) with qx[j][i] the west face of
 * cell i; the y-face array qy is (ny+1) x nx with qy[j][i] the south face of
 * cell (i, j).  Face fluxes are per unit width (m^2/s), positive towards +x
 * or +y.  Element type of every grid array passed in or out: float for
 * FLOOD_F32 handles, double for FLOOD_F64 handles.  Hydrograph tables,
 * fractions, slopes and ledger values are always double.
 *
 * Every function returns a flood_status (0 = FLOOD_OK, < 0 = error) and never
 * aborts or traps.  Errors are sticky per handle: after FLOOD_ERR_NONFINITE,
 * FLOOD_ERR_CFL, FLOOD_ERR_CUDA or FLOOD_ERR_TIMEOUT, stepping calls return
 * FLOOD_ERR_STATE until flood_write_state() installs a new state.  The message of the last
 * error is available from flood_last_error().
 *
 * Memory and streams: the handle owns all device memory (taken from the
 * PyTorch CUDA caching allocator) and issues all work on the stream given in
 * flood_opts (or the current PyTorch stream of the current device at
 * creation).  Input arrays are copied at the call; output arrays are
 * caller-owned.  A handle must not be used by two threads at once; different
 * handles may be used from different threads.  The kernels' shared-memory
 * limits and occupancy figures are set up once per process, on the device of
 * the first launch: a process drives one GPU (one process per GPU, as under
 * torchrun).
 */
#ifndef FLOOD_H
#define FLOOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLOOD_OK = 0,
    FLOOD_ERR_ARG = -1,          /* invalid argument (sizes, pointers, options, sections) */
    FLOOD_ERR_OOM = -2,          /* device allocation failed */
    FLOOD_ERR_CUDA = -3,         /* a CUDA call or kernel launch failed */
    FLOOD_ERR_NONFINITE = -4,    /* NaN or Inf depth detected at an epoch start */
    FLOOD_ERR_CFL = -5,          /* an epoch ended with its dt above the Courant limit dx / sqrt(g h_max) of the
                                    depth it ended with (reported at the next epoch start, sticky; also counted
                                    in FLOOD_LEDGER_CFL_EXCEED) */
    FLOOD_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
    FLOOD_ERR_STATE = -7,        /* handle is in an error state */
    FLOOD_ERR_UNSUPPORTED = -8   /* option not available for this precision or size */
} flood_status;

typedef enum { FLOOD_F32 = 0, FLOOD_F64 = 1 } flood_precision;

/* BoundarySide and the inflow/outflow kinds (Appendix, "Inputs"; Methods). */
typedef enum { FLOOD_XMIN = 0, FLOOD_XMAX = 1, FLOOD_YMIN = 2, FLOOD_YMAX = 3 } flood_side;
typedef enum { FLOOD_INFLOW = 0, FLOOD_OUTFLOW = 1 } flood_bc_kind;

/* Grid: nx x ny square cells of size dx (m) (Appendix "Inputs": unpadded_dem, resolution). */
typedef struct {
    int32_t nx, ny;
    double dx;
    int32_t precision;           /* flood_precision */
} flood_grid;

/*
 * One boundary section (Methods, inflow/outflow boundary conditions): the
 * contiguous cells [floor(frac_start L + 1/2), floor(frac_end L + 1/2)) along
 * `side` (L = ny for x sides, nx for y sides).  Inflow sections carry the
 * hydrograph Q_in(t) (m^3/s) as n_pts points (t_s ascending), interpolated
 * linearly and held constant past both ends, and the channel slope S_in.
 * Outflow sections carry S_out.  Sections must not share a boundary face.
 * The tables are copied at flood_create.
 */
typedef struct {
    int32_t side;                /* flood_side */
    int32_t kind;                /* flood_bc_kind */
    double frac_start, frac_end;
    double slope;
    const double *t_s, *q_m3s;   /* inflow only; host arrays of n_pts */
    int32_t n_pts;
} flood_bc_section;

/* Kernel families for the forward step (FLOOD_F32; FLOOD_F64 always uses REFERENCE). */
typedef enum {
    FLOOD_KERNEL_AUTO = 0,       /* TILED (K = 4) with E a multiple of 4 and no launch shape given (Eq. 3
                                    as printed and the scheme options alike); else TMA below 2^27 cells,
                                    else STREAM */
    FLOOD_KERNEL_REFERENCE = 1,  /* one thread per cell, IEEE ops in the oracle's order */
    FLOOD_KERNEL_ROWS = 2,       /* one warp per 128-column strip, float4 row streaming */
    FLOOD_KERNEL_TILED = 3,      /* pipeline of K warps per strip, K steps per launch (temporal blocking) */
    FLOOD_KERNEL_STREAM = 4,     /* one warp per 128-column strip, rows staged by bulk copies (default) */
    FLOOD_KERNEL_TMA = 5         /* as STREAM, rows staged as 2D tiles by tensor-map (TMA) copies */
} flood_kernel;

typedef struct {
    double g;                    /* 9.81 m/s^2 */
    double h_dry;                /* dry-face threshold on h_f (m), 1e-3 */
    double cfl_alpha;            /* 0.7 */
    double dt_cap;               /* upper bound of the CFL time step (s) */
    double dt_const;             /* constant time step (s), the paper's 0.1 */
    int32_t dt_mode;             /* 0 CFL epochs, 1 constant dt */
    int32_t epoch_steps;         /* E: steps per CFL epoch (1..1024) */
    int32_t bc_form;             /* 0 cell discharge dx h^(5/3) sqrt(S)/n, 1 literal dx^2 h^(2/3) sqrt(S)/n */
    int32_t kernel;              /* flood_kernel */
    int32_t steps_per_launch;    /* K for FLOOD_KERNEL_TILED: 1..4 or 8, must divide E (0 = 4) */
    int32_t tile_x, tile_y;      /* launch shape, 0 = chosen by the library.  STREAM: warps per block (1..4),
                                    rows per chunk.  TILED: at most tile_x pipelines (blocks), tile_y rows
                                    per work item (a chunk of one 120-column strip).  Negative: invalid. */
    int32_t use_graph;           /* 1: replay whole epochs from a captured CUDA graph */
    void *stream;                /* cudaStream_t, NULL = current PyTorch stream */
    double theta;                /* face-flux weighting (default 1 = Eq. 3 as printed).  theta in (0, 1):
                                    the numerator discharge of a face is theta q + (1 - theta)/2 times the
                                    sum of its two neighbours along the same axis (the theta scheme of
                                    de Almeida et al. 2012, cited in Methods); friction keeps |q| of the
                                    face.  theta != 1: kernels REFERENCE, STREAM, TMA, TILED (AUTO) and
                                    FP64, ensembles, the adjoint; not ROWS (FLOOD_ERR_UNSUPPORTED) */
    int32_t friction;            /* |q| in the friction term of Eq. 3.  0 (default): the face's own discharge
                                    component (the axis-by-axis integration of Methods).  1: the vector norm
                                    sqrt(q^2 + qo^2), qo the mean of the four faces of the other axis around
                                    the face.  1: kernels REFERENCE, STREAM, TMA, TILED (AUTO) and FP64,
                                    ensembles, the adjoint; not ROWS (FLOOD_ERR_UNSUPPORTED); other values
                                    FLOOD_ERR_ARG */
} flood_opts;

typedef struct flood_handle flood_handle;

/* Fields for flood_read. */
typedef enum {
    FLOOD_FIELD_H = 0, FLOOD_FIELD_QX = 1, FLOOD_FIELD_QY = 2, FLOOD_FIELD_Z = 3,
    FLOOD_FIELD_N = 4,
    FLOOD_FIELD_LEDGER = 5       /* FLOOD_LEDGER_LEN doubles, see flood_ledger_index */
} flood_field;

/* Ledger entries (doubles) returned by flood_read(FLOOD_FIELD_LEDGER). */
typedef enum {
    FLOOD_LEDGER_T = 0,          /* simulated time (s) */
    FLOOD_LEDGER_DT = 1,         /* time step in force (s) */
    FLOOD_LEDGER_V_IN = 2,       /* cumulative inflow volume sum dt Q_in (m^3) */
    FLOOD_LEDGER_V_OUT = 3,      /* cumulative outflow volume (m^3) */
    FLOOD_LEDGER_V_CLIP = 4,     /* cumulative volume added by the depth clip (m^3) */
    FLOOD_LEDGER_VOLUME = 5,     /* stored volume sum h dx^2 now (m^3) */
    FLOOD_LEDGER_H_MAX = 6,      /* max depth at the last epoch start (m) */
    FLOOD_LEDGER_STEP = 7,       /* steps taken */
    FLOOD_LEDGER_CFL_EXCEED = 8, /* epochs whose dt exceeded dx/sqrt(g h_max) at their end */
    FLOOD_LEDGER_LEN = 9
} flood_ledger_index;

/* Fill *o with the defaults listed beside each flood_opts field. */
void flood_default_opts(flood_opts *o);

/*
 * Create a simulation (Appendix "Inputs"; Methods "Data": the DEM grid).
 * dem, manning: host arrays of ny*nx elements of the grid's precision; manning
 * may be NULL for a uniform n = 0.03.  sections: n_sections descriptors (may
 * be 0).  opts may be NULL for defaults.  The initial state is dry (h = q = 0)
 * at t = 0.  On success *out receives the handle; on failure *out is NULL and
 * the error text is available from flood_last_error(NULL).
 */
flood_status flood_create(const flood_grid *grid, const void *dem, const void *manning,
                          const flood_bc_section *sections, int32_t n_sections,
                          const flood_opts *opts, flood_handle **out);

/* Advance n_steps >= 0 steps (Eq. 3-6, the time-step rule).  Asynchronous on the
 * handle's stream: a NaN/Inf depth or a broken Courant limit found at an
 * epoch start is reported by the next flood_sync (flood_read of the ledger
 * still returns the ledger and makes the error sticky). */
flood_status flood_step(flood_handle *h, int64_t n_steps);

/* Wait for the handle's stream and return its sticky status.  No counterpart
 * in the paper (its run loop is synchronous): the point where asynchronous
 * errors of flood_step surface. */
flood_status flood_sync(flood_handle *h);

/*
 * Copy a field out: the intermediate outputs of the paper's run loop
 * (Appendix, "Code Structure": the simulation manager returns intermediate
 * states of the simulation) and the mass ledger (not in the paper; the
 * invariant of Eq. 4).  dst holds `bytes` bytes (must equal the field's size:
 * ny*nx, ny*(nx+1) or (ny+1)*nx elements, or FLOOD_LEDGER_LEN doubles);
 * dst_on_device != 0 means a device pointer on the handle's device.
 * Synchronous on the handle's stream.
 */
flood_status flood_read(flood_handle *h, int32_t field, void *dst, size_t bytes, int32_t dst_on_device);

/*
 * Install a state (Appendix, "Code Structure": the initial conditions the
 * simulation manager hands to the cores; also a resume from a checkpoint): depth
 * (ny*nx), qx (ny*(nx+1)) and qy ((ny+1)*nx), host or device (src_on_device).
 * qx or qy may be NULL for zero fluxes.  Host input holding NaN or Inf is
 * rejected (FLOOD_ERR_ARG) and the state stays as it was (the check runs on
 * the GPU on a staged copy); device input is taken as it is (a non-finite
 * depth is then reported at the next epoch start).  Clears an error state.
 * The time, step count and volumes are not changed (see flood_set_clock).
 */
flood_status flood_write_state(flood_handle *h, const void *depth, const void *qx, const void *qy,
                               int32_t src_on_device);

/*
 * Advance to the simulated time t_end (seconds, >= the current time): whole
 * steps while they end at or before t_end, then one step shortened to end
 * exactly at t_end (the run loop's final-step truncation, Results "Running
 * the Simulation"); the current CFL epoch keeps its time step for the steps
 * after it.  *steps_taken (may be NULL) gets the number of steps.
 * FLOOD_ERR_ARG if t_end is not finite or lies before the current time.
 * Synchronous on the handle's stream.
 */
flood_status flood_advance(flood_handle *h, double t_end, int64_t *steps_taken);

/* Set time, step count and cumulative volumes (a checkpoint's ledger).  The
 * next step starts a new CFL epoch when step % E == 0. */
flood_status flood_set_clock(flood_handle *h, double t, int64_t step, double dt, double v_in,
                             double v_out, double v_clip);

/* Replace the per-cell Manning field (ny*nx, host or device). */
flood_status flood_set_manning(flood_handle *h, const void *manning, int32_t src_on_device);

/*
 * Advance n_steps and record the depth at n_gauges gauge cells after every
 * step: out[k*n_gauges + g] = h(gauge g) after step k, as doubles.  gauge_cells
 * are flat cell indices j*nx + i (host array).  out is host or device memory.
 */
flood_status flood_run_gauges(flood_handle *h, int64_t n_steps, const int64_t *gauge_cells,
                              int32_t n_gauges, double *out, int32_t out_on_device);

/*
 * Reverse-mode gradient (not in the paper; for the calibration use it names as
 * future work) of L = sum_k sum_g dLdh[k*n_gauges+g] * h_g(after step k) over
 * the next n_steps steps from the current state, with the time-step schedule
 * held fixed (chosen by the forward sweep).  Binomial checkpointing keeps at
 * most n_checkpoints states on the device (>= 1; 0: as many as half the free
 * device memory holds, up to n_steps, where every state is kept and no step is
 * replayed twice; the count is halved while that allocation fails).  The
 * snapshots and scratch return to the PyTorch caching allocator when the call
 * ends, which keeps them reserved for later allocations of the process
 * (torch.cuda.empty_cache() hands them back to the CUDA driver).  dLdh: host doubles.
 * dLdn_out: ny*nx elements of the grid's precision, host (out_on_device = 0)
 * or device.  dLdh0_out: optional (NULL) gradient with respect to the
 * starting depth.  The handle's state, clock and ledger are unchanged.
 * Branch conventions at non-smooth points: max() sends its derivative to the
 * lower-index cell on ties, d|q|/dq = 0 at q = 0 (for the vector norm the
 * derivative of |q| is 0 where |q| = 0), and the dry-face test, the outflow
 * dry test and the depth clip are held as constant masks; the Eq. 6 inflow
 * level is differentiated exactly (implicit function theorem).  With theta
 * weighting or vector-norm friction the reverse step runs as three passes
 * over global memory (11 scratch planes of the grid's size).
 */
flood_status flood_adjoint(flood_handle *h, int64_t n_steps, const int64_t *gauge_cells,
                           int32_t n_gauges, const double *dLdh, int32_t n_checkpoints,
                           void *dLdn_out, void *dLdh0_out, int32_t out_on_device);

/* Number of forward steps the last flood_adjoint call recomputed (revolve cost). */
int64_t flood_adjoint_forward_steps(const flood_handle *h);

/*
 * The checkpoint schedule of flood_adjoint without a grid or a device (not in
 * the paper; host only, runs without a GPU): the same binomial (revolve)
 * recursion reverses n_steps steps (1 .. 10^6) with min(n_checkpoints,
 * n_steps) snapshot slots (n_checkpoints >= 1; slot 0 holds the start
 * state), starting at global step start_step >= 0 of epochs of epoch_steps
 * steps, with replay launches of up to steps_per_replay steps that never
 * cross an epoch end (flood_adjoint uses 4 for FP32 grids with Eq. 3 as
 * printed, else 1).  Outputs: *forward_steps the steps replayed (what
 * flood_adjoint_forward_steps reports after the same sweep), *replay_launches
 * the launches they take, *in_order 1 if the steps were reversed exactly
 * from n_steps - 1 down to 0 with every snapshot slot free again at the end,
 * else 0.  A restore that would read a snapshot holding another step returns
 * FLOOD_ERR_STATE (flood_adjoint makes the same check).  FLOOD_ERR_ARG for
 * arguments out of range or NULL outputs.
 */
flood_status flood_revolve_plan(int64_t n_steps, int32_t n_checkpoints, int32_t epoch_steps,
                                int64_t start_step, int32_t steps_per_replay, int64_t *forward_steps,
                                int64_t *replay_launches, int32_t *in_order);

/* Profiling of flood_adjoint (off by default): when enabled, the next calls
 * bracket every reverse step and every forward replay with CUDA events, and
 * flood_adjoint_times reports their summed device time (ms) and counts. */
flood_status flood_adjoint_profile(flood_handle *h, int32_t enable);
flood_status flood_adjoint_times(const flood_handle *h, double *reverse_ms, int64_t *reverse_steps,
                                 double *forward_ms, int64_t *forward_steps);

/* Release all device memory of the handle (NULL is accepted).  Not in the
 * paper: resource management of this library. */
flood_status flood_destroy(flood_handle *h);

/* Text of the handle's last error ("" if none); with NULL, the calling thread's
 * last flood_create error.  Not in the paper: error reporting of this library. */
const char *flood_last_error(const flood_handle *h);

/*
 * Ensembles (not in the paper; its scenario sweeps over discharges, dam
 * release policies and climate scenarios are the use): n independent FP32
 * scenarios, each with its own grid, DEM, Manning field and boundary
 * sections (arguments as for flood_create, element k of each array), advanced
 * together: one step of the stream kernel over all their blocks per launch,
 * largest grid first (default), or, after flood_ensemble_set_kernel(TILED, K),
 * K steps of the temporal-blocking kernel over their (chunk, strip) items, the
 * scenarios in two groups of about equal cells, each group launching (and
 * starting its scenarios' epochs) on a stream of its own created here.  Each
 * scenario keeps its own CFL time step, Eq. 6 inflow and ledger.  Whole epochs
 * are captured once into a CUDA graph (steps_per_graph steps, a multiple of
 * epoch_steps) and replayed.  opts applies to every scenario (kernel and
 * use_graph are set by the ensemble; theta and friction apply to every
 * scenario); the scenarios share its stream, and flood_ensemble_step returns
 * with that stream waiting for both groups.  flood_ensemble_member returns
 * scenario k's handle for flood_read / flood_write_state / flood_set_clock
 * (do not destroy it or step it alone).  Errors: flood_ensemble_last_error.
 */
typedef struct flood_ensemble flood_ensemble;
flood_status flood_ensemble_create(int32_t n, const flood_grid *grids, const void *const *dems,
                                   const void *const *mannings, const flood_bc_section *const *sections,
                                   const int32_t *n_sections, const flood_opts *opts, flood_ensemble **out);
/* Launch shape: warps per block (1..4, stream kernel), rows per chunk (stream
 * blocks; for the tiled kernel the rows per (chunk, strip) item of a grid of
 * 2^20 cells, scaled by sqrt(cells / 2^20) for the others, at least 32 and at
 * most the grid's rows: the largest grids come first with the longest items
 * and the small ones fill the end of the launch), steps per graph replay,
 * graph on/off.  FLOOD_ERR_ARG on values out of range. */
flood_status flood_ensemble_set_launch(flood_ensemble *e, int32_t warps, int32_t rows, int32_t steps_per_graph,
                                       int32_t use_graph);
/* Kernel for the steps: FLOOD_KERNEL_STREAM (one step per launch) or
 * FLOOD_KERNEL_TILED with steps_per_launch K (1..4 or 8, dividing epoch_steps;
 * 0 = 4), the temporal blocking of Eq. 3-4 over K steps per launch; a launch
 * never crosses an epoch end.  FLOOD_ERR_ARG otherwise.  Drops the captured
 * graphs.  No counterpart in the paper: a launch-configuration choice. */
flood_status flood_ensemble_set_kernel(flood_ensemble *e, int32_t kernel, int32_t steps_per_launch);
flood_status flood_ensemble_step(flood_ensemble *e, int64_t n_steps);
flood_handle *flood_ensemble_member(flood_ensemble *e, int32_t k);
flood_status flood_ensemble_destroy(flood_ensemble *e);
const char *flood_ensemble_last_error(const flood_ensemble *e);

/*
 * Coarsen a cell field (DEM, Manning n or depth; ny*nx, row-major, x fastest,
 * FLOOD_F32 or FLOOD_F64) by block averaging, the way the paper derives its
 * coarser grids from the 1 m DEM (Methods, "Data"): dst is ceil(ny/factor) x
 * ceil(nx/factor), cell (J, I) the mean of the input cells of block
 * [J*factor, (J+1)*factor) x [I*factor, (I+1)*factor) that lie in the grid.
 * src and dst are both host (on_device = 0) or both device memory on the
 * current device; stream NULL = PyTorch's current stream.  Synchronous.
 * FLOOD_ERR_ARG for NULL pointers or sizes below 1 (message:
 * flood_last_error(NULL)).
 */
flood_status flood_coarsen(int32_t precision, const void *src, int32_t nx, int32_t ny, int32_t factor, void *dst,
                           int32_t on_device, void *stream);

/*
 * Domain decomposition (Methods, "TPU Implementation": the grid is split into
 * subgrids, one per core, and the borders of the discharge and then of the
 * depth are exchanged between neighbouring subgrids every step; Results,
 * "Scaling on TPU": 1 x N strips need the fewest exchanges).  The grid's ny
 * rows are split into n_parts row strips of full width; part r owns rows
 * [y0_r, y1_r) and stores rows [a_r, b_r) = [y0_r - halo, y1_r + halo) cut to
 * the grid, i.e. `halo` rows of each neighbour.  After an exchange a part can
 * take `halo` steps alone: one step spoils one more row next to each cut end,
 * so after `halo` steps its own rows are still exactly what the whole grid
 * gives (the same arithmetic on the same inputs, bit for bit).  Then the
 * halo rows of h, qx and qy are copied in again from the neighbours' own rows.
 * At each CFL epoch start every part takes the largest of the parts' depth
 * maxima; the ledger is the sum of the parts' own terms (inflow volume, time
 * and step count from part 0).  Inflow sections crossing a cut are solved
 * whole by every part (Eq. 6 needs only the section cells' z and n, copied to
 * each part at creation), so every part's boundary fluxes are the grid's.
 */

/* Row split of a decomposition (no device work; safe without a GPU).
 * part_rows: 4*n_parts ints, for part r {y0, y1, a, b} (owned rows [y0, y1),
 * stored rows [a, b), global row numbers): y0 = floor(r ny / n_parts).
 * copies: the halo copies that refresh every part's halo rows, at most
 * 6*n_parts entries (*n_copies: capacity in, count out; copies may be NULL
 * to ask for the count).  Rows of h and qx are row numbers, rows of qy face-row
 * numbers, both local to the source and destination parts' stored rows.
 * FLOOD_ERR_ARG if n_parts < 1, halo < 1, or a strip would have fewer than
 * max(halo, 1) rows. */
typedef struct {
    int32_t field;               /* FLOOD_FIELD_H, FLOOD_FIELD_QX or FLOOD_FIELD_QY */
    int32_t src_part, src_row;   /* first row in the source part's stored rows */
    int32_t dst_part, dst_row;   /* first row in the destination part's stored rows */
    int32_t rows;                /* rows (face rows for qy) copied */
} flood_halo_copy;
flood_status flood_decomp_plan(int32_t ny, int32_t n_parts, int32_t halo, int32_t *part_rows,
                               flood_halo_copy *copies, int32_t *n_copies);

/* Ledger of a decomposed grid from its parts' ledgers (n_parts rows of
 * FLOOD_LEDGER_LEN doubles, each the part's own terms as flood_read returns
 * them for a part): volumes summed, h_max the largest, time, time step, step
 * count and CFL count from part 0.  FLOOD_ERR_STATE if the parts disagree on
 * time, time step or step count.  No device work; safe without a GPU. */
flood_status flood_decomp_combine_ledgers(int32_t n_parts, const double *part_ledgers, double *out);

/* Create a grid of n_parts row strips on the current device (arguments as
 * for flood_create, plus n_parts and halo >= 1, the steps between exchanges).
 * The parts run the kernel family that flood_create chooses for the whole
 * grid; FP64 grids use the reference kernel.  use_graph is ignored.  Each part
 * steps on a stream of its own (created here); flood_decomp_step,
 * flood_decomp_write_state and flood_decomp_read order the parts' work after
 * what the caller queued on opts->stream, and flood_decomp_step returns with
 * opts->stream waiting for every part.  Errors: flood_last_error(NULL). */
typedef struct flood_decomp flood_decomp;
flood_status flood_decomp_create(const flood_grid *grid, const void *dem, const void *manning,
                                 const flood_bc_section *sections, int32_t n_sections, const flood_opts *opts,
                                 int32_t n_parts, int32_t halo, flood_decomp **out);
/* Advance every part n_steps >= 0 steps (exchanges and epoch starts included). */
flood_status flood_decomp_step(flood_decomp *d, int64_t n_steps);
/* flood_read of the whole grid, assembled from the parts' own rows. */
flood_status flood_decomp_read(flood_decomp *d, int32_t field, void *dst, size_t bytes, int32_t dst_on_device);
/* flood_write_state of the whole grid: each part takes its stored rows. */
flood_status flood_decomp_write_state(flood_decomp *d, const void *depth, const void *qx, const void *qy,
                                      int32_t src_on_device);
/* flood_sync of every part. */
flood_status flood_decomp_sync(flood_decomp *d);
/* Part k's handle (stored rows only; for flood_read; stepping calls on it
 * return FLOOD_ERR_STATE), or NULL. */
flood_handle *flood_decomp_part(flood_decomp *d, int32_t k);
flood_status flood_decomp_destroy(flood_decomp *d);
const char *flood_decomp_last_error(const flood_decomp *d);

/*
 * Debugging aids for tests of the failure paths (not in the paper).
 *
 * flood_debug_fail_alloc_after(n): the device allocation the library makes
 * after n more successful ones (n = 0: the next one) fails as if the device
 * were out of memory, in any handle, ensemble or decomposition of the process;
 * the hook then turns itself off.  n < 0 turns it off.  Calls that hit it
 * return FLOOD_ERR_OOM and release what they had allocated.
 * flood_debug_alloc_count(): device allocations the library has made so far.
 *
 * flood_debug_padding(h, fill, bad): the pitch padding of the handle's grid
 * planes (both state buffers, z and n: the elements past each row's last
 * element up to the row pitch, which no kernel may write and whose values no
 * result may depend on).  fill != 0: set every padding element to a NaN with a
 * fixed bit pattern (note that flood_write_state without qx or qy zeroes those
 * planes whole).  fill == 0: *bad = the number of padding elements whose bits
 * differ from that pattern.  Synchronous.
 */
void flood_debug_fail_alloc_after(int64_t n);
int64_t flood_debug_alloc_count(void);
flood_status flood_debug_padding(flood_handle *h, int32_t fill, int64_t *bad);

/*
 * flood_debug_tiled_split: the work items the temporal-blocking kernel would
 * split an nx x ny grid into (host only, no device): k_steps 1..4 or 8, mode
 * bit 0 theta weighting and bit 1 vector-norm friction (they narrow the
 * strips), resident >= 1 the pipelines the GPU holds at once (912 on a GB300
 * for K = 4 as printed).  *chunk_rows the rows per item, *blocks the
 * pipelines launched, *n_items the (chunk, strip) items.  FLOOD_ERR_ARG (no
 * message) for arguments out of range, NULL outputs or more than 2^31 - 1
 * items.
 */
flood_status flood_debug_tiled_split(int32_t nx, int32_t ny, int32_t k_steps, int32_t mode, int32_t resident,
                                     int32_t *chunk_rows, int32_t *blocks, int32_t *n_items);

/* Library version string. */
const char *flood_version(void);

/*
 * Stored water volume sum(h) dx^2 of a caller-owned device depth array: ny
 * rows of row_pitch elements with nx used per row (float for FLOOD_F32,
 * double for FLOOD_F64), written as one double to out_device, asynchronously
 * on `stream` (NULL = the legacy default stream).  The paper has no
 * counterpart; this entry point is for callers that cannot allocate device
 * memory when they need the number: code inside a CUDA-graph capture region,
 * callers whose device memory all belongs to their own pool, and hosts that
 * forbid allocation after start-up.  It allocates nothing: its scratch is a
 * fixed device array of 65536 row sums (512 KiB) that every GPU loading the
 * library keeps until exit, so ny > 65536 returns FLOOD_ERR_ARG.  The first
 * call on each device (with that device current) looks up the scratch's
 * address; make that call outside any stream capture.  The address is kept
 * for the life of the process and does not survive cudaDeviceReset on that
 * device: do not call this entry point on a device after resetting it.  All calls on a device
 * share the scratch, which keeps the last call's row sums: calls whose kernels
 * overlap on the GPU race.  Errors: flood_last_error(NULL).
 */
flood_status flood_volume_noalloc(const void *depth, int32_t nx, int32_t ny, int64_t row_pitch,
                                  int32_t precision, double dx, double *out_device, void *stream);

/*
 * Failure-detection check of the bounded device waits that every kernel's
 * copy waits use: one thread waits on a shared-memory mbarrier that nothing
 * arrives at, for budget_s seconds of device time (0 < budget_s <= 10), then
 * gives up the way the step kernels do on a copy that never lands.  Returns
 * FLOOD_ERR_TIMEOUT when the wait gave up (the expected outcome; the CUDA
 * context stays usable), FLOOD_OK if it did not, FLOOD_ERR_ARG for a budget
 * out of range, FLOOD_ERR_CUDA on a CUDA error.  Synchronous, on the current
 * device's default stream; allocates and frees 4 bytes of device memory.
 */
flood_status flood_check_bounded_wait(double budget_s);

#ifdef __cplusplus
}
#endif

#endif /* FLOOD_H */
