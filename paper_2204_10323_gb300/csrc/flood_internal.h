// flood_internal.h -- plain structs shared by the runtime (flood_api.cpp) and
// the CUDA kernels.  No PyTorch types; included by host C++ and by nvcc.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace flood {

constexpr int kMaxEpoch = 1024;       // largest E (steps per CFL epoch)
constexpr int kBcWall = 0, kBcInflow = 1, kBcOutflow = 2;
// An outflow face of a subdomain's halo row: its flux is computed like any
// outflow face but its volume is booked by the subdomain that owns the row.
constexpr int kBcOutflowHalo = 3;

// Device status bits (sticky, OR-ed by kernels).
constexpr int kStatusNonfinite = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusCfl = 4;          // an epoch's dt broke the Courant limit dx / sqrt(g h_max) at its end

// Device-resident control block of one simulation.
struct Ctrl {
    double t;                     // time at the start of the next step
    double dt;                    // time step of the current epoch
    double V_in, V_out, V_clip;   // cumulative volumes (m^3)
    double h_max;                 // depth maximum measured at the current epoch start
    double cfl_exceed;            // epochs whose dt broke dx / sqrt(g h_max) at their end
    unsigned long long hmax_bits; // running max of h (bits of a non-negative double)
    int status;                   // kStatus* bits
    int next_item;                // the temporal-blocking kernel's work-item counter (zeroed before each launch)
};

// One inflow section as seen by the Eq. 6 solver.
struct InflowSec {
    int ncell;                    // cells along the section
    int cell0;                    // offset into the section cell-index array
    int slot0;                    // first column of this section in the per-step flux rows
    int tab0, ntab;               // hydrograph table offset / length
    int side;                     // flood_side of the section
    double sqrtS;                 // sqrt(S_in)
};

// Geometry and physical constants (both precisions keep them in double here;
// kernels cast to their working type).
struct Geom {
    int nx, ny;
    int pitch;                    // elements per row of every grid array
    int bc_form;
    double dx, g, h_dry;
    float dx_f, h_dry_f;          // dx and h_dry rounded to FP32 once (the fast kernels' boundary faces)
    double theta;                 // face-flux weighting (1 = Eq. 3 as printed)
    int friction;                 // |q| of the friction term: 0 the face's own, 1 the vector norm
    double cfl_alpha, dt_cap, dt_const;
    int dt_mode, epoch_steps;
    int led_j0, led_j1;           // rows whose clipped volume and stored volume this grid books (all rows,
                                  // except for a subdomain of a decomposed grid: its own rows)
};

// Boundary description, one entry per boundary cell: sides laid out as
// [xmin: ny][xmax: ny][ymin: nx][ymax: nx].
struct Boundary {
    const int8_t *type;           // kBcWall / kBcInflow / kBcOutflow
    const int32_t *slot;          // inflow: column in the per-step inflow flux row
    const double *sqrtS;          // outflow: sqrt(S_out)
    const float *sqrtS_f;         // the same rounded to FP32 (fast kernels)
};

template <typename T>
struct StepArgs {
    Geom geo;
    const T *h, *qx, *qy, *z, *n;
    T *h_out, *qx_out, *qy_out;
    Boundary bc;
    const T *inflow_q;            // E x n_slots unit-width inflow fluxes (into the domain)
    int n_slots;
    const double *inflow_Q;       // E x n_inflow_sections discharges (for V_in)
    int n_inflow_sec;
    const double *t_list;         // E + 1 start times of the epoch's steps
    Ctrl *ctrl;
    int s;                        // step index inside the epoch (first step of the launch)
    int k_steps;                  // steps done by this launch (1 except the tiled kernel)
    int want_hmax;                // 1: record max depth after the launch's last step
    const int64_t *gauge_cells;   // flat j*nx+i; h after each step -> gauge_out
    int n_gauges;
    double *gauge_out;            // (k_steps) x n_gauges rows for this launch, or null
    int tile_x, tile_y;           // launch shape (stream/TMA: warps, rows; tiled: strips, rows per item)
};

// ---------------------------------------------------------------- launchers
// Each returns the cudaError_t of the launch.
template <typename T>
cudaError_t launch_step_reference(const StepArgs<T> &a, cudaStream_t st);
cudaError_t launch_step_rows(const StepArgs<float> &a, cudaStream_t st);
cudaError_t launch_step_stream(const StepArgs<float> &a, cudaStream_t st);
// Stream kernel over many grids: table of per-grid arguments (device), block
// prefix base[n+1] (device), one launch of total_blocks blocks.
// mode: the scheme options shared by every grid (bit 0 theta weighting, bit 1 vector-norm friction).
cudaError_t launch_step_stream_ensemble(const StepArgs<float> *table, const int *base, int n, int total_blocks,
                                        int warps, int rows, int step, int want_hmax, int mode, cudaStream_t st);
// Blocks of one grid for the stream kernel, and the (warps, rows) a tile pair selects.
int stream_blocks(const Geom &g, int warps, int rows);
cudaError_t launch_step_tma(const StepArgs<float> &a, cudaStream_t st);
// Temporal blocking over many grids: the (chunk, strip) items of grid k are
// base[k] .. base[k+1] - 1 (tiled_items per grid, table[k].tile_y rows per item), k_steps steps from s0.
int tiled_items(const Geom &g, int chunk_rows, int k_steps);
// next_item (device, zero before the launch): the pipelines take their items after
// the first from this counter (dynamic scheduling); null: block b takes b, b + grid, ...
cudaError_t launch_step_tiled_ensemble(const StepArgs<float> *table, const int *base, int n, int total_items,
                                       int k_steps, int s0, int want_hmax, int *next_item, int mode, cudaStream_t st);
void stream_launch_shape(const Geom &g, int tile_x, int tile_y, int *warps, int *rows);
cudaError_t launch_step_tiled(const StepArgs<float> &a, cudaStream_t st);

// Epoch start: choose dt from h_max (or constant, or fixed_dt[0] when given:
// the adjoint's replay of a logged epoch), fill t_list, reset the running
// maximum, count CFL exceedances, flag NaN/Inf.
cudaError_t launch_epoch_begin(const Geom &g, Ctrl *ctrl, double *t_list, int E, const double *fixed_dt,
                               cudaStream_t st);
// Decomposed grid: every part's running h_max (ctrls: n device pointers, on
// the device) set to the largest of them.
cudaError_t launch_hmax_allreduce(Ctrl *const *ctrls, int n, cudaStream_t st);
// Eq. 6 for every (step of the epoch, inflow section) pair.
template <typename T>
cudaError_t launch_inflow(const Geom &g, const InflowSec *secs, int nsec, const int64_t *sec_cells,
                          const int8_t *sec_side, const double *tab_t, const double *tab_q,
                          const T *z, const T *n, const double *t_list, int E, T *inflow_q,
                          int n_slots, double *inflow_Q, double *W_out, cudaStream_t st);
// Epoch bookkeeping of a batch of simulations in two launches: the time-step
// rule for each (one thread each), then Eq. 6 for every (step, section) task
// (task = {simulation, section}).
template <typename T>
struct EpochArgs {
    Geom geo;
    Ctrl *ctrl;
    double *t_list;
    const InflowSec *secs;
    int nsec;
    const int64_t *cells;
    const double *tab_t, *tab_q;
    const T *z, *n;
    T *inflow_q;
    int n_slots;
    double *inflow_Q, *inflow_W;
};
template <typename T>
cudaError_t launch_epoch_batched(const EpochArgs<T> *tab, int n, const int2 *tasks, int n_tasks, int E,
                                 cudaStream_t st);
// h_max of a state into ctrl->hmax_bits (max with what is there).
template <typename T>
cudaError_t launch_hmax(const Geom &g, const T *h, Ctrl *ctrl, cudaStream_t st);
// Block mean (f x f, partial blocks at the far edges) of a ny x nx field into ceil(ny/f) x ceil(nx/f).
template <typename T>
cudaError_t launch_coarsen(const T *src, int nx, int ny, int f, T *dst, cudaStream_t st);
// OR of "some element is NaN or Inf" over rows x cols of a pitched array into *flag (device).
template <typename T>
cudaError_t launch_nonfinite(const T *a, int rows, int cols, int pitch, int *flag, cudaStream_t st);
// Deterministic two-pass sum of h * dx^2 into *out (double, device).
template <typename T>
cudaError_t launch_volume(const Geom &g, const T *h, double *partials, int n_partials, double *out,
                          cudaStream_t st);
// ---------------------------------------------------------------- adjoint
// Buffers of one reverse step (all pitched like the state; gn in double).
template <typename T>
struct AdjArgs {
    StepArgs<T> fwd;              // forward state x_k (h, qx, qy, z, n), BCs, inflow row, ctrl (dt)
    const T *lh, *lqx, *lqy;      // adjoint of x_{k+1}
    T *lh_out, *lqx_out, *lqy_out;   // adjoint of x_k
    T *lhu;                       // scratch: adjoint of the unclipped depth
    double *gn;                   // dL/dn accumulator
    const InflowSec *secs;        // inflow sections (for the Eq. 6 derivative)
    const int64_t *sec_cells;
    const double *inflow_W;       // E x n_sec levels of this epoch
    const int64_t *gauge_cells;   // flat j*nx+i of the loss's gauges
    int n_gauges;
    const double *seed;           // dL/d(depth at gauge g after this step), n_gauges values (device)
    T *scratch;                   // scheme options only: 11 planes of pitch x (ny + 1) elements (face
                                  // contributions of both axes and the clip mask); null otherwise
    double *gn_in;                // FP32, Eq. 3 as printed: the inflow sections' dL/dn terms per section cell
                                  // (index cell0 + c), summed over the sweep, added to gn after it
                                  // (launch_gn_inflow_add); null: added to gn by each step
};
template <typename T>
cudaError_t launch_adjoint_step(const AdjArgs<T> &a, cudaStream_t st);
// 2D tensor map (a CUtensorMap, 64-byte aligned storage at map) of a pitched FP32
// field of width x height elements and a row pitch of `pitch` elements, for boxes
// of box_w x box_h elements; elements outside the field read as zeros.
cudaError_t encode_map_f32(void *map, const float *base, int width, int height, int pitch, int box_w, int box_h);
// dst (pitched, precision T) = gn (pitched doubles).
template <typename T>
cudaError_t launch_gn_out(const Geom &g, const double *gn, T *dst, cudaStream_t st);
// gn[sec_cells[c]] += gn_in[c] for c = 0 .. n_cells - 1, in that order.
cudaError_t launch_gn_inflow_add(double *gn, const double *gn_in, const int64_t *sec_cells, int n_cells,
                                 cudaStream_t st);

// Pitch padding (columns [cols, pitch) of rows x pitch elements of esz bytes):
// fill with the poison pattern, or count the elements whose bits differ from it.
cudaError_t launch_padding(void *a, size_t esz, int rows, int cols, int pitch, bool fill,
                           unsigned long long *count, cudaStream_t st);

// One thread waits budget_ns of device time on an mbarrier nothing arrives at;
// *gave_up (device) = 1 when the bounded wait gave up (the expected outcome).
cudaError_t launch_wait_probe(uint64_t budget_ns, int *gave_up, cudaStream_t st);

// Gather h at gauge cells into out[0..G).
template <typename T>
cudaError_t launch_gauges(const Geom &g, const T *h, const int64_t *cells, int G, double *out,
                          cudaStream_t st);

}  // namespace flood
