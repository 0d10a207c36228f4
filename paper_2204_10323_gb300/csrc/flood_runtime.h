// flood_runtime.h -- the handle behind the C ABI and the runtime's internal
// functions (host C++ only; uses no PyTorch types in its interface).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "flood.h"
#include "flood_internal.h"

#include <nvtx3/nvToolsExt.h>

struct flood_adjoint_state;   // adjoint work buffers (flood_adjoint.cpp)

struct flood_handle {
    flood::Geom geo{};
    int prec = 0;                 // flood_precision
    size_t esz = 4;               // bytes per grid element
    flood_opts opts{};
    int kernel = FLOOD_KERNEL_REFERENCE;
    int k_per_launch = 1;
    int tile_x = 0, tile_y = 0;   // stream kernel: warps per block, rows per chunk (0 = default)
    int device = 0;
    cudaStream_t stream = nullptr;

    // state (ping-pong) and static fields, pitched rows of geo.pitch elements
    void *h[2] = {nullptr, nullptr}, *qx[2] = {nullptr, nullptr}, *qy[2] = {nullptr, nullptr};
    int cur = 0;
    bool in_ensemble = false;     // a member of an ensemble (whose launch tables fix each member's cur)
    void *z = nullptr, *n = nullptr;

    // boundary description and the per-epoch inflow solution
    int8_t *bc_type = nullptr;
    int32_t *bc_slot = nullptr;
    double *bc_sqrtS = nullptr;
    float *bc_sqrtS_f = nullptr;
    flood::InflowSec *secs_dev = nullptr;
    int n_in = 0, n_slots = 1;
    int64_t *sec_cells = nullptr;
    double *tab_t = nullptr, *tab_q = nullptr;
    void *inflow_q = nullptr;     // E x n_slots
    double *inflow_Q = nullptr;   // E x n_in
    double *inflow_W = nullptr;   // E x n_in Eq. 6 water levels (for the adjoint)
    double *t_list = nullptr;     // E + 1
    flood::Ctrl *ctrl = nullptr;

    // reductions and gauges
    double *vol_partials = nullptr, *vol_out = nullptr;
    int *flag = nullptr;                  // device word for the non-finite check of flood_write_state
    int n_partials = 1024;
    int64_t *gauge_dev = nullptr;
    int gauge_cap = 0;
    double *gauge_buf = nullptr;
    size_t gauge_buf_cap = 0;

    int64_t step = 0;             // steps taken (host copy; defines the epoch position)
    int sticky = 0;               // flood_status of a sticky error
    std::string err;
    std::vector<void *> allocations;

    // captured epochs (use_graph): [parity of cur at the epoch start]
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};

    // subdomain of a decomposed grid (flood_decomp.cpp): the part's inflow sections are the whole
    // grid's, solved on copies of their cells' z and n; only part 0 books the inflow volume
    bool part = false;
    bool book_vin = true;
    void *sec_z = nullptr, *sec_n = nullptr;

    flood_adjoint_state *adj = nullptr;
    int64_t adj_forward_steps = 0;
    int adj_profile = 0;                      // flood_adjoint_profile
    double adj_prof_rev_ms = 0.0, adj_prof_fwd_ms = 0.0;
    int64_t adj_prof_rev_steps = 0, adj_prof_fwd_steps = 0;
};

namespace flood {

// One row strip of a grid decomposed into strips (flood_decomp.cpp): the part
// stores global rows [a, b) of a grid of ny_global rows and owns rows [y0, y1).
struct PartSpec {
    int ny_global;
    int a, b;
    int y0, y1;
    int index;                    // part number; part 0 books the inflow volume
};

// flood_create for a whole grid (part == nullptr) or for one part of it: dem and
// manning are the whole grid's host arrays, sections the whole grid's.
flood_status create_handle(const flood_grid *grid, const void *dem, const void *manning,
                           const flood_bc_section *sections, int32_t n_sections, const flood_opts *opts,
                           const PartSpec *part, flood_handle **out);
// Kernel family AUTO resolves to for a grid of nx x ny cells (flood_create's rule).
int auto_kernel(const flood_opts &o, int nx, int ny);
// Max of the depth over the rows [led_j0, led_j1) of the current state into the control block.
flood_status refresh_hmax_window(flood_handle *h);

// An NVTX range for the lifetime of the object: the runtime marks each stepping
// call, each epoch's bookkeeping, each adjoint sweep and each ensemble step, so
// a profiler's timeline shows them (no cost without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Every device allocation of the library (through PyTorch's caching allocator;
// NULL on failure, or when flood_debug_fail_alloc_after injects one).
void *raw_device_alloc(size_t bytes, cudaStream_t st);
void *dev_alloc(flood_handle *h, size_t bytes);
void dev_free(flood_handle *h, void *p);
flood_status fail(flood_handle *h, flood_status st, const std::string &msg);
flood_status cuda_fail(flood_handle *h, cudaError_t e, const char *where);

void section_range(const flood_bc_section &s, int nx, int ny, int *i0, int *i1);
size_t plane_elems(const flood_handle *h, int field);
void field_shape(const flood_handle *h, int field, int *rows, int *cols);
flood_status copy_in(flood_handle *h, void *dst_pitched, const void *src, int rows, int cols, int src_on_device);
flood_status copy_out(flood_handle *h, void *dst, const void *src_pitched, int rows, int cols, int dst_on_device);
flood_status refresh_hmax(flood_handle *h);
flood_status launch_inflow_epoch(flood_handle *h);
flood_status launch_steps(flood_handle *h, int s, int k, int want_hmax, const int64_t *gcells, int ng,
                          double *gout);
// One step at step-in-epoch s reading the state planes in[] = {h, qx, qy} and
// writing out[] (pitched like the handle's state; the handle's own buffers and
// its current index are not touched).
// k steps (k > 1: FP32, Eq. 3 as printed, at most 4 and within the epoch) from the planes `in`
// into the planes `out`, starting at step-in-epoch s.
flood_status launch_step_planes(flood_handle *h, int s, int k, const void *const in[3], void *const out[3]);
flood_status advance(flood_handle *h, int64_t n, const int64_t *gcells, int ng, double *gbuf,
                     const double *fixed_dt_log, bool epoch_open = false);
flood_status check_device_status(flood_handle *h);
StepArgs<float> step_args_f32(flood_handle *h, int s);
flood_status ensure_gauge_buffers(flood_handle *h, int ng, size_t n_values);

// CUDA-graph epochs (flood_graph.cpp)
flood_status advance_graph(flood_handle *h, int64_t n);
void invalidate_graphs(flood_handle *h);
void destroy_graphs(flood_handle *h);

// adjoint (flood_adjoint.cpp)
void destroy_adjoint(flood_handle *h);

}  // namespace flood
