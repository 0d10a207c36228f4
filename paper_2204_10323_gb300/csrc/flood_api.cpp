// flood_api.cpp -- the C ABI of include/flood.h: handle lifetime, device
// memory (PyTorch's CUDA caching allocator), streams, the epoch/step driver
// and host<->device copies.  All arithmetic of the method runs in the CUDA
// kernels declared in flood_internal.h.
#include "flood.h"

#include <c10/cuda/CUDACachingAllocator.h>
#include <c10/cuda/CUDAStream.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "flood_internal.h"
#include "flood_runtime.h"

using namespace flood;

namespace {

thread_local std::string g_create_error;

// Failure injection (flood_debug_fail_alloc_after): allocations left before the
// one that fails, -1 when off; and the number of allocations made so far.
std::atomic<int64_t> g_fail_countdown{-1};
std::atomic<int64_t> g_alloc_count{0};

}  // namespace

// ------------------------------------------------------------------ helpers
namespace flood {

void *raw_device_alloc(size_t bytes, cudaStream_t st)
{
    int64_t n = g_fail_countdown.load();
    while (n >= 0 && !g_fail_countdown.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 0) return nullptr;                 // the injected failure (the hook is now off)
    void *p = nullptr;
    try {
        p = c10::cuda::CUDACachingAllocator::raw_alloc_with_stream(bytes, st);
    } catch (...) {
        p = nullptr;
    }
    if (p) g_alloc_count++;
    return p;
}

void *dev_alloc(flood_handle *h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = raw_device_alloc(bytes, h->stream);
    if (p) h->allocations.push_back(p);
    return p;
}

void dev_free(flood_handle *h, void *p)
{
    if (!p) return;
    auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
    if (it != h->allocations.end()) h->allocations.erase(it);
    c10::cuda::CUDACachingAllocator::raw_delete(p);
}

flood_status fail(flood_handle *h, flood_status st, const std::string &msg)
{
    if (h) {
        h->err = msg;
        if (st == FLOOD_ERR_CUDA || st == FLOOD_ERR_NONFINITE || st == FLOOD_ERR_TIMEOUT || st == FLOOD_ERR_CFL)
            h->sticky = st;
    } else {
        g_create_error = msg;
    }
    return st;
}

flood_status cuda_fail(flood_handle *h, cudaError_t e, const char *where)
{
    return fail(h, FLOOD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace flood

#define CK(expr)                                                      \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr);        \
    } while (0)

extern "C" void flood_default_opts(flood_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->g = 9.81;
    o->h_dry = 1e-3;
    o->cfl_alpha = 0.7;
    o->dt_cap = 2.0;
    o->dt_const = 0.1;
    o->dt_mode = 0;
    o->epoch_steps = 16;
    o->bc_form = 0;
    o->kernel = FLOOD_KERNEL_AUTO;
    o->steps_per_launch = 0;
    o->tile_x = 0;
    o->tile_y = 0;
    o->use_graph = 0;
    o->stream = nullptr;
    o->theta = 1.0;
    o->friction = 0;
}

extern "C" flood_status flood_check_bounded_wait(double budget_s)
{
    if (!(budget_s > 0.0 && budget_s <= 10.0)) return fail(nullptr, FLOOD_ERR_ARG, "budget_s must lie in (0, 10]");
    int *d = nullptr;
    int gave_up = -1;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return fail(nullptr, FLOOD_ERR_CUDA, cudaGetErrorString(e));
    e = launch_wait_probe((uint64_t)(budget_s * 1e9), d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(&gave_up, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(nullptr, FLOOD_ERR_CUDA, cudaGetErrorString(e));
    if (gave_up == 1) return fail(nullptr, FLOOD_ERR_TIMEOUT, "the bounded wait gave up");
    return FLOOD_OK;
}

extern "C" const char *flood_version(void) { return "flood-gb300 0.1 (sm_103a)"; }

namespace flood {

// Cells [floor(fs L + 1/2), floor(fe L + 1/2)) along a side of L cells.
void section_range(const flood_bc_section &s, int nx, int ny, int *i0, int *i1)
{
    int L = (s.side == FLOOD_XMIN || s.side == FLOOD_XMAX) ? ny : nx;
    int a = (int)std::floor(s.frac_start * L + 0.5);
    int b = (int)std::floor(s.frac_end * L + 0.5);
    a = std::max(a, 0);
    b = std::min(b, L);
    b = std::max(b, a);
    *i0 = a;
    *i1 = b;
}

static int side_offset(int side, int nx, int ny)
{
    return side == FLOOD_XMIN ? 0 : side == FLOOD_XMAX ? ny : side == FLOOD_YMIN ? 2 * ny : 2 * ny + nx;
}

static int64_t side_cell_pitched(int side, int k, int nx, int ny, int pitch)
{
    int i, j;
    switch (side) {
    case FLOOD_XMIN: i = 0; j = k; break;
    case FLOOD_XMAX: i = nx - 1; j = k; break;
    case FLOOD_YMIN: i = k; j = 0; break;
    default: i = k; j = ny - 1; break;
    }
    return (int64_t)j * pitch + i;
}

size_t plane_elems(const flood_handle *h, int field)
{
    size_t P = (size_t)h->geo.pitch;
    return field == FLOOD_FIELD_QY ? P * (h->geo.ny + 1) : P * h->geo.ny;
}

// Host layout of a field: rows x cols.
void field_shape(const flood_handle *h, int field, int *rows, int *cols)
{
    *rows = h->geo.ny + (field == FLOOD_FIELD_QY ? 1 : 0);
    *cols = h->geo.nx + (field == FLOOD_FIELD_QX ? 1 : 0);
}

flood_status copy_in(flood_handle *h, void *dst_pitched, const void *src, int rows, int cols, int src_on_device)
{
    size_t e = h->esz;
    CK(cudaMemcpy2DAsync(dst_pitched, (size_t)h->geo.pitch * e, src, (size_t)cols * e, (size_t)cols * e, rows,
                         src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    return FLOOD_OK;
}

flood_status copy_out(flood_handle *h, void *dst, const void *src_pitched, int rows, int cols, int dst_on_device)
{
    size_t e = h->esz;
    CK(cudaMemcpy2DAsync(dst, (size_t)cols * e, src_pitched, (size_t)h->geo.pitch * e, (size_t)cols * e, rows,
                         dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    return FLOOD_OK;
}

// Re-measure h_max of the current state (epoch-start value for the next epoch).
flood_status refresh_hmax(flood_handle *h)
{
    CK(cudaMemsetAsync(&h->ctrl->hmax_bits, 0, sizeof(unsigned long long), h->stream));
    if (h->prec == FLOOD_F32) CK(launch_hmax<float>(h->geo, (const float *)h->h[h->cur], h->ctrl, h->stream));
    else CK(launch_hmax<double>(h->geo, (const double *)h->h[h->cur], h->ctrl, h->stream));
    return FLOOD_OK;
}

flood_status launch_inflow_epoch(flood_handle *h)
{
    if (h->n_in == 0) return FLOOD_OK;
    int E = h->geo.epoch_steps;
    // the section cells' z and n: in the grid's own planes, or a part's copies of them
    const void *z = h->sec_z ? h->sec_z : h->z, *n = h->sec_z ? h->sec_n : h->n;
    if (h->prec == FLOOD_F32)
        CK(launch_inflow<float>(h->geo, h->secs_dev, h->n_in, h->sec_cells, nullptr, h->tab_t, h->tab_q,
                                (const float *)z, (const float *)n, h->t_list, E, (float *)h->inflow_q,
                                h->n_slots, h->inflow_Q, h->inflow_W, h->stream));
    else
        CK(launch_inflow<double>(h->geo, h->secs_dev, h->n_in, h->sec_cells, nullptr, h->tab_t, h->tab_q,
                                 (const double *)z, (const double *)n, h->t_list, E, (double *)h->inflow_q,
                                 h->n_slots, h->inflow_Q, h->inflow_W, h->stream));
    return FLOOD_OK;
}

template <typename T>
StepArgs<T> make_args(flood_handle *h, int s, int k_steps, int want_hmax, const int64_t *gcells,
                             int ng, double *gout)
{
    StepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.geo = h->geo;
    int c = h->cur, o = 1 - h->cur;
    a.h = (const T *)h->h[c];
    a.qx = (const T *)h->qx[c];
    a.qy = (const T *)h->qy[c];
    a.z = (const T *)h->z;
    a.n = (const T *)h->n;
    a.h_out = (T *)h->h[o];
    a.qx_out = (T *)h->qx[o];
    a.qy_out = (T *)h->qy[o];
    a.bc.type = h->bc_type;
    a.bc.slot = h->bc_slot;
    a.bc.sqrtS = h->bc_sqrtS;
    a.bc.sqrtS_f = h->bc_sqrtS_f;
    a.inflow_q = (const T *)h->inflow_q;
    a.n_slots = h->n_slots;
    a.inflow_Q = h->inflow_Q;
    a.n_inflow_sec = h->book_vin ? h->n_in : 0;    // sections whose inflow volume this launch books
    a.t_list = h->t_list;
    a.ctrl = h->ctrl;
    a.s = s;
    a.k_steps = k_steps;
    a.want_hmax = want_hmax;
    a.gauge_cells = gcells;
    a.n_gauges = ng;
    a.gauge_out = gout;
    a.tile_x = h->tile_x;
    a.tile_y = h->tile_y;
    return a;
}

StepArgs<float> step_args_f32(flood_handle *h, int s) { return make_args<float>(h, s, 1, 0, nullptr, 0, nullptr); }

// The FP32 step of the handle's kernel family for prepared arguments.
static cudaError_t launch_f32(flood_handle *h, const StepArgs<float> &a)
{
    switch (h->kernel) {
    case FLOOD_KERNEL_REFERENCE: return launch_step_reference<float>(a, h->stream);
    case FLOOD_KERNEL_TILED:
        // gauge recording needs the depth after every step: single steps there
        if (a.gauge_out) {
            StepArgs<float> b = a;
            b.tile_x = b.tile_y = 0;
            return launch_step_stream(b, h->stream);
        }
        return launch_step_tiled(a, h->stream);
    case FLOOD_KERNEL_STREAM: return launch_step_stream(a, h->stream);
    case FLOOD_KERNEL_TMA: return launch_step_tma(a, h->stream);
    default: return launch_step_rows(a, h->stream);
    }
}

// One launch of k steps starting at step-in-epoch s.
flood_status launch_steps(flood_handle *h, int s, int k, int want_hmax, const int64_t *gcells, int ng,
                          double *gout)
{
    cudaError_t e;
    if (h->prec == FLOOD_F64)
        e = launch_step_reference<double>(make_args<double>(h, s, 1, want_hmax, gcells, ng, gout), h->stream);
    else
        e = launch_f32(h, make_args<float>(h, s, k, want_hmax, gcells, ng, gout));
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
    h->cur = 1 - h->cur;
    return FLOOD_OK;
}

template <typename T>
static void set_planes(StepArgs<T> &a, const void *const in[3], void *const out[3])
{
    a.h = (const T *)in[0];
    a.qx = (const T *)in[1];
    a.qy = (const T *)in[2];
    a.h_out = (T *)out[0];
    a.qx_out = (T *)out[1];
    a.qy_out = (T *)out[2];
}

flood_status launch_step_planes(flood_handle *h, int s, int k, const void *const in[3], void *const out[3])
{
    cudaError_t e;
    if (h->prec == FLOOD_F64) {
        if (k != 1) return fail(h, FLOOD_ERR_ARG, "FP64 planes advance one step per launch");
        StepArgs<double> a = make_args<double>(h, s, 1, 0, nullptr, 0, nullptr);
        set_planes(a, in, out);
        e = launch_step_reference<double>(a, h->stream);
    } else {
        StepArgs<float> a = make_args<float>(h, s, k, 0, nullptr, 0, nullptr);
        set_planes(a, in, out);
        if (k > 1) {                       // several steps: the temporal-blocking kernel (bitwise the single steps)
            a.tile_x = a.tile_y = 0;
            e = launch_step_tiled(a, h->stream);
        } else {
            e = launch_f32(h, a);
        }
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
    return FLOOD_OK;
}

// Advance n steps; if gcells, record gauges after each step into gbuf (device, n x ng).
// epoch_open: the current epoch was begun already (its dt, times and inflow rows
// are in place), so a first step at an epoch start does not begin it again.
flood_status advance(flood_handle *h, int64_t n, const int64_t *gcells, int ng, double *gbuf,
                     const double *fixed_dt_log, bool epoch_open)
{
    NvtxRange range("flood: steps");
    const int E = h->geo.epoch_steps;
    int64_t done = 0;
    while (done < n) {
        int s = (int)(h->step % E);
        if (s == 0 && !(epoch_open && done == 0)) {
            NvtxRange epoch("flood: epoch start (dt, Eq. 6 inflow)");
            const double *fdt = fixed_dt_log ? fixed_dt_log + done : nullptr;
            CK(launch_epoch_begin(h->geo, h->ctrl, h->t_list, E, fdt, h->stream));
            flood_status st = launch_inflow_epoch(h);
            if (st) return st;
        }
        int k = 1;
        if (h->prec == FLOOD_F32 && h->kernel == FLOOD_KERNEL_TILED && !gcells) {
            k = std::min<int64_t>(h->k_per_launch, std::min<int64_t>(E - s, n - done));
            if (k > 4 && k < 8) k = 4;   // the kernel exists for 1..4 and 8 steps per launch
        }
        int want = (s + k == E) ? 1 : 0;
        flood_status st = launch_steps(h, s, k, want, gcells, ng, gcells ? gbuf + done * ng : nullptr);
        if (st) return st;
        h->step += k;
        done += k;
    }
    return FLOOD_OK;
}

flood_status check_device_status(flood_handle *h)
{
    Ctrl c;
    CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (c.status & kStatusNonfinite) return fail(h, FLOOD_ERR_NONFINITE, "NaN or Inf depth at an epoch start");
    if (c.status & kStatusTimeout) return fail(h, FLOOD_ERR_TIMEOUT, "a bounded device wait gave up");
    if (c.status & kStatusCfl)
        return fail(h, FLOOD_ERR_CFL, "an epoch's time step broke the Courant limit dx / sqrt(g h_max) at its end");
    return FLOOD_OK;
}

}  // namespace flood

// ------------------------------------------------------------------ create / destroy
static flood_status validate(const flood_grid *grid, const flood_bc_section *secs, int nsec, const flood_opts &o)
{
    if (!grid) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (grid->nx < 1 || grid->ny < 1) return fail(nullptr, FLOOD_ERR_ARG, "nx and ny must be >= 1");
    if ((int64_t)grid->nx * grid->ny > (int64_t)1 << 34) return fail(nullptr, FLOOD_ERR_ARG, "grid too large");
    if (grid->nx > (1 << 24) || grid->ny > (1 << 24)) return fail(nullptr, FLOOD_ERR_ARG, "nx, ny must be <= 2^24");
    if (!(grid->dx > 0.0) || !std::isfinite(grid->dx)) return fail(nullptr, FLOOD_ERR_ARG, "dx must be > 0");
    if (grid->precision != FLOOD_F32 && grid->precision != FLOOD_F64)
        return fail(nullptr, FLOOD_ERR_ARG, "precision must be FLOOD_F32 or FLOOD_F64");
    if (nsec < 0 || (nsec > 0 && !secs)) return fail(nullptr, FLOOD_ERR_ARG, "bad section list");
    if (o.epoch_steps < 1 || o.epoch_steps > kMaxEpoch) return fail(nullptr, FLOOD_ERR_ARG, "epoch_steps must be 1..1024");
    if (!(o.g > 0) || !(o.h_dry > 0) || !(o.cfl_alpha > 0) || !(o.dt_cap > 0) || !(o.dt_const > 0))
        return fail(nullptr, FLOOD_ERR_ARG, "g, h_dry, cfl_alpha, dt_cap, dt_const must be > 0");
    if (o.dt_mode != 0 && o.dt_mode != 1) return fail(nullptr, FLOOD_ERR_ARG, "dt_mode must be 0 or 1");
    if (o.bc_form != 0 && o.bc_form != 1) return fail(nullptr, FLOOD_ERR_ARG, "bc_form must be 0 or 1");
    if (o.kernel < 0 || o.kernel > 5) return fail(nullptr, FLOOD_ERR_ARG, "unknown kernel");
    if (o.tile_x < 0 || o.tile_y < 0) return fail(nullptr, FLOOD_ERR_ARG, "tile_x and tile_y must be >= 0");
    if (!(o.theta > 0.0 && o.theta <= 1.0)) return fail(nullptr, FLOOD_ERR_ARG, "theta must lie in (0, 1]");
    if (o.theta != 1.0 && grid->precision == FLOOD_F32 && o.kernel == FLOOD_KERNEL_ROWS)
        return fail(nullptr, FLOOD_ERR_UNSUPPORTED, "theta != 1 needs the REFERENCE, STREAM, TMA or TILED kernel");
    if (o.friction != 0 && o.friction != 1) return fail(nullptr, FLOOD_ERR_ARG, "friction must be 0 or 1");
    if (o.friction != 0 && grid->precision == FLOOD_F32 && o.kernel == FLOOD_KERNEL_ROWS)
        return fail(nullptr, FLOOD_ERR_UNSUPPORTED,
                    "vector-norm friction needs the REFERENCE, STREAM, TMA or TILED kernel");
    if (o.kernel == FLOOD_KERNEL_TILED) {
        int K = o.steps_per_launch > 0 ? o.steps_per_launch : 4;
        if (!(K <= 4 || K == 8) || o.epoch_steps % K != 0)
            return fail(nullptr, FLOOD_ERR_ARG, "steps_per_launch must be 1..4 or 8 and divide epoch_steps");
    }
    std::vector<int> used(2 * (size_t)grid->nx + 2 * (size_t)grid->ny, 0);
    for (int k = 0; k < nsec; k++) {
        const flood_bc_section &s = secs[k];
        if (s.side < 0 || s.side > 3) return fail(nullptr, FLOOD_ERR_ARG, "section side must be 0..3");
        if (s.kind != FLOOD_INFLOW && s.kind != FLOOD_OUTFLOW) return fail(nullptr, FLOOD_ERR_ARG, "section kind");
        if (!(s.slope > 0) || !std::isfinite(s.slope)) return fail(nullptr, FLOOD_ERR_ARG, "section slope must be > 0");
        if (!(s.frac_start >= 0.0) || !(s.frac_end <= 1.0) || !(s.frac_end >= s.frac_start))
            return fail(nullptr, FLOOD_ERR_ARG, "section fractions must satisfy 0 <= start <= end <= 1");
        if (s.kind == FLOOD_INFLOW) {
            if (s.n_pts < 1 || !s.t_s || !s.q_m3s) return fail(nullptr, FLOOD_ERR_ARG, "inflow needs a hydrograph");
            for (int p = 0; p < s.n_pts; p++) {
                if (!std::isfinite(s.t_s[p]) || !std::isfinite(s.q_m3s[p]) || s.q_m3s[p] < 0.0)
                    return fail(nullptr, FLOOD_ERR_ARG, "hydrograph values must be finite, Q >= 0");
                if (p > 0 && !(s.t_s[p] > s.t_s[p - 1]))
                    return fail(nullptr, FLOOD_ERR_ARG, "hydrograph times must ascend");
            }
        }
        int i0, i1;
        section_range(s, grid->nx, grid->ny, &i0, &i1);
        int off = side_offset(s.side, grid->nx, grid->ny);
        for (int c = i0; c < i1; c++) {
            if (used[off + c]) return fail(nullptr, FLOOD_ERR_ARG, "sections overlap on a boundary face");
            used[off + c] = 1;
        }
    }
    return FLOOD_OK;
}

static int check_finite_host(const void *a, size_t n, int prec)
{
    if (prec == FLOOD_F32) {
        const float *f = (const float *)a;
        for (size_t k = 0; k < n; k++)
            if (!std::isfinite(f[k])) return 0;
    } else {
        const double *d = (const double *)a;
        for (size_t k = 0; k < n; k++)
            if (!std::isfinite(d[k])) return 0;
    }
    return 1;
}

namespace flood {

// AUTO: the temporal-blocking kernel with K = 4 where it applies (E a multiple
// of 4, no explicit launch shape), for Eq. 3 as printed and for the scheme
// options alike, else the tensor-tile kernel below 2^27 cells, else the
// row-staged stream kernel.  Measured on the fractal workload (us per step,
// epoch starts included): tiled K = 4 / TMA / stream 15.2 / 16.4 / 18.2 at
// 1024^2, 29.9 / 33.9 / 39.3 at 2048^2, 89.2 / 102.0 / 105.9 at 4096^2,
// 296 / 349 / 354 at 8192^2, 1059 / 1305 / 1302 at 16384^2; with vector-norm
// friction tiled / TMA 16.6 / 18.3, 36.1 / 41.0, 116.4 / 119.2, 385 / 381 and
// 1396 / 1425.  All of them are bitwise equal.
int auto_kernel(const flood_opts &o, int nx, int ny)
{
    const bool tiled = o.epoch_steps % 4 == 0 && o.tile_x == 0 && o.tile_y == 0;
    if (tiled) return FLOOD_KERNEL_TILED;
    return (int64_t)nx * ny < ((int64_t)1 << 27) ? FLOOD_KERNEL_TMA : FLOOD_KERNEL_STREAM;
}

flood_status refresh_hmax_window(flood_handle *h)
{
    Geom g = h->geo;
    g.ny = h->geo.led_j1 - h->geo.led_j0;
    const size_t off = (size_t)h->geo.led_j0 * h->geo.pitch * h->esz;
    CK(cudaMemsetAsync(&h->ctrl->hmax_bits, 0, sizeof(unsigned long long), h->stream));
    if (g.ny <= 0) return FLOOD_OK;
    const char *base = (const char *)h->h[h->cur] + off;
    if (h->prec == FLOOD_F32) CK(launch_hmax<float>(g, (const float *)base, h->ctrl, h->stream));
    else CK(launch_hmax<double>(g, (const double *)base, h->ctrl, h->stream));
    return FLOOD_OK;
}

flood_status create_handle(const flood_grid *grid, const void *dem, const void *manning,
                           const flood_bc_section *sections, int32_t n_sections, const flood_opts *opts,
                           const PartSpec *part, flood_handle **out)
{
    if (!out) return fail(nullptr, FLOOD_ERR_ARG, "out is NULL");
    *out = nullptr;
    flood_opts o;
    if (opts) o = *opts;
    else flood_default_opts(&o);
    flood_status vs = validate(grid, sections, n_sections, o);
    if (vs) return vs;
    if (!dem) return fail(nullptr, FLOOD_ERR_ARG, "dem is NULL");
    const size_t ncell = (size_t)grid->nx * grid->ny;
    const size_t esz = grid->precision == FLOOD_F32 ? 4 : 8;
    if (!check_finite_host(dem, ncell, grid->precision)) return fail(nullptr, FLOOD_ERR_ARG, "dem has NaN/Inf");
    if (manning) {
        if (!check_finite_host(manning, ncell, grid->precision)) return fail(nullptr, FLOOD_ERR_ARG, "manning has NaN/Inf");
        for (size_t k = 0; k < ncell; k++) {
            double v = grid->precision == FLOOD_F32 ? ((const float *)manning)[k] : ((const double *)manning)[k];
            if (!(v > 0.0)) return fail(nullptr, FLOOD_ERR_ARG, "manning must be > 0");
        }
    }
    // the rows this handle stores: all of them, or a part's global rows [a, b)
    const int ny_all = grid->ny;
    const int ra = part ? part->a : 0, rb = part ? part->b : ny_all;
    if (part && !(part->ny_global == ny_all && 0 <= ra && ra <= part->y0 && part->y0 < part->y1 &&
                  part->y1 <= rb && rb <= ny_all))
        return fail(nullptr, FLOOD_ERR_ARG, "bad part rows");
    flood_handle *h = new flood_handle();
    h->prec = grid->precision;
    h->esz = esz;
    h->opts = o;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        delete h;
        return fail(nullptr, FLOOD_ERR_CUDA, "no CUDA device");
    }
    h->device = dev;
    h->stream = o.stream ? (cudaStream_t)o.stream : c10::cuda::getCurrentCUDAStream(dev).stream();
    Geom &G = h->geo;
    G.nx = grid->nx;
    G.ny = rb - ra;
    G.pitch = (grid->nx + 1 + 31) / 32 * 32;
    G.bc_form = o.bc_form;
    G.theta = o.theta;
    G.friction = o.friction;
    G.dx = grid->dx;
    G.dx_f = (float)grid->dx;
    G.g = o.g;
    G.h_dry = o.h_dry;
    G.h_dry_f = (float)o.h_dry;
    G.cfl_alpha = o.cfl_alpha;
    G.dt_cap = o.dt_cap;
    G.dt_const = o.dt_const;
    G.dt_mode = o.dt_mode;
    G.epoch_steps = o.epoch_steps;
    G.led_j0 = part ? part->y0 - ra : 0;
    G.led_j1 = part ? part->y1 - ra : G.ny;
    const int E = o.epoch_steps;
    h->part = part != nullptr;
    h->book_vin = !part || part->index == 0;

    h->kernel = o.kernel == FLOOD_KERNEL_AUTO ? auto_kernel(o, grid->nx, ny_all) : o.kernel;
    if (h->prec == FLOOD_F64) h->kernel = FLOOD_KERNEL_REFERENCE;
    h->k_per_launch = 1;
    h->tile_x = o.tile_x;
    h->tile_y = o.tile_y;
    if (h->kernel == FLOOD_KERNEL_TILED)
        h->k_per_launch = (o.kernel == FLOOD_KERNEL_TILED && o.steps_per_launch > 0) ? o.steps_per_launch : 4;

    auto bail = [&](flood_status st, const char *msg) {
        std::string m = msg;
        flood_destroy(h);
        return fail(nullptr, st, m);
    };
#define ALLOC(ptr, type, bytes)                                                 \
    do {                                                                        \
        ptr = (type)dev_alloc(h, (bytes));                                      \
        if (!ptr) return bail(FLOOD_ERR_OOM, "device allocation failed");       \
    } while (0)

    const size_t plane = (size_t)G.pitch * G.ny * esz;
    const size_t plane_y = (size_t)G.pitch * (G.ny + 1) * esz;
    for (int b = 0; b < 2; b++) {
        ALLOC(h->h[b], void *, plane);
        ALLOC(h->qx[b], void *, plane);
        ALLOC(h->qy[b], void *, plane_y);
    }
    ALLOC(h->z, void *, plane);
    ALLOC(h->n, void *, plane);
    for (int b = 0; b < 2; b++) {
        if (cudaMemsetAsync(h->h[b], 0, plane, h->stream) || cudaMemsetAsync(h->qx[b], 0, plane, h->stream) ||
            cudaMemsetAsync(h->qy[b], 0, plane_y, h->stream))
            return bail(FLOOD_ERR_CUDA, "memset");
    }
    if (cudaMemsetAsync(h->z, 0, plane, h->stream) || cudaMemsetAsync(h->n, 0, plane, h->stream))
        return bail(FLOOD_ERR_CUDA, "memset");
    const size_t row_off = (size_t)ra * grid->nx * esz;
    if (copy_in(h, h->z, (const char *)dem + row_off, G.ny, G.nx, 0)) return bail(FLOOD_ERR_CUDA, "dem upload");
    std::vector<char> nbuf;
    const void *nsrc = manning;
    if (!manning) {
        nbuf.resize(ncell * esz);
        for (size_t k = 0; k < ncell; k++) {
            if (esz == 4) ((float *)nbuf.data())[k] = 0.03f;
            else ((double *)nbuf.data())[k] = 0.03;
        }
        nsrc = nbuf.data();
    }
    if (copy_in(h, h->n, (const char *)nsrc + row_off, G.ny, G.nx, 0)) return bail(FLOOD_ERR_CUDA, "manning upload");

    // boundary description of the stored rows.  A part keeps a border face of
    // the whole grid where it lies in its rows (an outflow face of a halo row
    // computes its flux without booking it); the rows' ends inside the grid are
    // walls (their neighbours' values arrive by the halo exchange).  Inflow
    // sections are always the whole grid's: a part solves Eq. 6 on copies of
    // the section cells' z and n, so every part obtains the same face fluxes.
    const int nb = 2 * G.nx + 2 * G.ny;
    std::vector<int8_t> btype(nb, kBcWall);
    std::vector<int32_t> bslot(nb, 0);
    std::vector<double> bsqrt(nb, 0.0);
    std::vector<InflowSec> isecs;
    std::vector<int64_t> icells;
    std::vector<char> secz, secn;
    std::vector<double> tt, tq;
    int slots = 0;
    // local boundary entry of global side cell c (-1 if the part does not store it) and its global row
    auto local_entry = [&](int side, int c, int *grow) -> int {
        const int off = side_offset(side, G.nx, G.ny);
        if (side == FLOOD_XMIN || side == FLOOD_XMAX) {
            *grow = c;
            return (c >= ra && c < rb) ? off + (c - ra) : -1;
        }
        *grow = side == FLOOD_YMIN ? 0 : ny_all - 1;
        if (side == FLOOD_YMIN && ra != 0) return -1;
        if (side == FLOOD_YMAX && rb != ny_all) return -1;
        return off + c;
    };
    const int own0 = part ? part->y0 : 0, own1 = part ? part->y1 : ny_all;
    for (int k = 0; k < n_sections; k++) {
        const flood_bc_section &s = sections[k];
        int i0, i1;
        section_range(s, grid->nx, ny_all, &i0, &i1);
        if (s.kind == FLOOD_OUTFLOW) {
            for (int c = i0; c < i1; c++) {
                int grow = 0;
                const int e = local_entry(s.side, c, &grow);
                if (e < 0) continue;
                btype[e] = (grow >= own0 && grow < own1) ? kBcOutflow : kBcOutflowHalo;
                bsqrt[e] = std::sqrt(s.slope);
            }
        } else {
            InflowSec S;
            std::memset(&S, 0, sizeof(S));
            S.ncell = i1 - i0;
            S.side = s.side;
            S.cell0 = (int)icells.size();
            S.slot0 = slots;
            S.tab0 = (int)tt.size();
            S.ntab = s.n_pts;
            S.sqrtS = std::sqrt(s.slope);
            for (int c = i0; c < i1; c++) {
                int grow = 0;
                const int e = local_entry(s.side, c, &grow);
                if (e >= 0) {
                    btype[e] = kBcInflow;
                    bslot[e] = slots + (c - i0);
                }
                const int64_t gcell = side_cell_pitched(s.side, c, G.nx, ny_all, G.nx);   // j * nx + i
                if (part) {
                    icells.push_back((int64_t)(secz.size() / esz));
                    const char *zc = (const char *)dem + gcell * esz;
                    const char *nc = (const char *)nsrc + gcell * esz;
                    secz.insert(secz.end(), zc, zc + esz);
                    secn.insert(secn.end(), nc, nc + esz);
                } else {
                    icells.push_back(side_cell_pitched(s.side, c, G.nx, G.ny, G.pitch));
                }
            }
            slots += i1 - i0;
            for (int p = 0; p < s.n_pts; p++) {
                tt.push_back(s.t_s[p]);
                tq.push_back(s.q_m3s[p]);
            }
            isecs.push_back(S);
        }
    }
    h->n_in = (int)isecs.size();
    h->n_slots = std::max(slots, 1);
    ALLOC(h->bc_type, int8_t *, nb);
    ALLOC(h->bc_slot, int32_t *, nb * sizeof(int32_t));
    ALLOC(h->bc_sqrtS, double *, nb * sizeof(double));
    ALLOC(h->bc_sqrtS_f, float *, nb * sizeof(float));
    std::vector<float> bsqrt_f(bsqrt.begin(), bsqrt.end());
    ALLOC(h->secs_dev, InflowSec *, std::max<size_t>(isecs.size(), 1) * sizeof(InflowSec));
    ALLOC(h->sec_cells, int64_t *, std::max<size_t>(icells.size(), 1) * sizeof(int64_t));
    if (part) {
        ALLOC(h->sec_z, void *, std::max<size_t>(secz.size(), esz));
        ALLOC(h->sec_n, void *, std::max<size_t>(secn.size(), esz));
    }
    ALLOC(h->tab_t, double *, std::max<size_t>(tt.size(), 1) * sizeof(double));
    ALLOC(h->tab_q, double *, std::max<size_t>(tq.size(), 1) * sizeof(double));
    ALLOC(h->inflow_q, void *, (size_t)E * h->n_slots * esz);
    ALLOC(h->inflow_Q, double *, (size_t)E * std::max(h->n_in, 1) * sizeof(double));
    ALLOC(h->inflow_W, double *, (size_t)E * std::max(h->n_in, 1) * sizeof(double));
    ALLOC(h->t_list, double *, (E + 1) * sizeof(double));
    ALLOC(h->ctrl, Ctrl *, sizeof(Ctrl));
    h->n_partials = 1024;
    ALLOC(h->vol_partials, double *, h->n_partials * sizeof(double));
    ALLOC(h->vol_out, double *, sizeof(double));
    ALLOC(h->flag, int *, sizeof(int));
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream);
    };
    if (up(h->bc_type, btype.data(), nb) || up(h->bc_slot, bslot.data(), nb * sizeof(int32_t)) ||
        up(h->bc_sqrtS, bsqrt.data(), nb * sizeof(double)) || up(h->bc_sqrtS_f, bsqrt_f.data(), nb * sizeof(float)) ||
        up(h->secs_dev, isecs.data(), isecs.size() * sizeof(InflowSec)) ||
        up(h->sec_cells, icells.data(), icells.size() * sizeof(int64_t)) ||
        up(h->tab_t, tt.data(), tt.size() * sizeof(double)) || up(h->tab_q, tq.data(), tq.size() * sizeof(double)))
        return bail(FLOOD_ERR_CUDA, "boundary upload");
    if (part && (up(h->sec_z, secz.data(), secz.size()) || up(h->sec_n, secn.data(), secn.size())))
        return bail(FLOOD_ERR_CUDA, "section upload");
    if (cudaMemsetAsync(h->inflow_q, 0, (size_t)E * h->n_slots * esz, h->stream) ||
        cudaMemsetAsync(h->inflow_Q, 0, (size_t)E * std::max(h->n_in, 1) * sizeof(double), h->stream) ||
        cudaMemsetAsync(h->t_list, 0, (E + 1) * sizeof(double), h->stream) ||
        cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream))
        return bail(FLOOD_ERR_CUDA, "memset");
    h->cur = 0;
    h->step = 0;
    h->sticky = FLOOD_OK;
    if (refresh_hmax(h)) return bail(FLOOD_ERR_CUDA, "h_max");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(FLOOD_ERR_CUDA, cudaGetErrorString(e));
#undef ALLOC
    *out = h;
    return FLOOD_OK;
}

}  // namespace flood

extern "C" flood_status flood_create(const flood_grid *grid, const void *dem, const void *manning,
                                     const flood_bc_section *sections, int32_t n_sections,
                                     const flood_opts *opts, flood_handle **out)
{
    return create_handle(grid, dem, manning, sections, n_sections, opts, nullptr, out);
}

extern "C" flood_status flood_destroy(flood_handle *h)
{
    if (!h) return FLOOD_OK;
    cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    destroy_adjoint(h);
    std::vector<void *> all = h->allocations;
    for (void *p : all) c10::cuda::CUDACachingAllocator::raw_delete(p);
    h->allocations.clear();
    delete h;
    return FLOOD_OK;
}

extern "C" const char *flood_last_error(const flood_handle *h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

// ------------------------------------------------------------------ stepping
extern "C" flood_status flood_step(flood_handle *h, int64_t n_steps)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    if (h->part) return fail(h, FLOOD_ERR_STATE, "a part of a decomposed grid is stepped by its decomposition");
    if (n_steps < 0) return fail(h, FLOOD_ERR_ARG, "n_steps must be >= 0");
    if (h->sticky) return fail(h, FLOOD_ERR_STATE, "handle is in an error state; write a new state first");
    if (h->opts.use_graph) return advance_graph(h, n_steps);
    return advance(h, n_steps, nullptr, 0, nullptr, nullptr);
}

extern "C" flood_status flood_coarsen(int32_t precision, const void *src, int32_t nx, int32_t ny, int32_t factor,
                                      void *dst, int32_t on_device, void *stream)
{
    if (!src || !dst) return fail(nullptr, FLOOD_ERR_ARG, "NULL argument");
    if (precision != FLOOD_F32 && precision != FLOOD_F64) return fail(nullptr, FLOOD_ERR_ARG, "bad precision");
    if (nx < 1 || ny < 1 || factor < 1) return fail(nullptr, FLOOD_ERR_ARG, "nx, ny and factor must be >= 1");
    if ((int64_t)nx * ny > (int64_t)1 << 34) return fail(nullptr, FLOOD_ERR_ARG, "grid too large");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, FLOOD_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = stream ? (cudaStream_t)stream : c10::cuda::getCurrentCUDAStream(dev).stream();
    const size_t esz = precision == FLOOD_F32 ? 4 : 8;
    const int mx = (nx + factor - 1) / factor, my = (ny + factor - 1) / factor;
    const size_t in_bytes = (size_t)nx * ny * esz, out_bytes = (size_t)mx * my * esz;
    void *d_src = const_cast<void *>(src), *d_dst = dst;
    if (!on_device) {
        d_src = raw_device_alloc(in_bytes, st);
        d_dst = d_src ? raw_device_alloc(out_bytes, st) : nullptr;
        if (!d_src || !d_dst) {
            if (d_src) c10::cuda::CUDACachingAllocator::raw_delete(d_src);
            return fail(nullptr, FLOOD_ERR_OOM, "coarsen buffers");
        }
        e = cudaMemcpyAsync(d_src, src, in_bytes, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess)
        e = precision == FLOOD_F32
                ? launch_coarsen<float>((const float *)d_src, nx, ny, factor, (float *)d_dst, st)
                : launch_coarsen<double>((const double *)d_src, nx, ny, factor, (double *)d_dst, st);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(dst, d_dst, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (!on_device) {
        c10::cuda::CUDACachingAllocator::raw_delete(d_src);
        c10::cuda::CUDACachingAllocator::raw_delete(d_dst);
    }
    if (e != cudaSuccess) return fail(nullptr, FLOOD_ERR_CUDA, cudaGetErrorString(e));
    return FLOOD_OK;
}

// Advance to the time t_end: whole steps while they end at or before t_end,
// then one step shortened to end exactly at t_end; the epoch keeps its time
// step for the steps after it (their start times are rebuilt from t_end and
// the epoch's inflow rows recomputed).
extern "C" flood_status flood_advance(flood_handle *h, double t_end, int64_t *steps_taken)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    if (h->sticky) return fail(h, FLOOD_ERR_STATE, "handle is in an error state; write a new state first");
    if (h->part) return fail(h, FLOOD_ERR_STATE, "a part of a decomposed grid is stepped by its decomposition");
    if (!std::isfinite(t_end)) return fail(h, FLOOD_ERR_ARG, "t_end must be finite");
    const int E = h->geo.epoch_steps;
    std::vector<double> tl(E + 1);
    int64_t taken = 0;
    Ctrl c;
    CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!(t_end >= c.t)) return fail(h, FLOOD_ERR_ARG, "t_end is before the current time");
    while (c.t < t_end) {
        const int s = (int)(h->step % E);
        const bool begun = s == 0;
        if (begun) {                                   // begin the epoch here: its dt decides the steps
            CK(launch_epoch_begin(h->geo, h->ctrl, h->t_list, E, nullptr, h->stream));
            flood_status st = launch_inflow_epoch(h);
            if (st) return st;
        }
        CK(cudaMemcpyAsync(tl.data(), h->t_list, (E + 1) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        int m = s;                                     // steps s .. m-1 end at or before t_end
        while (m < E && tl[m + 1] <= t_end) m++;
        if (m > s) {
            flood_status st = advance(h, m - s, nullptr, 0, nullptr, nullptr, begun);
            if (st) return st;
            taken += m - s;
        }
        if (tl[m] == t_end) break;
        if (m == E) {                                  // the epoch ended before t_end
            c.t = tl[E];
            continue;
        }
        // step m from tl[m] to t_end exactly
        const double dt = c.dt, dt_last = t_end - tl[m];
        CK(cudaMemcpyAsync(&h->ctrl->dt, &dt_last, sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->t_list + m + 1, &t_end, sizeof(double), cudaMemcpyHostToDevice, h->stream));
        flood_status st = advance(h, 1, nullptr, 0, nullptr, nullptr, begun && m == s);
        if (st) return st;
        taken += 1;
        // the rest of the epoch continues from t_end with the epoch's dt
        tl[m + 1] = t_end;
        for (int k = m + 1; k < E; k++) tl[k + 1] = tl[k] + dt;
        CK(cudaMemcpyAsync(&h->ctrl->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->t_list, tl.data(), (E + 1) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        if (m + 1 < E) {
            st = launch_inflow_epoch(h);
            if (st) return st;
        }
        CK(cudaStreamSynchronize(h->stream));          // host values above are in flight until here
        break;
    }
    CK(cudaStreamSynchronize(h->stream));
    if (steps_taken) *steps_taken = taken;
    return FLOOD_OK;
}

extern "C" flood_status flood_sync(flood_handle *h)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    if (h->sticky) return (flood_status)h->sticky;
    return check_device_status(h);
}

extern "C" flood_status flood_read(flood_handle *h, int32_t field, void *dst, size_t bytes, int32_t dst_on_device)
{
    if (!h || !dst) return fail(h, FLOOD_ERR_ARG, "NULL argument");
    if (field == FLOOD_FIELD_LEDGER) {
        if (bytes != FLOOD_LEDGER_LEN * sizeof(double)) return fail(h, FLOOD_ERR_ARG, "ledger needs 9 doubles");
        // stored volume of the rows this handle books (all rows, or a part's own)
        Geom vg = h->geo;
        vg.ny = h->geo.led_j1 - h->geo.led_j0;
        const char *hv = (const char *)h->h[h->cur] + (size_t)h->geo.led_j0 * h->geo.pitch * h->esz;
        if (h->prec == FLOOD_F32)
            CK(launch_volume<float>(vg, (const float *)hv, h->vol_partials, h->n_partials, h->vol_out, h->stream));
        else
            CK(launch_volume<double>(vg, (const double *)hv, h->vol_partials, h->n_partials, h->vol_out, h->stream));
        Ctrl c;
        double vol = 0.0;
        CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&vol, h->vol_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        double L[FLOOD_LEDGER_LEN] = {c.t, c.dt, c.V_in, c.V_out, c.V_clip, vol, c.h_max, (double)h->step,
                                      c.cfl_exceed};
        if (c.status & kStatusNonfinite) fail(h, FLOOD_ERR_NONFINITE, "NaN or Inf depth at an epoch start");
        else if (c.status & kStatusCfl)
            fail(h, FLOOD_ERR_CFL, "an epoch's time step broke the Courant limit dx / sqrt(g h_max) at its end");
        if (dst_on_device) CK(cudaMemcpy(dst, L, sizeof(L), cudaMemcpyHostToDevice));
        else std::memcpy(dst, L, sizeof(L));
        return FLOOD_OK;
    }
    const void *src;
    switch (field) {
    case FLOOD_FIELD_H: src = h->h[h->cur]; break;
    case FLOOD_FIELD_QX: src = h->qx[h->cur]; break;
    case FLOOD_FIELD_QY: src = h->qy[h->cur]; break;
    case FLOOD_FIELD_Z: src = h->z; break;
    case FLOOD_FIELD_N: src = h->n; break;
    default: return fail(h, FLOOD_ERR_ARG, "unknown field");
    }
    int rows, cols;
    field_shape(h, field, &rows, &cols);
    if (bytes != (size_t)rows * cols * h->esz) return fail(h, FLOOD_ERR_ARG, "dst size does not match the field");
    flood_status st = copy_out(h, dst, src, rows, cols, dst_on_device);
    if (st) return st;
    CK(cudaStreamSynchronize(h->stream));
    return FLOOD_OK;
}

extern "C" flood_status flood_write_state(flood_handle *h, const void *depth, const void *qx, const void *qy,
                                          int32_t src_on_device)
{
    if (!h || !depth) return fail(h, FLOOD_ERR_ARG, "NULL argument");
    CK(cudaStreamSynchronize(h->stream));
    // host input: stage the new state in the idle half of the ping-pong buffers
    // (the next step's output, free now) and check it on the device; only a
    // finite state becomes current, so a rejected one leaves the handle as it
    // was.  The staged half is made current by swapping the halves; an
    // ensemble member (whose launch tables fix its half) copies it over
    // instead.  Device input is taken as it is.
    const bool staged = !src_on_device;
    const int dst = staged ? 1 - h->cur : h->cur;
    const int nx = h->geo.nx, ny = h->geo.ny, P = h->geo.pitch;
    flood_status st = copy_in(h, h->h[dst], depth, ny, nx, src_on_device);
    if (st) return st;
    if (qx) st = copy_in(h, h->qx[dst], qx, ny, nx + 1, src_on_device);
    if (st) return st;
    if (qy) st = copy_in(h, h->qy[dst], qy, ny + 1, nx, src_on_device);
    if (st) return st;
    if (staged) {
        CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
        if (h->prec == FLOOD_F32) {
            CK(launch_nonfinite<float>((const float *)h->h[dst], ny, nx, P, h->flag, h->stream));
            if (qx) CK(launch_nonfinite<float>((const float *)h->qx[dst], ny, nx + 1, P, h->flag, h->stream));
            if (qy) CK(launch_nonfinite<float>((const float *)h->qy[dst], ny + 1, nx, P, h->flag, h->stream));
        } else {
            CK(launch_nonfinite<double>((const double *)h->h[dst], ny, nx, P, h->flag, h->stream));
            if (qx) CK(launch_nonfinite<double>((const double *)h->qx[dst], ny, nx + 1, P, h->flag, h->stream));
            if (qy) CK(launch_nonfinite<double>((const double *)h->qy[dst], ny + 1, nx, P, h->flag, h->stream));
        }
        int bad = 0;
        CK(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (bad) return fail(h, FLOOD_ERR_ARG, "depth or discharge has NaN/Inf");
        if (!h->in_ensemble) {
            h->cur = dst;
        } else {
            const int cur = h->cur;
            const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
            CK(cudaMemcpyAsync(h->h[cur], h->h[dst], plane_elems(h, FLOOD_FIELD_H) * h->esz, d2d, h->stream));
            if (qx) CK(cudaMemcpyAsync(h->qx[cur], h->qx[dst], plane_elems(h, FLOOD_FIELD_QX) * h->esz, d2d, h->stream));
            if (qy) CK(cudaMemcpyAsync(h->qy[cur], h->qy[dst], plane_elems(h, FLOOD_FIELD_QY) * h->esz, d2d, h->stream));
        }
    }
    if (!qx) CK(cudaMemsetAsync(h->qx[h->cur], 0, plane_elems(h, FLOOD_FIELD_QX) * h->esz, h->stream));
    if (!qy) CK(cudaMemsetAsync(h->qy[h->cur], 0, plane_elems(h, FLOOD_FIELD_QY) * h->esz, h->stream));
    // clear the device status word (keep the rest of the control block)
    CK(cudaMemsetAsync(&h->ctrl->status, 0, sizeof(int), h->stream));
    st = refresh_hmax(h);
    if (st) return st;
    CK(cudaStreamSynchronize(h->stream));
    h->sticky = FLOOD_OK;
    h->err.clear();
    return FLOOD_OK;
}

extern "C" flood_status flood_set_clock(flood_handle *h, double t, int64_t step, double dt, double v_in,
                                        double v_out, double v_clip)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    if (step < 0 || !std::isfinite(t) || !(dt >= 0.0)) return fail(h, FLOOD_ERR_ARG, "bad clock");
    Ctrl c;
    CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    c.t = t;
    c.dt = dt;
    c.V_in = v_in;
    c.V_out = v_out;
    c.V_clip = v_clip;
    CK(cudaMemcpyAsync(h->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
    h->step = step;
    // mid-epoch resume: rebuild the epoch's time list and inflow from (t, dt)
    int E = h->geo.epoch_steps, s = (int)(step % E);
    if (s != 0) {
        std::vector<double> tl(E + 1);
        tl[s] = t;
        for (int k = s - 1; k >= 0; k--) tl[k] = tl[k + 1] - dt;
        for (int k = s; k < E; k++) tl[k + 1] = tl[k] + dt;
        CK(cudaMemcpyAsync(h->t_list, tl.data(), (E + 1) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        flood_status st = launch_inflow_epoch(h);
        if (st) return st;
    }
    CK(cudaStreamSynchronize(h->stream));
    return FLOOD_OK;
}

extern "C" flood_status flood_set_manning(flood_handle *h, const void *manning, int32_t src_on_device)
{
    if (!h || !manning) return fail(h, FLOOD_ERR_ARG, "NULL argument");
    if (!src_on_device) {
        size_t nc = (size_t)h->geo.nx * h->geo.ny;
        if (!check_finite_host(manning, nc, h->prec)) return fail(h, FLOOD_ERR_ARG, "manning has NaN/Inf");
        for (size_t k = 0; k < nc; k++) {
            double v = h->prec == FLOOD_F32 ? ((const float *)manning)[k] : ((const double *)manning)[k];
            if (!(v > 0.0)) return fail(h, FLOOD_ERR_ARG, "manning must be > 0");
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    flood_status st = copy_in(h, h->n, manning, h->geo.ny, h->geo.nx, src_on_device);
    if (st) return st;
    if (h->step % h->geo.epoch_steps != 0) {
        st = launch_inflow_epoch(h);
        if (st) return st;
    }
    invalidate_graphs(h);
    CK(cudaStreamSynchronize(h->stream));
    return FLOOD_OK;
}

extern "C" flood_status flood_run_gauges(flood_handle *h, int64_t n_steps, const int64_t *gauge_cells,
                                         int32_t n_gauges, double *out, int32_t out_on_device)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    if (h->part) return fail(h, FLOOD_ERR_STATE, "a part of a decomposed grid is stepped by its decomposition");
    if (n_steps < 0 || n_gauges < 0 || (n_gauges > 0 && (!gauge_cells || !out)))
        return fail(h, FLOOD_ERR_ARG, "bad gauge arguments");
    if (h->sticky) return fail(h, FLOOD_ERR_STATE, "handle is in an error state; write a new state first");
    const int64_t nc = (int64_t)h->geo.nx * h->geo.ny;
    for (int g = 0; g < n_gauges; g++)
        if (gauge_cells[g] < 0 || gauge_cells[g] >= nc) return fail(h, FLOOD_ERR_ARG, "gauge cell out of range");
    if (n_gauges == 0 || n_steps == 0) return flood_step(h, n_steps);
    flood_status st = ensure_gauge_buffers(h, n_gauges, (size_t)n_steps * n_gauges);
    if (st) return st;
    CK(cudaMemcpyAsync(h->gauge_dev, gauge_cells, n_gauges * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    st = advance(h, n_steps, h->gauge_dev, n_gauges, h->gauge_buf, nullptr);
    if (st) return st;
    CK(cudaMemcpyAsync(out, h->gauge_buf, (size_t)n_steps * n_gauges * sizeof(double),
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FLOOD_OK;
}

namespace flood {

flood_status ensure_gauge_buffers(flood_handle *h, int ng, size_t n_values)
{
    if (ng > h->gauge_cap) {
        dev_free(h, h->gauge_dev);
        h->gauge_dev = (int64_t *)dev_alloc(h, (size_t)ng * sizeof(int64_t));
        if (!h->gauge_dev) return fail(h, FLOOD_ERR_OOM, "gauge list allocation");
        h->gauge_cap = ng;
    }
    if (n_values > h->gauge_buf_cap) {
        dev_free(h, h->gauge_buf);
        h->gauge_buf = (double *)dev_alloc(h, n_values * sizeof(double));
        if (!h->gauge_buf) return fail(h, FLOOD_ERR_OOM, "gauge series allocation");
        h->gauge_buf_cap = n_values;
    }
    return FLOOD_OK;
}

}  // namespace flood

// ------------------------------------------------------------------ debugging aids
extern "C" void flood_debug_fail_alloc_after(int64_t n) { g_fail_countdown = n < 0 ? -1 : n; }

extern "C" int64_t flood_debug_alloc_count(void) { return g_alloc_count.load(); }

extern "C" flood_status flood_debug_padding(flood_handle *h, int32_t fill, int64_t *bad)
{
    if (!h || (!fill && !bad)) return fail(h, FLOOD_ERR_ARG, "NULL argument");
    const int nx = h->geo.nx, ny = h->geo.ny, P = h->geo.pitch;
    unsigned long long *count = nullptr;
    if (!fill) {
        count = (unsigned long long *)dev_alloc(h, sizeof(unsigned long long));
        if (!count) return fail(h, FLOOD_ERR_OOM, "padding counter");
        CK(cudaMemsetAsync(count, 0, sizeof(unsigned long long), h->stream));
    }
    // (plane, rows, used columns): both state buffers, then z and n
    struct Plane { void *p; int rows, cols; };
    std::vector<Plane> planes;
    for (int b = 0; b < 2; b++) {
        planes.push_back({h->h[b], ny, nx});
        planes.push_back({h->qx[b], ny, nx + 1});
        planes.push_back({h->qy[b], ny + 1, nx});
    }
    planes.push_back({h->z, ny, nx});
    planes.push_back({h->n, ny, nx});
    cudaError_t e = cudaSuccess;
    for (const Plane &pl : planes) {
        e = launch_padding(pl.p, h->esz, pl.rows, pl.cols, P, fill != 0, count, h->stream);
        if (e != cudaSuccess) break;
    }
    unsigned long long n = 0;
    if (e == cudaSuccess && count) e = cudaMemcpyAsync(&n, count, sizeof(n), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (count) dev_free(h, count);
    if (e != cudaSuccess) return cuda_fail(h, e, "padding kernel");
    if (bad) *bad = (int64_t)n;
    return FLOOD_OK;
}
