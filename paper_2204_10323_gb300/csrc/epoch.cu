// epoch.cu -- per-epoch and bookkeeping kernels: the time-step rule, the
// Eq. 6 inflow distribution, and deterministic reductions (h_max, volume,
// gauge gathers).
#include <cfloat>

#include "device_common.cuh"

namespace flood {

namespace {

// Time-step rule at an epoch start: constant, frozen (adjoint replays), or
// dt = min(dt_cap, alpha dx / sqrt(g h_max)); h_max = 0 gives dt_cap.
__device__ void epoch_begin_body(const Geom &G, Ctrl *ctrl, double *t_list, int E, const double *fixed_dt)
{
    double hmax = __longlong_as_double((long long)ctrl->hmax_bits);
    if (!isfinite(hmax)) ctrl->status |= kStatusNonfinite;
    // the epoch that just ended: its dt against the Courant limit of the depth it ended with (not for
    // replays of a logged schedule, whose control block is restored after them)
    if (!fixed_dt && ctrl->dt > 0.0 && hmax > 0.0 && ctrl->dt * sqrt(G.g * hmax) > G.dx) {
        ctrl->cfl_exceed += 1.0;
        ctrl->status |= kStatusCfl;
    }
    double dt;
    if (fixed_dt) dt = *fixed_dt;
    else if (G.dt_mode == 1) dt = G.dt_const;
    else if (!(hmax > 0.0)) dt = G.dt_cap;
    else dt = fmin(G.dt_cap, G.cfl_alpha * G.dx / sqrt(G.g * hmax));
    ctrl->dt = dt;
    ctrl->h_max = hmax;
    ctrl->hmax_bits = 0ull;
    double t = ctrl->t;
    t_list[0] = t;
    for (int s = 0; s < E; s++) {
        t = t + dt;
        t_list[s + 1] = t;
    }
}

__global__ void epoch_begin_kernel(Geom G, Ctrl *ctrl, double *t_list, int E, const double *fixed_dt)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    epoch_begin_body(G, ctrl, t_list, E, fixed_dt);
}

// One thread per simulation of a batch.
template <typename T>
__global__ void epoch_begin_batched_kernel(const EpochArgs<T> *tab, int n, int E)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    epoch_begin_body(tab[k].geo, tab[k].ctrl, tab[k].t_list, E, nullptr);
}

// Linear interpolation in the hydrograph table, constant past both ends.
__device__ double hydrograph(const double *ts, const double *qs, int n, double t)
{
    if (n <= 0) return 0.0;
    if (t <= ts[0]) return qs[0];
    for (int k = 1; k < n; k++)
        if (t <= ts[k]) {
            double w = (t - ts[k - 1]) / (ts[k] - ts[k - 1]);
            return qs[k - 1] + w * (qs[k] - qs[k - 1]);
        }
    return qs[n - 1];
}

// Eq. 5 discharge of one cell (m^3/s) at depth hh.
__device__ __forceinline__ double manning_cell(double hh, double sqrtS, double n, double dx, int form)
{
    if (form == 0) return dx * pow(hh, 5.0 / 3.0) * sqrtS / n;
    return dx * dx * pow(hh, 2.0 / 3.0) * sqrtS / n;
}

// FP32 handles evaluate Eq. 5 in single precision inside the solve (the
// final rescale makes the section total exact either way); FP64 handles keep
// the double-precision evaluation of the plain definition.
__device__ __forceinline__ double manning_cell_t(double hh, double sqrtS, float n, double dx, int form)
{
    float h = (float)hh, p = form == 0 ? 5.0f / 3.0f : 2.0f / 3.0f;
    float a = form == 0 ? (float)dx : (float)(dx * dx);
    return (double)(a * powf(h, p) * (float)sqrtS / n);
}

__device__ __forceinline__ double manning_cell_t(double hh, double sqrtS, double n, double dx, int form)
{
    return manning_cell(hh, sqrtS, n, dx, form);
}

constexpr int kInflowThreads = 128;

// Sections of at most this many cells are solved by warp 0 alone: a bisection
// step then costs one warp reduction instead of two block barriers, and the
// solve is latency-bound (the sections of the workloads hold 12-512 cells).
// FP64 handles evaluate Eq. 5 with the slow double pow, so only the smallest
// sections go to one warp there.  The choice depends on the section alone, so
// a single grid and an ensemble member solve a section in the same order.
constexpr int kWarpCells = 1024;     // shared-memory copy of a one-warp section's z and n

template <typename T>
__device__ __forceinline__ bool one_warp(const InflowSec &S)
{
    return S.ncell <= (sizeof(T) == 4 ? kWarpCells : 32);
}

// Sum of a one-warp section's Eq. 5 discharges at level W from its cells' z
// and n staged in shared memory (every lane of warp 0 gets the sum).
template <typename T>
__device__ double section_total_warp(const InflowSec &S, const T *sz, const T *sn, double W, double dx,
                                     int form)
{
    double s = 0.0;
    for (int c = threadIdx.x; c < S.ncell; c += 32) {
        double hh = W - (double)sz[c];
        if (hh > 0.0) s += manning_cell_t(hh, S.sqrtS, sn[c], dx, form);
    }
    return warp_sum(s);
}

// FP32 handles, one-warp sections: Eq. 6 in single precision throughout the
// search (the level W, Eq. 5 per cell, the warp's butterfly sum), bisecting
// until the midpoint rounds to an end of the bracket (the double-precision
// search to 1e-12 m spends about twenty more halvings below the resolution of
// single-precision Eq. 5, each on the slow FP64 pipe); then each cell's
// discharge rescaled to Q_in in double.
__device__ void inflow_solve_warp_f32(const InflowSec &S, const float *sz, const float *sn, float zmin, double Q,
                                      double dx, int form, float *out, double *W_slot)
{
    const int lane = threadIdx.x;
    const float p = form == 0 ? 5.0f / 3.0f : 2.0f / 3.0f;
    const float a = form == 0 ? (float)dx : (float)(dx * dx);
    const float sq = (float)S.sqrtS;
    auto total = [&](float W) {
        float s = 0.0f;
        for (int c = lane; c < S.ncell; c += 32) {
            const float hh = W - sz[c];
            if (hh > 0.0f) s += a * powf(hh, p) * sq / sn[c];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
    };
    const float Qf = (float)Q;
    float Hb = 1.0f;
    while (total(zmin + Hb) < Qf && Hb < 1e12f) Hb *= 2.0f;
    float lo = zmin, hi = zmin + Hb;
    for (int it = 0; it < 200; it++) {
        const float mid = 0.5f * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (total(mid) < Qf) lo = mid;
        else hi = mid;
    }
    const float W = hi;
    if (lane == 0 && W_slot) *W_slot = (double)W;
    const double tot = (double)total(W);
    for (int c = lane; c < S.ncell; c += 32) {
        const float hh = W - sz[c];
        const float w = hh > 0.0f ? a * powf(hh, p) * sq / sn[c] : 0.0f;
        out[c] = (float)(((double)w * (Q / tot)) / dx);
    }
}

// Block-wide sum of the section's Eq. 5 discharges at level W (all threads get it).
template <typename T>
__device__ double section_total(const InflowSec &S, const int64_t *cells, const T *z, const T *n,
                                double W, double dx, int form, double *red)
{
    double s = 0.0;
    for (int c = threadIdx.x; c < S.ncell; c += kInflowThreads) {
        int64_t idx = cells[S.cell0 + c];
        double hh = W - (double)z[idx];
        if (hh > 0.0) s += manning_cell_t(hh, S.sqrtS, n[idx], dx, form);
    }
    s = warp_sum(s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kInflowThreads / 32; w++) t += red[w];
    return t;
}

// Eq. 6 for (step s of the epoch, inflow section k), by warp 0 or the whole
// block (one_warp): bisection for
// the level W with sum_c Q_c(W) = Q_in(t_s) on [min z, min z + H] (H doubled
// from 1 m), 200 halvings at most or a bracket below 1e-12 m, W = upper end;
// then each cell's discharge scaled by Q_in / sum, stored as unit-width flux.
template <typename T>
__device__ void inflow_body(const Geom &G, const InflowSec *secs, int nsec, const int64_t *cells,
                            const double *tab_t, const double *tab_q, const T *z, const T *n,
                            const double *t_list, T *inflow_q, int n_slots, double *inflow_Q, double *W_out,
                            const int s, const int k, double *red, T *sz, T *sn)
{
    const int tid = threadIdx.x;
    const InflowSec S = secs[k];
    const double t = t_list[s];
    const double Q = hydrograph(tab_t + S.tab0, tab_q + S.tab0, S.ntab, t);
    T *out = inflow_q + (size_t)s * n_slots + S.slot0;
    // a section that covers no cell carries no discharge
    if (tid == 0) inflow_Q[(size_t)s * nsec + k] = S.ncell > 0 ? Q : 0.0;
    double zmin = DBL_MAX;
    for (int c = tid; c < S.ncell; c += kInflowThreads) zmin = fmin(zmin, (double)z[cells[S.cell0 + c]]);
    for (int o = 16; o > 0; o >>= 1) zmin = fmin(zmin, __shfl_xor_sync(0xffffffffu, zmin, o));
    if ((tid & 31) == 0) red[tid >> 5] = zmin;
    __syncthreads();
    for (int w = 0; w < kInflowThreads / 32; w++) zmin = fmin(zmin, red[w]);
    if (!(Q > 0.0) || S.ncell == 0) {
        for (int c = tid; c < S.ncell; c += kInflowThreads) out[c] = T(0);
        return;
    }
    const bool warp_only = one_warp<T>(S);
    if (warp_only && tid >= 32) return;           // warp 0 solves and distributes
    const int nthreads = warp_only ? 32 : kInflowThreads;
    const double dx = G.dx;
    const int form = G.bc_form;
    if (warp_only) {                              // the section's z and n, read once
        for (int c = tid; c < S.ncell; c += 32) {
            const int64_t idx = cells[S.cell0 + c];
            sz[c] = z[idx];
            sn[c] = n[idx];
        }
        __syncwarp();
        if constexpr (sizeof(T) == 4) {
            inflow_solve_warp_f32(S, sz, sn, (float)zmin, Q, dx, form, out,
                                  W_out ? W_out + (size_t)s * nsec + k : nullptr);
            return;
        }
    }
    auto total_at = [&](double W) {
        return warp_only ? section_total_warp(S, sz, sn, W, dx, form) : section_total(S, cells, z, n, W, dx, form, red);
    };
    double Hb = 1.0;
    while (total_at(zmin + Hb) < Q && Hb < 1e12) Hb *= 2.0;
    double lo = zmin, hi = zmin + Hb;
    for (int it = 0; it < 200 && hi - lo >= 1e-12; it++) {
        double mid = 0.5 * (lo + hi);
        if (total_at(mid) < Q) lo = mid;
        else hi = mid;
    }
    const double W = hi;
    if (tid == 0 && W_out) W_out[(size_t)s * nsec + k] = W;
    const double total = total_at(W);
    for (int c = tid; c < S.ncell; c += nthreads) {
        int64_t idx = cells[S.cell0 + c];
        double hh = W - (double)z[idx];
        double w = hh > 0.0 ? manning_cell_t(hh, S.sqrtS, n[idx], dx, form) : 0.0;
        out[c] = T((w * (Q / total)) / dx);
    }
}

template <typename T>
__global__ void inflow_kernel(Geom G, const InflowSec *secs, int nsec, const int64_t *cells,
                              const double *tab_t, const double *tab_q, const T *z, const T *n,
                              const double *t_list, T *inflow_q, int n_slots, double *inflow_Q, double *W_out)
{
    __shared__ double red[kInflowThreads / 32];
    __shared__ T sz[kWarpCells], sn[kWarpCells];
    inflow_body<T>(G, secs, nsec, cells, tab_t, tab_q, z, n, t_list, inflow_q, n_slots, inflow_Q, W_out, blockIdx.x,
                   blockIdx.y, red, sz, sn);
}

// Eq. 6 for every (step, section) of a batch of simulations: block (s, task).
template <typename T>
__global__ void inflow_batched_kernel(const EpochArgs<T> *tab, const int2 *tasks)
{
    __shared__ double red[kInflowThreads / 32];
    __shared__ T sz[kWarpCells], sn[kWarpCells];
    const int2 t = tasks[blockIdx.y];
    const EpochArgs<T> &A = tab[t.x];
    inflow_body<T>(A.geo, A.secs, A.nsec, A.cells, A.tab_t, A.tab_q, A.z, A.n, A.t_list, A.inflow_q, A.n_slots,
                   A.inflow_Q, A.inflow_W, blockIdx.x, t.y, red, sz, sn);
}

// Rows over blocks, columns over threads; the maximum is exact in the state's
// own precision, and a NaN, once seen, is kept.
template <typename T>
__global__ void hmax_kernel(Geom G, const T *h, Ctrl *ctrl)
{
    __shared__ double red[32];
    T m = T(0);
    for (int j = blockIdx.x; j < G.ny; j += gridDim.x) {
        const T *row = h + (size_t)j * G.pitch;
        for (int i = threadIdx.x; i < G.nx; i += blockDim.x) {
            const T v = row[i];
            m = (v > m || v != v) ? v : m;
        }
    }
    const double bm = block_reduce<true>((double)m, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&ctrl->hmax_bits, bm);
}

// Sum of a thread's share of the depths: FP64 state in double; FP32 state as
// an unevaluated float pair (s, c) by Knuth's branch-free two-sum, each
// addition's rounding error carried in c, so the pair holds the exact sum to
// about n u^2 of the summands (n per thread, u = 2^-24) and the FP64 pipe is
// left out of the per-element work.
template <typename T>
struct ThreadSum;

template <>
struct ThreadSum<double> {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ double value() const { return s; }
};

template <>
struct ThreadSum<float> {
    float s = 0.0f, c = 0.0f;
    __device__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        c = __fadd_rn(c, e);
        s = t;
    }
    __device__ double value() const { return (double)s + (double)c; }
};

// Pass 1: block b sums rows b, b + nb, ... (fixed order for a fixed launch shape).
template <typename T>
__global__ void volume_partial_kernel(Geom G, const T *h, double *partials)
{
    __shared__ double red[32];
    ThreadSum<T> acc;
    for (int j = blockIdx.x; j < G.ny; j += gridDim.x) {
        const T *row = h + (size_t)j * G.pitch;
        for (int i = threadIdx.x; i < G.nx; i += blockDim.x) acc.add(row[i]);
    }
    const double s = block_reduce<false>(acc.value(), red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void volume_final_kernel(const double *partials, int np, double area, double *out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) s += partials[k];
    s = block_reduce<false>(s, red);
    if (threadIdx.x == 0) *out = s * area;
}

template <typename T>
__global__ void gauges_kernel(Geom G, const T *h, const int64_t *cells, int ng, double *out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    int64_t c = cells[k];
    out[k] = (double)h[(c / G.nx) * G.pitch + (c % G.nx)];
}

}  // namespace

// Parts of a decomposed grid: the largest of their running depth maxima
// (bits of non-negative doubles, or a NaN's larger bits) into every part, so
// that each part's epoch start takes the whole grid's h_max.
__global__ void hmax_allreduce_kernel(Ctrl *const *ctrls, int n)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long m = 0ull;
    for (int k = 0; k < n; k++) m = ctrls[k]->hmax_bits > m ? ctrls[k]->hmax_bits : m;
    for (int k = 0; k < n; k++) ctrls[k]->hmax_bits = m;
}

cudaError_t launch_hmax_allreduce(Ctrl *const *ctrls, int n, cudaStream_t st)
{
    hmax_allreduce_kernel<<<1, 32, 0, st>>>(ctrls, n);
    return cudaGetLastError();
}

cudaError_t launch_epoch_begin(const Geom &g, Ctrl *ctrl, double *t_list, int E, const double *fixed_dt,
                               cudaStream_t st)
{
    epoch_begin_kernel<<<1, 32, 0, st>>>(g, ctrl, t_list, E, fixed_dt);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_epoch_batched(const EpochArgs<T> *tab, int n, const int2 *tasks, int n_tasks, int E,
                                 cudaStream_t st)
{
    epoch_begin_batched_kernel<T><<<(n + 127) / 128, 128, 0, st>>>(tab, n, E);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n_tasks == 0) return e;
    inflow_batched_kernel<T><<<dim3(E, n_tasks), kInflowThreads, 0, st>>>(tab, tasks);
    return cudaGetLastError();
}

template cudaError_t launch_epoch_batched<float>(const EpochArgs<float> *, int, const int2 *, int, int, cudaStream_t);

template <typename T>
cudaError_t launch_inflow(const Geom &g, const InflowSec *secs, int nsec, const int64_t *sec_cells,
                          const int8_t * /*sec_side*/, const double *tab_t, const double *tab_q,
                          const T *z, const T *n, const double *t_list, int E, T *inflow_q, int n_slots,
                          double *inflow_Q, double *W_out, cudaStream_t st)
{
    if (nsec == 0) return cudaSuccess;
    dim3 grid(E, nsec);
    inflow_kernel<T><<<grid, kInflowThreads, 0, st>>>(g, secs, nsec, sec_cells, tab_t, tab_q, z, n, t_list, inflow_q,
                                          n_slots, inflow_Q, W_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hmax(const Geom &g, const T *h, Ctrl *ctrl, cudaStream_t st)
{
    const int blocks = g.ny < 152 * 8 ? g.ny : 152 * 8;
    hmax_kernel<T><<<blocks, 256, 0, st>>>(g, h, ctrl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_volume(const Geom &g, const T *h, double *partials, int n_partials, double *out,
                          cudaStream_t st)
{
    volume_partial_kernel<T><<<n_partials, 256, 0, st>>>(g, h, partials);
    volume_final_kernel<<<1, 256, 0, st>>>(partials, n_partials, g.dx * g.dx, out);
    return cudaGetLastError();
}

// Non-finite values among rows x cols elements of a pitched array: OR of the
// test into *flag (rows grid-strided over blocks, columns over threads).
template <typename T>
__global__ void nonfinite_kernel(const T *a, int rows, int cols, int pitch, int *flag)
{
    int bad = 0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const T *row = a + (size_t)r * pitch;
        for (int c = threadIdx.x; c < cols; c += blockDim.x) bad |= !isfinite(row[c]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

template <typename T>
cudaError_t launch_nonfinite(const T *a, int rows, int cols, int pitch, int *flag, cudaStream_t st)
{
    const int blocks = rows < 152 * 8 ? rows : 152 * 8;
    nonfinite_kernel<T><<<blocks, 256, 0, st>>>(a, rows, cols, pitch, flag);
    return cudaGetLastError();
}

// Poison of the pitch padding: quiet NaNs with a fixed payload, compared by bits.
template <typename U>
__global__ void padding_kernel(U *a, int rows, int cols, int pitch, U poison, int fill, unsigned long long *count)
{
    const int w = pitch - cols;
    unsigned long long bad = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)rows * w;
         k += (long long)gridDim.x * blockDim.x) {
        U *p = a + (size_t)(k / w) * pitch + cols + (k % w);
        if (fill) *p = poison;
        else bad += *p != poison;
    }
    if (!fill && bad) atomicAdd(count, bad);
}

cudaError_t launch_padding(void *a, size_t esz, int rows, int cols, int pitch, bool fill,
                           unsigned long long *count, cudaStream_t st)
{
    if (pitch <= cols || rows <= 0) return cudaSuccess;
    const long long n = (long long)rows * (pitch - cols);
    const int blocks = (int)(n < 152 * 8 * 256 ? (n + 255) / 256 : 152 * 8);
    if (esz == 4)
        padding_kernel<unsigned><<<blocks, 256, 0, st>>>((unsigned *)a, rows, cols, pitch, 0x7fc0deadu, fill ? 1 : 0,
                                                         count);
    else
        padding_kernel<unsigned long long><<<blocks, 256, 0, st>>>((unsigned long long *)a, rows, cols, pitch,
                                                                   0x7ff80000deadbeefull, fill ? 1 : 0, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gauges(const Geom &g, const T *h, const int64_t *cells, int G, double *out,
                          cudaStream_t st)
{
    if (G <= 0) return cudaSuccess;
    gauges_kernel<T><<<(G + 127) / 128, 128, 0, st>>>(g, h, cells, G, out);
    return cudaGetLastError();
}

#define FLOOD_INST(T)                                                                                      \
    template cudaError_t launch_inflow<T>(const Geom &, const InflowSec *, int, const int64_t *,             \
                                          const int8_t *, const double *, const double *, const T *,       \
                                          const T *, const double *, int, T *, int, double *, double *,      \
                                          cudaStream_t);                                                    \
    template cudaError_t launch_hmax<T>(const Geom &, const T *, Ctrl *, cudaStream_t);                     \
    template cudaError_t launch_volume<T>(const Geom &, const T *, double *, int, double *, cudaStream_t);   \
    template cudaError_t launch_gauges<T>(const Geom &, const T *, const int64_t *, int, double *, cudaStream_t); \
    template cudaError_t launch_nonfinite<T>(const T *, int, int, int, int *, cudaStream_t);
FLOOD_INST(float)
FLOOD_INST(double)
#undef FLOOD_INST

}  // namespace flood
