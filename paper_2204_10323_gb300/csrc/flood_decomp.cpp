// flood_decomp.cpp -- a grid split into 1 x N row strips with halo exchange
// (Methods, "TPU Implementation": one subgrid per core, borders exchanged
// between neighbours; Results, "Scaling on TPU": 1 x N strips).
//
// Each strip is an ordinary handle on the rows it stores (its own rows plus
// `halo` rows of each neighbour), so every step kernel runs on it unchanged.
// The ends of a strip inside the grid are walls to its kernels; a wall
// spoils one more row of the strip per step (the scheme's stencil reaches one
// cell), so after `halo` steps the strip's own rows -- and the face row on
// either side of them -- are still bit for bit what the whole grid computes.
// Then the halo rows are copied in again from the neighbours' own rows.  Here
// all strips live on one GPU, each stepping on a stream of its own (as each
// would on its own GPU); the copies are device-to-device copies on the
// decomposition's stream, between two joins of the strips' streams.  The copy
// list (flood_decomp_plan) names source and destination rows only, so a
// transport between GPUs would carry the same list (each row into the
// receiving GPU's own memory).
//
// Ledger: a strip books the clipped volume and outflow of its own rows only
// (Geom::led_j0/led_j1 and the halo outflow type), part 0 alone books the
// inflow volume, and h_max at an epoch end is the largest of the strips'
// own-row maxima, given to every strip before its epoch start.
#include "flood.h"

#include <c10/cuda/CUDACachingAllocator.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "flood_internal.h"
#include "flood_runtime.h"

using namespace flood;

struct flood_decomp {
    int n_parts = 0, halo = 1;
    int nx = 0, ny = 0, prec = 0, E = 16;
    size_t esz = 4;
    cudaStream_t stream = nullptr;           // the caller's: exchanges, h_max reduction, reads
    std::vector<cudaStream_t> lanes;         // one per part: the part's own work
    std::vector<cudaEvent_t> lane_ev;        // one per part
    cudaEvent_t main_ev = nullptr;
    std::vector<flood_handle *> parts;
    std::vector<int32_t> rows;               // 4 per part: y0, y1, a, b
    std::vector<flood_halo_copy> copies;
    Ctrl **ctrls_dev = nullptr;              // the parts' control blocks (device array)
    int64_t step = 0;
    int since = 0;                           // steps since the halos were last refreshed
    int sticky = 0;
    std::string err;
};

namespace {

thread_local std::string g_decomp_error;

flood_status dfail(flood_decomp *d, flood_status st, const std::string &msg)
{
    if (d) {
        d->err = msg;
        if (st == FLOOD_ERR_CUDA || st == FLOOD_ERR_NONFINITE || st == FLOOD_ERR_TIMEOUT || st == FLOOD_ERR_STATE ||
            st == FLOOD_ERR_CFL)
            d->sticky = st;
    } else {
        g_decomp_error = msg;
    }
    return st;
}

// A part's failure, reported with the part's own message.
flood_status part_fail(flood_decomp *d, int k, flood_status st)
{
    return dfail(d, st, "part " + std::to_string(k) + ": " + flood_last_error(d->parts[k]));
}

#define DCK(expr)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) return dfail(d, FLOOD_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void *field_plane(flood_handle *h, int field)
{
    switch (field) {
    case FLOOD_FIELD_H: return h->h[h->cur];
    case FLOOD_FIELD_QX: return h->qx[h->cur];
    default: return h->qy[h->cur];
    }
}

// The decomposition's stream waits for every part's stream.
flood_status join_lanes(flood_decomp *d)
{
    for (int r = 0; r < d->n_parts; r++) {
        DCK(cudaEventRecord(d->lane_ev[r], d->lanes[r]));
        DCK(cudaStreamWaitEvent(d->stream, d->lane_ev[r], 0));
    }
    return FLOOD_OK;
}

// Every part's stream waits for the decomposition's stream.
flood_status fork_lanes(flood_decomp *d)
{
    DCK(cudaEventRecord(d->main_ev, d->stream));
    for (int r = 0; r < d->n_parts; r++) DCK(cudaStreamWaitEvent(d->lanes[r], d->main_ev, 0));
    return FLOOD_OK;
}

// Refresh every part's halo rows from its neighbours' own rows (on the
// decomposition's stream, the parts' streams joined into it).
flood_status exchange(flood_decomp *d)
{
    NvtxRange range("flood: halo exchange");
    for (const flood_halo_copy &c : d->copies) {
        flood_handle *s = d->parts[c.src_part], *t = d->parts[c.dst_part];
        const size_t row_bytes = (size_t)s->geo.pitch * d->esz;
        const char *src = (const char *)field_plane(s, c.field) + (size_t)c.src_row * row_bytes;
        char *dst = (char *)field_plane(t, c.field) + (size_t)c.dst_row * row_bytes;
        DCK(cudaMemcpyAsync(dst, src, (size_t)c.rows * row_bytes, cudaMemcpyDeviceToDevice, d->stream));
    }
    d->since = 0;
    return FLOOD_OK;
}

}  // namespace

extern "C" flood_status flood_decomp_plan(int32_t ny, int32_t n_parts, int32_t halo, int32_t *part_rows,
                                          flood_halo_copy *copies, int32_t *n_copies)
{
    if (ny < 1 || n_parts < 1 || halo < 1 || !part_rows || !n_copies || *n_copies < 0)
        return dfail(nullptr, FLOOD_ERR_ARG, "ny, n_parts, halo must be >= 1; part_rows and n_copies non-NULL");
    if (n_parts > ny) return dfail(nullptr, FLOOD_ERR_ARG, "more parts than rows");
    for (int r = 0; r < n_parts; r++) {
        const int y0 = (int)((int64_t)r * ny / n_parts), y1 = (int)((int64_t)(r + 1) * ny / n_parts);
        if (n_parts > 1 && y1 - y0 < halo)
            return dfail(nullptr, FLOOD_ERR_ARG, "a strip would have fewer rows than the halo");
        part_rows[4 * r + 0] = y0;
        part_rows[4 * r + 1] = y1;
        part_rows[4 * r + 2] = r > 0 ? y0 - halo : 0;
        part_rows[4 * r + 3] = r < n_parts - 1 ? y1 + halo : ny;
    }
    std::vector<flood_halo_copy> list;
    for (int r = 0; r < n_parts; r++) {
        const int y0 = part_rows[4 * r], y1 = part_rows[4 * r + 1], a = part_rows[4 * r + 2], b = part_rows[4 * r + 3];
        if (r > 0) {               // rows [a, y0) and face rows [a, y0): the lower neighbour's own
            const int sa = part_rows[4 * (r - 1) + 2];
            for (int f : {FLOOD_FIELD_H, FLOOD_FIELD_QX, FLOOD_FIELD_QY})
                list.push_back({f, r - 1, a - sa, r, 0, y0 - a});
        }
        if (r < n_parts - 1) {     // rows [y1, b) and face rows [y1 + 1, b]: the upper neighbour's
            const int sa = part_rows[4 * (r + 1) + 2];
            for (int f : {FLOOD_FIELD_H, FLOOD_FIELD_QX})
                list.push_back({f, r + 1, y1 - sa, r, y1 - a, b - y1});
            list.push_back({FLOOD_FIELD_QY, r + 1, y1 + 1 - sa, r, y1 + 1 - a, b - y1});
        }
    }
    const int cap = *n_copies;
    *n_copies = (int32_t)list.size();
    if (copies) {
        if (cap < (int)list.size()) return dfail(nullptr, FLOOD_ERR_ARG, "copies holds too few entries");
        std::copy(list.begin(), list.end(), copies);
    }
    return FLOOD_OK;
}

extern "C" flood_status flood_decomp_combine_ledgers(int32_t n_parts, const double *L, double *out)
{
    if (n_parts < 1 || !L || !out) return dfail(nullptr, FLOOD_ERR_ARG, "bad ledger arguments");
    double r[FLOOD_LEDGER_LEN];
    std::memcpy(r, L, sizeof(r));
    for (int k = 1; k < n_parts; k++) {
        const double *p = L + (size_t)k * FLOOD_LEDGER_LEN;
        if (p[FLOOD_LEDGER_T] != r[FLOOD_LEDGER_T] || p[FLOOD_LEDGER_DT] != r[FLOOD_LEDGER_DT] ||
            p[FLOOD_LEDGER_STEP] != r[FLOOD_LEDGER_STEP])
            return dfail(nullptr, FLOOD_ERR_STATE, "parts disagree on time, time step or step count");
        for (int i : {FLOOD_LEDGER_V_IN, FLOOD_LEDGER_V_OUT, FLOOD_LEDGER_V_CLIP, FLOOD_LEDGER_VOLUME}) r[i] += p[i];
        r[FLOOD_LEDGER_H_MAX] = std::max(r[FLOOD_LEDGER_H_MAX], p[FLOOD_LEDGER_H_MAX]);
    }
    std::memcpy(out, r, sizeof(r));
    return FLOOD_OK;
}

extern "C" flood_status flood_decomp_create(const flood_grid *grid, const void *dem, const void *manning,
                                            const flood_bc_section *sections, int32_t n_sections,
                                            const flood_opts *opts, int32_t n_parts, int32_t halo, flood_decomp **out)
{
    if (!out) return dfail(nullptr, FLOOD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid) return dfail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    flood_opts o;
    if (opts) o = *opts;
    else flood_default_opts(&o);
    std::vector<int32_t> rows(4 * (size_t)std::max(n_parts, 1));
    int32_t ncopy = 0;
    flood_status st = flood_decomp_plan(grid->ny, n_parts, halo, rows.data(), nullptr, &ncopy);
    if (st) return st;
    flood_decomp *d = new flood_decomp();
    d->n_parts = n_parts;
    d->halo = halo;
    d->nx = grid->nx;
    d->ny = grid->ny;
    d->prec = grid->precision;
    d->esz = grid->precision == FLOOD_F32 ? 4 : 8;
    d->E = o.epoch_steps;
    d->rows = rows;
    d->copies.resize(ncopy);
    flood_decomp_plan(grid->ny, n_parts, halo, rows.data(), d->copies.data(), &ncopy);
    // every part runs the kernel family the whole grid would get
    if (o.kernel == FLOOD_KERNEL_AUTO && o.epoch_steps >= 1) o.kernel = auto_kernel(o, grid->nx, grid->ny);
    o.use_graph = 0;
    auto bail = [&](flood_status s, const std::string &m) {
        flood_decomp_destroy(d);
        return dfail(nullptr, s, m);
    };
    for (int r = 0; r < n_parts; r++) {
        PartSpec P{grid->ny, rows[4 * r + 2], rows[4 * r + 3], rows[4 * r], rows[4 * r + 1], r};
        flood_handle *h = nullptr;
        st = create_handle(grid, dem, manning, sections, n_sections, &o, &P, &h);
        if (st) return bail(st, std::string("part ") + std::to_string(r) + ": " + flood_last_error(nullptr));
        d->parts.push_back(h);
    }
    d->stream = d->parts[0]->stream;
    // a stream per part: the parts step side by side, as on separate GPUs
    d->lanes.assign(n_parts, nullptr);
    d->lane_ev.assign(n_parts, nullptr);
    if (cudaEventCreateWithFlags(&d->main_ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(FLOOD_ERR_CUDA, "event creation");
    for (int r = 0; r < n_parts; r++) {
        if (cudaStreamCreateWithFlags(&d->lanes[r], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&d->lane_ev[r], cudaEventDisableTiming) != cudaSuccess)
            return bail(FLOOD_ERR_CUDA, "stream creation");
    }
    // the parts' set-up on the caller's stream is done before their own streams start
    if (cudaStreamSynchronize(d->stream) != cudaSuccess) return bail(FLOOD_ERR_CUDA, "part set-up");
    for (int r = 0; r < n_parts; r++) d->parts[r]->stream = d->lanes[r];
    d->ctrls_dev = (Ctrl **)raw_device_alloc(n_parts * sizeof(Ctrl *), d->stream);
    if (!d->ctrls_dev) return bail(FLOOD_ERR_OOM, "device allocation failed");
    std::vector<Ctrl *> ctrls(n_parts);
    for (int r = 0; r < n_parts; r++) ctrls[r] = d->parts[r]->ctrl;
    if (cudaMemcpyAsync(d->ctrls_dev, ctrls.data(), n_parts * sizeof(Ctrl *), cudaMemcpyHostToDevice, d->stream) ||
        cudaStreamSynchronize(d->stream))
        return bail(FLOOD_ERR_CUDA, "control-block table upload");
    *out = d;
    return FLOOD_OK;
}

extern "C" flood_status flood_decomp_step(flood_decomp *d, int64_t n_steps)
{
    if (!d) return dfail(nullptr, FLOOD_ERR_ARG, "decomposition is NULL");
    if (n_steps < 0) return dfail(d, FLOOD_ERR_ARG, "n_steps must be >= 0");
    if (d->sticky) return dfail(d, FLOOD_ERR_STATE, "decomposition is in an error state; write a new state first");
    NvtxRange range("flood: decomposed steps");
    const int E = d->E;
    int64_t done = 0;
    {
        flood_status st = fork_lanes(d);      // whatever the caller queued comes first
        if (st) return st;
    }
    while (done < n_steps) {
        const int s = (int)(d->step % E);
        const bool due = d->since >= d->halo;
        if (s == 0 || due) {
            // every part's streams joined: the whole grid's h_max into every part at an
            // epoch start, the halo rows when due; then the parts go on side by side
            flood_status st = join_lanes(d);
            if (st) return st;
            if (s == 0) DCK(launch_hmax_allreduce(d->ctrls_dev, d->n_parts, d->stream));
            if (due && (st = exchange(d))) return st;
            if ((st = fork_lanes(d))) return st;
        }
        if (s == 0) {
            // epoch start: every part chooses dt from the whole grid's h_max, and solves Eq. 6
            for (int r = 0; r < d->n_parts; r++) {
                flood_handle *h = d->parts[r];
                DCK(launch_epoch_begin(h->geo, h->ctrl, h->t_list, E, nullptr, h->stream));
                flood_status st = launch_inflow_epoch(h);
                if (st) return part_fail(d, r, st);
            }
        }
        const int m = (int)std::min<int64_t>(std::min(d->halo - d->since, E - s), n_steps - done);
        for (int r = 0; r < d->n_parts; r++) {
            flood_handle *h = d->parts[r];
            for (int k_done = 0; k_done < m;) {
                int k = 1;
                if (h->prec == FLOOD_F32 && h->kernel == FLOOD_KERNEL_TILED) {
                    k = std::min(h->k_per_launch, m - k_done);
                    if (k > 4 && k < 8) k = 4;   // the kernel exists for 1..4 and 8 steps per launch
                }
                flood_status st = launch_steps(h, s + k_done, k, 0, nullptr, 0, nullptr);
                if (st) return part_fail(d, r, st);
                k_done += k;
            }
            h->step += m;
        }
        if (s + m == E) {
            // epoch end: each part's maximum over its own rows
            for (int r = 0; r < d->n_parts; r++) {
                flood_status st = refresh_hmax_window(d->parts[r]);
                if (st) return part_fail(d, r, st);
            }
        }
        d->step += m;
        d->since += m;
        done += m;
    }
    return join_lanes(d);                       // the caller's stream sees every part's steps
}

extern "C" flood_status flood_decomp_sync(flood_decomp *d)
{
    if (!d) return dfail(nullptr, FLOOD_ERR_ARG, "decomposition is NULL");
    if (d->sticky) return (flood_status)d->sticky;
    for (int r = 0; r < d->n_parts; r++) {
        flood_status st = flood_sync(d->parts[r]);
        if (st) return part_fail(d, r, st);
    }
    return FLOOD_OK;
}

extern "C" flood_status flood_decomp_read(flood_decomp *d, int32_t field, void *dst, size_t bytes,
                                          int32_t dst_on_device)
{
    if (!d || !dst) return dfail(d, FLOOD_ERR_ARG, "NULL argument");
    if (field == FLOOD_FIELD_LEDGER) {
        if (bytes != FLOOD_LEDGER_LEN * sizeof(double)) return dfail(d, FLOOD_ERR_ARG, "ledger needs 9 doubles");
        std::vector<double> L((size_t)d->n_parts * FLOOD_LEDGER_LEN);
        for (int r = 0; r < d->n_parts; r++) {
            flood_status st = flood_read(d->parts[r], FLOOD_FIELD_LEDGER, L.data() + (size_t)r * FLOOD_LEDGER_LEN,
                                         FLOOD_LEDGER_LEN * sizeof(double), 0);
            if (st) return part_fail(d, r, st);
        }
        double out[FLOOD_LEDGER_LEN];
        flood_status st = flood_decomp_combine_ledgers(d->n_parts, L.data(), out);
        if (st) return dfail(d, st, g_decomp_error);
        if (dst_on_device) DCK(cudaMemcpy(dst, out, sizeof(out), cudaMemcpyHostToDevice));
        else std::memcpy(dst, out, sizeof(out));
        return FLOOD_OK;
    }
    if (field < FLOOD_FIELD_H || field > FLOOD_FIELD_N) return dfail(d, FLOOD_ERR_ARG, "unknown field");
    {
        flood_status st = join_lanes(d);       // the parts' last writes come first
        if (st) return st;
    }
    const int rows_all = d->ny + (field == FLOOD_FIELD_QY ? 1 : 0);
    const int cols = d->nx + (field == FLOOD_FIELD_QX ? 1 : 0);
    if (bytes != (size_t)rows_all * cols * d->esz) return dfail(d, FLOOD_ERR_ARG, "dst size does not match the field");
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int r = 0; r < d->n_parts; r++) {
        flood_handle *h = d->parts[r];
        const int y0 = d->rows[4 * r], y1 = d->rows[4 * r + 1], a = d->rows[4 * r + 2];
        // own rows [y0, y1); the last part also the grid's north face row
        const int n = (y1 - y0) + ((field == FLOOD_FIELD_QY && r == d->n_parts - 1) ? 1 : 0);
        const void *plane = field == FLOOD_FIELD_Z ? h->z : field == FLOOD_FIELD_N ? h->n : field_plane(h, field);
        const size_t pitch_b = (size_t)h->geo.pitch * d->esz;
        DCK(cudaMemcpy2DAsync((char *)dst + (size_t)y0 * cols * d->esz, (size_t)cols * d->esz,
                              (const char *)plane + (size_t)(y0 - a) * pitch_b, pitch_b, (size_t)cols * d->esz, n, kind,
                              d->stream));
    }
    DCK(cudaStreamSynchronize(d->stream));
    return FLOOD_OK;
}

extern "C" flood_status flood_decomp_write_state(flood_decomp *d, const void *depth, const void *qx, const void *qy,
                                                 int32_t src_on_device)
{
    if (!d || !depth) return dfail(d, FLOOD_ERR_ARG, "NULL argument");
    const size_t e = d->esz;
    {
        flood_status st = fork_lanes(d);       // device sources the caller wrote on its stream come first
        if (st) return st;
    }
    for (int r = 0; r < d->n_parts; r++) {
        const int a = d->rows[4 * r + 2];
        const char *hp = (const char *)depth + (size_t)a * d->nx * e;
        const char *xp = qx ? (const char *)qx + (size_t)a * (d->nx + 1) * e : nullptr;
        const char *yp = qy ? (const char *)qy + (size_t)a * d->nx * e : nullptr;
        flood_status st = flood_write_state(d->parts[r], hp, xp, yp, src_on_device);
        if (st) {
            // parts before r hold the new state, the others the old one
            if (r > 0) d->sticky = FLOOD_ERR_STATE;
            return dfail(d, st, std::string("part ") + std::to_string(r) + ": " + flood_last_error(d->parts[r]));
        }
    }
    d->since = 0;
    d->sticky = FLOOD_OK;
    d->err.clear();
    return FLOOD_OK;
}

extern "C" flood_handle *flood_decomp_part(flood_decomp *d, int32_t k)
{
    if (!d || k < 0 || k >= d->n_parts) return nullptr;
    return d->parts[k];
}

extern "C" flood_status flood_decomp_destroy(flood_decomp *d)
{
    if (!d) return FLOOD_OK;
    for (cudaStream_t l : d->lanes)
        if (l) cudaStreamSynchronize(l);
    // the parts' memory goes back on the caller's stream, where it was taken
    for (size_t r = 0; r < d->parts.size(); r++) {
        flood_handle *h = d->parts[r];
        if (r < d->lanes.size() && d->lanes[r] && h->stream == d->lanes[r]) h->stream = d->stream;
        flood_destroy(h);
    }
    if (d->ctrls_dev) c10::cuda::CUDACachingAllocator::raw_delete(d->ctrls_dev);
    for (cudaEvent_t e : d->lane_ev)
        if (e) cudaEventDestroy(e);
    if (d->main_ev) cudaEventDestroy(d->main_ev);
    for (cudaStream_t l : d->lanes)
        if (l) cudaStreamDestroy(l);
    delete d;
    return FLOOD_OK;
}

extern "C" const char *flood_decomp_last_error(const flood_decomp *d)
{
    if (!d) return g_decomp_error.c_str();
    return d->err.c_str();
}
