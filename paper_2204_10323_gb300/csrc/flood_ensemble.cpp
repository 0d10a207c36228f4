// flood_ensemble.cpp -- many independent scenarios (own grid size, terrain,
// roughness, hydrograph) advanced together: one launch covers every scenario
// (largest first), either one step of the stream kernel over the blocks of
// all scenarios, or K steps of the temporal-blocking kernel over their
// (chunk, strip) items; whole CFL epochs (per-scenario time step and Eq. 6
// inflow, then the steps) are captured once into a CUDA graph and replayed.
// Each scenario is an ordinary FP32 handle, so flood_read / flood_write_state
// work on it.
#include "flood.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "flood_internal.h"
#include "flood_runtime.h"

using namespace flood;

struct flood_ensemble {
    std::vector<flood_handle *> members;   // creation order
    std::vector<int> order;                // block order: largest grid first
    int E = 16;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    int warps = 4, rows = 64, steps_per_graph = 16;
    int kernel = FLOOD_KERNEL_STREAM, k_steps = 4;   // TILED: k_steps per launch, rows per item
    int mode = 0;                          // scheme options: bit 0 theta weighting, bit 1 vector-norm friction
    StepArgs<float> *table[2] = {nullptr, nullptr};   // per parity of the ping-pong buffers
    int *base = nullptr;                   // block prefix, n + 1
    int total_blocks = 0;
    int *tbase = nullptr;                  // tiled item prefix, n + 1
    int total_items = 0;
    int *next_item = nullptr;              // tiled: the item counter of the launch (zeroed before each)
    // tiled: the members in two groups of about equal cells, each launched on a stream of its
    // own from one epoch start to the next, so that one group's launches fill the other's tails
    static constexpr int kGroups = 2;
    std::vector<int> group_of;             // per member
    StepArgs<float> *gtable[kGroups][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [group][parity]
    int *gtbase[kGroups] = {nullptr, nullptr};
    int *gnext[kGroups] = {nullptr, nullptr};
    int gn[kGroups] = {0, 0}, gtotal[kGroups] = {0, 0};
    EpochArgs<float> *getab[kGroups] = {nullptr, nullptr};   // the group's members' epoch arguments
    int2 *gtasks[kGroups] = {nullptr, nullptr};              // (member in the group, inflow section)
    int gntasks[kGroups] = {0, 0};
    cudaStream_t lane[kGroups] = {nullptr, nullptr};
    cudaEvent_t lane_ev[kGroups] = {nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr;
    bool forked = false;                   // the groups' streams run ahead of `stream`
    EpochArgs<float> *etab = nullptr;      // per member: epoch bookkeeping arguments
    int2 *tasks = nullptr;                 // (member, inflow section) pairs
    int n_tasks = 0;
    std::vector<cudaGraphExec_t> graphs;   // [parity]
    int graph_launches = 0;                // step launches in one graph (each flips the buffers)
    int use_graph = 1;
    std::string err;
    flood_handle *owner = nullptr;         // member 0: allocations for the tables
};

namespace {

thread_local std::string g_ens_error;

flood_status efail(flood_ensemble *e, flood_status st, const std::string &m)
{
    if (e) e->err = m;
    else g_ens_error = m;
    return st;
}

void drop_graphs(flood_ensemble *e)
{
    for (auto &g : e->graphs)
        if (g) cudaGraphExecDestroy(g);
    e->graphs.assign(2, nullptr);
}

// Epoch bookkeeping arguments of a member.
EpochArgs<float> epoch_args(const flood_handle *h)
{
    EpochArgs<float> A;
    A.geo = h->geo;
    A.ctrl = h->ctrl;
    A.t_list = h->t_list;
    A.secs = h->secs_dev;
    A.nsec = h->n_in;
    A.cells = h->sec_cells;
    A.tab_t = h->tab_t;
    A.tab_q = h->tab_q;
    A.z = (const float *)h->z;
    A.n = (const float *)h->n;
    A.inflow_q = (float *)h->inflow_q;
    A.n_slots = h->n_slots;
    A.inflow_Q = h->inflow_Q;
    A.inflow_W = h->inflow_W;
    return A;
}

// Rows per work item of the temporal-blocking kernel for a member grid: the
// launch shape's rows for a grid of 2^20 cells, scaled by the square root of
// the grid's cells over that, at least 32 and at most the grid's rows.  The
// grids come largest first, so the items shrink towards the end of a launch,
// where the pipelines, taking items as they come free, fill the tail with the
// small ones (the measured best of several rules on uneven scenario mixes).
int item_rows(const flood_ensemble *e, const Geom &g)
{
    const double cells = (double)g.nx * g.ny;
    const int r = (int)(e->rows * std::sqrt(cells / (double)(1 << 20)) + 0.5);
    return std::min(std::max(r, 32), g.ny);
}

flood_status build_tables(flood_ensemble *e)
{
    const int n = (int)e->members.size();
    std::vector<int> base(n + 1, 0), tbase(n + 1, 0);
    for (int k = 0; k < n; k++) {
        const Geom &g = e->members[e->order[k]]->geo;
        base[k + 1] = base[k] + stream_blocks(g, e->warps, e->rows);
        tbase[k + 1] = tbase[k] + tiled_items(g, item_rows(e, g), e->k_steps);
    }
    e->total_blocks = base[n];
    e->total_items = tbase[n];
    for (int p = 0; p < 2; p++) {
        std::vector<StepArgs<float>> t(n);
        for (int k = 0; k < n; k++) {
            flood_handle *h = e->members[e->order[k]];
            const int cur = h->cur;
            h->cur = p;
            t[k] = step_args_f32(h, 0);
            t[k].tile_y = item_rows(e, h->geo);
            h->cur = cur;
        }
        cudaError_t c = cudaMemcpyAsync(e->table[p], t.data(), n * sizeof(StepArgs<float>), cudaMemcpyHostToDevice,
                                        e->stream);
        if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    }
    cudaError_t c = cudaMemcpyAsync(e->base, base.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, e->stream);
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    c = cudaMemcpyAsync(e->tbase, tbase.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, e->stream);
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    // the groups: largest member first into the group with fewer cells so far
    {
        int64_t cells[flood_ensemble::kGroups] = {0, 0};
        std::vector<int> members[flood_ensemble::kGroups];
        for (int k = 0; k < n; k++) {
            const int m = e->order[k];
            const int g = cells[1] < cells[0] ? 1 : 0;
            members[g].push_back(m);
            cells[g] += (int64_t)e->members[m]->geo.nx * e->members[m]->geo.ny;
        }
        for (int g = 0; g < flood_ensemble::kGroups; g++) {
            const int ng = (int)members[g].size();
            std::vector<int> gb(ng + 1, 0);
            for (int i = 0; i < ng; i++) {
                const Geom &G = e->members[members[g][i]]->geo;
                gb[i + 1] = gb[i] + tiled_items(G, item_rows(e, G), e->k_steps);
            }
            e->gn[g] = ng;
            e->gtotal[g] = gb[ng];
            for (int p = 0; p < 2; p++) {
                std::vector<StepArgs<float>> t(ng);
                for (int i = 0; i < ng; i++) {
                    flood_handle *h = e->members[members[g][i]];
                    const int cur = h->cur;
                    h->cur = p;
                    t[i] = step_args_f32(h, 0);
                    t[i].tile_y = item_rows(e, h->geo);
                    h->cur = cur;
                }
                if (ng && (c = cudaMemcpyAsync(e->gtable[g][p], t.data(), ng * sizeof(StepArgs<float>),
                                               cudaMemcpyHostToDevice, e->stream)) != cudaSuccess)
                    return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
            }
            c = cudaMemcpyAsync(e->gtbase[g], gb.data(), (ng + 1) * sizeof(int), cudaMemcpyHostToDevice, e->stream);
            if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
            // the group's own epoch starts (dt, Eq. 6), on its stream
            std::vector<EpochArgs<float>> et(ng);
            std::vector<int2> tk;
            for (int i = 0; i < ng; i++) {
                const flood_handle *h = e->members[members[g][i]];
                et[i] = epoch_args(h);
                for (int sct = 0; sct < h->n_in; sct++) tk.push_back(make_int2(i, sct));
            }
            e->gntasks[g] = (int)tk.size();
            if (ng && (c = cudaMemcpyAsync(e->getab[g], et.data(), ng * sizeof(EpochArgs<float>), cudaMemcpyHostToDevice,
                                           e->stream)) != cudaSuccess)
                return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
            if (tk.size() && (c = cudaMemcpyAsync(e->gtasks[g], tk.data(), tk.size() * sizeof(int2),
                                                  cudaMemcpyHostToDevice, e->stream)) != cudaSuccess)
                return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
        }
    }
    c = cudaStreamSynchronize(e->stream);
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    drop_graphs(e);
    return FLOOD_OK;
}

// `st` waits for the groups' streams (after their launches since the last fork).
flood_status join_groups(flood_ensemble *e, cudaStream_t st)
{
    if (!e->forked) return FLOOD_OK;
    for (int g = 0; g < flood_ensemble::kGroups; g++) {
        cudaError_t c = cudaEventRecord(e->lane_ev[g], e->lane[g]);
        if (c == cudaSuccess) c = cudaStreamWaitEvent(st, e->lane_ev[g], 0);
        if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    }
    e->forked = false;
    return FLOOD_OK;
}

// The groups' streams wait for `st`.
flood_status fork_groups(flood_ensemble *e, cudaStream_t st)
{
    if (e->forked) return FLOOD_OK;
    cudaError_t c = cudaEventRecord(e->fork_ev, st);
    for (int g = 0; g < flood_ensemble::kGroups && c == cudaSuccess; g++) c = cudaStreamWaitEvent(e->lane[g], e->fork_ev, 0);
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    e->forked = true;
    return FLOOD_OK;
}

// One launch for every member: one step (stream kernel) or up to k_steps steps
// (temporal blocking), never past the end of the epoch or beyond `limit`
// steps; epoch bookkeeping per member when due.  Returns the steps taken in *k.
flood_status ensemble_step(flood_ensemble *e, int64_t limit, cudaStream_t st, int *k)
{
    const int E = e->E;
    const int s = (int)(e->step % E);
    const bool grouped = e->kernel == FLOOD_KERNEL_TILED && !(e->k_steps == 8 && (int)std::min<int64_t>(E - s, limit) < 8);
    if (s == 0 && grouped) {
        // each group starts its members' epoch on its own stream
        flood_status fs = fork_groups(e, st);
        if (fs) return fs;
        for (int g = 0; g < flood_ensemble::kGroups; g++) {
            if (e->gn[g] == 0) continue;
            cudaError_t c = launch_epoch_batched<float>(e->getab[g], e->gn[g], e->gtasks[g], e->gntasks[g], E, e->lane[g]);
            if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
        }
    } else if (s == 0) {
        flood_status fs = join_groups(e, st);
        if (fs) return fs;
        cudaError_t c = launch_epoch_batched<float>(e->etab, (int)e->members.size(), e->tasks, e->n_tasks, E, st);
        if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    }
    const int parity = e->members[0]->cur;
    const int n = (int)e->members.size();
    int steps = 1;
    cudaError_t c;
    if (e->kernel == FLOOD_KERNEL_TILED) {
        steps = (int)std::min<int64_t>(e->k_steps, std::min<int64_t>(E - s, limit));
    }
    // the item table is laid out for k_steps: 8-step tables (wider halos) take
    // only whole 8-step launches, anything shorter runs single stream steps
    if (e->kernel == FLOOD_KERNEL_TILED && !(e->k_steps == 8 && steps < 8)) {
        flood_status fs = fork_groups(e, st);
        if (fs) return fs;
        c = cudaSuccess;
        for (int g = 0; g < flood_ensemble::kGroups && c == cudaSuccess; g++) {
            if (e->gn[g] == 0) continue;
            c = cudaMemsetAsync(e->gnext[g], 0, sizeof(int), e->lane[g]);
            if (c == cudaSuccess)
                c = launch_step_tiled_ensemble(e->gtable[g][parity], e->gtbase[g], e->gn[g], e->gtotal[g], steps, s,
                                               s + steps == E ? 1 : 0, e->gnext[g], e->mode, e->lane[g]);
        }
    } else {
        flood_status fs = join_groups(e, st);
        if (fs) return fs;
        steps = 1;
        c = launch_step_stream_ensemble(e->table[parity], e->base, n, e->total_blocks, e->warps, e->rows, s,
                                        s == E - 1 ? 1 : 0, e->mode, st);
    }
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    for (flood_handle *h : e->members) {
        h->cur = 1 - h->cur;
        h->step += steps;
    }
    e->step += steps;
    *k = steps;
    return FLOOD_OK;
}

flood_status capture(flood_ensemble *e, int parity)
{
    cudaStream_t cap = nullptr;
    cudaError_t c = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    const int64_t step0 = e->step;
    std::vector<int> cur0;
    std::vector<int64_t> st0;
    for (flood_handle *h : e->members) {
        cur0.push_back(h->cur);
        st0.push_back(h->step);
    }
    c = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    flood_status fs = FLOOD_OK;
    int launches = 0;
    if (c == cudaSuccess) {
        for (int k = 0, taken = 0; k < e->steps_per_graph && !fs; k += taken, launches++)
            fs = ensemble_step(e, e->steps_per_graph - k, cap, &taken);
        if (!fs) fs = join_groups(e, cap);
    }
    e->forked = false;
    cudaGraph_t graph = nullptr;
    cudaError_t c2 = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    e->step = step0;
    for (size_t k = 0; k < e->members.size(); k++) {
        e->members[k]->cur = cur0[k];
        e->members[k]->step = st0[k];
    }
    if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    if (fs) {
        if (graph) cudaGraphDestroy(graph);
        return fs;
    }
    if (c2 != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c2));
    c = cudaGraphInstantiate(&e->graphs[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (c != cudaSuccess) {
        e->graphs[parity] = nullptr;
        return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
    }
    e->graph_launches = launches;
    return FLOOD_OK;
}

}  // namespace

extern "C" flood_status flood_ensemble_create(int32_t n, const flood_grid *grids, const void *const *dems,
                                              const void *const *mannings, const flood_bc_section *const *sections,
                                              const int32_t *n_sections, const flood_opts *opts,
                                              flood_ensemble **out)
{
    if (!out) return efail(nullptr, FLOOD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !dems || !n_sections) return efail(nullptr, FLOOD_ERR_ARG, "bad ensemble arguments");
    flood_opts o;
    if (opts) o = *opts;
    else flood_default_opts(&o);
    o.kernel = FLOOD_KERNEL_STREAM;
    o.use_graph = 0;
    flood_ensemble *e = new flood_ensemble();
    e->E = o.epoch_steps;
    e->mode = (o.theta != 1.0 ? 1 : 0) | (o.friction != 0 ? 2 : 0);
    e->graphs.assign(2, nullptr);
    for (int k = 0; k < n; k++) {
        if (grids[k].precision != FLOOD_F32) {
            flood_ensemble_destroy(e);
            return efail(nullptr, FLOOD_ERR_UNSUPPORTED, "ensembles are FP32");
        }
        flood_handle *h = nullptr;
        flood_status st = flood_create(&grids[k], dems[k], mannings ? mannings[k] : nullptr,
                                       sections ? sections[k] : nullptr, n_sections[k], &o, &h);
        if (st) {
            std::string m = std::string("member ") + std::to_string(k) + ": " + flood_last_error(nullptr);
            flood_ensemble_destroy(e);
            return efail(nullptr, st, m);
        }
        h->in_ensemble = true;
        e->members.push_back(h);
    }
    e->stream = e->members[0]->stream;
    e->owner = e->members[0];
    for (flood_handle *h : e->members)
        if (h->stream != e->stream) {
            flood_ensemble_destroy(e);
            return efail(nullptr, FLOOD_ERR_ARG, "members must share one stream");
        }
    e->order.resize(n);
    std::iota(e->order.begin(), e->order.end(), 0);
    std::stable_sort(e->order.begin(), e->order.end(), [&](int a, int b) {
        return (int64_t)e->members[a]->geo.nx * e->members[a]->geo.ny >
               (int64_t)e->members[b]->geo.nx * e->members[b]->geo.ny;
    });
    for (int p = 0; p < 2; p++) {
        e->table[p] = (StepArgs<float> *)dev_alloc(e->owner, n * sizeof(StepArgs<float>));
        if (!e->table[p]) {
            flood_ensemble_destroy(e);
            return efail(nullptr, FLOOD_ERR_OOM, "ensemble table");
        }
    }
    e->base = (int *)dev_alloc(e->owner, (n + 1) * sizeof(int));
    e->tbase = (int *)dev_alloc(e->owner, (n + 1) * sizeof(int));
    e->next_item = (int *)dev_alloc(e->owner, sizeof(int));
    for (int g = 0; g < flood_ensemble::kGroups; g++) {
        for (int p = 0; p < 2; p++) e->gtable[g][p] = (StepArgs<float> *)dev_alloc(e->owner, n * sizeof(StepArgs<float>));
        e->gtbase[g] = (int *)dev_alloc(e->owner, (n + 1) * sizeof(int));
        e->gnext[g] = (int *)dev_alloc(e->owner, sizeof(int));
        e->getab[g] = (EpochArgs<float> *)dev_alloc(e->owner, n * sizeof(EpochArgs<float>));
        int n_sec_all = 0;
        for (flood_handle *h : e->members) n_sec_all += h->n_in;
        e->gtasks[g] = (int2 *)dev_alloc(e->owner, std::max(n_sec_all, 1) * sizeof(int2));
        if (!e->gtable[g][0] || !e->gtable[g][1] || !e->gtbase[g] || !e->gnext[g] || !e->getab[g] || !e->gtasks[g] ||
            cudaStreamCreateWithFlags(&e->lane[g], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e->lane_ev[g], cudaEventDisableTiming) != cudaSuccess) {
            flood_ensemble_destroy(e);
            return efail(nullptr, FLOOD_ERR_OOM, "ensemble group tables and streams");
        }
    }
    if (cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
        flood_ensemble_destroy(e);
        return efail(nullptr, FLOOD_ERR_CUDA, "event creation");
    }
    e->etab = (EpochArgs<float> *)dev_alloc(e->owner, n * sizeof(EpochArgs<float>));
    std::vector<EpochArgs<float>> et(n);
    std::vector<int2> tk;
    for (int k = 0; k < n; k++) {
        flood_handle *h = e->members[k];
        EpochArgs<float> &A = et[k];
        A.geo = h->geo;
        A.ctrl = h->ctrl;
        A.t_list = h->t_list;
        A.secs = h->secs_dev;
        A.nsec = h->n_in;
        A.cells = h->sec_cells;
        A.tab_t = h->tab_t;
        A.tab_q = h->tab_q;
        A.z = (const float *)h->z;
        A.n = (const float *)h->n;
        A.inflow_q = (float *)h->inflow_q;
        A.n_slots = h->n_slots;
        A.inflow_Q = h->inflow_Q;
        A.inflow_W = h->inflow_W;
        for (int sct = 0; sct < h->n_in; sct++) tk.push_back(make_int2(k, sct));
    }
    e->n_tasks = (int)tk.size();
    e->tasks = (int2 *)dev_alloc(e->owner, std::max<size_t>(tk.size(), 1) * sizeof(int2));
    if (!e->base || !e->tbase || !e->next_item || !e->etab || !e->tasks ||
        cudaMemcpyAsync(e->etab, et.data(), n * sizeof(EpochArgs<float>), cudaMemcpyHostToDevice, e->stream) ||
        (tk.size() &&
         cudaMemcpyAsync(e->tasks, tk.data(), tk.size() * sizeof(int2), cudaMemcpyHostToDevice, e->stream))) {
        flood_ensemble_destroy(e);
        return efail(nullptr, FLOOD_ERR_OOM, "ensemble table");
    }
    flood_status st = build_tables(e);
    if (st) {
        std::string m = e->err;
        flood_ensemble_destroy(e);
        return efail(nullptr, st, m);
    }
    *out = e;
    return FLOOD_OK;
}

extern "C" flood_status flood_ensemble_set_launch(flood_ensemble *e, int32_t warps, int32_t rows,
                                                  int32_t steps_per_graph, int32_t use_graph)
{
    if (!e) return efail(nullptr, FLOOD_ERR_ARG, "ensemble is NULL");
    if (warps < 1 || warps > 4 || rows < 1 || steps_per_graph < 1 || steps_per_graph % e->E != 0)
        return efail(e, FLOOD_ERR_ARG, "warps 1..4, rows >= 1, steps_per_graph a multiple of epoch_steps");
    e->warps = warps;
    e->rows = rows;
    e->steps_per_graph = steps_per_graph;
    e->use_graph = use_graph ? 1 : 0;
    return build_tables(e);
}

extern "C" flood_status flood_ensemble_set_kernel(flood_ensemble *e, int32_t kernel, int32_t steps_per_launch)
{
    if (!e) return efail(nullptr, FLOOD_ERR_ARG, "ensemble is NULL");
    if (kernel != FLOOD_KERNEL_STREAM && kernel != FLOOD_KERNEL_TILED)
        return efail(e, FLOOD_ERR_ARG, "ensemble kernel must be FLOOD_KERNEL_STREAM or FLOOD_KERNEL_TILED");
    const int K = steps_per_launch > 0 ? steps_per_launch : 4;
    if (kernel == FLOOD_KERNEL_TILED && (!(K <= 4 || K == 8) || e->E % K != 0))
        return efail(e, FLOOD_ERR_ARG, "steps_per_launch must be 1..4 or 8 and divide epoch_steps");
    e->kernel = kernel;
    e->k_steps = kernel == FLOOD_KERNEL_TILED ? K : 1;
    return build_tables(e);                  // item counts depend on K; drops the graphs
}

extern "C" flood_status flood_ensemble_step(flood_ensemble *e, int64_t n_steps)
{
    if (!e) return efail(nullptr, FLOOD_ERR_ARG, "ensemble is NULL");
    NvtxRange range("flood: ensemble steps");
    if (n_steps < 0) return efail(e, FLOOD_ERR_ARG, "n_steps must be >= 0");
    for (flood_handle *h : e->members)
        if (h->sticky) return efail(e, FLOOD_ERR_STATE, "a member is in an error state");
    while (n_steps > 0) {
        const int s = (int)(e->step % e->E);
        if (e->use_graph && s == 0 && n_steps >= e->steps_per_graph) {
            const int parity = e->members[0]->cur;
            flood_status js = join_groups(e, e->stream);   // the groups' streams join before a capture or replay
            if (js) return js;
            if (!e->graphs[parity]) {
                flood_status st = capture(e, parity);
                if (st) return st;
            }
            cudaError_t c = cudaGraphLaunch(e->graphs[parity], e->stream);
            if (c != cudaSuccess) return efail(e, FLOOD_ERR_CUDA, cudaGetErrorString(c));
            const int flips = e->graph_launches & 1;
            for (flood_handle *h : e->members) {
                h->cur ^= flips;
                h->step += e->steps_per_graph;
            }
            e->step += e->steps_per_graph;
            n_steps -= e->steps_per_graph;
            continue;
        }
        int taken = 0;
        flood_status st = ensemble_step(e, n_steps, e->stream, &taken);
        if (st) return st;
        n_steps -= taken;
    }
    return join_groups(e, e->stream);           // the members' stream sees every step
}

extern "C" flood_handle *flood_ensemble_member(flood_ensemble *e, int32_t k)
{
    if (!e || k < 0 || k >= (int32_t)e->members.size()) return nullptr;
    return e->members[k];
}

extern "C" flood_status flood_ensemble_destroy(flood_ensemble *e)
{
    if (!e) return FLOOD_OK;
    if (e->stream) cudaStreamSynchronize(e->stream);
    for (int g = 0; g < flood_ensemble::kGroups; g++)
        if (e->lane[g]) cudaStreamSynchronize(e->lane[g]);
    drop_graphs(e);
    if (e->owner) {
        for (int p = 0; p < 2; p++)
            if (e->table[p]) dev_free(e->owner, e->table[p]);
        if (e->base) dev_free(e->owner, e->base);
        if (e->tbase) dev_free(e->owner, e->tbase);
        if (e->next_item) dev_free(e->owner, e->next_item);
        for (int g = 0; g < flood_ensemble::kGroups; g++) {
            for (int p = 0; p < 2; p++)
                if (e->gtable[g][p]) dev_free(e->owner, e->gtable[g][p]);
            if (e->gtbase[g]) dev_free(e->owner, e->gtbase[g]);
            if (e->gnext[g]) dev_free(e->owner, e->gnext[g]);
            if (e->getab[g]) dev_free(e->owner, e->getab[g]);
            if (e->gtasks[g]) dev_free(e->owner, e->gtasks[g]);
        }
        if (e->etab) dev_free(e->owner, e->etab);
        if (e->tasks) dev_free(e->owner, e->tasks);
    }
    for (flood_handle *h : e->members) flood_destroy(h);
    for (int g = 0; g < flood_ensemble::kGroups; g++) {
        if (e->lane_ev[g]) cudaEventDestroy(e->lane_ev[g]);
        if (e->lane[g]) cudaStreamDestroy(e->lane[g]);
    }
    if (e->fork_ev) cudaEventDestroy(e->fork_ev);
    delete e;
    return FLOOD_OK;
}

extern "C" const char *flood_ensemble_last_error(const flood_ensemble *e)
{
    return e ? e->err.c_str() : g_ens_error.c_str();
}
