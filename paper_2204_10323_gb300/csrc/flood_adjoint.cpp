// flood_adjoint.cpp -- reverse sweep driver of flood_adjoint: binomial
// checkpointing (Griewank & Walther, "Algorithm 799: revolve") over device
// resident snapshots, frozen time-step schedule, per-step adjoint kernels.
//
// Cost model: reversing l steps with the start state stored and s free
// snapshot slots takes F(l, s) forward steps, F(1, s) = 0, F(l, 0) =
// l(l-1)/2, F(l, s) = min_j [j + F(l-j, s-1) + F(j, s)]; the minimum equals
// the binomial closed form r l - C(c + r, c + 1) with c = s + 1 and r the
// least integer with C(c + r, c) >= l.  The schedule below places each
// snapshot at a split j attaining that minimum.
#include "flood.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "flood_internal.h"
#include "flood_runtime.h"

using namespace flood;

struct flood_adjoint_state {
    int dummy = 0;
};

namespace flood {

void destroy_adjoint(flood_handle *h)
{
    delete h->adj;
    h->adj = nullptr;
}

// C(c + r, c) with saturation.
static int64_t beta(int64_t c, int64_t r)
{
    double v = 1.0;
    for (int64_t k = 1; k <= r; k++) {
        v = v * (double)(c + k) / (double)k;
        if (v > 4e18) return (int64_t)4e18;
    }
    return (int64_t)(v + 0.5);
}

// Forward steps needed to reverse l steps with c snapshots including the start state's.
int64_t revolve_cost(int64_t l, int64_t c)
{
    if (l <= 1) return 0;
    if (c <= 1) return l * (l - 1) / 2;
    int64_t r = 0;
    while (beta(c, r) < l) r++;
    return r * l - beta(c + 1, r - 1);
}

namespace {

#define CKA(expr)                                                     \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr);        \
    } while (0)

struct Planes {
    void *h = nullptr, *qx = nullptr, *qy = nullptr;
};

struct Sweep {
    flood_handle *h = nullptr;
    bool profile = false;            // time every reverse step and forward replay with events
    std::vector<cudaEvent_t> ev_rev, ev_fwd;   // start/end pairs
    int64_t g0 = 0, N = 0;           // first global step, steps to reverse
    int E = 16;
    size_t plane = 0, plane_y = 0;
    std::vector<Planes> slots;
    std::vector<int> free_slots;
    Planes work[2];                  // the handle's two state buffers (replay outputs)
    Planes src;                      // where the state of work_step lives: a work buffer or a slot
    int64_t work_step = -1;          // local index of that state
    // epoch logs (device), one slice per epoch touched: dt, the E+1 start times
    // and the Eq. 6 rows (inflow_q, inflow_Q, inflow_W); the handle's epoch
    // pointers are aimed at the slice of the epoch in use
    double *dt_log = nullptr, *tl_log = nullptr;
    void *iq_log = nullptr;
    double *iQ_log = nullptr, *iW_log = nullptr;
    size_t iq_bytes = 0, nQ = 0;     // per epoch: bytes of inflow_q, doubles of inflow_Q / inflow_W
    std::vector<char> logged;
    int64_t e0 = 0;
    int64_t loaded = -1;             // epoch whose slice the handle's epoch pointers hold
    // adjoint buffers
    void *lh[2] = {nullptr, nullptr}, *lqx[2] = {nullptr, nullptr}, *lqy[2] = {nullptr, nullptr};
    void *lhu = nullptr;
    void *scratch = nullptr;      // the scheme options' reverse step: 11 planes of pitch x (ny + 1)
    double *gn = nullptr;
    double *gn_in = nullptr;      // FP32, Eq. 3 as printed, with inflow sections: their dL/dn terms per cell
    int n_in_cells = 0;
    int cur_l = 0;
    const int64_t *cells = nullptr;
    int G = 0;
    const double *seed = nullptr;    // device, N x G
    int64_t fwd_steps = 0;
    int64_t prof_fwd_steps = 0;      // forward steps inside the profiled launches
    int64_t launches = 0;            // forward replay launches
    int max_k = 1;                   // steps a replay launch may take at most
    std::vector<int64_t> slot_step;  // the step whose state each snapshot slot holds (-1: none)
    bool dry = false;                // the schedule alone, no device work (flood_revolve_plan)
    std::vector<int64_t> reversed;   // dry runs: the steps reversed, in order
};

flood_status copy_planes(flood_handle *h, const Planes &dst, const Planes &src, size_t plane, size_t plane_y)
{
    CKA(cudaMemcpyAsync(dst.h, src.h, plane, cudaMemcpyDeviceToDevice, h->stream));
    CKA(cudaMemcpyAsync(dst.qx, src.qx, plane, cudaMemcpyDeviceToDevice, h->stream));
    CKA(cudaMemcpyAsync(dst.qy, src.qy, plane_y, cudaMemcpyDeviceToDevice, h->stream));
    return FLOOD_OK;
}

Planes working(flood_handle *h)
{
    Planes p;
    p.h = h->h[h->cur];
    p.qx = h->qx[h->cur];
    p.qy = h->qy[h->cur];
    return p;
}

// Run fn between two events recorded on the handle's stream (profiling only).
template <typename Fn>
flood_status timed(Sweep &S, std::vector<cudaEvent_t> &evs, Fn fn)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return fail(S.h, FLOOD_ERR_CUDA, "event create");
    evs.push_back(a);
    evs.push_back(b);
    cudaEventRecord(a, S.h->stream);
    flood_status st = fn();
    cudaEventRecord(b, S.h->stream);
    return st;
}

double sum_pairs(std::vector<cudaEvent_t> &evs)
{
    double total = 0.0;
    for (size_t k = 0; k + 1 < evs.size(); k += 2) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, evs[k], evs[k + 1]) == cudaSuccess) total += ms;
    }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    evs.clear();
    return total;
}

// Aim the handle's epoch pointers at epoch e's slice; the first visit (the
// state of work_step is then the epoch's first state) chooses dt by the rule
// and solves Eq. 6 into the slice, later visits only set dt.
flood_status ensure_epoch(Sweep &S, int64_t e)
{
    flood_handle *h = S.h;
    if (S.loaded == e) return FLOOD_OK;
    const int64_t ie = e - S.e0;
    const int E = S.E;
    h->t_list = S.tl_log + ie * (E + 1);
    h->inflow_q = (char *)S.iq_log + ie * S.iq_bytes;
    h->inflow_Q = S.iQ_log + ie * S.nQ;
    h->inflow_W = S.iW_log + ie * S.nQ;
    double *dtl = S.dt_log + ie;
    if (!S.logged[ie]) {
        CKA(cudaMemsetAsync(&h->ctrl->hmax_bits, 0, sizeof(unsigned long long), h->stream));
        if (h->prec == FLOOD_F32) CKA(launch_hmax<float>(h->geo, (const float *)S.src.h, h->ctrl, h->stream));
        else CKA(launch_hmax<double>(h->geo, (const double *)S.src.h, h->ctrl, h->stream));
        CKA(launch_epoch_begin(h->geo, h->ctrl, h->t_list, E, nullptr, h->stream));
        CKA(cudaMemcpyAsync(dtl, &h->ctrl->dt, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        flood_status st = launch_inflow_epoch(h);
        if (st) return st;
        S.logged[ie] = 1;
    } else {
        CKA(cudaMemcpyAsync(&h->ctrl->dt, dtl, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    S.loaded = e;
    return FLOOD_OK;
}

bool same(const Planes &a, const Planes &b) { return a.h == b.h; }

// Steps the next replay launch may take towards `step`: up to S.max_k (4 for FP32
// grids running Eq. 3 as printed, whose temporal-blocking kernel gives the single
// steps' bits; 1 otherwise), never past the end of the epoch.
int replay_steps(const Sweep &S, int64_t step)
{
    if (S.max_k <= 1) return 1;
    const int s = (int)((S.g0 + S.work_step) % S.E);
    return (int)std::min<int64_t>(std::min<int64_t>(step - S.work_step, S.max_k), S.E - s);
}

// One forward replay launch of k steps (replay_steps) from S.src into `dst` (a
// free slot: a checkpoint being taken) or else into the work buffer that S.src
// is not.
flood_status forward_step(Sweep &S, const Planes *dst = nullptr, int k = 1)
{
    flood_handle *h = S.h;
    const int64_t g = S.g0 + S.work_step;
    const int64_t e = g / S.E;
    const int s = (int)(g % S.E);
    const Planes out = dst ? *dst : same(S.src, S.work[0]) ? S.work[1] : S.work[0];
    if (!S.dry) {
        if (s == 0 && !S.logged[e - S.e0]) S.loaded = -1;
        flood_status st = ensure_epoch(S, e);
        if (st) return st;
        const void *in[3] = {S.src.h, S.src.qx, S.src.qy};
        void *o[3] = {out.h, out.qx, out.qy};
        if (S.profile) st = timed(S, S.ev_fwd, [&] { return launch_step_planes(h, s, k, in, o); });
        else st = launch_step_planes(h, s, k, in, o);
        if (st) return st;
    }
    S.src = out;
    S.work_step += k;
    S.fwd_steps += k;
    S.launches++;
    if (dst) S.slot_step[dst - S.slots.data()] = S.work_step;
    if (S.profile) S.prof_fwd_steps += k;
    return FLOOD_OK;
}

// The state of `step` is the checkpoint in `slot`: read it in place.
flood_status restore(Sweep &S, int slot, int64_t step)
{
    if (S.work_step == step) return FLOOD_OK;
    if (S.slot_step[slot] != step) return fail(S.h, FLOOD_ERR_STATE, "revolve: a snapshot holds another step");
    S.src = S.slots[slot];
    S.work_step = step;
    return FLOOD_OK;
}

// Replay to `step`; the last step writes into `last_dst` when given.
flood_status advance_to(Sweep &S, int64_t step, const Planes *last_dst = nullptr)
{
    while (S.work_step < step) {
        // the launch that ends at `step` writes into last_dst
        const int k = replay_steps(S, step);
        flood_status st = forward_step(S, S.work_step + k == step ? last_dst : nullptr, k);
        if (st) return st;
    }
    return FLOOD_OK;
}

template <typename T>
flood_status reverse_step_t(Sweep &S)
{
    flood_handle *h = S.h;
    const int64_t k = S.work_step;
    const int64_t g = S.g0 + k;
    const int64_t e = g / S.E;
    const int s = (int)(g % S.E);
    if (s == 0 && !S.logged[e - S.e0]) S.loaded = -1;
    flood_status st = ensure_epoch(S, e);
    if (st) return st;
    const int c = S.cur_l, o = 1 - S.cur_l;
    AdjArgs<T> A;
    std::memset(&A, 0, sizeof(A));
    StepArgs<T> &a = A.fwd;
    a.geo = h->geo;
    a.h = (const T *)S.src.h;
    a.qx = (const T *)S.src.qx;
    a.qy = (const T *)S.src.qy;
    a.z = (const T *)h->z;
    a.n = (const T *)h->n;
    a.bc.type = h->bc_type;
    a.bc.slot = h->bc_slot;
    a.bc.sqrtS = h->bc_sqrtS;
    a.bc.sqrtS_f = h->bc_sqrtS_f;
    a.inflow_q = (const T *)h->inflow_q;
    a.n_slots = h->n_slots;
    a.inflow_Q = h->inflow_Q;
    a.n_inflow_sec = h->n_in;
    a.t_list = h->t_list;
    a.ctrl = h->ctrl;
    a.s = s;
    a.k_steps = 1;
    A.lh = (const T *)S.lh[c];
    A.lqx = (const T *)S.lqx[c];
    A.lqy = (const T *)S.lqy[c];
    A.lh_out = (T *)S.lh[o];
    A.lqx_out = (T *)S.lqx[o];
    A.lqy_out = (T *)S.lqy[o];
    A.lhu = (T *)S.lhu;
    A.gn = S.gn;
    A.secs = h->secs_dev;
    A.sec_cells = h->sec_cells;
    A.inflow_W = h->inflow_W;
    A.gauge_cells = S.cells;
    A.n_gauges = S.G;
    A.seed = S.seed + (size_t)k * S.G;      // dL/dh after step k, added to lambda_{k+1}
    A.scratch = (T *)S.scratch;
    A.gn_in = S.gn_in;
    if (S.profile) {
        flood_status ts = timed(S, S.ev_rev, [&] {
            cudaError_t e = launch_adjoint_step<T>(A, h->stream);
            return e == cudaSuccess ? FLOOD_OK : cuda_fail(h, e, "adjoint step");
        });
        if (ts) return ts;
    } else {
        CKA(launch_adjoint_step<T>(A, h->stream));
    }
    S.cur_l = o;
    return FLOOD_OK;
}

flood_status reverse_step(Sweep &S)
{
    if (S.dry) {
        S.reversed.push_back(S.work_step);
        return FLOOD_OK;
    }
    return S.h->prec == FLOOD_F32 ? reverse_step_t<float>(S) : reverse_step_t<double>(S);
}

// Reverse steps [a, b) with the state of step a in slot sa and S.free_slots free.
flood_status reverse_range(Sweep &S, int64_t a, int64_t b, int sa)
{
    flood_status st;
    if (b - a == 1) {
        if ((st = restore(S, sa, a))) return st;
        return reverse_step(S);
    }
    const int64_t s = (int64_t)S.free_slots.size();
    if (s == 0) {
        for (int64_t k = b - 1; k >= a; k--) {
            if (S.work_step > k || S.work_step < a)
                if ((st = restore(S, sa, a))) return st;
            if ((st = advance_to(S, k))) return st;
            if ((st = reverse_step(S))) return st;
        }
        return FLOOD_OK;
    }
    const int64_t l = b - a;
    int64_t best_j = 1, best = -1;
    for (int64_t j = 1; j < l; j++) {
        int64_t cst = j + revolve_cost(l - j, s) + revolve_cost(j, s + 1);
        if (best < 0 || cst < best) {
            best = cst;
            best_j = j;
        }
    }
    const int64_t m = a + best_j;
    if (S.work_step > m || S.work_step < a) {
        if ((st = restore(S, sa, a))) return st;
    }
    // checkpoint m in a free slot: the replay's last step writes it there
    const int sm = S.free_slots.back();
    S.free_slots.pop_back();
    if (S.work_step == m) {
        if (!S.dry && (st = copy_planes(S.h, S.slots[sm], S.src, S.plane, S.plane_y))) return st;
        S.src = S.slots[sm];
        S.slot_step[sm] = m;
    } else if ((st = advance_to(S, m, &S.slots[sm]))) {
        return st;
    }
    if ((st = reverse_range(S, m, b, sm))) return st;
    S.free_slots.push_back(sm);
    return reverse_range(S, a, m, sa);
}

}  // namespace

}  // namespace flood

extern "C" int64_t flood_adjoint_forward_steps(const flood_handle *h) { return h ? h->adj_forward_steps : 0; }

extern "C" flood_status flood_adjoint_profile(flood_handle *h, int32_t enable)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    h->adj_profile = enable ? 1 : 0;
    return FLOOD_OK;
}

extern "C" flood_status flood_adjoint_times(const flood_handle *h, double *reverse_ms, int64_t *reverse_steps,
                                            double *forward_ms, int64_t *forward_steps)
{
    if (!h || !reverse_ms || !reverse_steps || !forward_ms || !forward_steps)
        return fail(nullptr, FLOOD_ERR_ARG, "NULL argument");
    *reverse_ms = h->adj_prof_rev_ms;
    *reverse_steps = h->adj_prof_rev_steps;
    *forward_ms = h->adj_prof_fwd_ms;
    *forward_steps = h->adj_prof_fwd_steps;
    return FLOOD_OK;
}

extern "C" flood_status flood_adjoint(flood_handle *h, int64_t n_steps, const int64_t *gauge_cells,
                                      int32_t n_gauges, const double *dLdh, int32_t n_checkpoints,
                                      void *dLdn_out, void *dLdh0_out, int32_t out_on_device)
{
    if (!h) return fail(nullptr, FLOOD_ERR_ARG, "handle is NULL");
    if (h->part) return fail(h, FLOOD_ERR_STATE, "a part of a decomposed grid is stepped by its decomposition");
    NvtxRange range("flood: adjoint sweep");
    if (n_steps < 1 || n_gauges < 0 || n_checkpoints < 0 || !dLdn_out || (n_gauges > 0 && (!gauge_cells || !dLdh)))
        return fail(h, FLOOD_ERR_ARG, "bad adjoint arguments");
    if (h->sticky) return fail(h, FLOOD_ERR_STATE, "handle is in an error state; write a new state first");
    const int64_t nc = (int64_t)h->geo.nx * h->geo.ny;
    for (int g = 0; g < n_gauges; g++)
        if (gauge_cells[g] < 0 || gauge_cells[g] >= nc) return fail(h, FLOOD_ERR_ARG, "gauge cell out of range");
    const size_t esz = h->esz;
    const size_t P = (size_t)h->geo.pitch;
    Sweep S;
    S.h = h;
    S.profile = h->adj_profile != 0;
    S.g0 = h->step;
    S.N = n_steps;
    S.E = h->geo.epoch_steps;
    S.plane = P * h->geo.ny * esz;
    S.plane_y = P * (h->geo.ny + 1) * esz;
    // n_checkpoints = 0: as many snapshots as half the free device memory holds, at most
    // one per step (every state kept: no step is replayed twice)
    int64_t want = n_checkpoints;
    if (want == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(h, FLOOD_ERR_CUDA, "cudaMemGetInfo");
        want = std::max<int64_t>(1, (int64_t)(free_b / 2 / (2 * S.plane + S.plane_y)));
    }
    int C = (int)std::min<int64_t>(want, n_steps);
    std::vector<void *> mine;
    auto alloc = [&](size_t bytes) {
        void *p = dev_alloc(h, bytes);
        if (p) mine.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void *p : mine) dev_free(h, p);
        mine.clear();
    };
    // the snapshots in one allocation (planes are multiples of 128 bytes); a count
    // sized by the free memory is halved until the allocation succeeds
    {
        const size_t slot = 2 * S.plane + S.plane_y;
        char *block = (char *)alloc((size_t)C * slot);
        while (!block && n_checkpoints == 0 && C > 1) {
            C /= 2;
            block = (char *)alloc((size_t)C * slot);
        }
        if (!block) {
            release();
            return fail(h, FLOOD_ERR_OOM, "checkpoint allocation");
        }
        S.slots.resize(C);
        for (int c = 0; c < C; c++) {
            S.slots[c].h = block + (size_t)c * slot;
            S.slots[c].qx = block + (size_t)c * slot + S.plane;
            S.slots[c].qy = block + (size_t)c * slot + 2 * S.plane;
        }
    }
    for (int c = C - 1; c >= 1; c--) S.free_slots.push_back(c);
    S.slot_step.assign(C, -1);
    S.slot_step[0] = 0;                   // the start state, copied in before the sweep
    S.max_k = (h->prec == FLOOD_F32 && h->geo.theta == 1.0 && h->geo.friction == 0) ? 4 : 1;
    S.e0 = S.g0 / S.E;
    const int64_t n_ep = (S.g0 + n_steps - 1) / S.E - S.e0 + 1;
    S.logged.assign(n_ep, 0);
    const int E = S.E;
    S.iq_bytes = (size_t)E * h->n_slots * esz;
    S.nQ = (size_t)E * std::max(h->n_in, 1);
    S.dt_log = (double *)alloc(n_ep * sizeof(double));
    S.tl_log = (double *)alloc(n_ep * (E + 1) * sizeof(double));
    S.iq_log = alloc(n_ep * S.iq_bytes);
    S.iQ_log = (double *)alloc(n_ep * S.nQ * sizeof(double));
    S.iW_log = (double *)alloc(n_ep * S.nQ * sizeof(double));
    for (int b = 0; b < 2; b++) {
        S.lh[b] = alloc(S.plane);
        S.lqx[b] = alloc(S.plane);
        S.lqy[b] = alloc(S.plane_y);
    }
    S.lhu = alloc(S.plane);
    const bool opts = h->geo.theta != 1.0 || h->geo.friction != 0;
    if (opts) S.scratch = alloc(11 * S.plane_y);
    S.gn = (double *)alloc(P * h->geo.ny * sizeof(double));
    if (h->prec == FLOOD_F32 && !opts && h->n_in > 0) {      // the reverse step computes pass 3 beside its tiles
        S.n_in_cells = h->n_slots;
        S.gn_in = (double *)alloc((size_t)S.n_in_cells * sizeof(double));
        if (!S.gn_in) {
            release();
            return fail(h, FLOOD_ERR_OOM, "adjoint buffer allocation");
        }
    }
    double *seed_dev = (double *)alloc(std::max<size_t>((size_t)n_steps * n_gauges, 1) * sizeof(double));
    int64_t *cells_dev = (int64_t *)alloc(std::max(n_gauges, 1) * sizeof(int64_t));
    for (void *p : {(void *)S.dt_log, (void *)S.tl_log, S.iq_log, (void *)S.iQ_log, (void *)S.iW_log, S.lh[0],
                    S.lh[1], S.lqx[0], S.lqx[1], S.lqy[0], S.lqy[1], S.lhu, (void *)S.gn, (void *)seed_dev,
                    (void *)cells_dev})
        if (!p) {
            release();
            return fail(h, FLOOD_ERR_OOM, "adjoint buffer allocation");
        }
    if (opts && !S.scratch) {
        release();
        return fail(h, FLOOD_ERR_OOM, "adjoint buffer allocation");
    }
    // saved handle state: control block, kernel, state index and epoch pointers (the
    // sweep aims the epoch pointers at its own slices and writes nothing through the
    // handle's own epoch buffers)
    Ctrl saved_ctrl;
    const int saved_kernel = h->kernel;
    const int saved_cur = h->cur;
    const int64_t saved_step = h->step;
    void *const saved_iq = h->inflow_q;
    double *const saved_iQ = h->inflow_Q, *const saved_iW = h->inflow_W, *const saved_tl = h->t_list;
    auto finish = [&](flood_status st) {
        h->kernel = saved_kernel;
        h->inflow_q = saved_iq;
        h->inflow_Q = saved_iQ;
        h->inflow_W = saved_iW;
        h->t_list = saved_tl;
        release();
        return st;
    };
#define CKF(expr)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) return finish(cuda_fail(h, e_, #expr));              \
    } while (0)
    CKF(cudaMemcpyAsync(&saved_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    // the epoch in progress at the start is logged from the handle
    if (S.g0 % E != 0) {
        const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
        CKF(cudaMemcpyAsync(S.dt_log, &h->ctrl->dt, sizeof(double), d2d, h->stream));
        CKF(cudaMemcpyAsync(S.tl_log, h->t_list, (E + 1) * sizeof(double), d2d, h->stream));
        CKF(cudaMemcpyAsync(S.iq_log, h->inflow_q, S.iq_bytes, d2d, h->stream));
        CKF(cudaMemcpyAsync(S.iQ_log, h->inflow_Q, S.nQ * sizeof(double), d2d, h->stream));
        CKF(cudaMemcpyAsync(S.iW_log, h->inflow_W, S.nQ * sizeof(double), d2d, h->stream));
        S.logged[0] = 1;
    }
    if (n_gauges > 0) {
        CKF(cudaMemcpyAsync(seed_dev, dLdh, (size_t)n_steps * n_gauges * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream));
        CKF(cudaMemcpyAsync(cells_dev, gauge_cells, n_gauges * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    }
    for (int b = 0; b < 2; b++) {
        CKF(cudaMemsetAsync(S.lh[b], 0, S.plane, h->stream));
        CKF(cudaMemsetAsync(S.lqx[b], 0, S.plane, h->stream));
        CKF(cudaMemsetAsync(S.lqy[b], 0, S.plane_y, h->stream));
    }
    CKF(cudaMemsetAsync(S.lhu, 0, S.plane, h->stream));
    CKF(cudaMemsetAsync(S.gn, 0, P * h->geo.ny * sizeof(double), h->stream));
    if (S.gn_in) CKF(cudaMemsetAsync(S.gn_in, 0, (size_t)S.n_in_cells * sizeof(double), h->stream));
    S.cells = cells_dev;
    S.G = n_gauges;
    S.seed = seed_dev;
    // FP32 forward replays run the arithmetic the adjoint linearises: launches of
    // one step the tensor-tile kernel below 2^27 cells, the stream kernel above;
    // launches of up to four steps (replay_steps) the temporal-blocking kernel (all
    // bitwise equal)
    if (h->prec == FLOOD_F32)
        h->kernel = (int64_t)h->geo.nx * h->geo.ny < ((int64_t)1 << 27) ? FLOOD_KERNEL_TMA : FLOOD_KERNEL_STREAM;
    for (int b = 0; b < 2; b++) {
        S.work[b].h = h->h[b];
        S.work[b].qx = h->qx[b];
        S.work[b].qy = h->qy[b];
    }
    {
        flood_status st = copy_planes(h, S.slots[0], working(h), S.plane, S.plane_y);
        if (st) return finish(st);
    }
    S.src = S.slots[0];
    S.work_step = 0;
    {
        flood_status st = reverse_range(S, 0, n_steps, 0);
        if (st) return finish(st);
    }
    h->adj_forward_steps = S.fwd_steps;
    if (S.profile) {
        CKF(cudaStreamSynchronize(h->stream));
        h->adj_prof_rev_steps = (int64_t)S.ev_rev.size() / 2;
        h->adj_prof_fwd_steps = S.prof_fwd_steps;
        h->adj_prof_rev_ms = sum_pairs(S.ev_rev);
        h->adj_prof_fwd_ms = sum_pairs(S.ev_fwd);
    }
    // outputs
    if (S.gn_in) CKF(launch_gn_inflow_add(S.gn, S.gn_in, h->sec_cells, S.n_in_cells, h->stream));
    {
        flood_status st = FLOOD_OK;
        if (h->prec == FLOOD_F32) st = (flood_status)(launch_gn_out<float>(h->geo, S.gn, (float *)S.lhu, h->stream) ? FLOOD_ERR_CUDA : FLOOD_OK);
        else st = (flood_status)(launch_gn_out<double>(h->geo, S.gn, (double *)S.lhu, h->stream) ? FLOOD_ERR_CUDA : FLOOD_OK);
        if (st) return finish(fail(h, FLOOD_ERR_CUDA, "gradient conversion"));
        st = copy_out(h, dLdn_out, S.lhu, h->geo.ny, h->geo.nx, out_on_device);
        if (st) return finish(st);
        if (dLdh0_out) {
            st = copy_out(h, dLdh0_out, S.lh[S.cur_l], h->geo.ny, h->geo.nx, out_on_device);
            if (st) return finish(st);
        }
    }
    // put the handle back as it was
    h->cur = saved_cur;
    {
        flood_status st = copy_planes(h, working(h), S.slots[0], S.plane, S.plane_y);
        if (st) return finish(st);
    }
    h->step = saved_step;
    CKF(cudaMemcpyAsync(h->ctrl, &saved_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
    CKF(cudaStreamSynchronize(h->stream));
#undef CKF
    return finish(FLOOD_OK);
}

extern "C" flood_status flood_revolve_plan(int64_t n_steps, int32_t n_checkpoints, int32_t epoch_steps,
                                           int64_t start_step, int32_t steps_per_replay, int64_t *forward_steps,
                                           int64_t *replay_launches, int32_t *in_order)
{
    if (n_steps < 1 || n_steps > 1000000 || n_checkpoints < 1 || epoch_steps < 1 || start_step < 0 ||
        steps_per_replay < 1 || !forward_steps || !replay_launches || !in_order)
        return fail(nullptr, FLOOD_ERR_ARG, "bad revolve plan arguments");
    Sweep S;
    S.dry = true;
    S.g0 = start_step;
    S.N = n_steps;
    S.E = epoch_steps;
    S.max_k = steps_per_replay;
    const int C = (int)std::min<int64_t>(n_checkpoints, n_steps);
    S.slots.resize(C);
    S.slot_step.assign(C, -1);
    S.slot_step[0] = 0;
    for (int c = C - 1; c >= 1; c--) S.free_slots.push_back(c);
    S.work_step = 0;
    flood_status st = reverse_range(S, 0, n_steps, 0);
    if (st) return st;
    bool ok = (int64_t)S.reversed.size() == n_steps && (int)S.free_slots.size() == C - 1;
    for (int64_t k = 0; ok && k < n_steps; k++) ok = S.reversed[k] == n_steps - 1 - k;
    *forward_steps = S.fwd_steps;
    *replay_launches = S.launches;
    *in_order = ok ? 1 : 0;
    return FLOOD_OK;
}
