// step_tiled.cuh -- FP32 temporal blocking: K <= 4 (or 8) time steps per launch.
// The kernel templates; step_tiled.cu instantiates Eq. 3 as printed and
// step_tiled_opts.cu the scheme options (theta weighting, vector-norm friction).
//
// One block is a pipeline of K warps over output strips of 120 columns (128
// staged, 4 halo columns on each side held by lanes 0 and 31); warp s-1
// advances the strip by time level s.  The grid is persistent, one block per
// resident pipeline, and each block takes an equal contiguous share of the
// strip-major sequence of (strip, row) units, running the pipeline once per
// strip segment of its share, so that every SM gets the same work.  The warps move
// in lockstep ticks: at tick j, level s works on row r = j - 2(s-1), i.e. it
// computes the new south faces of row r, finishes row r-1 (Eq. 4) and
// computes the new west faces of row r, exactly like the single-step row
// kernels.  Level 1 reads its rows from a shared-memory ring filled by bulk
// copies (cp.async.bulk + mbarrier, a few rows ahead); level s > 1 reads the
// row that level s-1 finished at the previous tick from a double-buffered
// hand-off slot; only level K stores.  The dependency cone of K steps is K
// columns wide on each side, so the 120 inner columns are exact; in y the
// chunk needs K extra rows at each end.  HBM traffic per cell and step is
// about (20 B read + 12 B written) / K plus the 8/120 column overlap.
//
// Per cell and level the arithmetic is the single-step kernels' (the same
// explicitly rounded face function and depth update), so K levels give the
// same bits as K single steps.  Boundary faces (Eq. 5-6) use that level's
// inflow row; ledger volumes are booked only by the pipeline that owns the
// cell or boundary face.  Waits on the copies are bounded (about 2 s), after
// which the status word gets the timeout bit and the pipeline stops storing.
#pragma once

#include <atomic>

#include "fast_face.cuh"
#include "tma_util.cuh"

namespace flood {

// Rows per (chunk, strip) work item and the number of pipelines for a grid (step_tiled.cu):
// for items handed out round-robin, and for items taken from a counter.
void tiled_split(int n_strips, int ny, int resident, int K, int *chunk_rows, int *blocks);
void tiled_split_dynamic(int n_strips, int ny, int resident, int K, int *chunk_rows, int *blocks);

namespace {


// halo columns per side (at least K: the dependency cone of K steps) and
// output columns of a 128-column strip, per steps per launch K
__host__ __device__ constexpr int halo_cols(int K) { return K <= 4 ? 4 : 8; }
// Right-hand halo: the theta weighting of the strip's last face needs the face
// beyond the staged columns, so with it the cone reaches one column further on
// that side (K + 1 columns after K levels); the left edge loses nothing more.
// Rounded up to a multiple of 4 columns: a strip's first column x0 must stay
// a multiple of 4 (16-byte aligned bulk copies and float4 stores).
__host__ __device__ constexpr int halo_right(int K, int mode)
{
    return (mode & 1) && K + 1 > halo_cols(K) ? (K + 1 + 3) / 4 * 4 : halo_cols(K);
}
__host__ __device__ constexpr int out_cols(int K, int mode = 0) { return 128 - halo_cols(K) - halo_right(K, mode); }
static_assert(out_cols(4, 1) == 116 && out_cols(8, 1) == 108 && out_cols(4, 2) == 120, "strip widths");
static_assert(out_cols(1, 1) % 4 == 0 && out_cols(2, 1) % 4 == 0 && out_cols(3, 1) % 4 == 0 && out_cols(4, 1) % 4 == 0 &&
                  out_cols(8, 1) % 4 == 0 && halo_cols(4) % 4 == 0 && halo_cols(8) % 4 == 0,
              "strip origins must stay multiples of 4 columns");
// level-1 rows in flight, for one grid and for the ensemble kernel; six pipelines
// of 4 warps fit the registers and shared memory of an SM with either (tiled_min_blocks;
// the ensemble kernel's launch bounds).  One grid: 6 rows (3 and 6 measured alike, and
// 0.8 % faster than 4, which left 4 bytes of spill)
constexpr int kPF1 = 6, kPFE = 4;
constexpr uint64_t kBudgetNs = 2000000000ull;

constexpr int pow2_ceil(int v)
{
    int p = 1;
    while (p < v) p *= 2;
    return p;
}

template <int K, int kPF, int kHo = 3>
struct alignas(16) PipeSmem {
    // z,n rows kept: the lagging levels read 2(K-1)+1 rows back; a power of two,
    // so that the row's slot is a mask of its index
    static constexpr int kDZ = pow2_ceil(kPF + 2 * K);
    float hq[kPF][3][128];                  // level-1 input rows: h, qx, qy
    float zn[kDZ][2][128];                  // z, n of recent rows
    float ho[K > 1 ? K - 1 : 1][2][kHo][128];   // hand-off: level s -> s+1, double buffered by tick parity:
                                                // the finished row's h, qx, qy (and, for the scheme options,
                                                // the new qy of the row above it)
    uint64_t bar[kPF];
    double led[K][2];                       // per level (warp): boundary outflow volume, clipped volume,
                                            // summed over the runs of rows of the grid's items so far
};

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, const float4 &v) { *reinterpret_cast<float4 *>(p) = v; }

__device__ __forceinline__ float get(const float4 &v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

__device__ __forceinline__ void set(float4 &v, int k, float x)
{
    if (k == 0) v.x = x;
    else if (k == 1) v.y = x;
    else if (k == 2) v.z = x;
    else v.w = x;
}

// This thread's running depth maximum over one grid's cells of a launch (level K).
// The volume terms are kept in shared memory (PipeSmem::led), out of the registers
// of the pipeline's inner loop.
struct TiledLedger {
    float hmax = 0.0f;
    bool nan_seen = false;
};

__device__ __forceinline__ FastConst tiled_const(const StepArgs<float> &a)
{
    const Geom &G = a.geo;
    const float dt = (float)a.ctrl->dt, dx = (float)G.dx, g = (float)G.g;
    FastConst Kc;
    Kc.gdt = g * dt;
    Kc.a1 = Kc.gdt / dx;
    Kc.gdt4 = 0.25f * Kc.gdt;
    Kc.h_dry = (float)G.h_dry;
    Kc.dtdx = dt / dx;
    Kc.theta = (float)G.theta;
    Kc.w = (float)(0.5 * (1.0 - G.theta));
    return Kc;
}

// Hand-off fields per scheme mode: h, qx, qy of the finished row, plus the
// new qy of the row above it for the theta-weighting and the vector norm.
__host__ __device__ constexpr int hand_fields(int mode) { return mode ? 4 : 3; }

// One work item: the pipeline over strip `strip`, rows [y0, y1) of grid a, for
// steps s0 .. s0 + K - 1 of the epoch.  base counts the rows staged by earlier
// items (ring slot and phase of staged row idx are those of base + idx).
// Returns true (uniformly over the block) if a wait on a copy timed out; the
// copies in flight are then drained and the status word has the timeout bit.
//
// kMode bit 0: theta-weighted numerator discharges; bit 1: the vector norm in
// the friction term (the options of the stream kernel, with the same face
// arithmetic).  Both need the old qy of the row above the one being computed:
// level 1 reads it from the ring one row ahead (or from global memory past the
// staged rows), level s > 1 from the hand-off, where level s - 1 leaves the qy
// it computed for that row; and the old qy / qx of the row below, kept in
// registers.  Their faces are evaluated two per paired instruction, like
// Eq. 3 as printed, in the scalar option arithmetic's order.  The lanes at
// the strip's edges take their missing neighbour columns as garbage, like the
// plain arithmetic's edge lanes: the stencil still reaches one column per
// level, inside the halo.
template <int K, int kPF, int kMode = 0>
__device__ __forceinline__ bool tiled_item(const StepArgs<float> &a, const int s0, const FastConst &Kc,
                                           const int strip, const int y0, const int y1,
                                           PipeSmem<K, kPF, hand_fields(kMode)> &sm, uint32_t &base, TiledLedger &L)
{
    constexpr bool kTheta = (kMode & 1) != 0, kVec = (kMode & 2) != 0, kOpt = kMode != 0;
    constexpr int kHo = hand_fields(kMode);
    constexpr int kDZ = PipeSmem<K, kPF, kHo>::kDZ;
    const Geom &G = a.geo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lvl = warp + 1;                         // this warp's time level
    const int nx = G.nx, ny = G.ny, P = G.pitch;
    const int step = s0 + (lvl - 1);                  // this level's step in the epoch
    int issued = 0, consumed = 0;
    bool abort = false;
    constexpr int kOut = out_cols(K, kMode);
    const int x0 = strip * kOut - halo_cols(K);
    const int c0 = x0 + 4 * lane;
    const int own_lo = strip * kOut, own_hi = min(strip * kOut + kOut, nx);
    const int jb = max(y0 - K, 0);
    const int jload_hi = min(y1 + K - 1, ny - 1);     // last staged row
    const int nload = jload_hi - jb + 1;
    const int jlast = min(y1, ny) + 2 * (K - 1);      // last tick: level K reaches row min(y1, ny)
    const int rstart = jb == 0 ? 0 : jb + (lvl - 1);  // first row this level sees (halo row if jb > 0)
    const int cs = max(x0, 0);
    const int ce = min(x0 + 128, P);
    const int so = cs - x0;
    const uint32_t seg_bytes = (uint32_t)(ce - cs) * 4u;
    auto issue = [&](int idx) {
        const int j = jb + idx;
        const uint32_t slot = (base + (uint32_t)idx) % kPF;
        const size_t row = (size_t)j * P + cs;
        uint64_t *bar = &sm.bar[slot];
        mbar_arrive_expect_tx(bar, seg_bytes * 5u);
        float *hq = &sm.hq[slot][0][0];
        float *zn = &sm.zn[(unsigned)j % kDZ][0][0];
        bulk_copy_g2s(hq + 0 * 128 + so, a.h + row, seg_bytes, bar);
        bulk_copy_g2s(hq + 1 * 128 + so, a.qx + row, seg_bytes, bar);
        bulk_copy_g2s(hq + 2 * 128 + so, a.qy + row, seg_bytes, bar);
        bulk_copy_g2s(zn + 0 * 128 + so, a.z + row, seg_bytes, bar);
        bulk_copy_g2s(zn + 1 * 128 + so, a.n + row, seg_bytes, bar);
    };
    if (threadIdx.x == 0) {
        fence_proxy_async();                          // earlier items' reads of the rings come first
        for (; issued < min(kPF, nload); issued++) issue(issued);
    }

    bool own_cell[4], own_wface[4], in_col[4], in_wface[4], all_cell = true, all_wface = true;
    const bool edge_lane = c0 <= 0 || c0 + 3 >= nx;   // holds a column outside (0, nx)
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = c0 + k;
        in_col[k] = c >= 0 && c < nx;                 // a cell of the grid (its south face exists)
        in_wface[k] = c > 0 && c < nx;                // an interior west face
        own_cell[k] = c >= own_lo && c < own_hi;
        own_wface[k] = c >= own_lo && (c < own_hi || (c == nx && own_hi == nx));
        all_cell &= own_cell[k];
        all_wface &= own_wface[k];
    }

    // this level's previous row: input depth and the new faces computed for it
    // (and its old qy and qx, for the scheme options)
    float4 hp = make_float4(0, 0, 0, 0), qxw_p = hp, qys_p = hp, qyo_p = hp, qxo_p = hp;
    float qxe_p = 0.0f;
    // runs of up to 32 ticks; the float partial sums of the boundary outflow (fq)
    // and the clipped depth (fc) are summed over the warp in double after each run
    // and added to the warp's shared-memory sums (led)
    for (int j0 = jb; j0 <= jlast && !abort; j0 += 32) {
        float fq = 0.0f, fc = 0.0f;
        const int jend = min(j0 + 31, jlast);
        for (int j = j0; j <= jend; j++) {
            const int r = j - 2 * (lvl - 1);
            // ---- level 1 waits for its staged row; the other levels only read rows that
            // level 1 waited for at earlier ticks (ordered by the end-of-tick barrier)
            bool stop = false;
            if (lvl == 1 && r >= jb && r <= jload_hi) {
                const uint32_t g = base + (uint32_t)(r - jb);
                int ok = mbar_wait_bounded(&sm.bar[g % kPF], (g / kPF) & 1u, kBudgetNs) ? 1 : 0;
                if constexpr (kOpt) {                 // the row above, read one row ahead (issued already)
                    if (r + 1 <= jload_hi)
                        ok &= mbar_wait_bounded(&sm.bar[(g + 1) % kPF], ((g + 1) / kPF) & 1u, kBudgetNs) ? 1 : 0;
                }
                stop = !__all_sync(0xffffffffu, ok);
            }
            if (!stop && r >= rstart && r <= ny && r <= y1 + K - lvl) {
                // current row inputs
                float4 ch = make_float4(0, 0, 0, 0), cqx = ch, cqy = ch, cz = ch, cn = ch, pz = ch, pn = ch;
                if (r < ny) {
                    if (lvl == 1) {
                        const float *hq = &sm.hq[(base + (uint32_t)(r - jb)) % kPF][0][0];
                        ch = lds4(hq + 0 * 128 + 4 * lane);
                        cqx = lds4(hq + 1 * 128 + 4 * lane);
                        cqy = lds4(hq + 2 * 128 + 4 * lane);
                    } else {
                        const float *ho = &sm.ho[lvl - 2][(j - 1) & 1][0][0];
                        ch = lds4(ho + 0 * 128 + 4 * lane);
                        cqx = lds4(ho + 1 * 128 + 4 * lane);
                        cqy = lds4(ho + 2 * 128 + 4 * lane);
                    }
                    cz = lds4(&sm.zn[(unsigned)r % kDZ][0][4 * lane]);
                    cn = lds4(&sm.zn[(unsigned)r % kDZ][1][4 * lane]);
                }
                // old qy of the row above (the north faces of row r), for the scheme options
                float4 qyn = make_float4(0, 0, 0, 0);
                if constexpr (kOpt) {
                    if (r < ny) {
                        if (lvl > 1) {
                            qyn = lds4(&sm.ho[lvl - 2][(j - 1) & 1][3][4 * lane]);
                        } else if (r + 1 <= jload_hi) {
                            qyn = lds4(&sm.hq[(base + (uint32_t)(r + 1 - jb)) % kPF][2][4 * lane]);
                        } else {                      // past the staged rows: face row r + 1 <= ny
                            const float *row = a.qy + (size_t)(r + 1) * P;
                            if (c0 >= 0 && c0 + 3 < P) qyn = __ldg(reinterpret_cast<const float4 *>(row + c0));
                            else {
#pragma unroll
                                for (int k = 0; k < 4; k++)
                                    if (c0 + k >= 0 && c0 + k < P) set(qyn, k, __ldg(row + c0 + k));
                            }
                        }
                    }
                }
                if (r > 0) {
                    pz = lds4(&sm.zn[(unsigned)(r - 1) % kDZ][0][4 * lane]);
                    pn = lds4(&sm.zn[(unsigned)(r - 1) % kDZ][1][4 * lane]);
                }
                if (r == rstart && jb > 0) {
                    hp = ch;                          // halo row: only becomes the previous row
                    if constexpr (kOpt) {
                        qyo_p = cqy;
                        qxo_p = cqx;
                    }
                } else {
                    // ---- new south faces of row r (interior rows branch-free; the boundary
                    // rows, uniform over the warp, take the Eq. 5-6 path)
                    float4 qys;
                    if (r > 0 && r < ny && kOpt) {
                        // with the options (the stream kernel's arithmetic)
                        float xs4 = 0.0f, xn4 = 0.0f;  // old qx right of the lane's last column, rows r-1, r
                        if constexpr (kVec) {
                            xs4 = __shfl_down_sync(0xffffffffu, qxo_p.x, 1);
                            xn4 = __shfl_down_sync(0xffffffffu, cqx.x, 1);
                        }
                        // two faces per paired instruction (bitwise the scalar face_fast_sel_gen)
#pragma unroll
                        for (int k = 0; k < 4; k += 2) {
                            const unsigned long long q = f2pack(get(cqy, k), get(cqy, k + 1));
                            unsigned long long qn = q, qm;
                            if constexpr (kTheta)
                                qn = theta_q_x2(q, f2pack(get(qyo_p, k), get(qyo_p, k + 1)),
                                                f2pack(get(qyn, k), get(qyn, k + 1)), Kc);
                            if constexpr (kVec)
                                qm = q_norm_x2(q, f2pack(get(qxo_p, k), get(qxo_p, k + 1)),
                                               f2pack(get(qxo_p, k + 1), k + 1 < 3 ? get(qxo_p, k + 2) : xs4),
                                               f2pack(get(cqx, k), get(cqx, k + 1)),
                                               f2pack(get(cqx, k + 1), k + 1 < 3 ? get(cqx, k + 2) : xn4));
                            else
                                qm = f2pack(fabsf(get(cqy, k)), fabsf(get(cqy, k + 1)));
                            const unsigned long long eL = f2add(f2pack(get(hp, k), get(hp, k + 1)),
                                                                f2pack(get(pz, k), get(pz, k + 1)));
                            const unsigned long long eR = f2add(f2pack(get(ch, k), get(ch, k + 1)),
                                                                f2pack(get(cz, k), get(cz, k + 1)));
                            const unsigned long long ns = f2add(f2pack(get(pn, k), get(pn, k + 1)),
                                                                f2pack(get(cn, k), get(cn, k + 1)));
                            const float2 zm = make_float2(fmaxf(get(pz, k), get(cz, k)), fmaxf(get(pz, k + 1), get(cz, k + 1)));
                            const float2 v = face_fast_sel_x2_gen(qm, qn, eL, eR, zm, ns, Kc);
                            set(qys, k, v.x);
                            set(qys, k + 1, v.y);
                        }
                        if (edge_lane) {
#pragma unroll
                            for (int k = 0; k < 4; k++)
                                if (!in_col[k]) set(qys, k, 0.0f);
                        }
                    } else if (r > 0 && r < ny) {
                        // two faces per paired instruction (bitwise the scalar face_fast_sel)
#pragma unroll
                        for (int k = 0; k < 4; k += 2) {
                            const unsigned long long eL = f2add(f2pack(get(hp, k), get(hp, k + 1)),
                                                                f2pack(get(pz, k), get(pz, k + 1)));
                            const unsigned long long eR = f2add(f2pack(get(ch, k), get(ch, k + 1)),
                                                                f2pack(get(cz, k), get(cz, k + 1)));
                            const unsigned long long ns = f2add(f2pack(get(pn, k), get(pn, k + 1)),
                                                                f2pack(get(cn, k), get(cn, k + 1)));
                            const float2 zm = make_float2(fmaxf(get(pz, k), get(cz, k)), fmaxf(get(pz, k + 1), get(cz, k + 1)));
                            const float2 v = face_fast_sel_x2(make_float2(get(cqy, k), get(cqy, k + 1)), eL, eR, zm, ns, Kc);
                            set(qys, k, v.x);
                            set(qys, k + 1, v.y);
                        }
                        if (edge_lane) {
#pragma unroll
                            for (int k = 0; k < 4; k++)
                                if (!in_col[k]) set(qys, k, 0.0f);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const int c = c0 + k;
                            float v = 0.0f;
                            if (in_col[k]) {
                                float qo = 0.0f;
                                v = r == 0 ? boundary_fast_flux(a, step, 2, c, get(ch, k), get(cn, k), qo)
                                           : boundary_fast_flux(a, step, 3, c, get(hp, k), get(pn, k), qo);
                                if (own_cell[k] && ((r == 0 && y0 == 0) || (r == ny && y1 == ny))) fq += qo;
                            }
                            set(qys, k, v);
                        }
                    }
                    // ---- finish row r-1: Eq. 4 and the clip; hand it on (or store it at level K)
                    const bool has_prev = jb == 0 ? r > 0 : r > rstart + 1;
                    if (has_prev) {
                        const int rr = r - 1;
                        const bool own_row = rr >= y0 && rr < y1;
                        float4 fin;
                        bool neg = false;
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const float qe = k < 3 ? get(qxw_p, k + 1) : qxe_p;
                            const float dv = __fadd_rn(__fsub_rn(get(qxw_p, k), qe), __fsub_rn(get(qys_p, k), get(qys, k)));
                            const float v = __fmaf_rn(Kc.dtdx, dv, get(hp, k));
                            neg |= v < 0.0f;
                            set(fin, k, v);
                        }
                        if (neg) {                    // rare: clip to zero, book the removed volume
                            // (the ledger rows' bounds are read only here: the ensemble kernel's
                            // arguments live in global memory)
                            const bool led_row = own_row && rr >= G.led_j0 && rr < G.led_j1;
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                const float v = get(fin, k);
                                if (v < 0.0f) {
                                    if (led_row && own_cell[k]) fc -= v;
                                    set(fin, k, 0.0f);
                                }
                            }
                        }
                        if (lvl == K && own_row) {
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                const float v = get(fin, k);
                                if (own_cell[k]) {
                                    L.hmax = fmaxf(L.hmax, v);
                                    L.nan_seen |= (v != v);
                                }
                            }
                        }
                        if (lvl < K) {
                            float *ho = &sm.ho[lvl - 1][j & 1][0][0];
                            sts4(ho + 0 * 128 + 4 * lane, fin);
                            sts4(ho + 1 * 128 + 4 * lane, qxw_p);
                            sts4(ho + 2 * 128 + 4 * lane, qys_p);
                            if constexpr (kOpt) sts4(ho + 3 * 128 + 4 * lane, qys);   // the row above's new qy
                        } else if (own_row) {
                            const size_t ro = (size_t)rr * P + c0;
                            if (all_cell) {
                                *reinterpret_cast<float4 *>(a.h_out + ro) = fin;
                                *reinterpret_cast<float4 *>(a.qy_out + ro) = qys_p;
                                if (rr == ny - 1) *reinterpret_cast<float4 *>(a.qy_out + ro + P) = qys;
                            } else {
#pragma unroll
                                for (int k = 0; k < 4; k++)
                                    if (own_cell[k]) {
                                        a.h_out[ro + k] = get(fin, k);
                                        a.qy_out[ro + k] = get(qys_p, k);
                                        if (rr == ny - 1) a.qy_out[ro + P + k] = get(qys, k);
                                    }
                            }
                            if (all_wface) *reinterpret_cast<float4 *>(a.qx_out + ro) = qxw_p;
                            else {
#pragma unroll
                                for (int k = 0; k < 4; k++)
                                    if (own_wface[k]) a.qx_out[ro + k] = get(qxw_p, k);
                            }
                        }
                    }
                    // ---- new west faces of row r; row r becomes this level's previous row
                    if (r < ny) {
                        const bool own_row_r = r >= y0 && r < y1;
                        const float hl0 = __shfl_up_sync(0xffffffffu, ch.w, 1);
                        const float zl0 = __shfl_up_sync(0xffffffffu, cz.w, 1);
                        const float nl0 = __shfl_up_sync(0xffffffffu, cn.w, 1);
                        float4 qxw;
                        if constexpr (kOpt) {
                            // old qx left of the lane's first and right of its last column; old qy of
                            // rows r and r + 1 left of its first column
                            float ql0 = 0.0f, qr3 = 0.0f, ys0 = 0.0f, yn0 = 0.0f;
                            if constexpr (kTheta) {
                                ql0 = __shfl_up_sync(0xffffffffu, cqx.w, 1);
                                qr3 = __shfl_down_sync(0xffffffffu, cqx.x, 1);
                            }
                            if constexpr (kVec) {
                                ys0 = __shfl_up_sync(0xffffffffu, cqy.w, 1);
                                yn0 = __shfl_up_sync(0xffffffffu, qyn.w, 1);
                            }
                            // two faces per paired instruction (bitwise the scalar face_fast_sel_gen)
#pragma unroll
                            for (int k = 0; k < 4; k += 2) {
                                const float hla = k == 0 ? hl0 : get(ch, k - 1), hlb = get(ch, k);
                                const float zla = k == 0 ? zl0 : get(cz, k - 1), zlb = get(cz, k);
                                const float nla = k == 0 ? nl0 : get(cn, k - 1), nlb = get(cn, k);
                                const unsigned long long q = f2pack(get(cqx, k), get(cqx, k + 1));
                                unsigned long long qn = q, qm;
                                if constexpr (kTheta)
                                    qn = theta_q_x2(q, f2pack(k == 0 ? ql0 : get(cqx, k - 1), get(cqx, k)),
                                                    f2pack(get(cqx, k + 1), k + 1 == 3 ? qr3 : get(cqx, k + 2)), Kc);
                                if constexpr (kVec)
                                    qm = q_norm_x2(q, f2pack(k == 0 ? ys0 : get(cqy, k - 1), get(cqy, k)),
                                                   f2pack(get(cqy, k), get(cqy, k + 1)),
                                                   f2pack(k == 0 ? yn0 : get(qyn, k - 1), get(qyn, k)),
                                                   f2pack(get(qyn, k), get(qyn, k + 1)));
                                else
                                    qm = f2pack(fabsf(get(cqx, k)), fabsf(get(cqx, k + 1)));
                                const unsigned long long eL = f2add(f2pack(hla, hlb), f2pack(zla, zlb));
                                const unsigned long long eR = f2add(f2pack(get(ch, k), get(ch, k + 1)),
                                                                    f2pack(get(cz, k), get(cz, k + 1)));
                                const unsigned long long ns = f2add(f2pack(nla, nlb), f2pack(get(cn, k), get(cn, k + 1)));
                                const float2 zm = make_float2(fmaxf(zla, get(cz, k)), fmaxf(zlb, get(cz, k + 1)));
                                const float2 v = face_fast_sel_x2_gen(qm, qn, eL, eR, zm, ns, Kc);
                                set(qxw, k, v.x);
                                set(qxw, k + 1, v.y);
                            }
                        } else {
#pragma unroll
                        for (int k = 0; k < 4; k += 2) {
                            const float hla = k == 0 ? hl0 : get(ch, k - 1), hlb = get(ch, k);
                            const float zla = k == 0 ? zl0 : get(cz, k - 1), zlb = get(cz, k);
                            const float nla = k == 0 ? nl0 : get(cn, k - 1), nlb = get(cn, k);
                            const unsigned long long eL = f2add(f2pack(hla, hlb), f2pack(zla, zlb));
                            const unsigned long long eR = f2add(f2pack(get(ch, k), get(ch, k + 1)),
                                                                f2pack(get(cz, k), get(cz, k + 1)));
                            const unsigned long long ns = f2add(f2pack(nla, nlb), f2pack(get(cn, k), get(cn, k + 1)));
                            const float2 zm = make_float2(fmaxf(zla, get(cz, k)), fmaxf(zlb, get(cz, k + 1)));
                            const float2 v = face_fast_sel_x2(make_float2(get(cqx, k), get(cqx, k + 1)), eL, eR, zm, ns, Kc);
                            set(qxw, k, v.x);
                            set(qxw, k + 1, v.y);
                        }
                        }
                        if (edge_lane) {              // lanes at or beyond x = 0 or x = nx: Eq. 5-6, or no face
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                const int c = c0 + k;
                                if (!in_wface[k]) set(qxw, k, 0.0f);
                                if (c == 0 || c == nx) {
                                    float qo = 0.0f;
                                    const float hl = k == 0 ? hl0 : get(ch, k - 1);
                                    const float nl = k == 0 ? nl0 : get(cn, k - 1);
                                    const float v = c == 0 ? boundary_fast_flux(a, step, 0, r, get(ch, 0), get(cn, 0), qo)
                                                           : boundary_fast_flux(a, step, 1, r, hl, nl, qo);
                                    if (own_row_r && own_wface[k]) fq += qo;
                                    set(qxw, k, v);
                                }
                            }
                        }
                        qxe_p = __shfl_down_sync(0xffffffffu, qxw.x, 1);
                        hp = ch;
                        qxw_p = qxw;
                        qys_p = qys;
                        if constexpr (kOpt) {
                            qyo_p = cqy;
                            qxo_p = cqx;
                        }
                    }
                }
            }
            // ---- end of tick (shares a timeout); then level 1 refills the ring
            if (__syncthreads_or(stop ? 1 : 0)) {
                abort = true;
                break;
            }
            if (lvl == 1 && lane == 0 && r >= jb && r <= jload_hi) {
                consumed = r - jb + 1;
                if (issued < nload) {
                    fence_proxy_async();
                    issue(issued);
                    issued++;
                }
            }
        }
        // fold the run into the warp's double sums (rare: boundary faces, clipped cells)
        if (__any_sync(0xffffffffu, fq != 0.0f || fc != 0.0f)) {
            const double wq = warp_sum((double)fq), wc = warp_sum((double)fc);
            if (lane == 0) {
                sm.led[warp][0] += wq * G.dx;
                sm.led[warp][1] += wc * G.dx * G.dx;
            }
        }
    }
    if (!abort) {
        base += (uint32_t)nload;
    } else if (threadIdx.x == 0) {
        // leave no bulk copy writing into shared memory after exit
        for (int k = consumed; k < issued; k++) {
            const uint32_t g = base + (uint32_t)k;
            mbar_wait_bounded(&sm.bar[g % kPF], (g / kPF) & 1u, kBudgetNs);
        }
        atomicOr(&a.ctrl->status, kStatusTimeout);
    }
    return abort;
}

// Block-wide sums of the ledger terms into grid a's control block; the
// warps' volume sums (led, K levels) are reset for the next grid.
template <int K>
__device__ __forceinline__ void tiled_flush(const StepArgs<float> &a, const TiledLedger &L, const int want_hmax,
                                            double *red, double (*led)[2])
{
    __syncthreads();                                  // every warp's last run is in led
    if (threadIdx.x == 0) {
        double bo = 0.0, bc = 0.0;
        for (int w = 0; w < K; w++) {
            bo += led[w][0];
            bc += led[w][1];
            led[w][0] = led[w][1] = 0.0;
        }
        if (bo != 0.0) atomicAdd(&a.ctrl->V_out, a.ctrl->dt * bo);
        if (bc != 0.0) atomicAdd(&a.ctrl->V_clip, bc);
    }
    if (want_hmax) {
        const double bm = block_reduce<true>(L.nan_seen ? (double)NAN : (double)L.hmax, red);
        if (threadIdx.x == 0) atomic_max_nonneg(&a.ctrl->hmax_bits, bm);
    }
}

// Inflow volume of the K steps and the clock after them (one thread per grid).
template <int K>
__device__ __forceinline__ void tiled_finish(const StepArgs<float> &a, const int s0)
{
    const double dtd = a.ctrl->dt;
    double vin = a.ctrl->V_in;
    for (int s = 0; s < K; s++)
        for (int k = 0; k < a.n_inflow_sec; k++) {
            const double Q = a.inflow_Q[(size_t)(s0 + s) * a.n_inflow_sec + k];
            if (Q > 0.0) vin += dtd * Q;
        }
    a.ctrl->V_in = vin;
    a.ctrl->t = a.t_list[s0 + K];
}

template <int K, int kPF, int kHo>
__device__ __forceinline__ void init_ring(PipeSmem<K, kPF, kHo> &sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < kPF; s++) mbar_init(&sm.bar[s], 1);
        fence_mbar_init();
        for (int w = 0; w < K; w++) sm.led[w][0] = sm.led[w][1] = 0.0;
    }
    __syncthreads();
}

// One grid: work items (chunk, strip) in chunk-major order (a.tile_x strips,
// a.tile_y rows per chunk); block b takes item b first and then the next item
// of the launch's counter (a.ctrl->next_item) whenever it comes free.
// Pipelines per SM the launch bounds ask for: six for Eq. 3 as printed with
// K = 4 (80 registers), five with the scheme options' extra row state.
__host__ __device__ constexpr int tiled_min_blocks(int K, int mode) { return K == 4 ? (mode ? 5 : 6) : K == 8 ? 2 : 1; }

template <int K, int kMode>
__global__ void __launch_bounds__(K * 32, tiled_min_blocks(K, kMode)) step_tiled_kernel(const StepArgs<float> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    using Smem = PipeSmem<K, kPF1, hand_fields(kMode)>;
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    init_ring(sm);
    const int n_strips = a.tile_x, chunk_rows = a.tile_y;
    const int n_items = n_strips * ((a.geo.ny + chunk_rows - 1) / chunk_rows);
    const FastConst Kc = tiled_const(a);
    TiledLedger L;
    uint32_t base = 0;
    __shared__ int next;
    for (int item = blockIdx.x; item < n_items;) {
        const int strip = item % n_strips;
        const int y0 = (item / n_strips) * chunk_rows;
        const int y1 = min(y0 + chunk_rows, a.geo.ny);
        if (tiled_item<K, kPF1, kMode>(a, a.s, Kc, strip, y0, y1, sm, base, L)) break;
        if (threadIdx.x == 0) next = (int)gridDim.x + atomicAdd(&a.ctrl->next_item, 1);
        __syncthreads();
        item = next;
        __syncthreads();                              // read by every thread before thread 0 writes it again
    }
    tiled_flush<K>(a, L, a.want_hmax, red, sm.led);
    if (blockIdx.x == 0 && threadIdx.x == 0) tiled_finish<K>(a, a.s);
}

// Many grids: the items of grid k (its (chunk, strip) items, table[k].tile_y
// rows per chunk) are numbered base[k] .. base[k+1] - 1, grids ordered largest
// first; block b takes item b first and then, with next_item, the next
// unclaimed item of the counter (items grid, grid + 1, ... in the order the
// pipelines come free), else b + grid, b + 2 grid, ...  Either way a block's
// items ascend, so its grids do too.  A block sums a grid's
// ledger terms while its items belong to that grid and hands them to the
// grid's control block when it moves on; the grid's first item books its
// inflow volume and clock.
template <int K, int kMode>
__global__ void __launch_bounds__(K * 32, K == 4 ? (kMode ? 4 : 6) : K == 8 ? 2 : 1)
    step_tiled_ensemble_kernel(const StepArgs<float> *table, const int *base, const int n, const int s0,
                               const int want_hmax, int *next_item)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int next;
    using Smem = PipeSmem<K, kPFE, hand_fields(kMode)>;
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    init_ring(sm);
    const int total = base[n];
    TiledLedger L;
    uint32_t ring = 0;
    int cur = -1;
    for (int item = blockIdx.x; item < total;) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (base[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            if (cur >= 0) tiled_flush<K>(table[cur], L, want_hmax, red, sm.led);
            L = TiledLedger();
            cur = lo;
        }
        const StepArgs<float> &a = table[lo];
        const int local = item - base[lo];
        const int n_strips = (a.geo.nx + out_cols(K, kMode) - 1) / out_cols(K, kMode);
        const int strip = local % n_strips;
        const int y0 = (local / n_strips) * a.tile_y;
        const int y1 = min(y0 + a.tile_y, a.geo.ny);
        if (local == 0 && threadIdx.x == 0) tiled_finish<K>(a, s0);
        if (tiled_item<K, kPFE, kMode>(a, s0, tiled_const(a), strip, y0, y1, sm, ring, L)) break;
        if (threadIdx.x == 0) next = next_item ? (int)gridDim.x + atomicAdd(next_item, 1) : item + (int)gridDim.x;
        __syncthreads();
        item = next;
        __syncthreads();                              // read by every thread before thread 0 writes it again
    }
    if (cur >= 0) tiled_flush<K>(table[cur], L, want_hmax, red, sm.led);
}


// Blocks of `kernel` (K warps, `smem` bytes) resident on the GPU at once; the
// first call of a kernel sets its shared-memory limit and fills `cache` (threads
// that race here do the same work and store the same value).
template <typename Kern>
cudaError_t resident_blocks(Kern kernel, int threads, size_t smem, std::atomic<int> *cache, int *out)
{
    int v = cache->load(std::memory_order_acquire);
    if (!v) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
        if (e != cudaSuccess) return e;
        v = (per_sm < 1 ? 1 : per_sm) * sms;
        cache->store(v, std::memory_order_release);
    }
    *out = v;
    return cudaSuccess;
}

template <int K, int kMode>
cudaError_t launch_k(const StepArgs<float> &a0, cudaStream_t st)
{
    using Smem = PipeSmem<K, kPF1, hand_fields(kMode)>;
    static std::atomic<int> cache{0};
    int resident = 0;
    cudaError_t e = resident_blocks(step_tiled_kernel<K, kMode>, K * 32, sizeof(Smem), &cache, &resident);
    if (e != cudaSuccess) return e;
    StepArgs<float> a = a0;
    const int nx = a.geo.nx, ny = a.geo.ny;
    const int n_strips = (nx + out_cols(K, kMode) - 1) / out_cols(K, kMode);
    if (a0.tile_x > 0 && a0.tile_x < resident) resident = a0.tile_x;   // caller's cap on pipelines
    int chunk_rows = 0, blocks = 0;
    if (a0.tile_y > 0) {                                                // caller's rows per work item
        chunk_rows = a0.tile_y < ny ? a0.tile_y : ny;
        const long long items = (long long)n_strips * ((ny + chunk_rows - 1) / chunk_rows);
        blocks = (int)(items < resident ? items : resident);
    } else {
        tiled_split_dynamic(n_strips, ny, resident, K, &chunk_rows, &blocks);
    }
    a.tile_x = n_strips;
    a.tile_y = chunk_rows;
    e = cudaMemsetAsync(&a.ctrl->next_item, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    step_tiled_kernel<K, kMode><<<blocks, K * 32, sizeof(Smem), st>>>(a);
    return cudaGetLastError();
}

template <int K, int kMode>
cudaError_t launch_ens_k(const StepArgs<float> *table, const int *base, int n, int total_items, int s0,
                         int want_hmax, int *next_item, cudaStream_t st)
{
    using Smem = PipeSmem<K, kPFE, hand_fields(kMode)>;
    static std::atomic<int> cache{0};
    int resident = 0;
    cudaError_t e = resident_blocks(step_tiled_ensemble_kernel<K, kMode>, K * 32, sizeof(Smem), &cache, &resident);
    if (e != cudaSuccess) return e;
    const int blocks = total_items < resident ? total_items : resident;
    if (blocks < 1) return cudaSuccess;
    step_tiled_ensemble_kernel<K, kMode><<<blocks, K * 32, sizeof(Smem), st>>>(table, base, n, s0, want_hmax,
                                                                             next_item);
    return cudaGetLastError();
}


// Launchers of one scheme mode for every steps-per-launch K.
template <int kMode>
cudaError_t launch_tiled_mode(const StepArgs<float> &a, cudaStream_t st)
{
    switch (a.k_steps) {
    case 1: return launch_k<1, kMode>(a, st);
    case 2: return launch_k<2, kMode>(a, st);
    case 3: return launch_k<3, kMode>(a, st);
    case 4: return launch_k<4, kMode>(a, st);
    case 8: return launch_k<8, kMode>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int kMode>
cudaError_t launch_tiled_ensemble_mode(const StepArgs<float> *table, const int *base, int n, int total_items,
                                       int k_steps, int s0, int want_hmax, int *next_item, cudaStream_t st)
{
    switch (k_steps) {
    case 1: return launch_ens_k<1, kMode>(table, base, n, total_items, s0, want_hmax, next_item, st);
    case 2: return launch_ens_k<2, kMode>(table, base, n, total_items, s0, want_hmax, next_item, st);
    case 3: return launch_ens_k<3, kMode>(table, base, n, total_items, s0, want_hmax, next_item, st);
    case 4: return launch_ens_k<4, kMode>(table, base, n, total_items, s0, want_hmax, next_item, st);
    case 8: return launch_ens_k<8, kMode>(table, base, n, total_items, s0, want_hmax, next_item, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace flood
