// step_stream.cu -- FP32 single-step kernel fed by the bulk-copy engine.
//
// Same work split and arithmetic as the row-streaming kernel (one warp per
// 128-column strip and a chunk of rows, south to north, previous row in
// registers), but the rows arrive through a per-warp ring of kDepth shared
// memory stages filled by 1D bulk copies (cp.async.bulk, one per field and
// row, completion counted on an mbarrier per stage).  Lane 0 keeps kDepth
// rows in flight while the warp computes, so memory latency is hidden by
// copies in flight instead of by registers or extra warps.  Each staged row
// segment covers columns x0-4 .. x0+131, so the west and east neighbour
// columns of the strip come from shared memory as well.
//
// Waits are bounded: a stage that does not complete within ~2 s sets the
// timeout status bit, the warp waits (bounded) for its copies in flight and
// leaves without storing.
#include <cuda.h>

#include <atomic>
#include <type_traits>

#include "fast_face.cuh"
#include "tma_util.cuh"

namespace flood {

namespace {

constexpr int kMaxWarps = 4;     // warps (strips) per block at most
constexpr int kDepth = 4;        // rows in flight per warp
constexpr int kSeg = 136;        // floats per staged row segment (x0-4 .. x0+131)
constexpr int kFields = 5;       // h, z, n, qx, qy
constexpr uint64_t kBudgetNs = 2000000000ull;

// 16-byte aligned size: every warp's ring (bulk-copy destinations, float4
// loads) must start on a 16-byte boundary.
struct alignas(16) WarpRing {
    float buf[kDepth][kFields][kSeg];
    uint64_t bar[kDepth];
};

static_assert(sizeof(WarpRing) % 16 == 0, "per-warp ring must keep 16-byte alignment");

// The TMA-tile variant stages 2D tiles: per stage and field one tensor copy of
// kRowsT rows x kSeg columns (box origin x0-4, 16-byte aligned; elements
// outside the grid arrive as zeros).  A tensor copy's shared-memory
// destination must be 128-byte aligned, so each field's tile takes a slot of
// kSlotT floats (a multiple of 32) and the ring a multiple of 128 bytes.
constexpr int kRowsT = 2;        // rows per staged tile
constexpr int kStagesT = 2;      // tiles in flight per warp
constexpr int kSlotT = 288;      // >= kRowsT * kSeg, multiple of 32 floats
struct alignas(128) WarpRingT {
    float buf[kStagesT][kFields][kSlotT];
    uint64_t bar[kStagesT];
};
static_assert(kSlotT >= kRowsT * kSeg && kSlotT % 32 == 0, "tile slot must hold the box and keep 128 B alignment");
static_assert(sizeof(WarpRingT) % 128 == 0, "per-warp tile ring must keep 128-byte alignment");

// Tensor maps of h, z, n, qx, qy (the current buffers) for the TMA-tile kernel.
struct TmaMaps {
    CUtensorMap m[kFields];
};

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

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

// One block's work: warps cover consecutive 128-column strips of strip block
// bx, all on the row chunk by of `rows` rows; step is the step inside the epoch.
//
// ring_base counts the rows this warp staged in earlier calls (a persistent
// block calls it once per work item): the slot and phase of staged row idx are
// those of ring_base + idx.  fresh: the ring's barriers still need their
// initialisation.  Returns true if a wait on a copy timed out (the status word
// then has the timeout bit).
//
// kTensor: stage 2D tiles of kRowsT rows with tensor copies (maps: the grid's
// tensor maps; the ring counts tiles) instead of one 1D copy per row.
// kTheta: theta-weighted numerator discharges (FastConst theta, w): an x-face
// takes its row neighbours from the lane, the neighbouring lanes and the
// staged halo columns, a y-face the previous row's old qy (kept in registers)
// and the next row's (read from the ring one row ahead).
// kMode bit 0: kTheta.  Bit 1: vector-norm |q| in the friction term: an x-face
// takes the old qy of its two cells' south faces (this row, staged) and north
// faces (the next row's, read one row ahead as for kTheta), a y-face the old qx
// of its two cells' west and east faces (this row and the previous row's, kept
// in registers).
template <bool kTensor, int kMode = 0>
__device__ __forceinline__ bool stream_body(const StepArgs<float> &a, const int step, const int want_hmax, const int bx,
                                            const int by, const int rows, unsigned char *smem_raw, double *red,
                                            uint32_t &ring_base, const bool fresh, const TmaMaps *maps = nullptr)
{
    constexpr bool kTheta = (kMode & 1) != 0, kVec = (kMode & 2) != 0;
    constexpr int R = kTensor ? kRowsT : 1;            // rows per stage
    constexpr int NS = kTensor ? kStagesT : kDepth;    // stages in flight
    const Geom &G = a.geo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nx = G.nx, ny = G.ny;
    const int P = G.pitch;
    const int x0 = (bx * nwarps + warp) * 128;
    const int c0 = x0 + 4 * lane;
    const bool full = c0 + 3 < nx;                  // all four columns of the lane inside the grid
    const bool active = x0 < nx;
    const int y0 = by * rows;
    const int y1 = min(y0 + rows, ny);
    const int jstart = y0 > 0 ? y0 - 1 : 0;
    const int jlast = min(y1, ny - 1);             // last row that is staged
    const int nload = jlast - jstart + 1;
    const int nstage = (nload + R - 1) / R;        // stages (tiles) to stage
    using Ring = typename std::conditional<kTensor, WarpRingT, WarpRing>::type;
    Ring &ring = reinterpret_cast<Ring *>(smem_raw)[warp];
    // field f of staged row `sub` of stage slot s: columns x0-4 .. x0+131 at offsets 0 .. 135
    auto row_at = [&](uint32_t s, int f, int sub) -> const float * {
        if constexpr (kTensor) return &ring.buf[s][f][sub * kSeg];
        else return &ring.buf[s][f][0];
    };

    const double dtd = a.ctrl->dt;
    FastConst K;
    const float dt = (float)dtd, dx = (float)G.dx, g = (float)G.g;
    K.gdt = g * dt;
    K.a1 = K.gdt / dx;
    K.gdt4 = 0.25f * K.gdt;
    K.h_dry = (float)G.h_dry;
    K.dtdx = dt / dx;
    K.theta = (float)G.theta;
    K.w = (float)(0.5 * (1.0 - G.theta));

    double vout = 0.0, vclip = 0.0;
    float hmax = 0.0f;
    bool nan_seen = false;

    // staged segment: global columns [cs, ce) land at ring offset so
    const int cs = max(x0 - 4, 0);
    const int ce = min(x0 + 132, P);
    const int so = cs - (x0 - 4);
    const uint32_t seg_bytes = (uint32_t)(ce - cs) * 4u;
    const float *fields[kFields] = {a.h, a.z, a.n, a.qx, a.qy};

    if (fresh && lane == 0) {                 // every warp: it may be idle here and busy on a later item
        for (int s = 0; s < NS; s++) mbar_init(&ring.bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int st) {                // stage st covers staged rows st*R .. st*R + R - 1
        const uint32_t s = (ring_base + (uint32_t)st) % NS;
        if constexpr (kTensor) {
            mbar_arrive_expect_tx(&ring.bar[s], (uint32_t)(kFields * kRowsT * kSeg * 4));
#pragma unroll
            for (int f = 0; f < kFields; f++) tma_load_2d(&ring.buf[s][f][0], &maps->m[f], x0 - 4, jstart + st * R, &ring.bar[s]);
        } else {
            const size_t row = (size_t)(jstart + st) * P + cs;
            mbar_arrive_expect_tx(&ring.bar[s], seg_bytes * kFields);
#pragma unroll
            for (int f = 0; f < kFields; f++) bulk_copy_g2s(&ring.buf[s][f][so], fields[f] + row, seg_bytes, &ring.bar[s]);
        }
    };
    int issued = 0, consumed = 0;             // stages
    bool abort = false;
    if (active && lane == 0) {
        fence_proxy_async();              // this warp's reads of an earlier item come first
        for (; issued < min(NS, nstage); issued++) issue(issued);
    }

    float4 hp = make_float4(0, 0, 0, 0), zp = hp, np_ = hp;
    float4 qxw_p = hp, qys_p = hp;
    float4 qyo_p = hp;                            // old qy of the previous row (theta weighting)
    float4 qxo_p = hp;                            // old qx of the previous row (vector-norm friction)
    float qxEo_p = 0.0f;                          // lane 31: the previous row's old qx at x0 + 128
    float qxe_p3 = 0.0f;
    if (active) {
        for (int j = jstart; j <= y1; j++) {
            const int idx = j - jstart;
            float4 ch = make_float4(0, 0, 0, 0), cz = ch, cn = ch, cqx = ch, cqy = ch;
            float hW = 0.f, zW = 0.f, nW = 0.f, hE = 0.f, zE = 0.f, nE = 0.f, qxE = 0.f;
            float qxW = 0.f, qxEE = 0.f;              // old qx at x0-1 and x0+129 (theta weighting)
            float qyW = 0.f, qyE = 0.f;               // old qy at x0-1 and x0+128 (vector-norm friction)
            if (j < ny) {
                const int st = idx / R, sub = idx - st * R;
                const uint32_t g = ring_base + (uint32_t)st;
                const uint32_t s = g % NS;
                if (sub == 0) {               // first row of a stage: wait for its copies
                    bool ok = mbar_wait_bounded(&ring.bar[s], (g / NS) & 1u, kBudgetNs);
                    if (__any_sync(0xffffffffu, !ok)) {
                        abort = true;
                        break;
                    }
                    consumed = st + 1;
                }
                const int o = 4 + 4 * lane;
                ch = lds4(row_at(s, 0, sub) + o);
                cz = lds4(row_at(s, 1, sub) + o);
                cn = lds4(row_at(s, 2, sub) + o);
                cqx = lds4(row_at(s, 3, sub) + o);
                cqy = lds4(row_at(s, 4, sub) + o);
                if (lane == 0) {
                    hW = row_at(s, 0, sub)[3];
                    zW = row_at(s, 1, sub)[3];
                    nW = row_at(s, 2, sub)[3];
                    if constexpr (kTheta) qxW = row_at(s, 3, sub)[3];
                    if constexpr (kVec) qyW = row_at(s, 4, sub)[3];
                }
                if (lane == 31) {
                    hE = row_at(s, 0, sub)[132];
                    zE = row_at(s, 1, sub)[132];
                    nE = row_at(s, 2, sub)[132];
                    qxE = row_at(s, 3, sub)[132];
                    if constexpr (kTheta) qxEE = row_at(s, 3, sub)[133];
                    if constexpr (kVec) qyE = row_at(s, 4, sub)[132];
                }
                if (sub == R - 1) {           // stage read completely: refill it
                    __syncwarp();
                    if (lane == 0 && issued < nstage) {
                        fence_proxy_async();
                        issue(issued);
                        issued++;
                    }
                }
            }
            if (j < y0) {                 // halo row south of the chunk
                hp = ch;
                zp = cz;
                np_ = cn;
                qyo_p = cqy;
                qxo_p = cqx;
                qxEo_p = qxE;
                continue;
            }
            // old qy of row j + 1 <= ny (the north faces of row j), with lane 0's column
            // x0 - 1 and lane 31's x0 + 128 for the vector norm: a staged row is read from
            // the ring one row ahead (waiting for its copies if they have not landed), the
            // rows beyond the staged ones (the chunk's last, the grid's north edge) from
            // global memory
            float4 qyn = make_float4(0, 0, 0, 0);
            float qynW = 0.0f, qynE = 0.0f;
            if constexpr (kTheta || kVec) {
                const int jn = j + 1;
                if (jn <= jlast) {
                    const int idn = jn - jstart;
                    const int st = idn / R, sub = idn - st * R;
                    const uint32_t g = ring_base + (uint32_t)st;
                    const uint32_t s = g % NS;
                    if (sub == 0) {
                        bool ok = mbar_wait_bounded(&ring.bar[s], (g / NS) & 1u, kBudgetNs);
                        if (__any_sync(0xffffffffu, !ok)) {
                            abort = true;
                            break;
                        }
                        consumed = st + 1;
                    }
                    qyn = lds4(row_at(s, 4, sub) + 4 + 4 * lane);
                    if constexpr (kVec) {
                        if (lane == 0) qynW = row_at(s, 4, sub)[3];
                        if (lane == 31) qynE = row_at(s, 4, sub)[132];
                    }
                } else if (jn <= ny && (kTheta || j < y1)) {
                    const float *row = a.qy + (size_t)jn * P;
                    if (c0 < P) qyn = __ldg(reinterpret_cast<const float4 *>(row + c0));
                    if constexpr (kVec) {
                        if (lane == 0 && x0 > 0) qynW = __ldg(row + x0 - 1);
                        if (lane == 31 && x0 + 128 < nx) qynE = __ldg(row + x0 + 128);
                    }
                }
            }
            // ---- new south faces of row j
            // (interior rows branch-free; the boundary rows, uniform over the warp, take Eq. 5-6)
            float4 qys;
            if (j > 0 && j < ny) {
                if constexpr (kTheta || kVec) {
                    // old qx of rows j - 1 and j right of the lane's last column
                    float xs4 = 0.0f, xn4 = 0.0f;
                    if constexpr (kVec) {
                        xs4 = __shfl_down_sync(0xffffffffu, qxo_p.x, 1);
                        xn4 = __shfl_down_sync(0xffffffffu, cqx.x, 1);
                        if (lane == 31) {
                            xs4 = qxEo_p;
                            xn4 = qxE;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const float zl = get(zp, k), zr = get(cz, k), q = get(cqy, k);
                        const float qn = kTheta ? theta_q(q, get(qyo_p, k), get(qyn, k), K) : q;
                        const float qm = kVec ? q_norm(q, get(qxo_p, k), k < 3 ? get(qxo_p, k + 1) : xs4, get(cqx, k),
                                                       k < 3 ? get(cqx, k + 1) : xn4)
                                              : fabsf(q);
                        set(qys, k, face_fast_sel_gen(qm, qn, get(hp, k) + zl, get(ch, k) + zr, fmaxf(zl, zr),
                                                      get(np_, k) + get(cn, k), K));
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const float zl = get(zp, k), zr = get(cz, k);
                        set(qys, k, face_fast_sel(get(cqy, k), get(hp, k) + zl, get(ch, k) + zr, fmaxf(zl, zr),
                                                  get(np_, k) + get(cn, k), K));
                    }
                }
                if (!full) {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (c0 + k >= nx) set(qys, k, 0.0f);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    int c = c0 + k;
                    float v = 0.0f;
                    if (c < nx)
                        v = j == 0 ? boundary_fast_at(a, step, 2, c, get(ch, k), get(cn, k), vout)
                                   : boundary_fast_at(a, step, 3, c, get(hp, k), get(np_, k), vout);
                    set(qys, k, v);
                }
            }
            // ---- finish row j-1
            if (j > y0) {
                const int jr = j - 1;
                const size_t r = (size_t)jr * P + c0;
                float4 hn;
                bool neg = false;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    float qe = k < 3 ? get(qxw_p, k + 1) : qxe_p3;
                    float dv = __fadd_rn(__fsub_rn(get(qxw_p, k), qe), __fsub_rn(get(qys_p, k), get(qys, k)));
                    float v = __fmaf_rn(K.dtdx, dv, get(hp, k));
                    neg |= v < 0.0f;
                    set(hn, k, v);
                }
                if (neg) {                        // rare: clip to zero, book the removed volume
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const float v = get(hn, k);
                        if (v < 0.0f) {
                            if (c0 + k < nx && jr >= G.led_j0 && jr < G.led_j1) vclip += -(double)v * G.dx * G.dx;
                            set(hn, k, 0.0f);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float v = get(hn, k);
                    if (full || c0 + k < nx) {
                        hmax = fmaxf(hmax, v);
                        nan_seen |= (v != v);
                    }
                }
                if (c0 + 3 < nx) {
                    *reinterpret_cast<float4 *>(a.h_out + r) = hn;
                    *reinterpret_cast<float4 *>(a.qy_out + r) = qys_p;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (c0 + k < nx) {
                            a.h_out[r + k] = get(hn, k);
                            a.qy_out[r + k] = get(qys_p, k);
                        }
                }
                if (c0 + 3 <= nx) *reinterpret_cast<float4 *>(a.qx_out + r) = qxw_p;
                else {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (c0 + k <= nx) a.qx_out[r + k] = get(qxw_p, k);
                }
                if (lane == 31 && x0 + 128 == nx) a.qx_out[(size_t)jr * P + nx] = qxe_p3;
                if (jr == ny - 1) {
                    const size_t rn = (size_t)ny * P + c0;
                    if (c0 + 3 < nx) *reinterpret_cast<float4 *>(a.qy_out + rn) = qys;
                    else {
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            if (c0 + k < nx) a.qy_out[rn + k] = get(qys, k);
                    }
                }
            }
            if (j == y1) break;
            // ---- new west faces of row j
            float hl0 = __shfl_up_sync(0xffffffffu, ch.w, 1);
            float zl0 = __shfl_up_sync(0xffffffffu, cz.w, 1);
            float nl0 = __shfl_up_sync(0xffffffffu, cn.w, 1);
            if (lane == 0) {
                hl0 = hW;
                zl0 = zW;
                nl0 = nW;
            }
            float4 qxw;
            if constexpr (kTheta || kVec) {
                // old qx of the faces left of the lane's first and right of its last column
                float ql0 = 0.0f, qr3 = 0.0f;
                if constexpr (kTheta) {
                    ql0 = __shfl_up_sync(0xffffffffu, cqx.w, 1);
                    qr3 = __shfl_down_sync(0xffffffffu, cqx.x, 1);
                    if (lane == 0) ql0 = qxW;
                    if (lane == 31) qr3 = qxE;
                }
                // old qy of rows j and j + 1 left of the lane's first column
                float ys0 = 0.0f, yn0 = 0.0f;
                if constexpr (kVec) {
                    ys0 = __shfl_up_sync(0xffffffffu, cqy.w, 1);
                    yn0 = __shfl_up_sync(0xffffffffu, qyn.w, 1);
                    if (lane == 0) {
                        ys0 = qyW;
                        yn0 = qynW;
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float hl = k == 0 ? hl0 : get(ch, k - 1);
                    const float zl = k == 0 ? zl0 : get(cz, k - 1);
                    const float nl = k == 0 ? nl0 : get(cn, k - 1);
                    const float zr = get(cz, k), q = get(cqx, k);
                    const float qn = kTheta ? theta_q(q, k == 0 ? ql0 : get(cqx, k - 1), k == 3 ? qr3 : get(cqx, k + 1), K)
                                            : q;
                    const float qm = kVec ? q_norm(q, k == 0 ? ys0 : get(cqy, k - 1), get(cqy, k),
                                                   k == 0 ? yn0 : get(qyn, k - 1), get(qyn, k))
                                          : fabsf(q);
                    set(qxw, k, face_fast_sel_gen(qm, qn, hl + zl, get(ch, k) + zr, fmaxf(zl, zr), nl + get(cn, k), K));
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float hl = k == 0 ? hl0 : get(ch, k - 1);
                    const float zl = k == 0 ? zl0 : get(cz, k - 1);
                    const float nl = k == 0 ? nl0 : get(cn, k - 1);
                    const float zr = get(cz, k);
                    set(qxw, k, face_fast_sel(get(cqx, k), hl + zl, get(ch, k) + zr, fmaxf(zl, zr), nl + get(cn, k), K));
                }
            }
            if (c0 == 0 || !full) {               // lanes holding x = 0 or x >= nx: Eq. 5-6, or no face
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int c = c0 + k;
                    const float hl = k == 0 ? hl0 : get(ch, k - 1);
                    const float nl = k == 0 ? nl0 : get(cn, k - 1);
                    if (c == 0) set(qxw, k, boundary_fast_at(a, step, 0, j, get(ch, 0), get(cn, 0), vout));
                    else if (c == nx) set(qxw, k, boundary_fast_at(a, step, 1, j, hl, nl, vout));
                    else if (c > nx) set(qxw, k, 0.0f);
                }
            }
            float qe = __shfl_down_sync(0xffffffffu, qxw.x, 1);
            if (lane == 31) {
                const int c = x0 + 128;
                qe = 0.0f;
                if (c == nx) qe = boundary_fast_at(a, step, 1, j, ch.w, cn.w, vout);
                else if (c < nx) {
                    if constexpr (kTheta || kVec) {
                        const float qn = kTheta ? theta_q(qxE, cqx.w, qxEE, K) : qxE;
                        const float qm = kVec ? q_norm(qxE, cqy.w, qyE, qyn.w, qynE) : fabsf(qxE);
                        qe = face_fast_gen(qm, qn, ch.w + cz.w, hE + zE, fmaxf(cz.w, zE), cn.w + nE, K);
                    } else
                        qe = face_fast(qxE, ch.w + cz.w, hE + zE, fmaxf(cz.w, zE), cn.w + nE, K);
                }
            }
            hp = ch;
            zp = cz;
            np_ = cn;
            qyo_p = cqy;
            qxo_p = cqx;
            qxEo_p = qxE;
            qxw_p = qxw;
            qxe_p3 = qe;
            qys_p = qys;
        }
        if (abort) {
            // leave no bulk copy writing into shared memory after exit
            if (lane == 0) {
                for (int k = consumed; k < issued; k++) {
                    const uint32_t g = ring_base + (uint32_t)k;
                    mbar_wait_bounded(&ring.bar[g % NS], (g / NS) & 1u, kBudgetNs);
                }
                atomicOr(&a.ctrl->status, kStatusTimeout);
            }
            __syncwarp();
        }
        if (!abort) ring_base += (uint32_t)nstage;
    }
    double bo = block_reduce<false>(vout, red);
    if (threadIdx.x == 0 && bo != 0.0) atomicAdd(&a.ctrl->V_out, dtd * bo);
    double bc = block_reduce<false>(vclip, red);
    if (threadIdx.x == 0 && bc != 0.0) atomicAdd(&a.ctrl->V_clip, bc);
    if (want_hmax) {
        double bm = block_reduce<true>(nan_seen ? (double)NAN : (double)hmax, red);
        if (threadIdx.x == 0) atomic_max_nonneg(&a.ctrl->hmax_bits, bm);
    }
    if (bx == 0 && by == 0 && threadIdx.x == 0) {
        double vin = a.ctrl->V_in;
        for (int k = 0; k < a.n_inflow_sec; k++) {
            double Q = a.inflow_Q[(size_t)step * a.n_inflow_sec + k];
            if (Q > 0.0) vin += dtd * Q;
        }
        a.ctrl->V_in = vin;
        a.ctrl->t = a.t_list[step + 1];
    }
    return abort;
}

template <int kMode>
__global__ void __launch_bounds__(kMaxWarps * 32, 5) step_stream_kernel(const StepArgs<float> a, const int rows,
                                                                         const int nbx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    uint32_t ring_base = 0;
    stream_body<false, kMode>(a, a.s, a.want_hmax, (int)(blockIdx.x % (unsigned)nbx), (int)(blockIdx.x / (unsigned)nbx),
                              rows, smem_raw, red, ring_base, true);
}

// The same step with every warp's rows staged as 2D tiles by tensor copies.
template <int kMode>
__global__ void __launch_bounds__(kMaxWarps * 32, 4)
    step_tma_kernel(const StepArgs<float> a, const int rows, const int nbx, const __grid_constant__ TmaMaps maps)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    unsigned char *base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);   // 128-byte aligned rings
    uint32_t ring_base = 0;
    stream_body<true, kMode>(a, a.s, a.want_hmax, (int)(blockIdx.x % (unsigned)nbx), (int)(blockIdx.x / (unsigned)nbx),
                             rows, base, red, ring_base, true,
                              &maps);
}

// Many grids in one launch: block b belongs to the scenario whose block range
// [base[k], base[k+1]) holds it (scenarios ordered largest first); kMode as
// for one grid (the scenarios share their scheme options).
template <int kMode>
__global__ void __launch_bounds__(kMaxWarps * 32, 5)
    step_stream_ensemble_kernel(const StepArgs<float> *table, const int *base, const int n, const int rows,
                                const int step, const int want_hmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const int b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const StepArgs<float> &a = table[lo];
    const int nwarps = blockDim.x >> 5;
    const int strips = (a.geo.nx + 127) / 128;
    const int nbx = (strips + nwarps - 1) / nwarps;
    const int local = b - base[lo];
    uint32_t ring_base = 0;
    stream_body<false, kMode>(a, step, want_hmax, local % nbx, local / nbx, rows, smem_raw, red, ring_base, true);
}

// Variant of the stream/TMA kernels for a grid's options: bit 0 theta
// weighting, bit 1 vector-norm friction.
int kernel_mode(const Geom &g) { return (g.theta != 1.0 ? 1 : 0) | (g.friction != 0 ? 2 : 0); }

cudaError_t configure(int warps)
{
    static std::atomic<bool> configured{false};
    if (configured.load(std::memory_order_acquire)) return cudaSuccess;
    for (auto k : {step_stream_kernel<0>, step_stream_kernel<1>, step_stream_kernel<2>, step_stream_kernel<3>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(WarpRing) * kMaxWarps));
        if (e != cudaSuccess) return e;
    }
    for (auto k : {step_stream_ensemble_kernel<0>, step_stream_ensemble_kernel<1>, step_stream_ensemble_kernel<2>,
                   step_stream_ensemble_kernel<3>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(WarpRing) * kMaxWarps));
        if (e != cudaSuccess) return e;
    }
    configured.store(true, std::memory_order_release);
    (void)warps;
    return cudaSuccess;
}

}  // namespace

int stream_blocks(const Geom &g, int warps, int rows)
{
    const int strips = (g.nx + 127) / 128;
    return ((strips + warps - 1) / warps) * ((g.ny + rows - 1) / rows);
}

// Launch shape: the caller's (tile_x warps, tile_y rows) when given, else by
// the number of warps W = strips x chunks.  An SM holds 20 of these warps (the
// shared-memory rings of five 4-warp blocks), the GPU 3040.  Take the tallest
// chunk (fewer halo-row re-reads) whose W is at least two thirds of that and
// not between one and two and a half times it (a partly filled second wave
// leaves SMs idle at the tail); four warps per block once W passes 16 waves,
// else two.  Measured on the fractal workload against 14 shapes, this takes
// the fastest, or one within 1 %, at 1024^2, 2048^2, 4096^2, 8192^2 and
// 16384^2: (2, 4), (2, 16), (2, 16), (2, 32), (4, 32).
void stream_launch_shape(const Geom &g, int tile_x, int tile_y, int *warps, int *rows)
{
    const int strips = (g.nx + 127) / 128;
    int r = 4;
    for (int cand : {32, 16, 8, 4}) {
        const int64_t W = (int64_t)strips * ((g.ny + cand - 1) / cand);
        if (W >= 2000 && !(W > 3040 && W < 7600)) {
            r = cand;
            break;
        }
    }
    const int64_t W = (int64_t)strips * ((g.ny + r - 1) / r);
    int w = W >= 16 * 3040 ? 4 : 2;
    if (w > strips) w = strips;
    *warps = (tile_x >= 1 && tile_x <= kMaxWarps) ? tile_x : w;
    *rows = tile_y >= 1 ? tile_y : r;
}

cudaError_t launch_step_stream(const StepArgs<float> &a, cudaStream_t st)
{
    int warps, rows;
    stream_launch_shape(a.geo, a.tile_x, a.tile_y, &warps, &rows);
    cudaError_t e = configure(warps);
    if (e != cudaSuccess) return e;
    const int strips = (a.geo.nx + 127) / 128;
    const int nbx = (strips + warps - 1) / warps, nby = (a.geo.ny + rows - 1) / rows;
    const unsigned grid = (unsigned)((int64_t)nbx * nby);     // one-dimensional: (bx, by) from the block index
    const size_t smem = sizeof(WarpRing) * warps;
    switch (kernel_mode(a.geo)) {
    case 0: step_stream_kernel<0><<<grid, warps * 32, smem, st>>>(a, rows, nbx); break;
    case 1: step_stream_kernel<1><<<grid, warps * 32, smem, st>>>(a, rows, nbx); break;
    case 2: step_stream_kernel<2><<<grid, warps * 32, smem, st>>>(a, rows, nbx); break;
    default: step_stream_kernel<3><<<grid, warps * 32, smem, st>>>(a, rows, nbx); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.gauge_out) return launch_gauges<float>(a.geo, a.h_out, a.gauge_cells, a.n_gauges, a.gauge_out, st);
    return cudaSuccess;
}

// cuTensorMapEncodeTiled from the CUDA driver (through the runtime's entry-point
// query, so the library needs no link against the CUDA driver library).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_tiled()
{
    // looked up once per process (a function-local static: thread-safe initialisation)
    static const EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiled>(p);
        return (EncodeTiled) nullptr;
    }();
    return fn;
}

// Map of a pitched FP32 field of `height` rows: boxes of kRowsT rows x kSeg
// columns, zero fill outside [0, pitch) x [0, height).
static cudaError_t encode_field(EncodeTiled fn, CUtensorMap *m, const float *base, int pitch, int height)
{
    const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)height};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kSeg, (cuuint32_t)kRowsT};
    const cuuint32_t elem[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_map_f32(void *map, const float *base, int width, int height, int pitch, int box_w, int box_h)
{
    EncodeTiled fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t elem[2] = {1, 1};
    const CUresult r = fn(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base),
                          dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step_tma(const StepArgs<float> &a, cudaStream_t st)
{
    EncodeTiled fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    int warps, rows;
    stream_launch_shape(a.geo, a.tile_x, a.tile_y, &warps, &rows);
    const size_t smem = sizeof(WarpRingT) * warps + 128;
    static std::atomic<bool> configured{false};
    if (!configured.load(std::memory_order_acquire)) {
        for (auto k : {step_tma_kernel<0>, step_tma_kernel<1>, step_tma_kernel<2>, step_tma_kernel<3>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(sizeof(WarpRingT) * kMaxWarps + 128));
            if (e != cudaSuccess) return e;
        }
        configured.store(true, std::memory_order_release);
    }
    const int P = a.geo.pitch, ny = a.geo.ny;
    TmaMaps maps;
    const float *f[kFields] = {a.h, a.z, a.n, a.qx, a.qy};
    for (int k = 0; k < kFields; k++) {
        cudaError_t e = encode_field(fn, &maps.m[k], f[k], P, k == 4 ? ny + 1 : ny);
        if (e != cudaSuccess) return e;
    }
    const int strips = (a.geo.nx + 127) / 128;
    const int nbx = (strips + warps - 1) / warps, nby = (ny + rows - 1) / rows;
    const unsigned grid = (unsigned)((int64_t)nbx * nby);     // one-dimensional: (bx, by) from the block index
    switch (kernel_mode(a.geo)) {
    case 0: step_tma_kernel<0><<<grid, warps * 32, smem, st>>>(a, rows, nbx, maps); break;
    case 1: step_tma_kernel<1><<<grid, warps * 32, smem, st>>>(a, rows, nbx, maps); break;
    case 2: step_tma_kernel<2><<<grid, warps * 32, smem, st>>>(a, rows, nbx, maps); break;
    default: step_tma_kernel<3><<<grid, warps * 32, smem, st>>>(a, rows, nbx, maps); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.gauge_out) return launch_gauges<float>(a.geo, a.h_out, a.gauge_cells, a.n_gauges, a.gauge_out, st);
    return cudaSuccess;
}

cudaError_t launch_step_stream_ensemble(const StepArgs<float> *table, const int *base, int n, int total_blocks,
                                        int warps, int rows, int step, int want_hmax, int mode, cudaStream_t st)
{
    cudaError_t e = configure(warps);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(WarpRing) * warps;
    switch (mode) {
    case 0: step_stream_ensemble_kernel<0><<<total_blocks, warps * 32, smem, st>>>(table, base, n, rows, step, want_hmax); break;
    case 1: step_stream_ensemble_kernel<1><<<total_blocks, warps * 32, smem, st>>>(table, base, n, rows, step, want_hmax); break;
    case 2: step_stream_ensemble_kernel<2><<<total_blocks, warps * 32, smem, st>>>(table, base, n, rows, step, want_hmax); break;
    default: step_stream_ensemble_kernel<3><<<total_blocks, warps * 32, smem, st>>>(table, base, n, rows, step, want_hmax); break;
    }
    return cudaGetLastError();
}

}  // namespace flood
