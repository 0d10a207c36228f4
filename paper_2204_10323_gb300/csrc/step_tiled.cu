// step_tiled.cu -- FP32 temporal blocking: K <= 4 time steps per launch.
//
// Persistent, time-skewed row streaming.  Each warp owns one output strip of
// 120 columns and one chunk of rows; it stages 128 columns (4 halo columns on
// each side, held by lanes 0 and 31) row by row through shared memory with
// bulk copies (cp.async.bulk + mbarrier), and advances the rows through K
// time levels in a pipeline: when input row j arrives, level 1 finishes row
// j-1, level 2 finishes row j-2 from level 1's output of the same iteration,
// ..., and level K finishes row j-K, which is stored.  The dependency cone of
// K steps is K columns wide on each side, so the strip's 120 inner columns
// are exact after K levels; in y the skew only needs K extra rows at the two
// ends of a chunk, and chunks are as tall as the SM count allows.  HBM
// traffic per cell and step is about (20 B read + 12 B written) / K.
//
// Per cell and level the arithmetic is the single-step kernels' (the same
// explicitly rounded face function and depth update), so K levels give the
// same bits as K single steps.  Boundary faces (Eq. 5-6) are applied at every
// level with that level's inflow row; ledger volumes are booked only by the
// warp that owns the cell or boundary face.  Waits are bounded like the
// stream kernel's.
#include "fast_face.cuh"
#include "tma_util.cuh"

namespace flood {

namespace {

constexpr int kWarps = 4;                   // warps per block
constexpr int kHalo = 4;                    // halo columns per side (= largest K)
constexpr int kOut = 128 - 2 * kHalo;       // output columns per strip
constexpr int kPF = 3;                      // rows in flight
constexpr int kDZ = kPF + kHalo + 1;        // z,n ring depth: rows still read by lagging levels
constexpr uint64_t kBudgetNs = 2000000000ull;

// 16-byte aligned size: every warp's ring (bulk-copy destinations, float4
// loads) must start on a 16-byte boundary.
struct alignas(16) WarpRing {
    float hq[kPF][3][128];                  // h, qx, qy of staged rows
    float zn[kDZ][2][128];                  // z, n of the last kDZ rows
    uint64_t bar[kPF];
};

static_assert(sizeof(WarpRing) % 16 == 0, "per-warp ring must keep 16-byte alignment");
constexpr size_t kSmemBytes = sizeof(WarpRing) * kWarps;

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

// One level's pending row r-1: its input depth and the new faces computed for it.
struct Level {
    float4 hp, qxw, qys;
    float qxe;
};

template <int K>
__global__ void __launch_bounds__(kWarps * 32, 4) step_tiled_kernel(const StepArgs<float> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    const Geom &G = a.geo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = G.nx, ny = G.ny, P = G.pitch;
    const int n_strips = a.tile_x, chunk_rows = a.tile_y;
    const int gw = blockIdx.x * kWarps + warp;
    const int strip = gw % n_strips, chunk = gw / n_strips;
    const int y0 = chunk * chunk_rows;
    const bool active = y0 < ny;
    const int y1 = min(y0 + chunk_rows, ny);
    const int x0 = strip * kOut - kHalo;              // first staged column
    const int c0 = x0 + 4 * lane;
    const int own_lo = strip * kOut, own_hi = min(strip * kOut + kOut, nx);
    const int jb = max(y0 - K, 0);
    const int jend = y1 + K - 1;                      // last iteration (level K reaches row y1)
    const int jload_hi = min(y1 + K - 1, ny - 1);     // last staged row
    const int nload = jload_hi - jb + 1;
    WarpRing &ring = reinterpret_cast<WarpRing *>(smem_raw)[warp];

    const double dtd = a.ctrl->dt;
    FastConst Kc;
    const float dt = (float)dtd, dx = (float)G.dx, g = (float)G.g;
    Kc.gdt = g * dt;
    Kc.a1 = Kc.gdt / dx;
    Kc.h_dry = (float)G.h_dry;
    Kc.dtdx = dt / dx;

    double vout = 0.0, vclip = 0.0;
    float hmax = 0.0f;
    bool nan_seen = false;

    const int cs = max(x0, 0);
    const int ce = min(x0 + 128, P);
    const int so = cs - x0;
    const uint32_t seg_bytes = (uint32_t)(ce - cs) * 4u;

    if (active && lane == 0) {
        for (int s = 0; s < kPF; s++) mbar_init(&ring.bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int idx) {
        const int j = jb + idx;
        const size_t row = (size_t)j * P + cs;
        uint64_t *bar = &ring.bar[idx % kPF];
        mbar_arrive_expect_tx(bar, seg_bytes * 5u);
        float *hq = &ring.hq[idx % kPF][0][0];
        float *zn = &ring.zn[j % kDZ][0][0];
        bulk_copy_g2s(hq + 0 * 128 + so, a.h + row, seg_bytes, bar);
        bulk_copy_g2s(hq + 1 * 128 + so, a.qx + row, seg_bytes, bar);
        bulk_copy_g2s(hq + 2 * 128 + so, a.qy + row, seg_bytes, bar);
        bulk_copy_g2s(zn + 0 * 128 + so, a.z + row, seg_bytes, bar);
        bulk_copy_g2s(zn + 1 * 128 + so, a.n + row, seg_bytes, bar);
    };
    int issued = 0, consumed = 0;
    bool abort = false;
    if (active && lane == 0)
        for (; issued < min(kPF, nload); issued++) issue(issued);

    Level L[K];
#pragma unroll
    for (int s = 0; s < K; s++) {
        L[s].hp = L[s].qxw = L[s].qys = make_float4(0, 0, 0, 0);
        L[s].qxe = 0.0f;
    }
    bool own_cell[4], own_wface[4], all_cell = true, all_wface = true;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        int c = c0 + k;
        own_cell[k] = c >= own_lo && c < own_hi;
        own_wface[k] = c >= own_lo && (c < own_hi || (c == nx && own_hi == nx));
        all_cell &= own_cell[k];
        all_wface &= own_wface[k];
    }

    if (active) {
        for (int j = jb; j <= jend; j++) {
            // ---- input row j (level 0) from the ring
            float4 ho_h = make_float4(0, 0, 0, 0), ho_qx = ho_h, ho_qy = ho_h;   // hand-off to the next level
            bool ho_valid = false;
            if (j <= jload_hi) {
                const int idx = j - jb;
                bool ok = mbar_wait_bounded(&ring.bar[idx % kPF], (uint32_t)((idx / kPF) & 1), kBudgetNs);
                if (__any_sync(0xffffffffu, !ok)) {
                    abort = true;
                    break;
                }
                consumed = idx + 1;
                const float *hq = &ring.hq[idx % kPF][0][0];
                ho_h = lds4(hq + 0 * 128 + 4 * lane);
                ho_qx = lds4(hq + 1 * 128 + 4 * lane);
                ho_qy = lds4(hq + 2 * 128 + 4 * lane);
                ho_valid = true;
                __syncwarp();
                if (lane == 0 && issued < nload) {
                    fence_proxy_async();
                    issue(issued);
                    issued++;
                }
            }
#pragma unroll
            for (int s = 1; s <= K; s++) {
                const int r = j - (s - 1);                 // this level's current row
                const int rstart = jb == 0 ? 0 : jb + (s - 1);
                Level &S = L[s - 1];
                const float4 ch = ho_h, cqx = ho_qx, cqy = ho_qy;
                const bool cur_valid = ho_valid;
                ho_valid = false;
                if (r < rstart || r > ny) continue;
                if (r < ny && !cur_valid) continue;        // no input for this row (cannot happen)
                if (r == rstart && jb > 0) {               // halo row: only becomes the previous row
                    S.hp = ch;
                    continue;
                }
                const int step = a.s + (s - 1);
                float4 cz = make_float4(0, 0, 0, 0), cn = cz, pz = cz, pn = cz;
                if (r < ny) {
                    cz = lds4(&ring.zn[r % kDZ][0][4 * lane]);
                    cn = lds4(&ring.zn[r % kDZ][1][4 * lane]);
                }
                if (r > 0) {
                    pz = lds4(&ring.zn[(r - 1) % kDZ][0][4 * lane]);
                    pn = lds4(&ring.zn[(r - 1) % kDZ][1][4 * lane]);
                }
                // ---- new south faces of row r
                float4 qys;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int c = c0 + k;
                    float v = 0.0f;
                    if (c >= 0 && c < nx) {
                        double vo = 0.0;
                        if (r == 0) v = boundary_fast_at(a, step, 2, c, get(ch, k), get(cn, k), vo);
                        else if (r == ny) v = boundary_fast_at(a, step, 3, c, get(S.hp, k), get(pn, k), vo);
                        else {
                            float zl = get(pz, k), zr = get(cz, k);
                            v = face_fast(get(cqy, k), get(S.hp, k) + zl, get(ch, k) + zr, fmaxf(zl, zr),
                                          get(pn, k) + get(cn, k), Kc);
                        }
                        if (own_cell[k] && ((r == 0 && y0 == 0) || (r == ny && y1 == ny))) vout += vo;
                    }
                    set(qys, k, v);
                }
                // ---- finish row r-1 (Eq. 4, clip); hand it to the next level
                const bool has_prev = jb == 0 ? r > 0 : r > rstart + 1;
                if (has_prev) {
                    const int rr = r - 1;
                    const bool own_row = rr >= y0 && rr < y1;
                    float4 fin;
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        float qe = k < 3 ? get(S.qxw, k + 1) : S.qxe;
                        float dv = __fadd_rn(__fsub_rn(get(S.qxw, k), qe), __fsub_rn(get(S.qys, k), get(qys, k)));
                        float v = __fmaf_rn(Kc.dtdx, dv, get(S.hp, k));
                        if (v < 0.0f) {
                            if (own_row && own_cell[k]) vclip += -(double)v * G.dx * G.dx;
                            v = 0.0f;
                        }
                        if (s == K && own_row && own_cell[k]) {
                            hmax = fmaxf(hmax, v);
                            nan_seen |= (v != v);
                        }
                        set(fin, k, v);
                    }
                    if (s == K && own_row) {
                        const size_t ro = (size_t)rr * P + c0;
                        if (all_cell) {
                            *reinterpret_cast<float4 *>(a.h_out + ro) = fin;
                            *reinterpret_cast<float4 *>(a.qy_out + ro) = S.qys;
                            if (rr == ny - 1) *reinterpret_cast<float4 *>(a.qy_out + ro + P) = qys;
                        } else {
#pragma unroll
                            for (int k = 0; k < 4; k++)
                                if (own_cell[k]) {
                                    a.h_out[ro + k] = get(fin, k);
                                    a.qy_out[ro + k] = get(S.qys, k);
                                    if (rr == ny - 1) a.qy_out[ro + P + k] = get(qys, k);
                                }
                        }
                        if (all_wface) *reinterpret_cast<float4 *>(a.qx_out + ro) = S.qxw;
                        else {
#pragma unroll
                            for (int k = 0; k < 4; k++)
                                if (own_wface[k]) a.qx_out[ro + k] = get(S.qxw, k);
                        }
                    }
                    ho_h = fin;
                    ho_qx = S.qxw;
                    ho_qy = S.qys;
                    ho_valid = true;
                }
                // ---- new west faces of row r, then row r becomes this level's previous row
                if (r < ny) {
                    const bool own_row_r = r >= y0 && r < y1;
                    float hl0 = __shfl_up_sync(0xffffffffu, ch.w, 1);
                    float zl0 = __shfl_up_sync(0xffffffffu, cz.w, 1);
                    float nl0 = __shfl_up_sync(0xffffffffu, cn.w, 1);
                    float4 qxw;
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const int c = c0 + k;
                        float hl = k == 0 ? hl0 : get(ch, k - 1);
                        float zl = k == 0 ? zl0 : get(cz, k - 1);
                        float nl = k == 0 ? nl0 : get(cn, k - 1);
                        float v = 0.0f;
                        double vo = 0.0;
                        if (c == 0) v = boundary_fast_at(a, step, 0, r, get(ch, 0), get(cn, 0), vo);
                        else if (c == nx) v = boundary_fast_at(a, step, 1, r, hl, nl, vo);
                        else if (c > 0 && c < nx) {
                            float zr = get(cz, k);
                            v = face_fast(get(cqx, k), hl + zl, get(ch, k) + zr, fmaxf(zl, zr), nl + get(cn, k), Kc);
                        }
                        if (own_row_r && own_wface[k]) vout += vo;
                        set(qxw, k, v);
                    }
                    S.qxe = __shfl_down_sync(0xffffffffu, qxw.x, 1);
                    S.hp = ch;
                    S.qxw = qxw;
                    S.qys = qys;
                }
            }
        }
        if (abort) {
            if (lane == 0) {
                for (int k = consumed; k < issued; k++)
                    mbar_wait_bounded(&ring.bar[k % kPF], (uint32_t)((k / kPF) & 1), kBudgetNs);
                atomicOr(&a.ctrl->status, kStatusTimeout);
            }
            __syncwarp();
        }
    }
    double bo = block_reduce<false>(vout, red);
    if (threadIdx.x == 0 && bo != 0.0) atomicAdd(&a.ctrl->V_out, dtd * bo);
    double bc = block_reduce<false>(vclip, red);
    if (threadIdx.x == 0 && bc != 0.0) atomicAdd(&a.ctrl->V_clip, bc);
    if (a.want_hmax) {
        double bm = block_reduce<true>(nan_seen ? (double)NAN : (double)hmax, red);
        if (threadIdx.x == 0) atomic_max_nonneg(&a.ctrl->hmax_bits, bm);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double vin = a.ctrl->V_in;
        for (int s = 0; s < K; s++)
            for (int k = 0; k < a.n_inflow_sec; k++) {
                double Q = a.inflow_Q[(size_t)(a.s + s) * a.n_inflow_sec + k];
                if (Q > 0.0) vin += dtd * Q;
            }
        a.ctrl->V_in = vin;
        a.ctrl->t = a.t_list[a.s + K];
    }
}

template <int K>
cudaError_t launch_k(const StepArgs<float> &a0, cudaStream_t st)
{
    static int blocks_per_sm = 0, num_sms = 0;
    if (!blocks_per_sm) {
        cudaError_t e = cudaFuncSetAttribute(step_tiled_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, step_tiled_kernel<K>, kWarps * 32,
                                                          kSmemBytes);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    StepArgs<float> a = a0;
    const int nx = a.geo.nx, ny = a.geo.ny;
    const int n_strips = (nx + kOut - 1) / kOut;
    const int resident_warps = num_sms * blocks_per_sm * kWarps;
    // one chunk per resident warp, but no chunk shorter than 32 rows (the K-row skew overhead)
    int chunks = resident_warps / n_strips;
    chunks = chunks < 1 ? 1 : chunks;
    int max_chunks = (ny + 31) / 32;
    if (chunks > max_chunks) chunks = max_chunks;
    const int chunk_rows = (ny + chunks - 1) / chunks;
    chunks = (ny + chunk_rows - 1) / chunk_rows;
    a.tile_x = n_strips;
    a.tile_y = chunk_rows;
    const int warps = n_strips * chunks;
    const int blocks = (warps + kWarps - 1) / kWarps;
    step_tiled_kernel<K><<<blocks, kWarps * 32, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t tiled_smem_bytes(int, int, int) { return kSmemBytes; }

cudaError_t launch_step_tiled(const StepArgs<float> &a, cudaStream_t st)
{
    switch (a.k_steps) {
    case 1: return launch_k<1>(a, st);
    case 2: return launch_k<2>(a, st);
    case 3: return launch_k<3>(a, st);
    case 4: return launch_k<4>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace flood
