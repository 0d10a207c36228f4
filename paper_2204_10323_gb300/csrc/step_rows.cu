// step_rows.cu -- FP32 single-step kernel streaming rows through registers.
//
// One warp owns a strip of 128 columns (four per lane, float4 loads) and a
// chunk of R rows.  It walks the chunk from south to north keeping the
// previous row in registers: at row j it computes the new south faces of row
// j (Eq. 3 between rows j-1 and j) and the new west faces of row j, then
// finishes the depth of row j-1 (Eq. 4).  West neighbours come from the lane
// to the left by warp shuffle (lane 0 loads column x0-1), the east face of a
// lane's last column is the next lane's first west face (lane 31 computes the
// face at x0+128 itself).  Every cell value is read from HBM once per step
// apart from those strip and chunk edges, so the kernel moves close to the
// 32 bytes per cell-update of the method (20 read, 12 written).
//
// All face arithmetic uses explicitly rounded intrinsics, so the faces that
// two warps both evaluate (strip and chunk edges) come out bit-identical and
// the update conserves mass.
#include "fast_face.cuh"

namespace flood {

namespace {

constexpr int kWarps = 4;       // warps (strips) per block
constexpr int kRows = 32;       // rows per chunk

struct Row {
    float4 h, z, n, qx, qy;
};

__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

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

__global__ void __launch_bounds__(kWarps * 32) step_rows_kernel(const StepArgs<float> a, const int nbx)
{
    // one-dimensional grid (grids taller than 65535 blocks): block (bx, by) of nbx columns of blocks
    const int bx = (int)(blockIdx.x % (unsigned)nbx), by = (int)(blockIdx.x / (unsigned)nbx);
    __shared__ double red[32];
    const Geom &G = a.geo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = G.nx, ny = G.ny;
    const size_t P = (size_t)G.pitch;
    const int x0 = (bx * kWarps + warp) * 128;
    const int c0 = x0 + 4 * lane;
    const bool full = c0 + 3 < nx;                       // all four columns of the lane inside the grid
    const bool active = x0 < nx;
    const bool lane_in = active && c0 < (int)P;        // float4 lies inside the row pitch
    const int y0 = by * kRows;
    const int y1 = min(y0 + kRows, ny);
    const double dtd = a.ctrl->dt;
    FastConst K;
    const float dt = (float)dtd, dx = (float)G.dx, g = (float)G.g;
    K.gdt = g * dt;
    K.a1 = K.gdt / dx;
    K.gdt4 = 0.25f * K.gdt;
    K.h_dry = (float)G.h_dry;
    K.dtdx = dt / dx;
    const float *__restrict__ H = a.h;
    const float *__restrict__ Z = a.z;
    const float *__restrict__ N = a.n;
    const float *__restrict__ QX = a.qx;
    const float *__restrict__ QY = a.qy;

    double vout = 0.0, vclip = 0.0;
    float hmax = 0.0f;
    bool nan_seen = false;

    // previous row (j - 1): cells and the new faces computed for it
    float4 hp = make_float4(0, 0, 0, 0), zp = hp, np_ = hp;
    float4 qxw_p = hp, qys_p = hp;
    float qxe_p3 = 0.0f;
    if (active && y0 > 0 && lane_in) {
        size_t r = (size_t)(y0 - 1) * P + c0;
        hp = ld4(H + r);
        zp = ld4(Z + r);
        np_ = ld4(N + r);
    }
    Row nxt;
    nxt.h = nxt.z = nxt.n = nxt.qx = nxt.qy = make_float4(0, 0, 0, 0);
    if (active && lane_in && y0 < ny) {
        size_t r = (size_t)y0 * P + c0;
        nxt.h = ld4(H + r);
        nxt.z = ld4(Z + r);
        nxt.n = ld4(N + r);
        nxt.qx = ld4(QX + r);
        nxt.qy = ld4(QY + r);
    }
    if (active) {
        for (int j = y0; j <= y1; j++) {
            Row cur = nxt;
            // prefetch row j + 1 (row y1 itself only needs h, z, n, qy)
            if (j + 1 <= y1 && j + 1 < ny && lane_in) {
                size_t r = (size_t)(j + 1) * P + c0;
                nxt.h = ld4(H + r);
                nxt.z = ld4(Z + r);
                nxt.n = ld4(N + r);
                nxt.qy = ld4(QY + r);
                if (j + 1 < y1) nxt.qx = ld4(QX + r);
            }
            // ---- new south faces of row j (between rows j-1 and j)
            // (interior rows branch-free; the boundary rows, uniform over the warp, take Eq. 5-6)
            float4 qys;
            if (j > 0 && j < ny) {
                #pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float zl = get(zp, k), zr = get(cur.z, k);
                    set(qys, k, face_fast_sel(get(cur.qy, k), get(hp, k) + zl, get(cur.h, k) + zr, fmaxf(zl, zr),
                                              get(np_, k) + get(cur.n, k), K));
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
                        v = j == 0 ? boundary_fast_at(a, a.s, 2, c, get(cur.h, k), get(cur.n, k), vout)
                                   : boundary_fast_at(a, a.s, 3, c, get(hp, k), get(np_, k), vout);
                    set(qys, k, v);
                }
            }
            // ---- finish row j-1: Eq. 4, clip, stores
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
                else
                    #pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (c0 + k <= nx) a.qx_out[r + k] = get(qxw_p, k);
                if (lane == 31 && x0 + 128 == nx) a.qx_out[(size_t)jr * P + nx] = qxe_p3;
                if (jr == ny - 1) {
                    const size_t rn = (size_t)ny * P + c0;
                    if (c0 + 3 < nx) *reinterpret_cast<float4 *>(a.qy_out + rn) = qys;
                    else
                        #pragma unroll
                        for (int k = 0; k < 4; k++)
                            if (c0 + k < nx) a.qy_out[rn + k] = get(qys, k);
                }
            }
            if (j == y1) break;
            // ---- new west faces of row j
            float hW = __shfl_up_sync(0xffffffffu, cur.h.w, 1);
            float zW = __shfl_up_sync(0xffffffffu, cur.z.w, 1);
            float nW = __shfl_up_sync(0xffffffffu, cur.n.w, 1);
            if (lane == 0) {
                if (x0 > 0) {
                    size_t r = (size_t)j * P + (x0 - 1);
                    hW = __ldg(H + r);
                    zW = __ldg(Z + r);
                    nW = __ldg(N + r);
                } else {
                    hW = zW = nW = 0.0f;
                }
            }
            float4 qxw;
            #pragma unroll
            for (int k = 0; k < 4; k++) {
                const float hl = k == 0 ? hW : get(cur.h, k - 1);
                const float zl = k == 0 ? zW : get(cur.z, k - 1);
                const float nl = k == 0 ? nW : get(cur.n, k - 1);
                const float zr = get(cur.z, k);
                set(qxw, k, face_fast_sel(get(cur.qx, k), hl + zl, get(cur.h, k) + zr, fmaxf(zl, zr),
                                          nl + get(cur.n, k), K));
            }
            if (c0 == 0 || !full) {               // lanes holding x = 0 or x >= nx: Eq. 5-6, or no face
                #pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int c = c0 + k;
                    const float hl = k == 0 ? hW : get(cur.h, k - 1);
                    const float nl = k == 0 ? nW : get(cur.n, k - 1);
                    if (c == 0) set(qxw, k, boundary_fast_at(a, a.s, 0, j, get(cur.h, 0), get(cur.n, 0), vout));
                    else if (c == nx) set(qxw, k, boundary_fast_at(a, a.s, 1, j, hl, nl, vout));
                    else if (c > nx) set(qxw, k, 0.0f);
                }
            }
            // east face of the lane's last column = next lane's first west face
            float qe = __shfl_down_sync(0xffffffffu, qxw.x, 1);
            if (lane == 31) {
                const int c = x0 + 128;
                qe = 0.0f;
                if (c == nx) qe = boundary_fast_at(a, a.s, 1, j, cur.h.w, cur.n.w, vout);
                else if (c < nx) {
                    size_t r = (size_t)j * P + c;
                    float hr = __ldg(H + r), zr = __ldg(Z + r), nr = __ldg(N + r);
                    float zl = cur.z.w;
                    qe = face_fast(__ldg(QX + r), cur.h.w + zl, hr + zr, fmaxf(zl, zr), cur.n.w + nr, K);
                }
            }
            // shift
            hp = cur.h;
            zp = cur.z;
            np_ = cur.n;
            qxw_p = qxw;
            qxe_p3 = qe;
            qys_p = qys;
        }
    }
    // ledger and h_max (all threads take part in the block reductions)
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
        for (int k = 0; k < a.n_inflow_sec; k++) {
            double Q = a.inflow_Q[(size_t)a.s * a.n_inflow_sec + k];
            if (Q > 0.0) vin += dtd * Q;
        }
        a.ctrl->V_in = vin;
        a.ctrl->t = a.t_list[a.s + 1];
    }
}

}  // namespace

cudaError_t launch_step_rows(const StepArgs<float> &a, cudaStream_t st)
{
    const int strips = (a.geo.nx + 127) / 128;
    const int nbx = (strips + kWarps - 1) / kWarps, nby = (a.geo.ny + kRows - 1) / kRows;
    step_rows_kernel<<<(unsigned)((int64_t)nbx * nby), kWarps * 32, 0, st>>>(a, nbx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.gauge_out) return launch_gauges<float>(a.geo, a.h_out, a.gauge_cells, a.n_gauges, a.gauge_out, st);
    return cudaSuccess;
}

}  // namespace flood
