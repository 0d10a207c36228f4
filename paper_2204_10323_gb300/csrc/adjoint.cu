// adjoint.cu -- reverse of one time step (not in the paper; its calibration
// use is named as future work).  Given the forward state x_k and the adjoint
// lambda_{k+1} of the state after the step, produce lambda_k and accumulate
// dL/dn.  The forward step is h' = max(h + dt/dx div q'(x_k, n), 0) with q'
// from Eq. 3 on interior faces and Eq. 5-6 on boundary faces, so
//
//   lambda_hu(c) = lambda_h'(c) * [h'_unclipped(c) >= 0]
//   mu_f         = lambda_q'(f) + dt/dx (lambda_hu(R) - lambda_hu(L))     (face f between L and R)
//   lambda_h(c)  = lambda_hu(c) + sum_f mu_f dq'_f/dh_c
//   lambda_q(f)  = mu_f dq'_f/dq_f                                          (interior faces)
//   dL/dn(c)    += sum_f mu_f dq'_f/dn_c
//
// Branch conventions: max(eta_L, eta_R) sends its derivative to L on ties;
// d|q|/dq = 0 at q = 0; the dry-face test, the outflow dry test and the clip
// are held as masks; the Eq. 6 level is differentiated exactly through the
// implicit function theorem.  Each cell gathers the contributions of its
// four faces (both cells of a face evaluate its derivatives), so no atomics
// are needed and the result is deterministic.
//
// The clip mask is recomputed with the forward kernels' own arithmetic (IEEE
// order for FP64, the fast FP32 face for FP32), so the clip and wet/dry
// decisions are exactly the forward's.
#include <algorithm>
#include <cstddef>
#include <type_traits>

#include <cuda.h>

#include "fast_face.cuh"
#include "tma_util.cuh"

namespace flood {

namespace {

constexpr int BX = 32, BY = 8;

// ---------------------------------------------------------------- forward faces per precision
template <typename T> struct Fwd;

template <> struct Fwd<double> {
    double g, dt, dx, hd;
    __device__ Fwd(const Geom &G, double dt_) : g(G.g), dt(dt_), dx(G.dx), hd(G.h_dry) {}
    __device__ double face(double q, double hL, double zL, double nL, double hR, double zR, double nR) const
    {
        return face_update_ieee<double>(q, fabs(q), hL, zL, nL, hR, zR, nR, g, dt, dx, hd);
    }
    __device__ double hf(double hL, double zL, double hR, double zR) const
    {
        using O = R<double>;
        return O::sub(O::max(O::add(hL, zL), O::add(hR, zR)), O::max(zL, zR));
    }
    __device__ double outflow(double h, double sqrtS, double n, int form) const
    {
        return outflow_flux_ieee<double>(h, sqrtS, n, dx, hd, form);
    }
    __device__ double update(double h, double qW, double qE, double qS, double qN) const
    {
        using O = R<double>;
        double dv = O::add(O::sub(qW, qE), O::sub(qS, qN));
        return O::add(h, O::div(O::mul(dt, dv), dx));
    }
    __device__ static double rcp_(double x) { return 1.0 / x; }
    __device__ static double pow_m73_(double x) { const double m = ::rcbrt(x), r = 1.0 / x; return m * r * r; }
};

template <> struct Fwd<float> {
    FastConst K;
    float dx, hd;
    __device__ Fwd(const Geom &G, double dt_)
    {
        const float dt = (float)dt_;
        dx = (float)G.dx;
        K.gdt = (float)G.g * dt;
        K.a1 = K.gdt / dx;
        K.gdt4 = 0.25f * K.gdt;
        K.h_dry = (float)G.h_dry;
        K.dtdx = dt / dx;
        hd = K.h_dry;
    }
    __device__ float face(float q, float hL, float zL, float nL, float hR, float zR, float nR) const
    {
        return face_fast(q, hL + zL, hR + zR, fmaxf(zL, zR), nL + nR, K);
    }
    __device__ float hf(float hL, float zL, float hR, float zR) const
    {
        return __fsub_rn(fmaxf(hL + zL, hR + zR), fmaxf(zL, zR));
    }
    __device__ float outflow(float h, float sqrtS, float n, int form) const
    {
        return outflow_fast(h, sqrtS, n, dx, hd, form);
    }
    __device__ float update(float h, float qW, float qE, float qS, float qN) const
    {
        float dv = __fadd_rn(__fsub_rn(qW, qE), __fsub_rn(qS, qN));
        return __fmaf_rn(K.dtdx, dv, h);
    }
    __device__ static float rcp_(float x) { return rcp_fast(x); }
    __device__ static float pow_m73_(float x) { return pow_m73(x); }
};

// Partial derivatives of one wet face's Eq. 3 value.
template <typename T> struct FaceLin {
    T dq, dhL, dhR, dn;     // dn = dq'/dn_L = dq'/dn_R
};

template <typename T>
__device__ __forceinline__ FaceLin<T> face_lin(T q, T hL, T zL, T nL, T hR, T zR, T nR, T hf, T g, T dt, T dx)
{
    FaceLin<T> r;
    const T etaL = hL + zL, etaR = hR + zR;
    const T nf = T(0.5) * (nL + nR);
    const T gdt = g * dt, a1 = gdt / dx;
    const T inv_hf = Fwd<T>::rcp_(hf);
    const T hf_m73 = Fwd<T>::pow_m73_(hf);
    const T c0 = gdt * nf * nf * hf_m73;     // friction per |q|
    const T fric = c0 * (q < T(0) ? -q : q);
    const T inv_den = Fwd<T>::rcp_(T(1) + fric);
    const T slope = etaR - etaL;
    const T F = (q - a1 * hf * slope) * inv_den;
    const T sg = q > T(0) ? T(1) : (q < T(0) ? T(-1) : T(0));
    r.dq = (T(1) - F * c0 * sg) * inv_den;
    const T dF_dhf = (-a1 * slope + F * (T(7) / T(3)) * fric * inv_hf) * inv_den;
    const T d_expl = a1 * hf * inv_den;
    const bool left = etaL >= etaR;
    r.dhL = d_expl + (left ? dF_dhf : T(0));
    r.dhR = -d_expl + (left ? T(0) : dF_dhf);
    r.dn = -F * fric * inv_den * Fwd<T>::rcp_(nf);
    return r;
}

template <typename T>
__device__ __forceinline__ int bc_off(const Geom &G, int side)
{
    return side == 0 ? 0 : side == 1 ? G.ny : side == 2 ? 2 * G.ny : 2 * G.ny + G.nx;
}

// Forward boundary face value (same rules as the forward kernels).
template <typename T>
__device__ __forceinline__ T bface(const StepArgs<T> &a, const Fwd<T> &F, int side, int k, T h, T n)
{
    const Geom &G = a.geo;
    const int off = bc_off<T>(G, side);
    const int type = a.bc.type[off + k];
    if (type == kBcWall) return T(0);
    const T inward = T(inward_sign(side));
    if (type == kBcInflow) return inward * a.inflow_q[(size_t)a.s * a.n_slots + a.bc.slot[off + k]];
    return -inward * F.outflow(h, T(a.bc.sqrtS[off + k]), n, G.bc_form);
}

// Adjoint of an outflow boundary face: contributions to lambda_h(c) and dL/dn(c).
template <typename T>
__device__ __forceinline__ void outflow_adj(const StepArgs<T> &a, const Fwd<T> &F, int side, int k, T h, T n,
                                            T mu, T &lh, T &gn)
{
    const Geom &G = a.geo;
    const int off = bc_off<T>(G, side);
    if (a.bc.type[off + k] != kBcOutflow) return;
    const T q = F.outflow(h, T(a.bc.sqrtS[off + k]), n, G.bc_form);
    if (!(q > T(0))) return;                    // dry boundary cell: held at zero
    const T nu = -T(inward_sign(side)) * mu;   // adjoint of the outflow magnitude
    const T pe = G.bc_form == 0 ? T(5.0 / 3.0) : T(2.0 / 3.0);
    lh += nu * pe * q / h;
    gn += -nu * q / n;
}

// One launch per reverse step, face-centric within a BX x 8 tile (256
// threads: 32 registers and 19 KB of shared memory in FP32 let eight blocks
// share an SM, so one block's barriers and loads overlap the others' work;
// 32 x 16 and 32 x 4 tiles measured 12 % and 15 % slower at 1024^2):
//  0. the tile's cells with a two-cell halo (h, z, n) and the faces around it
//     (old q) are staged in shared memory;
//  A. every face around the tile and its one-cell halo gets its new value q'
//     (the forward arithmetic);
//  B. the tile and halo cells get the adjoint of their unclipped depth
//     (lambda_h' plus the gauge seeds, zero where the depth was clipped);
//  C. every face touching a tile cell gets mu and its derivatives once,
//     leaving its contributions to the two cells and the adjoint of its old q;
//  D. every tile cell gathers the contributions of its four faces.
template <typename T> struct TileRows { static constexpr int v = 8; };
constexpr int kTileGauges = 32;

template <typename T>
__global__ void __launch_bounds__(BX * TileRows<T>::v) adj_step_kernel(const AdjArgs<T> A, const int nbx)
{
    constexpr int BYT = TileRows<T>::v;
    constexpr int NT = BX * BYT;
    __shared__ T sh[BYT + 4][BX + 4], sz[BYT + 4][BX + 4], sn[BYT + 4][BX + 4];   // cells I0-2.., J0-2..
    __shared__ T sqx[BYT + 2][BX + 3], sX[BYT + 2][BX + 3];   // x-faces: columns I0-1 .., rows J0-1 ..
    __shared__ T sqy[BYT + 3][BX + 2], sY[BYT + 3][BX + 2];   // y-faces: rows J0-1 .., columns I0-1 ..
    __shared__ T sL[BYT + 2][BX + 2];                          // cells I0-1 .., J0-1 ..
    __shared__ T cXl[BYT][BX + 1], cXr[BYT][BX + 1], cXn[BYT][BX + 1];
    __shared__ T cYl[BYT + 1][BX], cYr[BYT + 1][BX], cYn[BYT + 1][BX];
    __shared__ int s_ng, s_gk[kTileGauges];                     // gauges inside the tile and its halo
    const StepArgs<T> &a = A.fwd;
    const Geom &G = a.geo;
    const int nx = G.nx, ny = G.ny;
    const size_t P = (size_t)G.pitch;
    const double dtd = a.ctrl->dt;
    const Fwd<T> F(G, dtd);
    const T dt = T(dtd), dx = T(G.dx), g = T(G.g), hd = T(G.h_dry), dtdx = dt / dx;
    const int tid = threadIdx.y * BX + threadIdx.x;
    // one-dimensional grid (grids taller than 65535 tiles): tile (bx, by) of nbx columns of tiles
    const int I0 = (int)(blockIdx.x % (unsigned)nbx) * BX, J0 = (int)(blockIdx.x / (unsigned)nbx) * BYT;

    // 0. stage cells and old face fluxes (zeros outside the domain)
    for (int t = tid; t < (BYT + 4) * (BX + 4); t += NT) {
        const int lj = t / (BX + 4), li = t % (BX + 4);
        const int j = J0 - 2 + lj, i = I0 - 2 + li;
        T hv = T(0), zv = T(0), nv = T(0);
        if (i >= 0 && i < nx && j >= 0 && j < ny) {
            const size_t c = (size_t)j * P + i;
            hv = a.h[c];
            zv = a.z[c];
            nv = a.n[c];
        }
        sh[lj][li] = hv;
        sz[lj][li] = zv;
        sn[lj][li] = nv;
    }
    for (int t = tid; t < (BYT + 2) * (BX + 3); t += NT) {
        const int lj = t / (BX + 3), li = t % (BX + 3);
        const int j = J0 - 1 + lj, fi = I0 - 1 + li;
        sqx[lj][li] = (j >= 0 && j < ny && fi >= 0 && fi <= nx) ? a.qx[(size_t)j * P + fi] : T(0);
    }
    for (int t = tid; t < (BYT + 3) * (BX + 2); t += NT) {
        const int lj = t / (BX + 2), li = t % (BX + 2);
        const int fj = J0 - 1 + lj, i = I0 - 1 + li;
        sqy[lj][li] = (i >= 0 && i < nx && fj >= 0 && fj <= ny) ? a.qy[(size_t)fj * P + i] : T(0);
    }
    __syncthreads();
    // A. new face values.  x-face (lj, li) lies between cells (lj+1, li) and (lj+1, li+1) of the staging.
    for (int t = tid; t < (BYT + 2) * (BX + 3); t += NT) {
        const int lj = t / (BX + 3), li = t % (BX + 3);
        const int j = J0 - 1 + lj, fi = I0 - 1 + li;
        T v = T(0);
        if (j >= 0 && j < ny && fi >= 0 && fi <= nx) {
            const int sj = lj + 1, sl = li, sr = li + 1;
            if (fi == 0) v = bface(a, F, 0, j, sh[sj][sr], sn[sj][sr]);
            else if (fi == nx) v = bface(a, F, 1, j, sh[sj][sl], sn[sj][sl]);
            else v = F.face(sqx[lj][li], sh[sj][sl], sz[sj][sl], sn[sj][sl], sh[sj][sr], sz[sj][sr], sn[sj][sr]);
        }
        sX[lj][li] = v;
    }
    // y-face (lj, li) lies between cells (lj, li+1) and (lj+1, li+1) of the staging.
    for (int t = tid; t < (BYT + 3) * (BX + 2); t += NT) {
        const int lj = t / (BX + 2), li = t % (BX + 2);
        const int fj = J0 - 1 + lj, i = I0 - 1 + li;
        T v = T(0);
        if (i >= 0 && i < nx && fj >= 0 && fj <= ny) {
            const int sc = li + 1, sb = lj, st = lj + 1;
            if (fj == 0) v = bface(a, F, 2, i, sh[st][sc], sn[st][sc]);
            else if (fj == ny) v = bface(a, F, 3, i, sh[sb][sc], sn[sb][sc]);
            else v = F.face(sqy[lj][li], sh[sb][sc], sz[sb][sc], sn[sb][sc], sh[st][sc], sz[st][sc], sn[st][sc]);
        }
        sY[lj][li] = v;
    }
    __syncthreads();
    // B. adjoint of the unclipped depth (gauge seeds included).  The gauges inside
    // the tile and its halo are listed first (flags in gauge order), so that a
    // cell scans only those; a tile holding more than kTileGauges scans them all.
    if (tid == 0) s_ng = 0;
    __syncthreads();
    for (int gk = tid; gk < A.n_gauges; gk += NT) {
        const int64_t flat = A.gauge_cells[gk];
        const int gj = (int)(flat / nx), gi = (int)(flat - (int64_t)gj * nx);
        if (gj >= J0 - 1 && gj <= J0 + BYT && gi >= I0 - 1 && gi <= I0 + BX) {
            const int slot = atomicAdd(&s_ng, 1);
            if (slot < kTileGauges) s_gk[slot] = gk;
        }
    }
    __syncthreads();
    if (tid == 0 && s_ng > 1 && s_ng <= kTileGauges) {   // restore gauge order: repeated gauges add up in order
        for (int x = 1; x < s_ng; x++)
            for (int y = x; y > 0 && s_gk[y - 1] > s_gk[y]; y--) {
                const int tmp = s_gk[y];
                s_gk[y] = s_gk[y - 1];
                s_gk[y - 1] = tmp;
            }
    }
    __syncthreads();
    const int ng_tile = s_ng;
    for (int t = tid; t < (BYT + 2) * (BX + 2); t += NT) {
        const int lj = t / (BX + 2), li = t % (BX + 2);
        const int j = J0 - 1 + lj, i = I0 - 1 + li;
        T v = T(0);
        if (i >= 0 && i < nx && j >= 0 && j < ny) {
            const T hu = F.update(sh[lj + 1][li + 1], sX[lj][li], sX[lj][li + 1], sY[lj][li], sY[lj + 1][li]);
            if (!(hu < T(0))) {
                v = A.lh[(size_t)j * P + i];
                if (ng_tile > 0) {
                    const int64_t flat = (int64_t)j * nx + i;
                    if (ng_tile <= kTileGauges) {
                        for (int x = 0; x < ng_tile; x++)
                            if (A.gauge_cells[s_gk[x]] == flat) v = v + T(A.seed[s_gk[x]]);
                    } else {
                        for (int gk = 0; gk < A.n_gauges; gk++)
                            if (A.gauge_cells[gk] == flat) v = v + T(A.seed[gk]);
                    }
                }
            }
        }
        sL[lj][li] = v;
    }
    __syncthreads();
    // C. each face touching the tile once.  x-face column li = fi - I0, row lj = j - J0.
    for (int t = tid; t < BYT * (BX + 1); t += NT) {
        const int lj = t / (BX + 1), li = t % (BX + 1);
        const int j = J0 + lj, fi = I0 + li;
        T cl = T(0), cr = T(0), cn = T(0);
        if (j < ny && fi <= nx) {
            const size_t r = (size_t)j * P;
            const T lR = sL[lj + 1][li + 1], lL = sL[lj + 1][li];
            const int sj = lj + 2, sl = li + 1, sr = li + 2;     // staging coordinates of L and R
            if (fi == 0) {
                const T mu = A.lqx[r] + dtdx * lR;
                outflow_adj(a, F, 0, j, sh[sj][sr], sn[sj][sr], mu, cr, cn);
                A.lqx_out[r] = T(0);
            } else if (fi == nx) {
                const T mu = A.lqx[r + nx] - dtdx * lL;
                outflow_adj(a, F, 1, j, sh[sj][sl], sn[sj][sl], mu, cl, cn);
                A.lqx_out[r + nx] = T(0);
            } else {
                const T mu = A.lqx[r + fi] + dtdx * (lR - lL);
                const T hL = sh[sj][sl], zL = sz[sj][sl], nL = sn[sj][sl];
                const T hR = sh[sj][sr], zR = sz[sj][sr], nR = sn[sj][sr];
                const T hf = F.hf(hL, zL, hR, zR);
                T lq = T(0);
                if (hf > hd && mu != T(0)) {
                    FaceLin<T> d = face_lin<T>(sqx[lj + 1][li + 1], hL, zL, nL, hR, zR, nR, hf, g, dt, dx);
                    cl = mu * d.dhL;
                    cr = mu * d.dhR;
                    cn = mu * d.dn;
                    lq = mu * d.dq;
                }
                if (li < BX) A.lqx_out[r + fi] = lq;        // the tile owns the west faces of its cells
            }
        }
        cXl[lj][li] = cl;
        cXr[lj][li] = cr;
        cXn[lj][li] = cn;
    }
    // y-face row lj = fj - J0, column li = i - I0.
    for (int t = tid; t < (BYT + 1) * BX; t += NT) {
        const int lj = t / BX, li = t % BX;
        const int fj = J0 + lj, i = I0 + li;
        T cl = T(0), cr = T(0), cn = T(0);
        if (i < nx && fj <= ny) {
            const T lR = sL[lj + 1][li + 1], lL = sL[lj][li + 1];
            const int sc = li + 2, sb = lj + 1, st = lj + 2;     // staging coordinates of L (below) and R
            if (fj == 0) {
                const T mu = A.lqy[i] + dtdx * lR;
                outflow_adj(a, F, 2, i, sh[st][sc], sn[st][sc], mu, cr, cn);
                A.lqy_out[i] = T(0);
            } else if (fj == ny) {
                const size_t c = (size_t)(ny - 1) * P + i;
                const T mu = A.lqy[c + P] - dtdx * lL;
                outflow_adj(a, F, 3, i, sh[sb][sc], sn[sb][sc], mu, cl, cn);
                A.lqy_out[c + P] = T(0);
            } else {
                const size_t c = (size_t)fj * P + i;
                const T mu = A.lqy[c] + dtdx * (lR - lL);
                const T hL = sh[sb][sc], zL = sz[sb][sc], nL = sn[sb][sc];
                const T hR = sh[st][sc], zR = sz[st][sc], nR = sn[st][sc];
                const T hf = F.hf(hL, zL, hR, zR);
                T lq = T(0);
                if (hf > hd && mu != T(0)) {
                    FaceLin<T> d = face_lin<T>(sqy[lj + 1][li + 1], hL, zL, nL, hR, zR, nR, hf, g, dt, dx);
                    cl = mu * d.dhL;
                    cr = mu * d.dhR;
                    cn = mu * d.dn;
                    lq = mu * d.dq;
                }
                if (lj < BYT) A.lqy_out[c] = lq;            // the tile owns the south faces of its cells
            }
        }
        cYl[lj][li] = cl;
        cYr[lj][li] = cr;
        cYn[lj][li] = cn;
    }
    __syncthreads();
    // D. gather per tile cell
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = I0 + tx, j = J0 + ty;
    if (i >= nx || j >= ny) return;
    const size_t c = (size_t)j * P + i;
    const T lu = sL[ty + 1][tx + 1];
    const T lh = lu + cXr[ty][tx] + cXl[ty][tx + 1] + cYr[ty][tx] + cYl[ty + 1][tx];
    // this step's dL/dn of the cell in the working precision, then one add into the
    // double accumulator over the sweep
    const T gs = (cXn[ty][tx] + cXn[ty][tx + 1]) + (cYn[ty][tx] + cYn[ty + 1][tx]);
    A.lh_out[c] = lh;
    A.gn[c] += (double)gs;
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) A.lhu[c] = lu;   // read by the inflow pass
}

// Pass 3: the inflow faces of each section depend on every section cell's n
// through the Eq. 6 level W: with w_c the cell discharge (sum_c w_c = Q),
// pe its depth exponent and hh_c = W - z_c,
//   dw_c/dn_j = -delta_cj w_c/n_c + (pe w_c/hh_c) dW/dn_j,
//   dW/dn_j   = (w_j/n_j) / sum_c (pe w_c/hh_c),
// so dL/dn_j += (w_j/n_j) (sum_c nu_c pe w_c/hh_c / sum_c pe w_c/hh_c - nu_j).

// Adjoint of the unclipped depth of cell (i, j) from global memory: its four new
// faces, the update and the clip test with the arithmetic of the tile kernels'
// phases A and B, the gauge seeds in gauge order.
template <typename T>
__device__ T cell_lhu(const AdjArgs<T> &A, const Fwd<T> &F, const int i, const int j)
{
    const StepArgs<T> &a = A.fwd;
    const int nx = a.geo.nx, ny = a.geo.ny;
    const size_t P = (size_t)a.geo.pitch, c = (size_t)j * P + i;
    const T h = a.h[c], z = a.z[c], n = a.n[c];
    T qW, qE, qS, qN;
    if (i == 0) qW = bface(a, F, 0, j, h, n);
    else qW = F.face(a.qx[c], a.h[c - 1], a.z[c - 1], a.n[c - 1], h, z, n);
    if (i == nx - 1) qE = bface(a, F, 1, j, h, n);
    else qE = F.face(a.qx[c + 1], h, z, n, a.h[c + 1], a.z[c + 1], a.n[c + 1]);
    if (j == 0) qS = bface(a, F, 2, i, h, n);
    else qS = F.face(a.qy[c], a.h[c - P], a.z[c - P], a.n[c - P], h, z, n);
    if (j == ny - 1) qN = bface(a, F, 3, i, h, n);
    else qN = F.face(a.qy[c + P], h, z, n, a.h[c + P], a.z[c + P], a.n[c + P]);
    const T hu = F.update(h, qW, qE, qS, qN);
    if (hu < T(0)) return T(0);
    T v = A.lh[c];
    const int64_t flat = (int64_t)j * nx + i;
    for (int gk = 0; gk < A.n_gauges; gk++)
        if (A.gauge_cells[gk] == flat) v = v + T(A.seed[gk]);
    return v;
}

// Section k of pass 3 on the calling block.  kFused: the block runs beside the
// tiles of the same launch, so it derives each cell's adjoint of the unclipped
// depth itself (cell_lhu) and adds its dL/dn terms to gn_in (one double per
// section cell, added to gn after the sweep); otherwise it reads lhu from the
// finished tiles and adds into gn.
template <typename T, bool kFused>
__device__ void inflow_adjoint(const AdjArgs<T> &A, const int k, double *red)
{
    const StepArgs<T> &a = A.fwd;
    const Geom &G = a.geo;
    const InflowSec S = A.secs[k];
    const double Q = a.inflow_Q[(size_t)a.s * a.n_inflow_sec + k];
    if (!(Q > 0.0) || S.ncell == 0) return;
    const double W = A.inflow_W[(size_t)a.s * a.n_inflow_sec + k];
    const double dx = G.dx, dtdx = a.ctrl->dt / G.dx;
    const double pe = G.bc_form == 0 ? 5.0 / 3.0 : 2.0 / 3.0;
    const double inward = (double)inward_sign(S.side);
    const size_t P = (size_t)G.pitch;
    const Fwd<T> F(G, a.ctrl->dt);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    auto lhu_of = [&](int64_t idx) -> double {
        if constexpr (kFused) return (double)cell_lhu<T>(A, F, (int)(idx % (int64_t)P), (int)(idx / (int64_t)P));
        else return (double)A.lhu[idx];
    };
    auto lq_of = [&](int64_t idx) -> double {
        switch (S.side) {
        case 0: return (double)A.lqx[idx];
        case 1: return (double)A.lqx[idx + 1];
        case 2: return (double)A.lqy[idx];
        default: return (double)A.lqy[idx + P];
        }
    };
    double D = 0.0, Nn = 0.0, nu0 = 0.0;             // nu0: this thread's first cell (reused below)
    for (int c = tid; c < S.ncell; c += nt) {
        const int64_t idx = A.sec_cells[S.cell0 + c];
        const double hh = W - (double)a.z[idx];
        if (!(hh > 0.0)) continue;
        const double w = (double)a.inflow_q[(size_t)a.s * a.n_slots + S.slot0 + c] * dx;
        const double mu = lq_of(idx) + inward * dtdx * lhu_of(idx);
        const double nu = inward * mu / dx;
        if (c == tid) nu0 = nu;
        D += pe * w / hh;
        Nn += nu * pe * w / hh;
    }
    D = block_reduce<false>(D, red);
    __syncthreads();
    if (tid == 0) red[31] = D;
    __syncthreads();
    D = red[31];
    __syncthreads();
    Nn = block_reduce<false>(Nn, red);
    __syncthreads();
    if (tid == 0) red[30] = Nn;
    __syncthreads();
    Nn = red[30];
    if (!(D > 0.0)) return;
    for (int c = tid; c < S.ncell; c += nt) {
        const int64_t idx = A.sec_cells[S.cell0 + c];
        const double hh = W - (double)a.z[idx];
        if (!(hh > 0.0)) continue;
        const double w = (double)a.inflow_q[(size_t)a.s * a.n_slots + S.slot0 + c] * dx;
        const double nu = c == tid ? nu0 : inward * (lq_of(idx) + inward * dtdx * lhu_of(idx)) / dx;
        const double term = (w / (double)a.n[idx]) * (Nn / D - nu);
        if constexpr (kFused) A.gn_in[S.cell0 + c] += term;
        else A.gn[idx] += term;
    }
}

// The fused form's entry, kept out of line: its double-precision section sums
// would otherwise raise the register count of the tile kernel that calls it.
__device__ __noinline__ void inflow_adjoint_fused(const AdjArgs<float> &A, const int k, double *red)
{
    inflow_adjoint<float, true>(A, k, red);
}

template <typename T>
__global__ void adj_inflow_kernel(const AdjArgs<T> A)
{
    __shared__ double red[32];
    inflow_adjoint<T, false>(A, blockIdx.x, red);
}

// The FP32 reverse step with its inputs staged by the tensor-memory accelerator:
// one thread issues eight 2D tensor copies (the forward state h, z, n, qx, qy and
// the adjoint after the step lh, lqx, lqy, each box with its halo, zeros outside
// the grid) onto one mbarrier, so the tile's staging costs no per-element index
// arithmetic or load latency in the threads; phases A-D are those of
// adj_step_kernel.  Staged rows start at column I0 - 4 (16-byte aligned) and
// are kAW = 40 wide.
struct AdjMaps {
    CUtensorMap m[8];            // h, z, n, qx, qy, lh, lqx, lqy
};
enum { kMh = 0, kMz, kMn, kMqx, kMqy, kMlh, kMlqx, kMlqy };
constexpr int kAW = 40;
// A tensor copy's shared-memory destination must be 128-byte aligned: every box
// starts on its own 128-byte boundary.  TB: rows of the tile.
template <int TB>
struct alignas(128) AdjStage {
    alignas(128) float h[TB + 4][kAW];      // cells: rows J0-2 .., columns I0-4 ..
    alignas(128) float z[TB + 4][kAW];
    alignas(128) float n[TB + 4][kAW];
    alignas(128) float qx[TB + 2][kAW];     // x-faces: rows J0-1 .., face columns I0-4 ..
    alignas(128) float qy[TB + 3][kAW];     // y-faces: face rows J0-1 .., columns I0-4 ..
    alignas(128) float lh[TB + 2][kAW];     // lambda_h': rows J0-1 .., columns I0-4 ..
    alignas(128) float lqx[TB][kAW];        // lambda_qx': rows J0 .., face columns I0 ..
    alignas(128) float lqy[TB + 1][BX];     // lambda_qy': face rows J0 .., columns I0 ..
    uint64_t bar;
};
template <int TB>
__host__ __device__ constexpr bool adj_stage_aligned()
{
    using S = AdjStage<TB>;
    return offsetof(S, z) % 128 == 0 && offsetof(S, n) % 128 == 0 && offsetof(S, qx) % 128 == 0 &&
           offsetof(S, qy) % 128 == 0 && offsetof(S, lh) % 128 == 0 && offsetof(S, lqx) % 128 == 0 &&
           offsetof(S, lqy) % 128 == 0 && offsetof(S, bar) % 8 == 0;
}
static_assert(adj_stage_aligned<8>() && adj_stage_aligned<16>(), "tensor-copy destinations must be 128-byte aligned");
// bytes the eight boxes deliver (the barrier's transaction count)
template <int TB>
__host__ __device__ constexpr uint32_t adj_bytes()
{
    return (uint32_t)sizeof(float) *
           (3 * (TB + 4) * kAW + (TB + 2) * kAW + (TB + 3) * kAW + (TB + 2) * kAW + TB * kAW + (TB + 1) * BX);
}
// rows of the FP32 reverse step's tile, and its blocks per SM at 40 registers
constexpr int kAdjTB = 8;
constexpr uint64_t kAdjBudgetNs = 2000000000ull;

template <int TB>
__global__ void __launch_bounds__(BX * TB, TB == 8 ? 6 : 3) adj_step_tma_kernel(const AdjArgs<float> A, const int nbx,
                                                                 const int n_tiles,
                                                                 const __grid_constant__ AdjMaps maps)
{
    using T = float;
    const int n_sec = (int)gridDim.x - n_tiles;
    if ((int)blockIdx.x < n_sec) {                   // the first blocks: pass 3, one section each, beside the tiles
        __shared__ double red_in[32];
        inflow_adjoint_fused(A, (int)blockIdx.x, red_in);
        return;
    }
    const int tile = (int)blockIdx.x - n_sec;
    __shared__ AdjStage<TB> S;
    __shared__ T sX[TB + 2][BX + 3];   // new x-faces: rows J0-1 .., face columns I0-1 ..
    __shared__ T sY[TB + 3][BX + 2];   // new y-faces: face rows J0-1 .., columns I0-1 ..
    __shared__ T sL[TB + 2][BX + 2];   // cells I0-1 .., J0-1 ..
    __shared__ T cXl[TB][BX + 1], cXr[TB][BX + 1], cXn[TB][BX + 1];
    __shared__ T cYl[TB + 1][BX], cYr[TB + 1][BX], cYn[TB + 1][BX];
    __shared__ int s_ng, s_gk[kTileGauges];
    const StepArgs<T> &a = A.fwd;
    const Geom &G = a.geo;
    const int nx = G.nx, ny = G.ny;
    const size_t P = (size_t)G.pitch;
    const double dtd = a.ctrl->dt;
    const Fwd<T> F(G, dtd);
    const T dt = T(dtd), dx = T(G.dx), g = T(G.g), hd = T(G.h_dry), dtdx = dt / dx;
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int I0 = (tile % nbx) * BX, J0 = (tile / nbx) * TB;

    // 0. the eight boxes onto one barrier; the gauge list is built meanwhile
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
        s_ng = 0;
        mbar_arrive_expect_tx(&S.bar, adj_bytes<TB>());
        tma_load_2d(&S.h[0][0], &maps.m[kMh], I0 - 4, J0 - 2, &S.bar);
        tma_load_2d(&S.z[0][0], &maps.m[kMz], I0 - 4, J0 - 2, &S.bar);
        tma_load_2d(&S.n[0][0], &maps.m[kMn], I0 - 4, J0 - 2, &S.bar);
        tma_load_2d(&S.qx[0][0], &maps.m[kMqx], I0 - 4, J0 - 1, &S.bar);
        tma_load_2d(&S.qy[0][0], &maps.m[kMqy], I0 - 4, J0 - 1, &S.bar);
        tma_load_2d(&S.lh[0][0], &maps.m[kMlh], I0 - 4, J0 - 1, &S.bar);
        tma_load_2d(&S.lqx[0][0], &maps.m[kMlqx], I0, J0, &S.bar);
        tma_load_2d(&S.lqy[0][0], &maps.m[kMlqy], I0, J0, &S.bar);
    }
    __syncthreads();
    // B prelude: the gauges inside the tile and its halo, in gauge order (repeated
    // gauges add up in order); a tile holding more than kTileGauges scans them all
    for (int gk = tid; gk < A.n_gauges; gk += BX * TB) {
        const int64_t flat = A.gauge_cells[gk];
        const int gj = (int)(flat / nx), gi = (int)(flat - (int64_t)gj * nx);
        if (gj >= J0 - 1 && gj <= J0 + TB && gi >= I0 - 1 && gi <= I0 + BX) {
            const int slot = atomicAdd(&s_ng, 1);
            if (slot < kTileGauges) s_gk[slot] = gk;
        }
    }
    const bool ok = mbar_wait_bounded(&S.bar, 0u, kAdjBudgetNs);
    if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) {
            atomicOr(&a.ctrl->status, kStatusTimeout);
            mbar_wait_bounded(&S.bar, 0u, kAdjBudgetNs);   // no copy may land after the block is gone
        }
        return;
    }
    if (tid == 0 && s_ng > 1 && s_ng <= kTileGauges) {
        for (int x = 1; x < s_ng; x++)
            for (int y = x; y > 0 && s_gk[y - 1] > s_gk[y]; y--) {
                const int tmp = s_gk[y];
                s_gk[y] = s_gk[y - 1];
                s_gk[y - 1] = tmp;
            }
    }
    // A. new face values.  x-face (lj, li): row J0-1+lj, face column fi = I0-1+li, between
    // cells at staged columns li+2 (L) and li+3 (R) of staged row lj+1.
    for (int t = tid; t < (TB + 2) * (BX + 3); t += BX * TB) {
        const int lj = t / (BX + 3), li = t % (BX + 3);
        const int j = J0 - 1 + lj, fi = I0 - 1 + li;
        T v = T(0);
        if (j >= 0 && j < ny && fi >= 0 && fi <= nx) {
            const int sj = lj + 1, sl = li + 2, sr = li + 3;
            if (fi == 0) v = bface(a, F, 0, j, S.h[sj][sr], S.n[sj][sr]);
            else if (fi == nx) v = bface(a, F, 1, j, S.h[sj][sl], S.n[sj][sl]);
            else
                v = F.face(S.qx[lj][li + 3], S.h[sj][sl], S.z[sj][sl], S.n[sj][sl], S.h[sj][sr], S.z[sj][sr],
                           S.n[sj][sr]);
        }
        sX[lj][li] = v;
    }
    // y-face (lj, li): face row fj = J0-1+lj, column i = I0-1+li, between cells of
    // staged rows lj (below) and lj+1 (above) at staged column li+3.
    for (int t = tid; t < (TB + 3) * (BX + 2); t += BX * TB) {
        const int lj = t / (BX + 2), li = t % (BX + 2);
        const int fj = J0 - 1 + lj, i = I0 - 1 + li;
        T v = T(0);
        if (i >= 0 && i < nx && fj >= 0 && fj <= ny) {
            const int sc = li + 3, sb = lj, st = lj + 1;
            if (fj == 0) v = bface(a, F, 2, i, S.h[st][sc], S.n[st][sc]);
            else if (fj == ny) v = bface(a, F, 3, i, S.h[sb][sc], S.n[sb][sc]);
            else
                v = F.face(S.qy[lj][li + 3], S.h[sb][sc], S.z[sb][sc], S.n[sb][sc], S.h[st][sc], S.z[st][sc],
                           S.n[st][sc]);
        }
        sY[lj][li] = v;
    }
    __syncthreads();
    // B. adjoint of the unclipped depth (gauge seeds included)
    const int ng_tile = s_ng;
    for (int t = tid; t < (TB + 2) * (BX + 2); t += BX * TB) {
        const int lj = t / (BX + 2), li = t % (BX + 2);
        const int j = J0 - 1 + lj, i = I0 - 1 + li;
        T v = T(0);
        if (i >= 0 && i < nx && j >= 0 && j < ny) {
            const T hu = F.update(S.h[lj + 1][li + 3], sX[lj][li], sX[lj][li + 1], sY[lj][li], sY[lj + 1][li]);
            if (!(hu < T(0))) {
                v = S.lh[lj][li + 3];
                if (ng_tile > 0) {
                    const int64_t flat = (int64_t)j * nx + i;
                    if (ng_tile <= kTileGauges) {
                        for (int x = 0; x < ng_tile; x++)
                            if (A.gauge_cells[s_gk[x]] == flat) v = v + T(A.seed[s_gk[x]]);
                    } else {
                        for (int gk = 0; gk < A.n_gauges; gk++)
                            if (A.gauge_cells[gk] == flat) v = v + T(A.seed[gk]);
                    }
                }
            }
        }
        sL[lj][li] = v;
    }
    __syncthreads();
    // C. each face touching the tile once.  x-face (lj, li): row J0+lj, face column
    // fi = I0+li; cells at staged columns li+3 (L) and li+4 (R) of staged row lj+2.
    for (int t = tid; t < TB * (BX + 1); t += BX * TB) {
        const int lj = t / (BX + 1), li = t % (BX + 1);
        const int j = J0 + lj, fi = I0 + li;
        T cl = T(0), cr = T(0), cn = T(0);
        if (j < ny && fi <= nx) {
            const size_t r = (size_t)j * P;
            const T lR = sL[lj + 1][li + 1], lL = sL[lj + 1][li];
            const int sj = lj + 2, sl = li + 3, sr = li + 4;
            if (fi == 0) {
                const T mu = S.lqx[lj][li] + dtdx * lR;
                outflow_adj(a, F, 0, j, S.h[sj][sr], S.n[sj][sr], mu, cr, cn);
                A.lqx_out[r] = T(0);
            } else if (fi == nx) {
                const T mu = S.lqx[lj][li] - dtdx * lL;
                outflow_adj(a, F, 1, j, S.h[sj][sl], S.n[sj][sl], mu, cl, cn);
                A.lqx_out[r + nx] = T(0);
            } else {
                const T mu = S.lqx[lj][li] + dtdx * (lR - lL);
                const T hL = S.h[sj][sl], zL = S.z[sj][sl], nL = S.n[sj][sl];
                const T hR = S.h[sj][sr], zR = S.z[sj][sr], nR = S.n[sj][sr];
                const T hf = F.hf(hL, zL, hR, zR);
                T lq = T(0);
                if (hf > hd && mu != T(0)) {
                    FaceLin<T> d = face_lin<T>(S.qx[lj + 1][li + 4], hL, zL, nL, hR, zR, nR, hf, g, dt, dx);
                    cl = mu * d.dhL;
                    cr = mu * d.dhR;
                    cn = mu * d.dn;
                    lq = mu * d.dq;
                }
                if (li < BX) A.lqx_out[r + fi] = lq;        // the tile owns the west faces of its cells
            }
        }
        cXl[lj][li] = cl;
        cXr[lj][li] = cr;
        cXn[lj][li] = cn;
    }
    // y-face (lj, li): face row fj = J0+lj, column i = I0+li; cells of staged rows
    // lj+1 (below) and lj+2 (above) at staged column li+4.
    for (int t = tid; t < (TB + 1) * BX; t += BX * TB) {
        const int lj = t / BX, li = t % BX;
        const int fj = J0 + lj, i = I0 + li;
        T cl = T(0), cr = T(0), cn = T(0);
        if (i < nx && fj <= ny) {
            const T lR = sL[lj + 1][li + 1], lL = sL[lj][li + 1];
            const int sc = li + 4, sb = lj + 1, st = lj + 2;
            if (fj == 0) {
                const T mu = S.lqy[lj][li] + dtdx * lR;
                outflow_adj(a, F, 2, i, S.h[st][sc], S.n[st][sc], mu, cr, cn);
                A.lqy_out[i] = T(0);
            } else if (fj == ny) {
                const size_t c = (size_t)(ny - 1) * P + i;
                const T mu = S.lqy[lj][li] - dtdx * lL;
                outflow_adj(a, F, 3, i, S.h[sb][sc], S.n[sb][sc], mu, cl, cn);
                A.lqy_out[c + P] = T(0);
            } else {
                const size_t c = (size_t)fj * P + i;
                const T mu = S.lqy[lj][li] + dtdx * (lR - lL);
                const T hL = S.h[sb][sc], zL = S.z[sb][sc], nL = S.n[sb][sc];
                const T hR = S.h[st][sc], zR = S.z[st][sc], nR = S.n[st][sc];
                const T hf = F.hf(hL, zL, hR, zR);
                T lq = T(0);
                if (hf > hd && mu != T(0)) {
                    FaceLin<T> d = face_lin<T>(S.qy[lj + 1][li + 4], hL, zL, nL, hR, zR, nR, hf, g, dt, dx);
                    cl = mu * d.dhL;
                    cr = mu * d.dhR;
                    cn = mu * d.dn;
                    lq = mu * d.dq;
                }
                if (lj < TB) A.lqy_out[c] = lq;             // the tile owns the south faces of its cells
            }
        }
        cYl[lj][li] = cl;
        cYr[lj][li] = cr;
        cYn[lj][li] = cn;
    }
    __syncthreads();
    // D. gather per tile cell
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = I0 + tx, j = J0 + ty;
    if (i >= nx || j >= ny) return;
    const size_t c = (size_t)j * P + i;
    const T lu = sL[ty + 1][tx + 1];
    const T lh = lu + cXr[ty][tx] + cXl[ty][tx + 1] + cYr[ty][tx] + cYl[ty + 1][tx];
    const T gs = (cXn[ty][tx] + cXn[ty][tx + 1]) + (cYn[ty][tx] + cYn[ty + 1][tx]);
    A.lh_out[c] = lh;
    A.gn[c] += (double)gs;
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) A.lhu[c] = lu;   // read by the inflow pass
}

// ---------------------------------------------------------------- the scheme options
// With the theta weighting or the vector norm a face's new value also depends
// on its two neighbours along the axis and on the four faces of the other axis
// around it, so their adjoints receive contributions too.  The reverse step
// then runs in three passes over global memory (each face's derivatives once):
//  R1 per cell: the new faces (the forward kernels' own arithmetic, so the clip
//     and wet/dry decisions are the forward's), the clip mask, and the adjoint
//     of the unclipped depth (gauge seeds added by a one-thread pass after it);
//  R2 per face: mu and the face's derivatives, stored as its contributions to
//     the two cells (depth, Manning n), to its own old discharge, to its axis
//     neighbours (theta) and to the orthogonal faces (vector norm);
//  R3 per cell: the gathers, for the cell and for the faces it owns (its west
//     and south faces; the last column and row also the east and north ones).
// Scratch planes (pitch x (ny + 1) each): 0..4 x-faces (to L, to R, dL/dn,
// to the axis neighbours, to the orthogonal faces), 5..9 the same for y-faces,
// 10 the clip mask.
template <typename T> struct OptFace;

template <> struct OptFace<float> {
    FastConst K;
    __device__ OptFace(const Geom &G, double dt_)
    {
        const float dt = (float)dt_, dx = (float)G.dx;
        K.gdt = (float)G.g * dt;
        K.a1 = K.gdt / dx;
        K.gdt4 = 0.25f * K.gdt;
        K.h_dry = (float)G.h_dry;
        K.dtdx = dt / dx;
        K.theta = (float)G.theta;
        K.w = (float)(0.5 * (1.0 - G.theta));
    }
    __device__ float qn(float q, float qp, float qx, bool th) const { return th ? theta_q(q, qp, qx, K) : q; }
    __device__ float qm(float q, float a, float b, float c, float d, bool vec) const
    {
        return vec ? q_norm(q, a, b, c, d) : fabsf(q);
    }
    __device__ float qo(float a, float b, float c, float d) const
    {
        return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(a, b), __fadd_rn(c, d)));
    }
    __device__ float face(float qmag, float qnum, float hL, float zL, float nL, float hR, float zR, float nR) const
    {
        return face_fast_gen(qmag, qnum, hL + zL, hR + zR, fmaxf(zL, zR), nL + nR, K);
    }
};

template <> struct OptFace<double> {
    double g, dt, dx, hd, th, w;
    __device__ OptFace(const Geom &G, double dt_)
        : g(G.g), dt(dt_), dx(G.dx), hd(G.h_dry), th(G.theta), w(0.5 * (1.0 - G.theta)) {}
    __device__ double qn(double q, double qp, double qx, bool t) const { return theta_q_ieee<double>(q, qp, qx, th, w, t); }
    __device__ double qm(double q, double a, double b, double c, double d, bool vec) const
    {
        return q_norm_ieee<double>(q, a, b, c, d, vec);
    }
    __device__ double qo(double a, double b, double c, double d) const
    {
        using O = R<double>;
        return O::mul(0.25, O::add(O::add(a, b), O::add(c, d)));
    }
    __device__ double face(double qmag, double qnum, double hL, double zL, double nL, double hR, double zR,
                           double nR) const
    {
        return face_update_ieee<double>(qnum, qmag, hL, zL, nL, hR, zR, nR, g, dt, dx, hd);
    }
};

// Inputs of an interior face: its old q, the numerator discharge, the friction
// magnitude and the mean orthogonal discharge, with the forward step's neighbours.
template <typename T>
struct OptIn {
    T q, qn, qm, qo;
};

template <typename T>
__device__ __forceinline__ OptIn<T> opt_x_in(const StepArgs<T> &a, const OptFace<T> &O, int j, int fi, bool th,
                                             bool vec)
{
    const size_t P = (size_t)a.geo.pitch, r = (size_t)j * P;
    OptIn<T> v;
    v.q = a.qx[r + fi];
    v.qn = O.qn(v.q, a.qx[r + fi - 1], a.qx[r + fi + 1], th);
    const T qa = a.qy[r + fi - 1], qb = a.qy[r + fi], qc = a.qy[r + P + fi - 1], qd = a.qy[r + P + fi];
    v.qm = O.qm(v.q, qa, qb, qc, qd, vec);
    v.qo = vec ? O.qo(qa, qb, qc, qd) : T(0);
    return v;
}

template <typename T>
__device__ __forceinline__ OptIn<T> opt_y_in(const StepArgs<T> &a, const OptFace<T> &O, int fj, int i, bool th,
                                             bool vec)
{
    const size_t P = (size_t)a.geo.pitch, r = (size_t)fj * P;
    OptIn<T> v;
    v.q = a.qy[r + i];
    v.qn = O.qn(v.q, a.qy[r - P + i], a.qy[r + P + i], th);
    const T qa = a.qx[r - P + i], qb = a.qx[r - P + i + 1], qc = a.qx[r + i], qd = a.qx[r + i + 1];
    v.qm = O.qm(v.q, qa, qb, qc, qd, vec);
    v.qo = vec ? O.qo(qa, qb, qc, qd) : T(0);
    return v;
}

// New value of x-face (j, fi), fi in [0, nx], and of y-face (fj, i), fj in [0, ny].
template <typename T>
__device__ __forceinline__ T opt_new_x(const StepArgs<T> &a, const Fwd<T> &F, const OptFace<T> &O, int j, int fi,
                                       bool th, bool vec)
{
    const Geom &G = a.geo;
    const size_t r = (size_t)j * G.pitch;
    if (fi == 0) return bface(a, F, 0, j, a.h[r], a.n[r]);
    if (fi == G.nx) return bface(a, F, 1, j, a.h[r + G.nx - 1], a.n[r + G.nx - 1]);
    const OptIn<T> v = opt_x_in(a, O, j, fi, th, vec);
    return O.face(v.qm, v.qn, a.h[r + fi - 1], a.z[r + fi - 1], a.n[r + fi - 1], a.h[r + fi], a.z[r + fi], a.n[r + fi]);
}

template <typename T>
__device__ __forceinline__ T opt_new_y(const StepArgs<T> &a, const Fwd<T> &F, const OptFace<T> &O, int fj, int i,
                                       bool th, bool vec)
{
    const Geom &G = a.geo;
    const size_t P = (size_t)G.pitch, r = (size_t)fj * P;
    if (fj == 0) return bface(a, F, 2, i, a.h[i], a.n[i]);
    if (fj == G.ny) return bface(a, F, 3, i, a.h[r - P + i], a.n[r - P + i]);
    const OptIn<T> v = opt_y_in(a, O, fj, i, th, vec);
    return O.face(v.qm, v.qn, a.h[r - P + i], a.z[r - P + i], a.n[r - P + i], a.h[r + i], a.z[r + i], a.n[r + i]);
}

// Derivatives of one wet face F = (qn - a1 hf (eta_R - eta_L)) / (1 + cc qmag),
// cc = g dt nf^2 hf^(-7/3): own old q, each axis neighbour (theta), each of
// the four orthogonal faces (vector norm), h_L, h_R and n (per cell).
template <typename T> struct OptLin {
    T dq, dnb, dorth, dhL, dhR, dn;
};

template <typename T>
__device__ __forceinline__ OptLin<T> opt_lin(const OptIn<T> &v, T hL, T zL, T nL, T hR, T zR, T nR, T hf, T g, T dt,
                                             T dx, T th, T w, bool vec)
{
    OptLin<T> r;
    const T etaL = hL + zL, etaR = hR + zR;
    const T nf = T(0.5) * (nL + nR);
    const T gdt = g * dt, a1 = gdt / dx;
    const T cc = gdt * nf * nf * Fwd<T>::pow_m73_(hf);
    const T fric = cc * v.qm;
    const T inv_den = Fwd<T>::rcp_(T(1) + fric);
    const T F = (v.qn - a1 * hf * (etaR - etaL)) * inv_den;
    const T dF_dqm = -F * cc * inv_den;
    T dqm_dq, dqm_dqo;
    if (!vec) {
        dqm_dq = v.q > T(0) ? T(1) : (v.q < T(0) ? T(-1) : T(0));
        dqm_dqo = T(0);
    } else if (v.qm > T(0)) {
        const T inv = Fwd<T>::rcp_(v.qm);
        dqm_dq = v.q * inv;
        dqm_dqo = v.qo * inv;
    } else {
        dqm_dq = dqm_dqo = T(0);
    }
    r.dq = th * inv_den + dF_dqm * dqm_dq;
    r.dnb = w * inv_den;
    r.dorth = T(0.25) * dF_dqm * dqm_dqo;
    const T dF_dhf = (-a1 * (etaR - etaL) + F * (T(7) / T(3)) * fric * Fwd<T>::rcp_(hf)) * inv_den;
    const T d_expl = a1 * hf * inv_den;
    const bool left = etaL >= etaR;
    r.dhL = d_expl + (left ? dF_dhf : T(0));
    r.dhR = -d_expl + (left ? T(0) : dF_dhf);
    r.dn = -F * fric * inv_den * Fwd<T>::rcp_(nf);
    return r;
}

template <typename T>
__device__ __forceinline__ T *opt_plane(const AdjArgs<T> &A, int k)
{
    return A.scratch + (size_t)k * A.fwd.geo.pitch * (A.fwd.geo.ny + 1);
}

// R1: clip mask and the adjoint of the unclipped depth of every cell.
template <typename T>
__global__ void __launch_bounds__(256) adj_opt_cells_kernel(const AdjArgs<T> A, const int nbx)
{
    const StepArgs<T> &a = A.fwd;
    const Geom &G = a.geo;
    const int i = (int)(blockIdx.x % (unsigned)nbx) * BX + threadIdx.x;
    const int j = (int)(blockIdx.x / (unsigned)nbx) * 8 + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const bool th = G.theta != 1.0, vec = G.friction != 0;
    const Fwd<T> F(G, a.ctrl->dt);
    const OptFace<T> O(G, a.ctrl->dt);
    const size_t c = (size_t)j * G.pitch + i;
    const T qW = opt_new_x(a, F, O, j, i, th, vec), qE = opt_new_x(a, F, O, j, i + 1, th, vec);
    const T qS = opt_new_y(a, F, O, j, i, th, vec), qN = opt_new_y(a, F, O, j + 1, i, th, vec);
    const T hu = F.update(a.h[c], qW, qE, qS, qN);
    const bool keep = !(hu < T(0));
    A.lhu[c] = keep ? A.lh[c] : T(0);
    opt_plane(A, 10)[c] = keep ? T(1) : T(0);
}

// Gauge seeds into the unclipped depth's adjoint, in gauge order (repeated gauges add up in order).
template <typename T>
__global__ void adj_opt_seeds_kernel(const AdjArgs<T> A)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const Geom &G = A.fwd.geo;
    for (int k = 0; k < A.n_gauges; k++) {
        const int64_t flat = A.gauge_cells[k];
        const size_t c = (size_t)(flat / G.nx) * G.pitch + (size_t)(flat % G.nx);
        if (opt_plane(A, 10)[c] != T(0)) A.lhu[c] = A.lhu[c] + T(A.seed[k]);
    }
}

// R2: every face's contributions (axis 0: x-faces, rows ny, faces nx + 1; axis 1: y-faces).
template <typename T>
__global__ void __launch_bounds__(256) adj_opt_faces_kernel(const AdjArgs<T> A, const int axis, const int nbx)
{
    const StepArgs<T> &a = A.fwd;
    const Geom &G = a.geo;
    const int nx = G.nx, ny = G.ny;
    const int fi = (int)(blockIdx.x % (unsigned)nbx) * BX + threadIdx.x;
    const int fj = (int)(blockIdx.x / (unsigned)nbx) * 8 + threadIdx.y;
    const int ncol = axis == 0 ? nx + 1 : nx, nrow = axis == 0 ? ny : ny + 1;
    if (fi >= ncol || fj >= nrow) return;
    const bool th = G.theta != 1.0, vec = G.friction != 0;
    const Fwd<T> F(G, a.ctrl->dt);
    const OptFace<T> O(G, a.ctrl->dt);
    const T dt = T(a.ctrl->dt), dx = T(G.dx), g = T(G.g), hd = T(G.h_dry), dtdx = dt / dx;
    const T tw = T(G.theta), ww = T(0.5 * (1.0 - G.theta));
    const size_t P = (size_t)G.pitch, f = (size_t)fj * P + fi;
    // the face's two cells (L lower index, R) as flat pitched indices, and whether they exist
    const bool hasL = axis == 0 ? fi > 0 : fj > 0, hasR = axis == 0 ? fi < nx : fj < ny;
    const size_t cL = axis == 0 ? f - 1 : f - P, cR = f;
    const T lL = hasL ? A.lhu[cL] : T(0), lR = hasR ? A.lhu[cR] : T(0);
    const T mu = (axis == 0 ? A.lqx[f] : A.lqy[f]) + dtdx * (lR - lL);
    T cl = T(0), cr = T(0), cn = T(0), lq = T(0), lt = T(0), lo = T(0);
    if (!hasL || !hasR) {                                    // a border face: Eq. 5-6 or a wall
        const int side = axis == 0 ? (hasL ? 1 : 0) : (hasL ? 3 : 2);
        const int k = axis == 0 ? fj : fi;
        const size_t cell = hasL ? cL : cR;
        outflow_adj(a, F, side, k, a.h[cell], a.n[cell], mu, hasL ? cl : cr, cn);
    } else {
        const OptIn<T> v = axis == 0 ? opt_x_in(a, O, fj, fi, th, vec) : opt_y_in(a, O, fj, fi, th, vec);
        const T hL = a.h[cL], zL = a.z[cL], nL = a.n[cL], hR = a.h[cR], zR = a.z[cR], nR = a.n[cR];
        const T hf = F.hf(hL, zL, hR, zR);
        if (hf > hd && mu != T(0)) {
            const OptLin<T> d = opt_lin<T>(v, hL, zL, nL, hR, zR, nR, hf, g, dt, dx, tw, ww, vec);
            cl = mu * d.dhL;
            cr = mu * d.dhR;
            cn = mu * d.dn;
            lq = mu * d.dq;
            lt = th ? mu * d.dnb : T(0);
            lo = vec ? mu * d.dorth : T(0);
        }
    }
    const int b = axis == 0 ? 0 : 5;
    opt_plane(A, b + 0)[f] = cl;
    opt_plane(A, b + 1)[f] = cr;
    opt_plane(A, b + 2)[f] = cn;
    opt_plane(A, b + 3)[f] = lt;
    opt_plane(A, b + 4)[f] = lo;
    (axis == 0 ? A.lqx_out : A.lqy_out)[f] = lq;
}

// R3: per cell, its own adjoint and dL/dn, and the gathers of the faces it owns.
template <typename T>
__global__ void __launch_bounds__(256) adj_opt_gather_kernel(const AdjArgs<T> A, const int nbx)
{
    const Geom &G = A.fwd.geo;
    const int nx = G.nx, ny = G.ny;
    const int i = (int)(blockIdx.x % (unsigned)nbx) * BX + threadIdx.x;
    const int j = (int)(blockIdx.x / (unsigned)nbx) * 8 + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const size_t P = (size_t)G.pitch, c = (size_t)j * P + i;
    const T *XL = opt_plane(A, 0), *XR = opt_plane(A, 1), *XN = opt_plane(A, 2), *XT = opt_plane(A, 3),
            *XO = opt_plane(A, 4);
    const T *YL = opt_plane(A, 5), *YR = opt_plane(A, 6), *YN = opt_plane(A, 7), *YT = opt_plane(A, 8),
            *YO = opt_plane(A, 9);
    A.lh_out[c] = A.lhu[c] + XR[c] + XL[c + 1] + YR[c] + YL[c + P];
    const T gs = (XN[c] + XN[c + 1]) + (YN[c] + YN[c + P]);
    A.gn[c] += (double)gs;
    // x-face (j, fi): theta from x-faces fi - 1 and fi + 1; vector norm from the y-faces
    // (j, fi - 1), (j, fi), (j + 1, fi - 1), (j + 1, fi) that read its old value
    auto gather_x = [&](int fi) {
        const size_t f = (size_t)j * P + fi;
        T s = T(0);
        if (fi > 0) s += XT[f - 1];
        if (fi < nx) s += XT[f + 1];
        if (fi > 0) s += YO[f - 1] + YO[f + P - 1];
        if (fi < nx) s += YO[f] + YO[f + P];
        A.lqx_out[f] += s;
    };
    // y-face (fj, i): theta from y-faces fj - 1 and fj + 1; vector norm from the x-faces
    // (fj - 1, i), (fj - 1, i + 1), (fj, i), (fj, i + 1) that read its old value
    auto gather_y = [&](int fj) {
        const size_t f = (size_t)fj * P + i;
        T s = T(0);
        if (fj > 0) s += YT[f - P];
        if (fj < ny) s += YT[f + P];
        if (fj > 0) s += XO[f - P] + XO[f - P + 1];
        if (fj < ny) s += XO[f] + XO[f + 1];
        A.lqy_out[f] += s;
    };
    gather_x(i);
    if (i == nx - 1) gather_x(nx);
    gather_y(j);
    if (j == ny - 1) gather_y(ny);
}

template <typename T>
__global__ void gn_out_kernel(Geom G, const double *gn, T *dst)
{
    const size_t N = (size_t)G.nx * G.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = (k / G.nx) * G.pitch + k % G.nx;
        dst[c] = T(gn[c]);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gn_out(const Geom &g, const double *gn, T *dst, cudaStream_t st)
{
    const size_t N = (size_t)g.nx * g.ny;
    const int blocks = (int)std::min<size_t>((N + 255) / 256, 152 * 16);
    gn_out_kernel<T><<<blocks, 256, 0, st>>>(g, gn, dst);
    return cudaGetLastError();
}

template cudaError_t launch_gn_out<float>(const Geom &, const double *, float *, cudaStream_t);

namespace {
__global__ void gn_inflow_add_kernel(double *gn, const double *gn_in, const int64_t *cells, int n)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int c = 0; c < n; c++) gn[cells[c]] += gn_in[c];     // in section-cell order (a corner cell may repeat)
}
}  // namespace

cudaError_t launch_gn_inflow_add(double *gn, const double *gn_in, const int64_t *sec_cells, int n_cells,
                                 cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    gn_inflow_add_kernel<<<1, 32, 0, st>>>(gn, gn_in, sec_cells, n_cells);
    return cudaGetLastError();
}
template cudaError_t launch_gn_out<double>(const Geom &, const double *, double *, cudaStream_t);

template <typename T>
cudaError_t launch_adjoint_step(const AdjArgs<T> &A, cudaStream_t st)
{
    const Geom &G = A.fwd.geo;
    cudaError_t e0 = cudaSuccess;
    if (G.theta != 1.0 || G.friction != 0) {
        if (!A.scratch) return cudaErrorInvalidValue;
        const dim3 block(BX, 8);
        const int nbx = (G.nx + BX - 1) / BX, nby = (G.ny + 7) / 8;
        adj_opt_cells_kernel<T><<<(unsigned)((int64_t)nbx * nby), block, 0, st>>>(A, nbx);
        if (A.n_gauges > 0) adj_opt_seeds_kernel<T><<<1, 32, 0, st>>>(A);
        const int nbx0 = (G.nx + 1 + BX - 1) / BX;
        adj_opt_faces_kernel<T><<<(unsigned)((int64_t)nbx0 * nby), block, 0, st>>>(A, 0, nbx0);
        const int nby1 = (G.ny + 1 + 7) / 8;
        adj_opt_faces_kernel<T><<<(unsigned)((int64_t)nbx * nby1), block, 0, st>>>(A, 1, nbx);
        adj_opt_gather_kernel<T><<<(unsigned)((int64_t)nbx * nby), block, 0, st>>>(A, nbx);
    } else if constexpr (std::is_same<T, float>::value) {
        // FP32: the tile's inputs staged by tensor copies (maps of this step's buffers)
        const int P = G.pitch, nx = G.nx, ny = G.ny;
        const StepArgs<float> &f = A.fwd;
        AdjMaps maps;
        constexpr int TB = kAdjTB;
        const struct {
            const float *base;
            int w, h, bw, bh;
        } fields[8] = {{f.h, nx, ny, kAW, TB + 4},          {f.z, nx, ny, kAW, TB + 4},
                       {f.n, nx, ny, kAW, TB + 4},          {f.qx, nx + 1, ny, kAW, TB + 2},
                       {f.qy, nx, ny + 1, kAW, TB + 3},     {A.lh, nx, ny, kAW, TB + 2},
                       {A.lqx, nx + 1, ny, kAW, TB},        {A.lqy, nx, ny + 1, BX, TB + 1}};
        for (int k = 0; k < 8; k++) {
            const cudaError_t e = encode_map_f32(&maps.m[k], fields[k].base, fields[k].w, fields[k].h, P,
                                                 fields[k].bw, fields[k].bh);
            if (e != cudaSuccess) return e;
        }
        const int nbx = (nx + BX - 1) / BX, nby = (ny + TB - 1) / TB;
        const int n_tiles = nbx * nby, n_sec = A.gn_in ? A.fwd.n_inflow_sec : 0;
        adj_step_tma_kernel<TB><<<(unsigned)(n_tiles + n_sec), dim3(BX, TB), 0, st>>>(A, nbx, n_tiles, maps);
        e0 = cudaGetLastError();
        if (e0 != cudaSuccess || n_sec > 0) return e0;   // pass 3 ran in the same launch
        if (A.fwd.n_inflow_sec > 0) adj_inflow_kernel<T><<<A.fwd.n_inflow_sec, 256, 0, st>>>(A);
        return cudaGetLastError();
    } else {
        constexpr int BYT = TileRows<T>::v;
        dim3 block(BX, BYT);
        const int nbx = (G.nx + BX - 1) / BX, nby = (G.ny + BYT - 1) / BYT;
        adj_step_kernel<T><<<(unsigned)((int64_t)nbx * nby), block, 0, st>>>(A, nbx);
    }
    if (A.fwd.n_inflow_sec > 0) adj_inflow_kernel<T><<<A.fwd.n_inflow_sec, 256, 0, st>>>(A);
    return cudaGetLastError();
}

template cudaError_t launch_adjoint_step<float>(const AdjArgs<float> &, cudaStream_t);
template cudaError_t launch_adjoint_step<double>(const AdjArgs<double> &, cudaStream_t);

}  // namespace flood
