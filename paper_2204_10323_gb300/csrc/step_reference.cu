// step_reference.cu -- one thread per cell, every operation IEEE-rounded in
// the order of the plain definition (Methods, Eq. 3-4, boundary faces by
// Eq. 5-6).  This is the FP64 path and the FP32 cross-check; each cell
// evaluates its four faces itself, and because the arithmetic is never
// contracted both cells of an interior face obtain the same bits, so the
// update conserves mass exactly like the face-by-face definition.
#include "device_common.cuh"

namespace flood {

namespace {

constexpr int BX = 32, BY = 8;

template <typename T>
__device__ __forceinline__ T boundary_face(const StepArgs<T> &a, int side, int k, T h_cell, T n_cell,
                                           double &vout)
{
    const Geom &G = a.geo;
    int off = side == 0 ? 0 : side == 1 ? G.ny : side == 2 ? 2 * G.ny : 2 * G.ny + G.nx;
    int type = a.bc.type[off + k];
    if (type == kBcWall) return T(0);
    T inward = T(inward_sign(side));
    if (type == kBcInflow) return inward * a.inflow_q[(size_t)a.s * a.n_slots + a.bc.slot[off + k]];
    T q = outflow_flux_ieee<T>(h_cell, T(a.bc.sqrtS[off + k]), n_cell, T(G.dx), T(G.h_dry), G.bc_form);
    if (type == kBcOutflow) vout += (double)q * G.dx;
    return -inward * q;
}

template <typename T>
__global__ void __launch_bounds__(BX *BY) step_reference_kernel(const StepArgs<T> a, const int nbx)
{
    // one-dimensional grid (grids taller than 65535 blocks): block (bx, by) of nbx columns of blocks
    const int bx = (int)(blockIdx.x % (unsigned)nbx), by = (int)(blockIdx.x / (unsigned)nbx);
    using O = R<T>;
    __shared__ double red[32];
    __shared__ T tile[BY][BX];
    const Geom &G = a.geo;
    const int i = bx * BX + threadIdx.x;
    const int j = by * BY + threadIdx.y;
    const bool in = i < G.nx && j < G.ny;
    const T dt = T(a.ctrl->dt), dx = T(G.dx), g = T(G.g), hd = T(G.h_dry);
    const bool wt = G.theta != 1.0;                   // theta-weighted numerator discharges
    const bool vec = G.friction != 0;                 // vector-norm |q| in the friction term
    const T th = T(G.theta), w = T(0.5 * (1.0 - G.theta));
    double vout = 0.0, vclip = 0.0, hmax = 0.0;
    T hn = T(0);
    if (in) {
        const size_t P = (size_t)G.pitch;
        const size_t c = (size_t)j * P + i;
        const T hC = a.h[c], zC = a.z[c], nC = a.n[c];
        T qW, qE, qS, qN;
        // (interior x-faces i in 1..nx-1 have neighbours i-1 >= 0 and i+1 <= nx in the row and
        // y-faces of columns i-1, i in rows j, j+1 <= ny; interior y-faces j in 1..ny-1 neighbours
        // j-1 >= 0 and j+1 <= ny and x-faces of columns i, i+1 <= nx in rows j-1, j)
        const T *qx = a.qx, *qy = a.qy;
        if (i == 0) qW = boundary_face(a, 0, j, hC, nC, vout);
        else qW = face_update_ieee<T>(wt ? theta_q_ieee<T>(qx[c], qx[c - 1], qx[c + 1], th, w, true) : qx[c],
                                      vec ? q_norm_ieee<T>(qx[c], qy[c - 1], qy[c], qy[c + P - 1], qy[c + P], true)
                                          : R<T>::abs(qx[c]),
                                      a.h[c - 1], a.z[c - 1], a.n[c - 1], hC, zC, nC, g, dt, dx, hd);
        if (i == G.nx - 1) qE = boundary_face(a, 1, j, hC, nC, vout);
        else qE = face_update_ieee<T>(wt ? theta_q_ieee<T>(qx[c + 1], qx[c], qx[c + 2], th, w, true) : qx[c + 1],
                                      vec ? q_norm_ieee<T>(qx[c + 1], qy[c], qy[c + 1], qy[c + P], qy[c + P + 1], true)
                                          : R<T>::abs(qx[c + 1]),
                                      hC, zC, nC, a.h[c + 1], a.z[c + 1], a.n[c + 1], g, dt, dx, hd);
        if (j == 0) qS = boundary_face(a, 2, i, hC, nC, vout);
        else qS = face_update_ieee<T>(wt ? theta_q_ieee<T>(qy[c], qy[c - P], qy[c + P], th, w, true) : qy[c],
                                      vec ? q_norm_ieee<T>(qy[c], qx[c - P], qx[c - P + 1], qx[c], qx[c + 1], true)
                                          : R<T>::abs(qy[c]),
                                      a.h[c - P], a.z[c - P], a.n[c - P], hC, zC, nC, g, dt, dx, hd);
        if (j == G.ny - 1) qN = boundary_face(a, 3, i, hC, nC, vout);
        else qN = face_update_ieee<T>(wt ? theta_q_ieee<T>(qy[c + P], qy[c], qy[c + 2 * P], th, w, true) : qy[c + P],
                                      vec ? q_norm_ieee<T>(qy[c + P], qx[c], qx[c + 1], qx[c + P], qx[c + P + 1], true)
                                          : R<T>::abs(qy[c + P]),
                                      hC, zC, nC, a.h[c + P], a.z[c + P], a.n[c + P], g, dt, dx, hd);
        // Eq. 4 with the new fluxes, then the depth clip
        T dv = O::add(O::sub(qW, qE), O::sub(qS, qN));
        hn = O::add(hC, O::div(O::mul(dt, dv), dx));
        if (hn < T(0)) {
            if (j >= G.led_j0 && j < G.led_j1) vclip += -(double)hn * G.dx * G.dx;
            hn = T(0);
        }
        a.h_out[c] = hn;
        a.qx_out[c] = qW;
        a.qy_out[c] = qS;
        if (i == G.nx - 1) a.qx_out[c + 1] = qE;
        if (j == G.ny - 1) a.qy_out[c + P] = qN;
        hmax = (double)hn;
    }
    // ledger: outflow and clip volumes (one atomic per block that has any)
    double bo = block_reduce<false>(vout, red);
    if (threadIdx.x == 0 && threadIdx.y == 0 && bo != 0.0) atomicAdd(&a.ctrl->V_out, (double)dt * bo);
    double bc = block_reduce<false>(vclip, red);
    if (threadIdx.x == 0 && threadIdx.y == 0 && bc != 0.0) atomicAdd(&a.ctrl->V_clip, bc);
    if (a.want_hmax) {
        double bm = block_reduce<true>(hmax, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) atomic_max_nonneg(&a.ctrl->hmax_bits, bm);
    }
    if (a.gauge_out) {
        tile[threadIdx.y][threadIdx.x] = hn;
        __syncthreads();
        int tid = threadIdx.y * BX + threadIdx.x;
        for (int k = tid; k < a.n_gauges; k += BX * BY) {
            int64_t cell = a.gauge_cells[k];
            int gi = (int)(cell % G.nx), gj = (int)(cell / G.nx);
            int li = gi - bx * BX, lj = gj - by * BY;
            if (li >= 0 && li < BX && lj >= 0 && lj < BY) a.gauge_out[k] = (double)tile[lj][li];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        double vin = a.ctrl->V_in;
        for (int k = 0; k < a.n_inflow_sec; k++) {
            double Q = a.inflow_Q[(size_t)a.s * a.n_inflow_sec + k];
            if (Q > 0.0) vin += a.ctrl->dt * Q;
        }
        a.ctrl->V_in = vin;
        a.ctrl->t = a.t_list[a.s + 1];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_step_reference(const StepArgs<T> &a, cudaStream_t st)
{
    dim3 block(BX, BY);
    const int nbx = (a.geo.nx + BX - 1) / BX, nby = (a.geo.ny + BY - 1) / BY;
    step_reference_kernel<T><<<(unsigned)((int64_t)nbx * nby), block, 0, st>>>(a, nbx);
    return cudaGetLastError();
}

template cudaError_t launch_step_reference<float>(const StepArgs<float> &, cudaStream_t);
template cudaError_t launch_step_reference<double>(const StepArgs<double> &, cudaStream_t);

}  // namespace flood
