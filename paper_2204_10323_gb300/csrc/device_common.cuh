// device_common.cuh -- device helpers of the flood kernels: IEEE-rounded
// arithmetic wrappers (never contracted by the compiler, so every call site
// computing the same face from the same inputs returns the same bits), the
// Eq. 3 face update, the Eq. 5 boundary discharge and warp/block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "flood_internal.h"

namespace flood {

template <typename T> struct R;

template <> struct R<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float cbrt(float a) { return cbrtf(a); }
    static __device__ __forceinline__ float pw(float a, float b) { return powf(a, b); }
    static __device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
};

template <> struct R<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double cbrt(double a) { return ::cbrt(a); }
    static __device__ __forceinline__ double pw(double a, double b) { return ::pow(a, b); }
    static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double max(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double abs(double a) { return fabs(a); }
};

// Eq. 3 at one interior face between cell L (lower index) and R, with the
// time step in the numerator and h_f = max(eta_L, eta_R) - max(z_L, z_R);
// 0 when h_f <= h_dry.  qn is the discharge in the numerator (q itself unless
// theta-weighted), qmag the |q| of the friction term (q_norm_ieee).
// Operations in the order of the plain definition, each rounded once (no
// contraction).
template <typename T>
__device__ __forceinline__ T face_update_ieee(T qn, T qmag, T hL, T zL, T nL, T hR, T zR, T nR, T g, T dt,
                                              T dx, T h_dry)
{
    using O = R<T>;
    T etaL = O::add(hL, zL), etaR = O::add(hR, zR);
    T hf = O::sub(O::max(etaL, etaR), O::max(zL, zR));
    if (!(hf > h_dry)) return T(0);
    T nf = O::mul(T(0.5), O::add(nL, nR));
    T gdt = O::mul(g, dt);
    T slope_term = O::div(O::mul(O::mul(gdt, hf), O::sub(etaR, etaL)), dx);
    T hf_m73 = O::div(T(1), O::mul(O::mul(hf, hf), O::cbrt(hf)));
    T friction = O::mul(O::mul(O::mul(O::mul(gdt, nf), nf), qmag), hf_m73);
    return O::div(O::sub(qn, slope_term), O::add(T(1), friction));
}

// |q| of the friction term of a face: its own |q|, or with vec the vector
// norm sqrt(q^2 + qo^2), qo = ((a + b) + (c + d)) / 4 the mean of the four
// faces of the other axis around it (a, b on the lower-index side).
template <typename T>
__device__ __forceinline__ T q_norm_ieee(T q, T a, T b, T c, T d, bool vec)
{
    using O = R<T>;
    if (!vec) return O::abs(q);
    const T qo = O::mul(T(0.25), O::add(O::add(a, b), O::add(c, d)));
    return O::sqrt(O::add(O::mul(q, q), O::mul(qo, qo)));
}

// Numerator discharge of a face (qn of face_update_ieee): q itself, or with
// theta < 1 the weighted theta q + w (q_prev + q_next), w = (1 - theta)/2, of
// the face and its two neighbours along the same axis.
template <typename T>
__device__ __forceinline__ T theta_q_ieee(T q, T q_prev, T q_next, T theta, T w, bool weighted)
{
    using O = R<T>;
    return weighted ? O::add(O::mul(theta, q), O::mul(w, O::add(q_prev, q_next))) : q;
}

// Eq. 5 per boundary cell as a unit-width flux (m^2/s): bc_form 0 uses the
// flow area dx*h (q = h^(5/3) sqrt(S)/n), bc_form 1 the literal A = dx^2
// (q = dx h^(2/3) sqrt(S)/n).  0 on a dry cell.
template <typename T>
__device__ __forceinline__ T outflow_flux_ieee(T h, T sqrtS, T n, T dx, T h_dry, int bc_form)
{
    using O = R<T>;
    if (!(h > h_dry)) return T(0);
    if (bc_form == 0)
        return O::div(O::div(O::mul(O::mul(dx, O::pw(h, T(5.0 / 3.0))), sqrtS), n), dx);
    return O::div(O::div(O::mul(O::mul(O::mul(dx, dx), O::pw(h, T(2.0 / 3.0))), sqrtS), n), dx);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// max that keeps a NaN (fmax would drop it), so a NaN depth reaches the epoch check
__device__ __forceinline__ double nanmax(double a, double b)
{
    if (a != a) return a;
    if (b != b) return b;
    return a > b ? a : b;
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum/max (every thread of the block must call; result valid in thread 0).
template <bool kMax>
__device__ __forceinline__ double block_reduce(double v, double *smem32)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nthreads = blockDim.x * blockDim.y * blockDim.z;
    int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    lane = tid & 31;
    wid = tid >> 5;
    v = kMax ? warp_max(v) : warp_sum(v);
    __syncthreads();
    if (lane == 0) smem32[wid] = v;
    __syncthreads();
    int nw = (nthreads + 31) >> 5;
    if (wid == 0) {
        v = lane < nw ? smem32[lane] : (kMax ? 0.0 : 0.0);
        v = kMax ? warp_max(v) : warp_sum(v);
    }
    return v;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v)
{
    // Non-negative doubles (and NaNs, whose bit patterns are larger) order as unsigned integers.
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Inward unit sign of a side: +1 on xmin / ymin, -1 on xmax / ymax.
__device__ __forceinline__ int inward_sign(int side) { return (side == 0 || side == 2) ? 1 : -1; }

}  // namespace flood
