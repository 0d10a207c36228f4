// fast_face.cuh -- FP32 face arithmetic shared by the bandwidth kernels
// (rows, stream, tiled).  Every operation is an explicitly rounded intrinsic
// or a CUDA math function, never contracted by the compiler, so two kernels
// or two call sites that evaluate the same face from the same inputs obtain
// the same bits (the face shared by two warps or tiles stays conservative).
#pragma once

#include "device_common.cuh"

namespace flood {

struct FastConst {
    float a1;       // g dt / dx   (slope term factor)
    float gdt;      // g dt        (friction factor)
    float gdt4;     // g dt / 4    (friction factor of the Manning sum n_L + n_R: n_f^2 = (n_L + n_R)^2 / 4)
    float h_dry;
    float dtdx;     // dt / dx
    float theta, w; // face-flux weighting theta and (1 - theta)/2
};

// Numerator discharge of a theta-weighted face from its own and its two
// neighbours' discharge along the same axis: theta q + w (q_prev + q_next) as
// one fused multiply-add (the paired form below is the same operation; a paired
// multiply followed by a paired add is fused by the hardware, so both forms
// write the fusion out).
__device__ __forceinline__ float theta_q(float q, float q_prev, float q_next, const FastConst &k)
{
    return __fmaf_rn(k.theta, q, __fmul_rn(k.w, __fadd_rn(q_prev, q_next)));
}

// x^(-7/3) for x > 0 as 2^(-7/3 log2 x) with the hardware base-2 logarithm
// and exponential (relative error below 1e-6 for the depths of a flood).
__device__ __forceinline__ float pow_m73(float x)
{
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    l = __fmul_rn(l, -7.0f / 3.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(l));
    return r;
}

// 1/x by the hardware reciprocal approximation (about 1 ulp); Eq. 3 divides
// by 1 + friction >= 1 only.
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Square root by the hardware approximation (a few ulp; sqrt(0) = 0 without
// the special-case path of the IEEE-rounded square root).
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// |q| of a face in the friction term as the vector norm: the face's discharge q
// and the mean of the four faces of the other axis around it (a, b on the
// lower-index side, c, d on the other).
__device__ __forceinline__ float q_norm(float q, float a, float b, float c, float d)
{
    const float qo = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(a, b), __fadd_rn(c, d)));
    return sqrt_fast(__fmaf_rn(q, q, __fmul_rn(qo, qo)));
}

// Eq. 3 for a wet face of flow depth hf: qmag the |q| of the friction term
// (the face's own |q| unless the vector norm is asked for), qn the numerator
// discharge (q itself unless theta-weighted).  The numerator
// qn - (a1 hf)(eta_R - eta_L) and the denominator 1 + friction are each one
// fused multiply-add (one rounding), as the paired form below computes them.
// Called with hf <= 0 the result is NaN or garbage, never a trap;
// face_fast_sel discards it.
__device__ __forceinline__ float face_wet(float qmag, float qn, float etaL, float etaR, float hf, float nsum,
                                          const FastConst &k)
{
    float r7 = pow_m73(hf);
    // g dt n_f^2 |q| with n_f = nsum / 2 as (g dt / 4)(nsum^2)|q|: the scalings by
    // powers of two are exact, so this is the same number with one product fewer
    float aq = __fmul_rn(__fmul_rn(k.gdt4, __fmul_rn(nsum, nsum)), qmag);
    float num = __fmaf_rn(__fmul_rn(-k.a1, hf), __fsub_rn(etaR, etaL), qn);
    return __fmul_rn(num, rcp_fast(__fmaf_rn(aq, r7, 1.0f)));
}

// ---- two faces at once on the paired single-precision instructions
// (add/sub/mul .f32x2: one instruction for two lanes of a 64-bit register
// pair, each rounded as the scalar instruction), for the issue-bound
// temporal-blocking kernel.  face_fast_sel_x2 returns exactly the two values
// face_fast_sel returns for (x, y): the same operations in the same order.
__device__ __forceinline__ unsigned long long f2pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float2 f2unpack(unsigned long long r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ float lg2_fast(float x)
{
    float l;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    return l;
}

__device__ __forceinline__ float ex2_fast(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// face_fast_sel_gen for two faces: qmag and qn packed (|q| of the friction term,
// numerator discharge), etaL, etaR, nsum packed, zmax the two faces' max(z_L, z_R).
__device__ __forceinline__ float2 face_fast_sel_x2_gen(unsigned long long qmag, unsigned long long qn,
                                                       unsigned long long etaL, unsigned long long etaR, float2 zmax,
                                                       unsigned long long nsum, const FastConst &k)
{
    const float2 eL = f2unpack(etaL), eR = f2unpack(etaR);
    const unsigned long long hf = f2sub(f2pack(fmaxf(eL.x, eR.x), fmaxf(eL.y, eR.y)), f2pack(zmax.x, zmax.y));
    const float2 h = f2unpack(hf);
    const unsigned long long l = f2mul(f2pack(lg2_fast(h.x), lg2_fast(h.y)), f2pack(-7.0f / 3.0f, -7.0f / 3.0f));
    const float2 lv = f2unpack(l);
    const unsigned long long r7 = f2pack(ex2_fast(lv.x), ex2_fast(lv.y));
    const unsigned long long aq = f2mul(f2mul(f2pack(k.gdt4, k.gdt4), f2mul(nsum, nsum)), qmag);
    const unsigned long long num = f2fma(f2mul(f2pack(-k.a1, -k.a1), hf), f2sub(etaR, etaL), qn);
    const float2 den = f2unpack(f2fma(aq, r7, f2pack(1.0f, 1.0f)));
    const float2 v = f2unpack(f2mul(num, f2pack(rcp_fast(den.x), rcp_fast(den.y))));
    return make_float2(h.x > k.h_dry ? v.x : 0.0f, h.y > k.h_dry ? v.y : 0.0f);
}

// etaL, etaR, zmax, nsum, q: the two faces' arguments of face_fast_sel.
__device__ __forceinline__ float2 face_fast_sel_x2(float2 q, unsigned long long etaL, unsigned long long etaR,
                                                   float2 zmax, unsigned long long nsum, const FastConst &k)
{
    return face_fast_sel_x2_gen(f2pack(fabsf(q.x), fabsf(q.y)), f2pack(q.x, q.y), etaL, etaR, zmax, nsum, k);
}

// theta_q for two faces (packed q, previous and next neighbours).
__device__ __forceinline__ unsigned long long theta_q_x2(unsigned long long q, unsigned long long q_prev,
                                                         unsigned long long q_next, const FastConst &k)
{
    return f2fma(f2pack(k.theta, k.theta), q, f2mul(f2pack(k.w, k.w), f2add(q_prev, q_next)));
}

// q_norm for two faces (packed q and the four orthogonal neighbours a, b, c, d).
__device__ __forceinline__ unsigned long long q_norm_x2(unsigned long long q, unsigned long long a,
                                                        unsigned long long b, unsigned long long c,
                                                        unsigned long long d)
{
    const unsigned long long qo = f2mul(f2pack(0.25f, 0.25f), f2add(f2add(a, b), f2add(c, d)));
    const float2 s = f2unpack(f2fma(q, q, f2mul(qo, qo)));
    return f2pack(sqrt_fast(s.x), sqrt_fast(s.y));
}

// Eq. 3 at one face: eta_L, eta_R water levels, zmax = max(z_L, z_R),
// nsum = n_L + n_R.
__device__ __forceinline__ float face_fast(float q, float etaL, float etaR, float zmax, float nsum,
                                           const FastConst &k)
{
    float hf = __fsub_rn(fmaxf(etaL, etaR), zmax);
    if (!(hf > k.h_dry)) return 0.0f;
    return face_wet(fabsf(q), q, etaL, etaR, hf, nsum, k);
}

// face_fast with the friction magnitude qmag and the numerator discharge qn
// given (vector-norm friction, theta-weighted faces).
__device__ __forceinline__ float face_fast_gen(float qmag, float qn, float etaL, float etaR, float zmax, float nsum,
                                               const FastConst &k)
{
    float hf = __fsub_rn(fmaxf(etaL, etaR), zmax);
    if (!(hf > k.h_dry)) return 0.0f;
    return face_wet(qmag, qn, etaL, etaR, hf, nsum, k);
}

// The same value as face_fast without a branch: a dry face is evaluated too
// and its result discarded, so that the faces of a lane can be interleaved by
// the compiler.
__device__ __forceinline__ float face_fast_sel(float q, float etaL, float etaR, float zmax, float nsum,
                                               const FastConst &k)
{
    float hf = __fsub_rn(fmaxf(etaL, etaR), zmax);
    float v = face_wet(fabsf(q), q, etaL, etaR, hf, nsum, k);
    return hf > k.h_dry ? v : 0.0f;
}

// face_fast_sel with qmag and qn given (vector-norm friction, theta-weighted faces).
__device__ __forceinline__ float face_fast_sel_gen(float qmag, float qn, float etaL, float etaR, float zmax,
                                                   float nsum, const FastConst &k)
{
    float hf = __fsub_rn(fmaxf(etaL, etaR), zmax);
    float v = face_wet(qmag, qn, etaL, etaR, hf, nsum, k);
    return hf > k.h_dry ? v : 0.0f;
}

// Eq. 5 boundary flux magnitude (m^2/s) of a cell of depth h.
__device__ __forceinline__ float outflow_fast(float h, float sqrtS, float n, float dx, float h_dry, int form)
{
    if (!(h > h_dry)) return 0.0f;
    float c = cbrtf(h);
    float p = form == 0 ? __fmul_rn(h, __fmul_rn(c, c)) : __fmul_rn(dx, __fmul_rn(c, c));
    return __fdividef(__fmul_rn(p, sqrtS), n);
}

// Boundary face value on `side` at index k along it, for the adjacent cell
// (h, n), at step `step` of the epoch (selects the Eq. 6 inflow row).
__device__ __forceinline__ float boundary_fast_at(const StepArgs<float> &a, int step, int side, int k, float h,
                                                  float n, double &vout)
{
    const Geom &G = a.geo;
    int off = side == 0 ? 0 : side == 1 ? G.ny : side == 2 ? 2 * G.ny : 2 * G.ny + G.nx;
    int type = a.bc.type[off + k];
    if (type == kBcWall) return 0.0f;
    float inward = (side == 0 || side == 2) ? 1.0f : -1.0f;
    if (type == kBcInflow) return inward * a.inflow_q[(size_t)step * a.n_slots + a.bc.slot[off + k]];
    float q = outflow_fast(h, a.bc.sqrtS_f[off + k], n, G.dx_f, G.h_dry_f, G.bc_form);
    if (type == kBcOutflow) vout += (double)q * G.dx;
    return -inward * q;
}

// As boundary_fast_at, booking the outflow flux magnitude (m^2/s, not yet
// times dx) into a float partial sum that the caller folds into its double
// ledger every few rows.
__device__ __forceinline__ float boundary_fast_flux(const StepArgs<float> &a, int step, int side, int k, float h,
                                                    float n, float &qout)
{
    const Geom &G = a.geo;
    int off = side == 0 ? 0 : side == 1 ? G.ny : side == 2 ? 2 * G.ny : 2 * G.ny + G.nx;
    int type = a.bc.type[off + k];
    if (type == kBcWall) return 0.0f;
    float inward = (side == 0 || side == 2) ? 1.0f : -1.0f;
    if (type == kBcInflow) return inward * a.inflow_q[(size_t)step * a.n_slots + a.bc.slot[off + k]];
    float q = outflow_fast(h, a.bc.sqrtS_f[off + k], n, G.dx_f, G.h_dry_f, G.bc_form);
    if (type == kBcOutflow) qout += q;
    return -inward * q;
}

}  // namespace flood
