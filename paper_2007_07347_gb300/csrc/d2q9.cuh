// d2q9.cuh -- D2Q9 lattice constants, the discrete equilibrium and the storage
// codecs of f shared by the CUDA translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include "sdugks_internal.h"

namespace sdugks {

// Velocity a: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
__host__ __device__ constexpr int EX(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0); }
__host__ __device__ constexpr int EY(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0); }

// Mirror image of velocity a in a line of constant x (xi_x -> -xi_x) and of constant y.
__host__ __device__ constexpr int MIRROR_X(int a) {
    return a == 1 ? 3 : a == 3 ? 1 : a == 5 ? 6 : a == 6 ? 5 : a == 7 ? 8 : a == 8 ? 7 : a;
}
__host__ __device__ constexpr int MIRROR_Y(int a) {
    return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}

template <class R> __device__ __forceinline__ R wq(int a) {
    return a == 0 ? R(4) / R(9) : (a < 5 ? R(1) / R(9) : R(1) / R(36));
}
template <class R> __device__ __forceinline__ R inv_wq(int a) {
    return a == 0 ? R(9) / R(4) : (a < 5 ? R(9) : R(36));
}

// xi_a . v with the lattice components folded in at compile time.
template <class R> __device__ __forceinline__ R xdot(int a, R vx, R vy) {
    const int ex = EX(a), ey = EY(a);
    R s = R(0);
    if (ex == 1) s = vx; else if (ex == -1) s = -vx;
    if (ey == 1) s = (ex == 0) ? vy : s + vy;
    else if (ey == -1) s = (ex == 0) ? -vy : s - vy;
    return s;
}

// Discrete equilibrium (second-order Hermite expansion of the Maxwellian, Eq. Feq on
// the nine-velocity lattice): w rho [1 + 3 xi.u + 4.5 (xi.u)^2 - 1.5 |u|^2].
template <class R> __device__ __forceinline__ void feq9(R rho, R ux, R uy, R out[NQ]) {
    const R base = R(1) - R(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int a = 0; a < NQ; a++) {
        const R eu = xdot<R>(a, ux, uy);
        out[a] = wq<R>(a) * rho * (base + eu * (R(3) + R(4.5) * eu));
    }
}

// The same equilibrium with the shared terms factored out of the nine velocities
// (opposite velocities share w rho [1 - 1.5 |u|^2 + 4.5 (xi.u)^2] and differ in the
// sign of 3 w rho xi.u).  Used by the hot kernels.
template <class R> __device__ __forceinline__ R recip(R x) { return R(1) / x; }
// FP32: the hardware reciprocal (rcp.approx, at most 1 ulp from 1/x; subnormals flush
// to zero, which the densities here never are)
template <> __device__ __forceinline__ float recip<float>(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// feq9fd(b0, rho, u): w [b0 + rho (3 xi.u + 4.5 (xi.u)^2 - 1.5 |u|^2)].  With b0 = rho
// this is the equilibrium itself (feq9f); with b0 = rho - 1 it is the equilibrium's
// deviation from the rest equilibrium of unit density, feq(rho, u) - w, the form the
// FP32 kernels compute in (each term then has the size of the deviation, not of f).
template <class R> __device__ __forceinline__ void feq9fd(R b0, R rho, R ux, R uy, R out[NQ]) {
    const R base = b0 - R(1.5) * rho * (ux * ux + uy * uy);
    const R r3 = R(3) * rho, r45 = R(4.5) * rho;
    const R w0 = R(4) / R(9), w1 = R(1) / R(9), w5 = R(1) / R(36);
    out[0] = w0 * base;
    {
        const R t = base + r45 * ux * ux, l = r3 * ux;
        out[1] = w1 * (t + l); out[3] = w1 * (t - l);
    }
    {
        const R t = base + r45 * uy * uy, l = r3 * uy;
        out[2] = w1 * (t + l); out[4] = w1 * (t - l);
    }
    {
        const R e = ux + uy, t = base + r45 * e * e, l = r3 * e;
        out[5] = w5 * (t + l); out[7] = w5 * (t - l);
    }
    {
        const R e = uy - ux, t = base + r45 * e * e, l = r3 * e;
        out[6] = w5 * (t + l); out[8] = w5 * (t - l);
    }
}

// FP32: the same equilibrium with the four velocity pairs (1,2) (3,4) (5,6) (7,8)
// evaluated by paired FP32 instructions (FFMA2/FMUL2; each lane rounds as the scalar
// operation would): t = base + 4.5 rho e^2 and l = 3 rho e for e = (u_x, u_y) and for
// e = (u_x + u_y, u_y - u_x), then w (t + l) and w (t - l).
template <> __device__ __forceinline__ void feq9fd<float>(float b0, float rho, float ux, float uy, float out[NQ]) {
    const float base = b0 - 1.5f * rho * (ux * ux + uy * uy);
    const float r3 = 3.0f * rho, r45 = 4.5f * rho;
    const float2 B = make_float2(base, base), R45 = make_float2(r45, r45), R3 = make_float2(r3, r3);
    const float2 w1 = make_float2(1.0f / 9.0f, 1.0f / 9.0f), w5 = make_float2(1.0f / 36.0f, 1.0f / 36.0f);
    const float2 m1 = make_float2(-1.0f, -1.0f);
    out[0] = (4.0f / 9.0f) * base;
    {
        const float2 e = make_float2(ux, uy);
        const float2 t = __ffma2_rn(__fmul2_rn(R45, e), e, B), l = __fmul2_rn(R3, e);
        const float2 p = __fmul2_rn(w1, __fadd2_rn(t, l)), q = __fmul2_rn(w1, __ffma2_rn(l, m1, t));
        out[1] = p.x; out[2] = p.y; out[3] = q.x; out[4] = q.y;
    }
    {
        const float2 e = make_float2(ux + uy, uy - ux);
        const float2 t = __ffma2_rn(__fmul2_rn(R45, e), e, B), l = __fmul2_rn(R3, e);
        const float2 p = __fmul2_rn(w5, __fadd2_rn(t, l)), q = __fmul2_rn(w5, __ffma2_rn(l, m1, t));
        out[5] = p.x; out[6] = p.y; out[7] = q.x; out[8] = q.y;
    }
}

template <class R> __device__ __forceinline__ void feq9f(R rho, R ux, R uy, R out[NQ]) {
    feq9fd<R>(rho, rho, ux, uy, out);
}

// (u_x, u_y) from rho, rho u in the compute precision (FP32: one hardware reciprocal;
// FP64: two IEEE divisions).
template <class R> __device__ __forceinline__ void vel_of(R rho, R m1, R m2, R &ux, R &uy) {
    const R inv = recip<R>(rho);
    ux = m1 * inv;
    uy = m2 * inv;
}
template <> __device__ __forceinline__ void vel_of<double>(double rho, double m1, double m2, double &ux, double &uy) {
    ux = m1 / rho;
    uy = m2 / rho;
}

// Deviation form.  The FP32-compute kernels (FP32, bf16 and fp16 storage) store the
// conserved variables as W = (rho - 1, rho u_x, rho u_y) (FP64) and work with g = f - w,
// the distribution's deviation from the rest equilibrium of unit density, and with
// equilibria in the same form (feq9fd with b0 = rho - 1).  FP64 keeps W = (rho, rho u)
// and f itself.  Every step
// of the update is linear in f or uses a moment of it, and a constant field has no
// gradient and no net flux through a closed cell, so the update of g is the update of
// f with w taken out; but the face fluxes and their moments are then sums of small
// terms instead of differences of O(w) terms, and their FP32 rounding error shrinks in
// proportion (it sets the floor of the FP32 residual).
template <int P> struct Dev { static constexpr bool ON = P != P_FP64; };
// the density the stored W[0] is measured from: rho = rho_ref + W[0]
template <int P> __host__ __device__ constexpr double rho_ref() { return P == P_FP64 ? 0.0 : 1.0; }

// Storage codecs.  FP64 stores f; FP32 stores g = f - w.  BF16DEV stores the scaled
// deviation d = (f - feq(W)) / w from the equilibrium of the same time level (the feq
// passed is in the kernel's form, so dec returns g and enc takes g).
template <int P> struct Store;
template <> struct Store<P_FP64> {
    using T = double; using R = double;
    static __device__ __forceinline__ R dec(T v, R, int) { return v; }
    static __device__ __forceinline__ T enc(R f, R, int) { return f; }
};
template <> struct Store<P_FP32> {
    using T = float; using R = float;
    static __device__ __forceinline__ R dec(T v, R, int) { return v; }
    static __device__ __forceinline__ T enc(R f, R, int) { return f; }
};
template <> struct Store<P_BF16DEV> {
    using T = __nv_bfloat16; using R = float;
    static __device__ __forceinline__ R dec(T v, R feq, int a) { return feq + wq<R>(a) * __bfloat162float(v); }
    static __device__ __forceinline__ T enc(R f, R feq, int a) { return __float2bfloat16_rn((f - feq) * inv_wq<R>(a)); }
};
// FP16DEV stores d / s with the power of two s = 2^-10: binary16 keeps 11 significant
// bits over [6.1e-5, 65504], so scaled deviations |d| from 6e-8 to 64 stay normal.
constexpr float FP16DEV_SCALE = 1.0f / 1024.0f;
template <> struct Store<P_FP16DEV> {
    using T = __half; using R = float;
    static __device__ __forceinline__ R dec(T v, R feq, int a) {
        return feq + (wq<R>(a) * FP16DEV_SCALE) * __half2float(v);
    }
    static __device__ __forceinline__ T enc(R f, R feq, int a) {
        return __float2half_rn((f - feq) * (inv_wq<R>(a) * (1.0f / FP16DEV_SCALE)));
    }
};

// IEEE-754 format conversions by field arithmetic on the integer pipe (the FP64 unit of
// this GPU is narrow, and the FP32 kernels only need FP32 copies of the FP64 W).
// binary64 -> binary32: the exponent field is rebiased by 896 and the mantissa is
// truncated to 23 bits (error < 1 ulp of binary32); magnitudes below the binary32
// normal range become signed zero.  Intended for the finite, normal-range conserved
// variables: NaN and values beyond the binary32 range give unspecified finite results
// (the FP64 W they come from keeps the NaN, which the residual reduction reports).
__device__ __forceinline__ float d2f_fields(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned s = hi & 0x80000000u, a = hi & 0x7fffffffu;
    const unsigned m = ((a - 0x38000000u) << 3) | (lo >> 29);
    return __uint_as_float(a < 0x38100000u ? s : (s | m));
}
// binary32 -> binary64, exact for normal numbers, zero, infinity and NaN; binary32
// subnormals (below 1.2e-38) become signed zero.
__device__ __forceinline__ double f2d_fields(float f)
{
    const unsigned u = __float_as_uint(f), s = u & 0x80000000u, a = u & 0x7fffffffu;
    unsigned hi = s | ((a >> 3) + 0x38000000u), lo = a << 29;
    if (a < 0x00800000u) { hi = s; lo = 0u; }
    if (a >= 0x7f800000u) { hi = s | 0x7ff00000u | (a > 0x7f800000u ? 0x80000u : 0u); lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}
template <class R> __device__ __forceinline__ R from_f64(double d) { return R(d); }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return d2f_fields(d); }
template <class R> __device__ __forceinline__ double to_f64(R x) { return double(x); }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return f2d_fields(x); }

// Stored conserved variables -> rho - 1, rho and u in the compute precision.  FP32
// compute: W = (rho - 1, rho u); rho - 1 converted from FP64 keeps its own relative
// precision.  FP64: W = (rho, rho u) (drho is then rho - 1 rounded, unused by the
// FP64 kernels).
template <class R> __device__ __forceinline__ void macro_of(double w0, double w1, double w2, R &drho, R &rho, R &ux,
                                                           R &uy) {
    drho = from_f64<R>(w0);
    rho = R(1) + drho;
    vel_of<R>(rho, from_f64<R>(w1), from_f64<R>(w2), ux, uy);
}
template <> __device__ __forceinline__ void macro_of<double>(double w0, double w1, double w2, double &drho,
                                                             double &rho, double &ux, double &uy) {
    rho = w0;
    drho = w0 - 1.0;
    ux = w1 / w0;
    uy = w2 / w0;
}

}  // namespace sdugks
