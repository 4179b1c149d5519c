// ahs_stencil.cuh -- building blocks of the z-marching step kernels: the storage
// type of a kernel instance, field access of one step (kernel-parameter pointers
// or a batch member's arena), complex products, the plaquette of Eq. 15 as a
// product of link phases, and the compensated momentum update.
#pragma once

#include "ahs_device.cuh"

#include <cstddef>
#include <type_traits>

namespace eng {
namespace {

// Storage and arithmetic type of a kernel instance: float32 (the default path) or
// FP64 (the reference precision mode) -- its complex pair, coefficients and link
// phases (the polynomial link_sincos of that precision).
template <class R>
struct Real;
template <>
struct Real<float> {
    using V2 = float2;
    using Coef = StepCoef;
    static __device__ __forceinline__ float2 v2(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ void link(float th, float &s, float &c) { link_sincos(th, s, c); }
};
template <>
struct Real<double> {
    using V2 = double2;
    using Coef = StepCoef64;
    static __device__ __forceinline__ double2 v2(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ void link(double th, double &s, double &c) { link_sincos(th, s, c); }
};

template <class R>
struct Raw {
    R tx, ty, tz, pr, pi;
};

template <class R>
struct PE {
    R qr, qi, ex, ey, ez;
    R qrl, qil, exl, eyl, ezl;   // low words (compensated precision)
};

__device__ __forceinline__ int wrapN(int v, int N)
{
    v %= N;
    return v < 0 ? v + N : v;
}

// Field access of one step, in the plane order of a buffer: 0 Re phi, 1 Im phi,
// 2 Re Pi, 3 Im Pi, 4-6 theta_xyz, 7-9 E_xyz; `in` reads the time-n buffer,
// `out` writes the n+1 buffer.  ParamFields takes the twenty plane pointers of a
// single lattice (kernel parameters, constant bank); ArenaFields addresses the
// two buffers of one member of a batch from one base pointer with 32-bit plane
// offsets (requires 20 N^3 < 2^32).
enum { FPR = 0, FPI, FQR, FQI, FTX, FTY, FTZ, FEX, FEY, FEZ, FQRL, FQIL, FEXL, FEYL, FEZL };

struct ParamFields {
    using real = float;
    const StepPtrs &P;
    uint32_t V;   // sites per plane (N^3): the extent of the bounds-check build's offset checks
    __device__ __forceinline__ const float *src(int f) const
    {
        return f == FPR ? P.pr : f == FPI ? P.pim : f == FQR ? P.qr : f == FQI ? P.qi : f == FTX ? P.tx
             : f == FTY ? P.ty : f == FTZ ? P.tz : f == FEX ? P.ex : f == FEY ? P.ey : f == FEZ ? P.ez
             : f == FQRL ? P.qrl : f == FQIL ? P.qil : f == FEXL ? P.exl : f == FEYL ? P.eyl : P.ezl;
    }
    __device__ __forceinline__ float *dst(int f) const
    {
        return f == FPR ? P.pr1 : f == FPI ? P.pim1 : f == FQR ? P.qr1 : f == FQI ? P.qi1 : f == FTX ? P.tx1
             : f == FTY ? P.ty1 : f == FTZ ? P.tz1 : f == FEX ? P.ex1 : f == FEY ? P.ey1 : f == FEZ ? P.ez1
             : f == FQRL ? P.qrl1 : f == FQIL ? P.qil1 : f == FEXL ? P.exl1 : f == FEYL ? P.eyl1 : P.ezl1;
    }
    __device__ __forceinline__ float in(int f, uint32_t o) const { return __ldg(src(f) + AHS_INDEX(o, V)); }
    __device__ __forceinline__ void out(int f, uint32_t o, float v) const { dst(f)[AHS_INDEX(o, V)] = v; }
    // sites o and o+1 as one 8-byte access (o even, planes 8-byte aligned)
    __device__ __forceinline__ float2 in2(int f, uint32_t o) const
    {
        return __ldg(reinterpret_cast<const float2 *>(src(f) + AHS_INDEX(o, V - 1)));
    }
    __device__ __forceinline__ void out2(int f, uint32_t o, float a, float b) const
    {
        *reinterpret_cast<float2 *>(dst(f) + AHS_INDEX(o, V - 1)) = make_float2(a, b);
    }
};

struct ArenaFields {
    using real = float;
    const float *base;       // the member's first plane (buffer 0, Re phi)
    uint32_t in0, out0, V;   // plane offsets of the read and write buffers, plane size
    __device__ __forceinline__ const float *src(int f) const { return base + (in0 + (uint32_t)f * V); }
    __device__ __forceinline__ float in(int f, uint32_t o) const
    {
        return __ldg(base + (in0 + (uint32_t)f * V + AHS_INDEX(o, V)));
    }
    __device__ __forceinline__ void out(int f, uint32_t o, float v) const
    {
        const_cast<float *>(base)[out0 + (uint32_t)f * V + AHS_INDEX(o, V)] = v;
    }
    // sites o and o+1 as one 8-byte access (o even; every member's planes start on
    // an 8-byte boundary when its N is even)
    __device__ __forceinline__ float2 in2(int f, uint32_t o) const
    {
        return __ldg(reinterpret_cast<const float2 *>(base + (in0 + (uint32_t)f * V + AHS_INDEX(o, V - 1))));
    }
    __device__ __forceinline__ void out2(int f, uint32_t o, float a, float b) const
    {
        *reinterpret_cast<float2 *>(const_cast<float *>(base) + (out0 + (uint32_t)f * V + AHS_INDEX(o, V - 1))) =
            make_float2(a, b);
    }
};

// the twenty FP64 planes of a single lattice in FP64 precision (no low words)
struct ParamFields64 {
    using real = double;
    const StepPtrs64 &P;
    uint32_t V;   // sites per plane (N^3)
    __device__ __forceinline__ const double *src(int f) const
    {
        return f == FPR ? P.pr : f == FPI ? P.pim : f == FQR ? P.qr : f == FQI ? P.qi : f == FTX ? P.tx
             : f == FTY ? P.ty : f == FTZ ? P.tz : f == FEX ? P.ex : f == FEY ? P.ey : P.ez;
    }
    __device__ __forceinline__ double in(int f, uint32_t o) const { return __ldg(src(f) + AHS_INDEX(o, V)); }
    __device__ __forceinline__ void out(int f, uint32_t o, double v) const
    {
        double *p = f == FPR ? P.pr1 : f == FPI ? P.pim1 : f == FQR ? P.qr1 : f == FQI ? P.qi1 : f == FTX ? P.tx1
                  : f == FTY ? P.ty1 : f == FTZ ? P.tz1 : f == FEX ? P.ex1 : f == FEY ? P.ey1 : P.ez1;
        p[AHS_INDEX(o, V)] = v;
    }
};

template <class FA>
__device__ __forceinline__ Raw<typename FA::real> load_raw(const FA &P, uint32_t o)
{
    Raw<typename FA::real> a;
    a.tx = P.in(FTX, o);
    a.ty = P.in(FTY, o);
    a.tz = P.in(FTZ, o);
    a.pr = P.in(FPR, o);
    a.pi = P.in(FPI, o);
    return a;
}

template <bool COMP, class FA>
__device__ __forceinline__ PE<typename FA::real> load_pe(const FA &P, uint32_t o)
{
    PE<typename FA::real> a;
    a.qr = P.in(FQR, o);
    a.qi = P.in(FQI, o);
    a.ex = P.in(FEX, o);
    a.ey = P.in(FEY, o);
    a.ez = P.in(FEZ, o);
    if constexpr (COMP) {
        a.qrl = P.in(FQRL, o);
        a.qil = P.in(FQIL, o);
        a.exl = P.in(FEXL, o);
        a.eyl = P.in(FEYL, o);
        a.ezl = P.in(FEZL, o);
    } else {
        a.qrl = a.qil = a.exl = a.eyl = a.ezl = 0;
    }
    return a;
}

// Compensated damped update of one momentum component held as hi + lo:
// (hi', lo') = c (hi + lo) + d with the rounding errors of the product c hi (by
// FMA) and of the sum (TwoSum, Knuth) carried in the low word, then renormalised
// (Fast2Sum, Dekker).
__device__ __forceinline__ void comp_update(float c, float hi, float lo, float d, float &nhi, float &nlo)
{
    const float p = c * hi;
    const float e1 = fmaf(c, hi, -p);
    const float s = p + d;
    const float bb = s - p;
    const float e2 = (p - (s - bb)) + (d - bb);
    const float l = fmaf(c, lo, e1 + e2);
    nhi = s + l;
    nlo = l - (nhi - s);
}

// complex helpers: a * b and a * conj(b)
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b)
{
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Q = V_i(x) conj(V_j(x)) * V_j(x+i) conj(V_i(x+j)); the last product's roundings are
// explicit, since its real part (cos of the plaquette) is a diagnostic only
template <class V2>
__device__ __forceinline__ V2 plaquette(V2 vi, V2 vj, V2 vjp, V2 vip)
{
    const V2 a = cmulc(vi, vj), b = cmulc(vjp, vip);
    V2 q;
    q.x = rn_fma(a.x, b.x, -rn_mul(a.y, b.y));
    q.y = rn_fma(a.x, b.y, rn_mul(a.y, b.x));
    return q;
}

__device__ __forceinline__ int next_plane(int z, int N) { return z + 1 == N ? 0 : z + 1; }

}  // namespace
}  // namespace eng
