// ahs_device.cuh -- device helpers shared by the engine's kernels: the gauge-
// invariant link phase and plaquette wrap of the winding count, and site indexing.
#pragma once

#include "ahs_internal.cuh"

namespace eng {

constexpr float kPiF = 3.14159265358979f;
constexpr float kTwoPiF = 6.28318530717959f;
constexpr float kInvTwoPiF = 0.159154943091895f;
constexpr double kPiD = 3.141592653589793238;
// A float32 complex number whose imaginary part exceeds kTie times its real part
// has the same sign as its FP64 counterpart, so its arg lies on the same side of the
// branch cut: the float32 link phase conj(p) U q is within 5e-7 |z| of the exact one
// (link phases V within 1.5e-7, two rounded complex products), a plaquette product
// of four link phases within 7e-7, a margin of at least 14 below kTie.  Closer to the
// cut the value is recomputed in FP64.
constexpr float kTie = 1e-5f;

// ---------------------------------------------------------------- index checks
// The bounds-check build of the library (-DAHS_BOUNDS_CHECK, _ahs_check.so) checks
// every global offset of the step kernels' tile loaders, rings and stores and every
// shared-memory index of their tiles against the extent it addresses.  An index
// outside it is counted in g_bounds_errors (one counter per translation unit, read
// by ahs_bounds_check) and replaced by 0, so the access stays in range: nothing
// traps, and nothing is read or written outside its array.  The production build
// compiles the checks away.
#ifdef AHS_BOUNDS_CHECK
static __device__ unsigned long long g_bounds_errors;
static __device__ __forceinline__ uint32_t checked_index(uint32_t i, uint32_t n)
{
    if (i >= n) {
        atomicAdd(&g_bounds_errors, 1ull);
        return 0u;
    }
    return i;
}
static __device__ __forceinline__ int checked_index(int i, int n)
{
    if (i < 0 || i >= n) {
        atomicAdd(&g_bounds_errors, 1ull);
        return 0;
    }
    return i;
}
#define AHS_INDEX(i, n) ::eng::checked_index((i), (n))
// host side: this translation unit's counter on the current device (read, then
// zeroed if reset), and a self-test launch that passes one index outside its extent
// through the check (touching no memory)
static __global__ void bounds_selftest_kernel()
{
    (void)checked_index(7, 3);
}
#define AHS_BOUNDS_COUNTER(name)                                                                     \
    cudaError_t name(unsigned long long *count, int op)                                            \
    {                                                                                              \
        if (op == 2) {                                                                             \
            bounds_selftest_kernel<<<1, 1>>>();                                                    \
            cudaError_t e = cudaDeviceSynchronize();                                               \
            if (e != cudaSuccess) return e;                                                        \
        }                                                                                          \
        cudaError_t e = cudaMemcpyFromSymbol(count, g_bounds_errors, sizeof(*count));              \
        if (e != cudaSuccess || op == 0) return e;                                                 \
        const unsigned long long zero = 0;                                                         \
        return cudaMemcpyToSymbol(g_bounds_errors, &zero, sizeof(zero));                           \
    }
#else
#define AHS_INDEX(i, n) (i)
#define AHS_BOUNDS_COUNTER(name)                                                                     \
    cudaError_t name(unsigned long long *count, int)                                               \
    {                                                                                              \
        *count = 0;                                                                                \
        return cudaErrorNotSupported;                                                              \
    }
#endif

// ---------------------------------------------------------------- link phases
// (cos th, sin th) of a link angle (Eq. 13) without the library sincosf: th is
// reduced to r = th - k pi, |r| <= pi/2, k = rint(th / pi), with pi split into two
// float32 parts (Cody & Waite, "Software Manual for the Elementary Functions",
// 1980) so that the fused multiply-adds leave r accurate to about an ulp for
// |th| up to ~1e5; then sin r = r + r^3 S(r^2) and cos r = 1 + r^2 C(r^2) with the
// near-minimax polynomials of gen_link_sincos.py (degrees 9 and 10), and both
// change sign for odd k.  Error: at most 1.3e-7 (sin) and 1.5e-7 (cos) absolute,
// i.e. 1-2 ulp of values near 1; |V|^2 - 1 is unbiased to 4e-9.  No branches, no
// special-function unit and no conversion: 16 instructions on the FMA and ALU pipes.
constexpr float kLinkS0 = -0.16666659712791443f, kLinkS1 = 0.00833306647837162f,
                kLinkS2 = -0.0001980959059437737f, kLinkS3 = 2.605750751172309e-06f;
constexpr float kLinkC0 = -0.5f, kLinkC1 = 0.04166664183139801f, kLinkC2 = -0.00138884037733078f,
                kLinkC3 = 2.476187000866048e-05f, kLinkC4 = -2.607681608424173e-07f;
constexpr float kLinkInvPi = 0.31830987334251404f;   // float32(1/pi)
constexpr float kLinkPiA = 3.1415927410125732f;      // float32(pi)
constexpr float kLinkPiB = -8.742277657347586e-08f;  // float32(pi - kLinkPiA)
constexpr float kLinkRound = 12582912.0f;             // 1.5 * 2^23

static __device__ __forceinline__ void link_sincos(float th, float &s, float &c)
{
    // k = rint(th / pi) by the rounding of one fused multiply-add: t = 1.5 * 2^23 +
    // th / pi lies in [2^23, 2^24) for |th| < 2^22 pi, where float32 spacing is 1,
    // so t - 1.5 * 2^23 is the nearest integer and t's last bit is k's parity
    const float t = fmaf(th, kLinkInvPi, kLinkRound);
    const float k = t - kLinkRound;
    float r = fmaf(-k, kLinkPiA, th);
    r = fmaf(-k, kLinkPiB, r);
    const float r2 = r * r;
    float ps = fmaf(r2, kLinkS3, kLinkS2);
    ps = fmaf(r2, ps, kLinkS1);
    ps = fmaf(r2, ps, kLinkS0);
    float pc = fmaf(r2, kLinkC4, kLinkC3);
    pc = fmaf(r2, pc, kLinkC2);
    pc = fmaf(r2, pc, kLinkC1);
    pc = fmaf(r2, pc, kLinkC0);
    const float sv = fmaf(r * r2, ps, r);
    const float cv = fmaf(r2, pc, 1.0f);
    const unsigned flip = __float_as_uint(t) << 31;   // (-1)^k as a sign bit
    s = __uint_as_float(__float_as_uint(sv) ^ flip);
    c = __uint_as_float(__float_as_uint(cv) ^ flip);
}

// The FP64 precision mode's link phases, built the same way in double: pi in two
// FP64 parts, sin r = r + r^3 S(r^2) and cos r = 1 + r^2 C(r^2) of degrees 17 and
// 16 (gen_link_sincos.py --double; fit errors 3e-19 and 4e-18), sign flipped for
// odd k.  Error about 1 ulp of values near 1 for |th| up to ~1e5; 24 FP64
// instructions, no branches and no conversion.
__device__ constexpr double kLinkS64[8] = {-0.16666666666666666,     0.008333333333333194,   -0.0001984126984120922,
                                2.7557319211137538e-06,   -2.505210687282421e-08, 1.6058939706909938e-10,
                                -7.642991513761023e-13,   2.7211752032504598e-15};
__device__ constexpr double kLinkC64[8] = {-0.49999999999999983,     0.04166666666666437,    -0.0013888888888785656,
                                2.480158727914948e-05,    -2.755731652526679e-07, 2.087656774286206e-09,
                                -1.1463039414469496e-11,  4.610294611228809e-14};
constexpr double kLinkInvPi64 = 0.3183098861837907;        // double(1/pi)
constexpr double kLinkPiA64 = 3.141592653589793;           // double(pi)
constexpr double kLinkPiB64 = 1.2246467991473532e-16;      // double(pi - kLinkPiA64)
constexpr double kLinkRound64 = 6755399441055744.0;         // 1.5 * 2^52

static __device__ __forceinline__ void link_sincos(double th, double &s, double &c)
{
    // k = rint(th / pi) and its parity from one fused multiply-add, as in float32
    const double t = fma(th, kLinkInvPi64, kLinkRound64);
    const double k = t - kLinkRound64;
    double r = fma(-k, kLinkPiA64, th);
    r = fma(-k, kLinkPiB64, r);
    const double r2 = r * r;
    double ps = kLinkS64[7], pc = kLinkC64[7];
#pragma unroll
    for (int i = 6; i >= 0; --i) {
        ps = fma(r2, ps, kLinkS64[i]);
        pc = fma(r2, pc, kLinkC64[i]);
    }
    const double sv = fma(r * r2, ps, r);
    const double cv = fma(r2, pc, 1.0);
    const unsigned long long flip = (unsigned long long)__double_as_longlong(t) << 63;
    s = __longlong_as_double(__double_as_longlong(sv) ^ (long long)flip);
    c = __longlong_as_double(__double_as_longlong(cv) ^ (long long)flip);
}

// ---------------------------------------------------------------- windings
// Y_i(x) = arg(phi^*(x) U_i(x) phi(x+i)), U_i = exp(-i theta_i).
template <class In>
static __device__ __noinline__ double link_phase_fp64(In pr, In pi, In qr, In qi, In th)
{
    double s, c;
    sincos((double)th, &s, &c);
    double ur = c, ui = -s;
    double hr = __dsub_rn(__dmul_rn(ur, (double)qr), __dmul_rn(ui, (double)qi));
    double hi = __dadd_rn(__dmul_rn(ur, (double)qi), __dmul_rn(ui, (double)qr));
    double zr = __dsub_rn(__dmul_rn((double)pr, hr), __dmul_rn(-(double)pi, hi));
    double zi = __dadd_rn(__dmul_rn((double)pr, hi), __dmul_rn(-(double)pi, hr));
    return atan2(zi, zr);
}

// [alpha]_pi of alpha = a + b - c - d: wrapped into (-pi, pi] by
// alpha + 2 pi floor((pi - alpha)/(2 pi)).
template <class In>
static __device__ __noinline__ double wrap_plaq_fp64(In a, In b, In c, In d)
{
    double al = __dsub_rn(__dsub_rn(__dadd_rn((double)a, (double)b), (double)c), (double)d);
    double k = floor(__ddiv_rn(__dsub_rn(kPiD, al), 2.0 * kPiD));
    return __dadd_rn(al, __dmul_rn(2.0 * kPiD, k));
}

// true when the complex number z = (zr, zi) is too close to the branch cut of arg
// (the negative real axis, or z = 0) for the sign of its computed imaginary part to
// decide the branch (float32; FP64 fields use the same margin): zr <= 0 and
// |zi| <= kTie |zr|, evaluated as the one fused multiply-add kTie zr + |zi| <= 0
// (which also flags a positive zr so small that kTie zr underflows while zi = 0: a
// flag only sends the value to the FP64 path)
template <class R>
static __device__ __forceinline__ bool near_cut(R zr, R zi)
{
    return fma(R(kTie), zr, fabs(zi)) <= R(0);
}

// Octant code o of an angle in (-pi, pi]: the angle lies in [o pi/4, (o+1) pi/4],
// o in -4..3, and o pi/4 + pi/8 is within pi/8 of it.  From a complex number: the
// signs of its parts and which is larger in magnitude; from an FP64 angle: floor.
// A float32 number can get a different code than its exact value only within its
// rounding (~1e-6 rad) of an octant boundary, and then a neighbouring one, so the
// centre stays within pi/8 + 1e-6 of the exact angle; at the branch cut (+-pi) a
// wrong sign would move it by 2 pi instead, which the near_cut fallback rules out.
template <class R>
static __device__ __forceinline__ int octant(R zr, R zi)
{
    const bool steep = fabs(zi) > fabs(zr);
    if (zi >= R(0)) return zr >= R(0) ? (steep ? 1 : 0) : (steep ? 2 : 3);
    return zr >= R(0) ? (steep ? -2 : -1) : (steep ? -3 : -4);
}
static __device__ __forceinline__ int octant(double a)
{
    const int o = (int)floor(a * (4.0 / kPiD));
    return o < -4 ? -4 : o > 3 ? 3 : o;
}

// Y_i(x) from a precomputed link phase V_i = (cos theta_i, sin theta_i) = conj(U_i),
// as an octant code; the FP64 fallback recomputes from theta_i, which the caller
// loads only then.
template <class R, class ThetaFn>
static __device__ __forceinline__ int link_phase_v(R pr, R pi, R qr, R qi, R vc, R vs, ThetaFn theta)
{
    const R hr = vc * qr + vs * qi;   // U_i q with U_i = vc - i vs
    const R hi = vc * qi - vs * qr;
    const R zr = pr * hr + pi * hi;   // conj(p) U_i q
    const R zi = pr * hi - pi * hr;
    if (near_cut(zr, zi)) return octant(link_phase_fp64(pr, pi, qr, qi, theta()));
    return octant(zr, zi);
}

// [alpha]_pi from the plaquette product Q = exp(i alpha) (Eq. 15 conjugated), as an
// octant code; the FP64 fallback recomputes alpha = a + b - c - d from the four
// link angles.
template <class R, class AnglesFn>
static __device__ __forceinline__ int wrap_from_q(R qr, R qi, AnglesFn angles)
{
    if (near_cut(qr, qi)) {
        R a, b, c, d;
        angles(a, b, c, d);
        return octant(wrap_plaq_fp64(a, b, c, d));
    }
    return octant(qr, qi);
}

// W = (Y1 + Y2 - Y3 - Y4 + [alpha]_pi) / 2 pi is an integer (the five phases add
// up to the argument of a positive real number); with each angle replaced by its
// octant centre (o + 1/2) pi/4 the sum is off by at most 5 (pi/8 + 1e-6) < pi, so
// W is the integer nearest to (2T + 1)/16, T = o1 + o2 - o3 - o4 + o_alpha, i.e.
// floor((2T + 9)/16) (never a tie: 2T + 1 is odd).
static __device__ __forceinline__ int winding(int o1, int o2, int o3, int o4, int oa)
{
    const int t = o1 + o2 - o3 - o4 + oa;
    return (2 * t + 9) >> 4;
}

// ---------------------------------------------------------------- flagged codes
// The fused measurement keeps each angle as a flagged code: bits 0-2 its octant + 4
// (0..7, from the float value), bit 3 set when the value is too close to the branch
// cut for that octant to be trusted (near_cut).  A plaquette whose five codes carry
// no flag has the winding winding_codes gives; a site any of whose phases is flagged
// (a few in 10^4 sites) recomputes the flagged ones in FP64 (site_windings_flagged).
// Both give the winding of the definition: the octants of the exact angles agree with
// these to within one octant, which the pi/5 margin of winding() absorbs, and at the
// cut FP64 decides.
// The code without branches: with b = (zr < 0) and s = (|zi| > |zr|), octant + 4 is
// 4 + 2b + (b xor s) for zi >= 0 (4, 5 in the first quadrant, 7, 6 in the second),
// and conjugation maps octant o to -1 - o, i.e. code c to 7 - c -- the same codes as
// octant() + 4, signed zeros included.
template <class R>
static __device__ __forceinline__ int flagged_octant(R zr, R zi)
{
    const int b = zr < R(0), s = fabs(zi) > fabs(zr);
    const int c = 4 + 2 * b + (b ^ s);
    return (zi < R(0) ? 7 - c : c) | (near_cut(zr, zi) ? 8 : 0);
}

// Y_i(x) as a flagged code from V_i = (cos theta_i, sin theta_i): arg of conj(p) U_i q
template <class R>
static __device__ __forceinline__ int link_code(R pr, R pi, R qr, R qi, R vc, R vs)
{
    const R hr = vc * qr + vs * qi;   // U_i q with U_i = vc - i vs
    const R hi = vc * qi - vs * qr;
    const R zr = pr * hr + pi * hi;   // conj(p) U_i q
    const R zi = pr * hi - pi * hr;
    return flagged_octant(zr, zi);
}

// winding() of five codes without flags (the caller has checked that none is set,
// so each is its octant + 4); the offsets of 4 cancel in c1 + c2 - c3 - c4 and one
// is left from ca
static __device__ __forceinline__ int winding_codes(int c1, int c2, int c3, int c4, int ca)
{
    const int t = c1 + c2 - c3 - c4 + ca - 4;
    return (2 * t + 9) >> 4;
}

// Octant code of an FP64 complex number with the signs taken as atan2 takes them
// (a signed zero decides the side of the branch cut: arg(-1 + 0i) = pi, arg(-1 - 0i)
// = -pi), so no arctangent is needed.
static __device__ __forceinline__ int octant_signed(double zr, double zi)
{
    const bool steep = fabs(zi) > fabs(zr), ny = signbit(zi), nx = signbit(zr);
    if (!ny) return !nx ? (steep ? 1 : 0) : (steep ? 2 : 3);
    return !nx ? (steep ? -2 : -1) : (steep ? -3 : -4);
}

// The windings W_xy, W_xz, W_yz of the plaquettes with lower corner x from the flagged
// codes of their phases, each flagged phase recomputed in FP64 from the fields (planes
// pr, pi, tx, ty, tz of N^3 = V sites, read at the offsets o0 .. o6 of x, x+x, x+y,
// x+z, x+x+y, x+x+z, x+y+z): a link phase from the FP64 polynomial link phase of its
// angle and the FP64 product conj(p) U q, a plaquette angle by wrap_plaq_fp64 of its
// four link angles.  codes holds twelve 4-bit codes (code k in bits 4k..4k+3) in the
// order Y_x, Y_y, Y_z at x; Y_y at x+x; Y_x at x+y; Y_z at x+x; Y_z at x+y; Y_x at
// x+z; Y_y at x+z; alpha_xy, alpha_xz, alpha_yz.  The rare path of the fused
// measurement: plain pointers and values only, so that the caller keeps its field
// access in registers.
template <class In>
static __device__ __noinline__ int3 site_windings_flagged(const In *pr, const In *pim, const In *tx, const In *ty,
                                                          const In *tz, uint32_t V, uint32_t o0, uint32_t o1,
                                                          uint32_t o2, uint32_t o3, uint32_t o4, uint32_t o5,
                                                          uint32_t o6, unsigned long long codes)
{
    const uint32_t o[7] = {AHS_INDEX(o0, V), AHS_INDEX(o1, V), AHS_INDEX(o2, V), AHS_INDEX(o3, V),
                           AHS_INDEX(o4, V), AHS_INDEX(o5, V), AHS_INDEX(o6, V)};
    const In *th[3] = {tx, ty, tz};
    auto code = [&](int k) { return (int)((codes >> (4 * k)) & 15u); };
    auto Y = [&](int k, int a, int b, int f) {   // Y_f at site a, towards site b = a + f
        const int c = code(k);
        if (!(c & 8)) return (c & 7) - 4;
        double sn, cs;
        link_sincos((double)th[f][o[a]], sn, cs);
        const double p0 = pr[o[a]], p1 = pim[o[a]], q0 = pr[o[b]], q1 = pim[o[b]];
        const double hr = __dadd_rn(__dmul_rn(cs, q0), __dmul_rn(sn, q1));   // U q, U = cos - i sin
        const double hi = __dsub_rn(__dmul_rn(cs, q1), __dmul_rn(sn, q0));
        const double zr = __dadd_rn(__dmul_rn(p0, hr), __dmul_rn(p1, hi));   // conj(p) U q
        const double zi = __dsub_rn(__dmul_rn(p0, hi), __dmul_rn(p1, hr));
        return octant_signed(zr, zi);
    };
    auto A = [&](int k, int i, int j) {   // [alpha_ij]_pi at x: links i, j at x, x+i, x+j
        const int c = code(k);
        if (!(c & 8)) return (c & 7) - 4;
        const int oi = i == 0 ? 1 : 2, oj = j == 1 ? 2 : 3;   // x+i, x+j
        return octant(wrap_plaq_fp64(th[i][o[0]], th[j][o[oi]], th[i][o[oj]], th[j][o[0]]));
    };
    const int yx = Y(0, 0, 1, 0), yy = Y(1, 0, 2, 1), yz = Y(2, 0, 3, 2);
    int3 w;
    w.x = winding(yx, Y(3, 1, 4, 1), Y(4, 2, 4, 0), yy, A(9, 0, 1));
    w.y = winding(yx, Y(5, 1, 5, 2), Y(7, 3, 5, 0), yz, A(10, 0, 2));
    w.z = winding(yy, Y(6, 2, 6, 2), Y(8, 3, 6, 1), yz, A(11, 1, 2));
    return w;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): one step from state v.
static __device__ __forceinline__ uint64_t splitmix64_device(uint64_t v)
{
    uint64_t z = v + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static __device__ __forceinline__ size_t sidx(int x, int y, int z, int N)
{
    return (size_t)x + (size_t)N * ((size_t)y + (size_t)N * (size_t)z);
}

// ---------------------------------------------------------------- explicit roundings
// Arithmetic that the compiler may not contract into fused multiply-adds of its own
// choosing: the diagnostics of a measuring step are evaluated with these, so that
// every kernel that measures -- the fused measuring step, its batched form, the
// separate Gauss launch -- gives the same bits whatever the surrounding code.
static __device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
static __device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
static __device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
static __device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
static __device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
static __device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
static __device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
static __device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------- Gauss residual
// G(x) = sum_i (E_i(x) - E_i(x-i)) / dx - m_gauss Im(conj(phi) Pi) of one site (the
// stored momenta at n - 1/2 with phi^n), every rounding explicit.
template <class R>
static __device__ __forceinline__ R gauss_site(R ex, R exm, R ey, R eym, R ez, R ezm, R inv_dx, R m_gauss, R pr,
                                               R pim, R qr, R qi)
{
    const R div = rn_mul(rn_add(rn_add(rn_sub(ex, exm), rn_sub(ey, eym)), rn_sub(ez, ezm)), inv_dx);
    return rn_sub(div, rn_mul(m_gauss, rn_sub(rn_mul(pr, qi), rn_mul(pim, qr))));
}
template <class R>
static __device__ __forceinline__ R square_add(R g, R acc) { return rn_fma(g, g, acc); }

// ---------------------------------------------------------------- reduction
// per-thread sums of one tile: float32 (FP64 for the FP64 mode) along the z-march
template <class R>
struct AccT {
    R s[NSUM];
    R gmax;
    int wind, nf;
};
using Acc = AccT<float>;

template <class R>
static __device__ __forceinline__ void acc_zero(AccT<R> &a)
{
#pragma unroll
    for (int q = 0; q < NSUM; ++q) a.s[q] = R(0);
    a.gmax = R(0);
    a.wind = 0;
    a.nf = 0;
}

// Block reduction of the sums to one row of FP64 partials: in the sums' type within
// a warp, FP64 across warps in a fixed order (deterministic for a launch shape).
// which slots of the partial row a block writes
enum { ROW_ALL = 0, ROW_NO_GAUSS = 1, ROW_GAUSS_ONLY = 2 };

template <int NT, class R>
static __device__ void block_reduce_store(AccT<R> &a, double *out, int slots = ROW_ALL)
{
    constexpr int NW = NT / 32;
    __shared__ double red[NW][NQ];
    const int lane = threadIdx.x & 31;
    const int wid = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < NSUM; ++q) a.s[q] += __shfl_xor_sync(0xffffffffu, a.s[q], off);
        a.gmax = fmax(a.gmax, __shfl_xor_sync(0xffffffffu, a.gmax, off));
        a.wind += __shfl_xor_sync(0xffffffffu, a.wind, off);
        a.nf += __shfl_xor_sync(0xffffffffu, a.nf, off);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NSUM; ++q) red[wid][q] = (double)a.s[q];
        red[wid][Q_GMAX] = (double)a.gmax;
        red[wid][Q_WIND] = (double)a.wind;
        red[wid][Q_NF] = (double)a.nf;
        red[wid][14] = 0.0;
        red[wid][15] = 0.0;
    }
    __syncthreads();
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    const bool gauss_slot = t == Q_G2 || t == Q_GMAX;
    if (t < NQ && (slots == ROW_ALL || (slots == ROW_NO_GAUSS) != gauss_slot)) {
        double v = red[0][t];
        for (int w = 1; w < NW; ++w) v = (t == Q_GMAX) ? fmax(v, red[w][t]) : v + red[w][t];
        out[t] = v;
    }
}

}  // namespace eng
