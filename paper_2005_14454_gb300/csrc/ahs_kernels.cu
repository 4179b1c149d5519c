// ahs_kernels.cu -- sm_103a kernels of the lattice Abelian-Higgs engine.
//
// The step kernel fuses the kick of Eqs. 7-8 (covariant Laplacian of Eq. 14,
// compact plaquette curl of Eqs. 15-16, current Im[phi^* D^+ phi]) with the
// drift of Eqs. 9-10, and on measurement steps the diagnostics of Eqs. diagxi /
// diagvel plus the Gauss residual, reduced to FP64 block partials.
#include "ahs_internal.cuh"

#include <cmath>

namespace eng {

namespace {

constexpr float kPiF = 3.14159265358979f;
constexpr float kTwoPiF = 6.28318530717959f;
constexpr float kInvTwoPiF = 0.159154943091895f;
constexpr double kPiD = 3.141592653589793238;
// Below pi - kTie the float32 branch decision of atan2 / of the wrap is the same
// as the FP64 one (the float32 error is < 1e-6 rad); at and above it the value is
// recomputed in FP64 with the operations in the order of the definition.
constexpr float kTie = 1e-4f;

// ---------------------------------------------------------------- windings
// Y_i(x) = arg(phi^*(x) U_i(x) phi(x+i)), U_i = exp(-i theta_i).
__device__ __noinline__ double link_phase_fp64(float pr, float pi, float qr, float qi, float th)
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

__device__ __forceinline__ float link_phase(float pr, float pi, float qr, float qi, float th)
{
    float s, c;
    sincosf(th, &s, &c);
    float hr = c * qr + s * qi;
    float hi = c * qi - s * qr;
    float zr = pr * hr + pi * hi;
    float zi = pr * hi - pi * hr;
    float y = atan2f(zi, zr);
    if (fabsf(y) > kPiF - kTie) y = (float)link_phase_fp64(pr, pi, qr, qi, th);
    return y;
}

// [alpha]_pi of alpha = a + b - c - d: wrapped into (-pi, pi] by
// alpha + 2 pi floor((pi - alpha)/(2 pi)).
__device__ __noinline__ double wrap_plaq_fp64(float a, float b, float c, float d)
{
    double al = __dsub_rn(__dsub_rn(__dadd_rn((double)a, (double)b), (double)c), (double)d);
    double k = floor(__ddiv_rn(__dsub_rn(kPiD, al), 2.0 * kPiD));
    return __dadd_rn(al, __dmul_rn(2.0 * kPiD, k));
}

__device__ __forceinline__ float wrap_plaq(float a, float b, float c, float d)
{
    float al = ((a + b) - c) - d;
    float w = al + kTwoPiF * floorf((kPiF - al) * kInvTwoPiF);
    float mag = fabsf(a) + fabsf(b) + fabsf(c) + fabsf(d);
    if (fabsf(w) > kPiF - (kTie + 1e-6f * mag)) w = (float)wrap_plaq_fp64(a, b, c, d);
    return w;
}

__device__ __forceinline__ int winding(float y1, float y2, float y3, float y4, float aw)
{
    float sum = ((((y1 + y2) - y3) - y4) + aw);
    return __float2int_rn(sum * kInvTwoPiF);
}

__device__ __forceinline__ size_t sidx(int x, int y, int z, int N)
{
    return (size_t)x + (size_t)N * ((size_t)y + (size_t)N * (size_t)z);
}

// ---------------------------------------------------------------- reduction
struct Acc {
    float s[NSUM];
    float gmax;
    int wind, nf;
};

__device__ __forceinline__ void acc_zero(Acc &a)
{
#pragma unroll
    for (int q = 0; q < NSUM; ++q) a.s[q] = 0.f;
    a.gmax = 0.f;
    a.wind = 0;
    a.nf = 0;
}

// Block reduction of Acc to one row of FP64 partials: float32 within a warp,
// FP64 across warps in a fixed order (deterministic for a fixed launch shape).
template <int NT>
__device__ void block_reduce_store(Acc &a, double *out)
{
    constexpr int NW = NT / 32;
    __shared__ double red[NW][NQ];
    const int lane = threadIdx.x & 31;
    const int wid = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < NSUM; ++q) a.s[q] += __shfl_xor_sync(0xffffffffu, a.s[q], off);
        a.gmax = fmaxf(a.gmax, __shfl_xor_sync(0xffffffffu, a.gmax, off));
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
    if (t < NQ) {
        double v = red[0][t];
        for (int w = 1; w < NW; ++w) v = (t == Q_GMAX) ? fmax(v, red[w][t]) : v + red[w][t];
        out[t] = v;
    }
}

// ---------------------------------------------------------------- step kernel
// One thread per (x, y) column of a 32 x 8 tile, looping over a chunk of z.
constexpr int BX = 32, BY = 8, NT = BX * BY, ZCHUNK = 16;

template <bool MEASURE, bool STORE>
__global__ void __launch_bounds__(NT) step_kernel(StepPtrs P, StepCoef k, int N, double *partials)
{
    const int x = blockIdx.x * BX + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    const bool active = (x < N) && (y < N);
    const int z0 = blockIdx.z * ZCHUNK;
    const int z1 = min(z0 + ZCHUNK, N);

    Acc acc;
    if (MEASURE) acc_zero(acc);

    if (active) {
        const int xm = (x == 0) ? N - 1 : x - 1, xp = (x == N - 1) ? 0 : x + 1;
        const int ym = (y == 0) ? N - 1 : y - 1, yp = (y == N - 1) ? 0 : y + 1;
        for (int z = z0; z < z1; ++z) {
            const int zm = (z == 0) ? N - 1 : z - 1, zp = (z == N - 1) ? 0 : z + 1;
            const size_t s = sidx(x, y, z, N);
            const size_t sxp = sidx(xp, y, z, N), sxm = sidx(xm, y, z, N);
            const size_t syp = sidx(x, yp, z, N), sym = sidx(x, ym, z, N);
            const size_t szp = sidx(x, y, zp, N), szm = sidx(x, y, zm, N);

            const float p0r = __ldg(P.pr + s), p0i = __ldg(P.pim + s);
            const float tx0 = __ldg(P.tx + s), ty0 = __ldg(P.ty + s), tz0 = __ldg(P.tz + s);

            // covariant Laplacian (Eq. 14) and link currents J_i = Im(phi^* U_i phi(x+i))
            float hsr = 0.f, hsi = 0.f;
            float J[3], Hr[3], Hi[3];
            {
                const float th0[3] = {tx0, ty0, tz0};
                const float *T[3] = {P.tx, P.ty, P.tz};
                const size_t sp[3] = {sxp, syp, szp}, sm[3] = {sxm, sym, szm};
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float sn, cs;
                    sincosf(th0[i], &sn, &cs);
                    const float qr = __ldg(P.pr + sp[i]), qi = __ldg(P.pim + sp[i]);
                    const float hr = cs * qr + sn * qi;          // U_i(x) phi(x+i)
                    const float hi = cs * qi - sn * qr;
                    Hr[i] = hr;
                    Hi[i] = hi;
                    J[i] = p0r * hi - p0i * hr;
                    float sn2, cs2;
                    sincosf(__ldg(T[i] + sm[i]), &sn2, &cs2);
                    const float mr = __ldg(P.pr + sm[i]), mi = __ldg(P.pim + sm[i]);
                    hsr += hr + (cs2 * mr - sn2 * mi);           // U_i(x-i)^* phi(x-i)
                    hsi += hi + (cs2 * mi + sn2 * mr);
                }
            }
            const float mod2 = p0r * p0r + p0i * p0i;
            const float q0r = __ldg(P.qr + s), q0i = __ldg(P.qi + s);
            const float potf = k.kpi_pot * (mod2 - k.sigma2);
            const float qnr = k.cpi * q0r + k.kpi_lap * (hsr - 6.f * p0r) - potf * p0r;
            const float qni = k.cpi * q0i + k.kpi_lap * (hsi - 6.f * p0i) - potf * p0i;

            // plaquette sines alpha_ij(b) = th_i(b) + th_j(b+i) - th_i(b+j) - th_j(b)
            const float txyp = __ldg(P.tx + syp), txzp = __ldg(P.tx + szp);
            const float tyxp = __ldg(P.ty + sxp), tyzp = __ldg(P.ty + szp);
            const float tzxp = __ldg(P.tz + sxp), tzyp = __ldg(P.tz + syp);
            const float txxm = __ldg(P.tx + sxm), tyxm = __ldg(P.ty + sxm), tzxm = __ldg(P.tz + sxm);
            const float txym = __ldg(P.tx + sym), tyym = __ldg(P.ty + sym), tzym = __ldg(P.tz + sym);
            const float txzm = __ldg(P.tx + szm), tyzm = __ldg(P.ty + szm), tzzm = __ldg(P.tz + szm);
            const float a_xy = ((tx0 + tyxp) - txyp) - ty0;
            const float a_xz = ((tx0 + tzxp) - txzp) - tz0;
            const float a_yz = ((ty0 + tzyp) - tyzp) - tz0;
            const float a_xy_ym = ((txym + __ldg(P.ty + sidx(xp, ym, z, N))) - tx0) - tyym;
            const float a_xy_xm = ((txxm + ty0) - __ldg(P.tx + sidx(xm, yp, z, N))) - tyxm;
            const float a_xz_zm = ((txzm + __ldg(P.tz + sidx(xp, y, zm, N))) - tx0) - tzzm;
            const float a_xz_xm = ((txxm + tz0) - __ldg(P.tx + sidx(xm, y, zp, N))) - tzxm;
            const float a_yz_zm = ((tyzm + __ldg(P.tz + sidx(x, yp, zm, N))) - ty0) - tzzm;
            const float a_yz_ym = ((tyym + tz0) - __ldg(P.ty + sidx(x, ym, zp, N))) - tzym;
            float s_xy, c_xy, s_xz, c_xz, s_yz, c_yz;
            sincosf(a_xy, &s_xy, &c_xy);
            sincosf(a_xz, &s_xz, &c_xz);
            sincosf(a_yz, &s_yz, &c_yz);
            const float cx = -(s_xy - sinf(a_xy_ym)) - (s_xz - sinf(a_xz_zm));
            const float cy = (s_xy - sinf(a_xy_xm)) - (s_yz - sinf(a_yz_zm));
            const float cz = (s_xz - sinf(a_xz_xm)) + (s_yz - sinf(a_yz_ym));
            const float e0x = __ldg(P.ex + s), e0y = __ldg(P.ey + s), e0z = __ldg(P.ez + s);
            const float enx = k.ce * e0x + k.ke_curl * cx + k.ke_cur * J[0];
            const float eny = k.ce * e0y + k.ke_curl * cy + k.ke_cur * J[1];
            const float enz = k.ce * e0z + k.ke_curl * cz + k.ke_cur * J[2];

            if (MEASURE) {
                const float pbr = 0.5f * (q0r + qnr), pbi = 0.5f * (q0i + qni);
                const float K = pbr * pbr + pbi * pbi;
                float G = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float dr = Hr[i] - p0r, di = Hi[i] - p0i;
                    G += dr * dr + di * di;
                }
                G *= k.m_grad;
                const float dm = mod2 - k.sigma2;
                const float V = k.m_pot * dm * dm;
                const float ebx = 0.5f * (e0x + enx), eby = 0.5f * (e0y + eny), ebz = 0.5f * (e0z + enz);
                const float El = k.m_el * (ebx * ebx + eby * eby + ebz * ebz);
                const float B = k.m_mag * ((1.f - c_xy) + (1.f - c_xz) + (1.f - c_yz));
                const float L = K - G - V + El - B;
                const float rho = K + G + V + El + B;
                const float pres = K - G * (1.f / 3.f) - V + (El + B) * (1.f / 3.f);
                // Gauss residual of the stored momenta (time n - 1/2) with phi^n
                const float div = ((e0x - __ldg(P.ex + sxm)) + (e0y - __ldg(P.ey + sym)) + (e0z - __ldg(P.ez + szm))) * k.inv_dx;
                const float g = div - k.m_gauss * (p0r * q0i - p0i * q0r);
                acc.s[Q_K] += K; acc.s[Q_G] += G; acc.s[Q_V] += V; acc.s[Q_EL] += El;
                acc.s[Q_B] += B; acc.s[Q_L] += L; acc.s[Q_KL] += K * L; acc.s[Q_GL] += G * L;
                acc.s[Q_PL] += pres * L; acc.s[Q_RL] += rho * L; acc.s[Q_G2] += g * g;
                acc.gmax = fmaxf(acc.gmax, fabsf(g));
                if (!isfinite(rho) || !isfinite(L) || !isfinite(g)) acc.nf += 1;

                // plaquette windings with lower corner x
                const float pxr = __ldg(P.pr + sxp), pxi = __ldg(P.pim + sxp);
                const float pyr = __ldg(P.pr + syp), pyi = __ldg(P.pim + syp);
                const float pzr = __ldg(P.pr + szp), pzi = __ldg(P.pim + szp);
                const size_t sxy = sidx(xp, yp, z, N), sxz = sidx(xp, y, zp, N), syz = sidx(x, yp, zp, N);
                const float pxyr = __ldg(P.pr + sxy), pxyi = __ldg(P.pim + sxy);
                const float pxzr = __ldg(P.pr + sxz), pxzi = __ldg(P.pim + sxz);
                const float pyzr = __ldg(P.pr + syz), pyzi = __ldg(P.pim + syz);
                const float Yx = link_phase(p0r, p0i, pxr, pxi, tx0);
                const float Yy = link_phase(p0r, p0i, pyr, pyi, ty0);
                const float Yz = link_phase(p0r, p0i, pzr, pzi, tz0);
                const float Yy_x = link_phase(pxr, pxi, pxyr, pxyi, tyxp);
                const float Yz_x = link_phase(pxr, pxi, pxzr, pxzi, tzxp);
                const float Yx_y = link_phase(pyr, pyi, pxyr, pxyi, txyp);
                const float Yz_y = link_phase(pyr, pyi, pyzr, pyzi, tzyp);
                const float Yx_z = link_phase(pzr, pzi, pxzr, pxzi, txzp);
                const float Yy_z = link_phase(pzr, pzi, pyzr, pyzi, tyzp);
                const int wxy = winding(Yx, Yy_x, Yx_y, Yy, wrap_plaq(tx0, tyxp, txyp, ty0));
                const int wxz = winding(Yx, Yz_x, Yx_z, Yz, wrap_plaq(tx0, tzxp, txzp, tz0));
                const int wyz = winding(Yy, Yz_y, Yy_z, Yz, wrap_plaq(ty0, tzyp, tyzp, tz0));
                acc.wind += abs(wxy) + abs(wxz) + abs(wyz);
            }

            if (STORE) {
                P.qr1[s] = qnr;
                P.qi1[s] = qni;
                P.ex1[s] = enx;
                P.ey1[s] = eny;
                P.ez1[s] = enz;
                P.pr1[s] = p0r + k.dphi * qnr;
                P.pim1[s] = p0i + k.dphi * qni;
                float t1x = tx0 + k.dtheta * enx, t1y = ty0 + k.dtheta * eny, t1z = tz0 + k.dtheta * enz;
                if (k.wrap) {
                    t1x += kTwoPiF * floorf((kPiF - t1x) * kInvTwoPiF);
                    t1y += kTwoPiF * floorf((kPiF - t1y) * kInvTwoPiF);
                    t1z += kTwoPiF * floorf((kPiF - t1z) * kInvTwoPiF);
                }
                P.tx1[s] = t1x;
                P.ty1[s] = t1y;
                P.tz1[s] = t1z;
            }
        }
    }
    if (MEASURE) {
        const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
        block_reduce_store<NT>(acc, partials + b * NQ);
    }
}

// ---------------------------------------------------------------- init
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): one step from state v.
__device__ __forceinline__ uint64_t splitmix64(uint64_t v)
{
    uint64_t z = v + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void init_kernel(float *pr, float *pim, size_t V, uint64_t seed, double sigma)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
        const double u = (double)(splitmix64(seed ^ splitmix64((uint64_t)i)) >> 11) * (1.0 / 9007199254740992.0);
        const double th = __dmul_rn(2.0 * kPiD, u);
        double s, c;
        sincos(th, &s, &c);
        pr[i] = (float)__dmul_rn(sigma, c);
        pim[i] = (float)__dmul_rn(sigma, s);
    }
}

// ---------------------------------------------------------------- windings field
__global__ void windings_kernel(const float *__restrict__ pr, const float *__restrict__ pim,
                                const float *__restrict__ tx, const float *__restrict__ ty,
                                const float *__restrict__ tz, int N, int8_t *W)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (x >= N || y >= N) return;
    const int xp = (x == N - 1) ? 0 : x + 1, yp = (y == N - 1) ? 0 : y + 1, zp = (z == N - 1) ? 0 : z + 1;
    const size_t V = (size_t)N * N * N;
    const size_t s = sidx(x, y, z, N), sxp = sidx(xp, y, z, N), syp = sidx(x, yp, z, N), szp = sidx(x, y, zp, N);
    const size_t sxy = sidx(xp, yp, z, N), sxz = sidx(xp, y, zp, N), syz = sidx(x, yp, zp, N);
    const float p0r = pr[s], p0i = pim[s];
    const float pxr = pr[sxp], pxi = pim[sxp], pyr = pr[syp], pyi = pim[syp], pzr = pr[szp], pzi = pim[szp];
    const float tx0 = tx[s], ty0 = ty[s], tz0 = tz[s];
    const float Yx = link_phase(p0r, p0i, pxr, pxi, tx0);
    const float Yy = link_phase(p0r, p0i, pyr, pyi, ty0);
    const float Yz = link_phase(p0r, p0i, pzr, pzi, tz0);
    const float Yy_x = link_phase(pxr, pxi, pr[sxy], pim[sxy], ty[sxp]);
    const float Yz_x = link_phase(pxr, pxi, pr[sxz], pim[sxz], tz[sxp]);
    const float Yx_y = link_phase(pyr, pyi, pr[sxy], pim[sxy], tx[syp]);
    const float Yz_y = link_phase(pyr, pyi, pr[syz], pim[syz], tz[syp]);
    const float Yx_z = link_phase(pzr, pzi, pr[sxz], pim[sxz], tx[szp]);
    const float Yy_z = link_phase(pzr, pzi, pr[syz], pim[syz], ty[szp]);
    W[s] = (int8_t)winding(Yx, Yy_x, Yx_y, Yy, wrap_plaq(tx0, ty[sxp], tx[syp], ty0));
    W[V + s] = (int8_t)winding(Yx, Yz_x, Yx_z, Yz, wrap_plaq(tx0, tz[sxp], tx[szp], tz0));
    W[2 * V + s] = (int8_t)winding(Yy, Yz_y, Yy_z, Yz, wrap_plaq(ty0, tz[syp], ty[szp], tz0));
}

// ---------------------------------------------------------------- box gather
struct PlaneList { const float *p[10]; };

__global__ void gather_box_kernel(PlaneList L, int nplanes, int N, int x0, int y0, int z0, int nx, int ny,
                                  int nz, float *dst)
{
    const size_t per = (size_t)nx * ny * nz;
    const size_t total = per * nplanes;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int pl = (int)(i / per);
        size_t r = i - (size_t)pl * per;
        const int bx = (int)(r % nx);
        r /= nx;
        const int by = (int)(r % ny);
        const int bz = (int)(r / ny);
        const int x = (x0 + bx) % N, y = (y0 + by) % N, z = (z0 + bz) % N;
        dst[i] = L.p[pl][sidx(x, y, z, N)];
    }
}

// ---------------------------------------------------------------- final reduction
constexpr int RT = 256;

__global__ void __launch_bounds__(RT) reduce_kernel(const double *__restrict__ part, int nb, ObsScalars sc,
                                                    ahs_obs_t *rec)
{
    __shared__ double sh[RT][NQ + 1];
    const int t = threadIdx.x;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int b = t; b < nb; b += RT) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double x = part[(size_t)b * NQ + q];
            v[q] = (q == Q_GMAX) ? fmax(v[q], x) : v[q] + x;
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[t][q] = v[q];
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (t < w) {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                sh[t][q] = (q == Q_GMAX) ? fmax(sh[t][q], sh[t + w][q]) : sh[t][q] + sh[t + w][q];
        }
        __syncthreads();
    }
    if (t == 0) {
        const double *S = sh[0];
        const double dx3 = sc.dx * sc.dx * sc.dx;
        ahs_obs_t o;
        o.step = sc.step;
        o.tau = sc.tau;
        o.a = sc.a;
        o.sum_K = S[Q_K]; o.sum_G = S[Q_G]; o.sum_V = S[Q_V]; o.sum_El = S[Q_EL]; o.sum_B = S[Q_B];
        o.sum_L = S[Q_L]; o.sum_KL = S[Q_KL]; o.sum_GL = S[Q_GL]; o.sum_pL = S[Q_PL]; o.sum_rhoL = S[Q_RL];
        o.e_kin = dx3 * S[Q_K];
        o.e_grad = dx3 * S[Q_G];
        o.e_pot = dx3 * S[Q_V];
        o.e_elec = dx3 * S[Q_EL];
        o.e_mag = dx3 * S[Q_B];
        o.e_total = o.e_kin + o.e_grad + o.e_pot + o.e_elec + o.e_mag;
        o.lagrangian = dx3 * S[Q_L];
        o.xi_l = (o.lagrangian < 0.0) ? sqrt(-sc.mu * sc.volume / o.lagrangian) : INFINITY;
        const double R = S[Q_KL] / S[Q_GL];
        o.v2_phi = 2.0 * R / (1.0 + R);
        o.v2_omega = 0.5 * (1.0 + 3.0 * S[Q_PL] / S[Q_RL]);
        o.n_wind = (int64_t)S[Q_WIND];
        o.string_length = sc.dx * (double)o.n_wind;
        o.xi_w = (o.n_wind > 0) ? sqrt(sc.volume / o.string_length) : INFINITY;
        o.gauss_rms = sqrt(S[Q_G2] / sc.sites);
        o.gauss_max = S[Q_GMAX];
        o.nonfinite = (int64_t)S[Q_NF];
        *rec = o;
    }
}

}  // namespace

int step_blocks(int N)
{
    const int gx = (N + BX - 1) / BX, gy = (N + BY - 1) / BY, gz = (N + ZCHUNK - 1) / ZCHUNK;
    return gx * gy * gz;
}

cudaError_t launch_step(const StepPtrs &p, const StepCoef &k, int N, bool measure, bool store,
                        double *partials, int *nblocks, cudaStream_t st)
{
    dim3 block(BX, BY);
    dim3 grid((N + BX - 1) / BX, (N + BY - 1) / BY, (N + ZCHUNK - 1) / ZCHUNK);
    if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
    if (measure && store)
        step_kernel<true, true><<<grid, block, 0, st>>>(p, k, N, partials);
    else if (measure)
        step_kernel<true, false><<<grid, block, 0, st>>>(p, k, N, partials);
    else if (store)
        step_kernel<false, true><<<grid, block, 0, st>>>(p, k, N, partials);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_init(float *pr, float *pim, int N, uint64_t seed, double sigma, cudaStream_t st)
{
    const size_t V = (size_t)N * N * N;
    const int threads = 256;
    const size_t want = (V + threads - 1) / threads;
    const int blocks = (int)(want < (size_t)152 * 64 ? want : (size_t)152 * 64);
    init_kernel<<<blocks, threads, 0, st>>>(pr, pim, V, seed, sigma);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partials, int nblocks, const ObsScalars &sc, ahs_obs_t *rec,
                          cudaStream_t st)
{
    reduce_kernel<<<1, RT, 0, st>>>(partials, nblocks, sc, rec);
    return cudaGetLastError();
}

cudaError_t launch_windings(const float *pr, const float *pim, const float *tx, const float *ty, const float *tz,
                            int N, int8_t *W, cudaStream_t st)
{
    dim3 block(32, 8);
    dim3 grid((N + 31) / 32, (N + 7) / 8, N);
    windings_kernel<<<grid, block, 0, st>>>(pr, pim, tx, ty, tz, N, W);
    return cudaGetLastError();
}

cudaError_t launch_gather_box(const float *const *planes, int nplanes, int N, int x0, int y0, int z0, int nx,
                              int ny, int nz, float *dst, cudaStream_t st)
{
    PlaneList L;
    for (int i = 0; i < 10; ++i) L.p[i] = (i < nplanes) ? planes[i] : nullptr;
    const size_t total = (size_t)nx * ny * nz * nplanes;
    const int threads = 256;
    const size_t want = (total + threads - 1) / threads;
    const int blocks = (int)(want < 4096 ? (want > 0 ? want : 1) : 4096);
    gather_box_kernel<<<blocks, threads, 0, st>>>(L, nplanes, N, x0, y0, z0, nx, ny, nz, dst);
    return cudaGetLastError();
}

}  // namespace eng
