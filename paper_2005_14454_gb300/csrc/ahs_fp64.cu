// ahs_fp64.cu -- FP64 storage and arithmetic on the GPU, the reference precision
// mode of the engine (precision studies; GB300's FP64 rate makes it ~10x slower
// than the float32 path).
//
// A direct stencil, one thread per (x, y) column marching a z-chunk: the kick of
// Eqs. 7-8 with the plaquette sines summed from the link angles (Eqs. 15-16), the
// drift of Eqs. 9-10, and on measurement steps the diagnostics, Gauss residual and
// windings -- everything in FP64, windings with FP64 atan2, reduced to the same FP64
// partial rows as the float32 kernels.
#include "ahs_device.cuh"

namespace eng {
namespace {

constexpr int BX = 32, BY = 8, NT = BX * BY;

__device__ __forceinline__ size_t at(int x, int y, int z, int N)
{
    return (size_t)x + (size_t)N * ((size_t)y + (size_t)N * (size_t)z);
}

// arg(conj(p) U q), U = exp(-i th)
__device__ __forceinline__ double yphase(double pr, double pi, double qr, double qi, double th)
{
    double s, c;
    sincos(th, &s, &c);
    const double hr = c * qr + s * qi, hi = c * qi - s * qr;
    return atan2(pr * hi - pi * hr, pr * hr + pi * hi);
}

__device__ __forceinline__ double wrap_pi(double a) { return a + 2.0 * kPiD * floor((kPiD - a) / (2.0 * kPiD)); }

__device__ __forceinline__ int wnum(double y1, double y2, double y3, double y4, double aw)
{
    return (int)rint((y1 + y2 - y3 - y4 + aw) / (2.0 * kPiD));
}

struct AccD {
    double s[NSUM];
    double gmax;
    int wind, nf;
};

template <bool MEASURE, bool STORE>
__global__ void __launch_bounds__(NT) step_fp64(StepPtrs64 P, StepCoef64 k, int N, int Dz, double *partials)
{
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    const bool active = x < N && y < N;
    const int z0 = blockIdx.z * Dz, z1 = min(z0 + Dz, N);
    AccD acc;
    if (MEASURE) {
        for (int q = 0; q < NSUM; ++q) acc.s[q] = 0.0;
        acc.gmax = 0.0;
        acc.wind = 0;
        acc.nf = 0;
    }
    if (active) {
        const int xm = x == 0 ? N - 1 : x - 1, xp = x == N - 1 ? 0 : x + 1;
        const int ym = y == 0 ? N - 1 : y - 1, yp = y == N - 1 ? 0 : y + 1;
        for (int z = z0; z < z1; ++z) {
            const int zm = z == 0 ? N - 1 : z - 1, zp = z == N - 1 ? 0 : z + 1;
            const size_t s = at(x, y, z, N);
            const size_t sp[3] = {at(xp, y, z, N), at(x, yp, z, N), at(x, y, zp, N)};
            const size_t sm[3] = {at(xm, y, z, N), at(x, ym, z, N), at(x, y, zm, N)};
            const double *T[3] = {P.tx, P.ty, P.tz};
            const double fr = P.pr[s], fi = P.pim[s];
            double lr = 0.0, li = 0.0, J[3], G = 0.0;
            for (int i = 0; i < 3; ++i) {
                double sn, cs;
                sincos(T[i][s], &sn, &cs);
                const double qr = P.pr[sp[i]], qi = P.pim[sp[i]];
                const double hr = cs * qr + sn * qi, hi = cs * qi - sn * qr;   // U_i(x) phi(x+i)
                J[i] = fr * hi - fi * hr;
                if (MEASURE) G += (hr - fr) * (hr - fr) + (hi - fi) * (hi - fi);
                sincos(T[i][sm[i]], &sn, &cs);
                const double mr = P.pr[sm[i]], mi = P.pim[sm[i]];
                lr += hr + (cs * mr - sn * mi) - 2.0 * fr;                    // + U_i(x-i)^* phi(x-i)
                li += hi + (cs * mi + sn * mr) - 2.0 * fi;
            }
            const double m2 = fr * fr + fi * fi - k.sigma2;
            const double q0r = P.qr[s], q0i = P.qi[s];
            const double qnr = k.cpi * q0r + k.kpi_lap * lr - k.kpi_pot * m2 * fr;
            const double qni = k.cpi * q0i + k.kpi_lap * li - k.kpi_pot * m2 * fi;
            // plaquette angles alpha_ij(b) = th_i(b) + th_j(b+i) - th_i(b+j) - th_j(b)
            auto alpha = [&](int i, int j, int bx, int by, int bz) {
                const int bxi = (bx + (i == 0)) % N, byi = (by + (i == 1)) % N, bzi = (bz + (i == 2)) % N;
                const int bxj = (bx + (j == 0)) % N, byj = (by + (j == 1)) % N, bzj = (bz + (j == 2)) % N;
                return T[i][at(bx, by, bz, N)] + T[j][at(bxi, byi, bzi, N)] - T[i][at(bxj, byj, bzj, N)] -
                       T[j][at(bx, by, bz, N)];
            };
            const double axy = alpha(0, 1, x, y, z), axz = alpha(0, 2, x, y, z), ayz = alpha(1, 2, x, y, z);
            const double sxy = sin(axy), sxz = sin(axz), syz = sin(ayz);
            const double cx = -(sxy - sin(alpha(0, 1, x, ym, z))) - (sxz - sin(alpha(0, 2, x, y, zm)));
            const double cy = (sxy - sin(alpha(0, 1, xm, y, z))) - (syz - sin(alpha(1, 2, x, y, zm)));
            const double cz = (sxz - sin(alpha(0, 2, xm, y, z))) + (syz - sin(alpha(1, 2, x, ym, z)));
            const double e0x = P.ex[s], e0y = P.ey[s], e0z = P.ez[s];
            const double enx = k.ce * e0x + k.ke_curl * cx + k.ke_cur * J[0];
            const double eny = k.ce * e0y + k.ke_curl * cy + k.ke_cur * J[1];
            const double enz = k.ce * e0z + k.ke_curl * cz + k.ke_cur * J[2];
            if (MEASURE) {
                const double pbr = 0.5 * (q0r + qnr), pbi = 0.5 * (q0i + qni);
                const double K = pbr * pbr + pbi * pbi;
                G *= k.m_grad;
                const double V = k.m_pot * m2 * m2;
                const double bx = 0.5 * (e0x + enx), by = 0.5 * (e0y + eny), bz = 0.5 * (e0z + enz);
                const double El = k.m_el * (bx * bx + by * by + bz * bz);
                const double B = k.m_mag * ((1.0 - cos(axy)) + (1.0 - cos(axz)) + (1.0 - cos(ayz)));
                const double L = K - G - V + El - B, rho = K + G + V + El + B;
                const double pres = K - G / 3.0 - V + (El + B) / 3.0;
                const double div = ((e0x - P.ex[sm[0]]) + (e0y - P.ey[sm[1]]) + (e0z - P.ez[sm[2]])) * k.inv_dx;
                const double g = div - k.m_gauss * (fr * q0i - fi * q0r);
                acc.s[Q_K] += K; acc.s[Q_G] += G; acc.s[Q_V] += V; acc.s[Q_EL] += El; acc.s[Q_B] += B;
                acc.s[Q_L] += L; acc.s[Q_KL] += K * L; acc.s[Q_GL] += G * L; acc.s[Q_PL] += pres * L;
                acc.s[Q_RL] += rho * L; acc.s[Q_G2] += g * g;
                acc.gmax = fmax(acc.gmax, fabs(g));
                if (!isfinite(rho) || !isfinite(L) || !isfinite(g)) acc.nf += 1;
                // windings of the plaquettes with lower corner x
                auto Y = [&](int i, int bx, int by, int bz) {
                    const size_t b0 = at(bx, by, bz, N);
                    const size_t b1 = at((bx + (i == 0)) % N, (by + (i == 1)) % N, (bz + (i == 2)) % N, N);
                    return yphase(P.pr[b0], P.pim[b0], P.pr[b1], P.pim[b1], T[i][b0]);
                };
                const double Yx = Y(0, x, y, z), Yy = Y(1, x, y, z), Yz = Y(2, x, y, z);
                const int nxy = wnum(Yx, Y(1, xp, y, z), Y(0, x, yp, z), Yy, wrap_pi(axy));
                const int nxz = wnum(Yx, Y(2, xp, y, z), Y(0, x, y, zp), Yz, wrap_pi(axz));
                const int nyz = wnum(Yy, Y(2, x, yp, z), Y(1, x, y, zp), Yz, wrap_pi(ayz));
                acc.wind += abs(nxy) + abs(nxz) + abs(nyz);
            }
            if (STORE) {
                P.qr1[s] = qnr; P.qi1[s] = qni;
                P.ex1[s] = enx; P.ey1[s] = eny; P.ez1[s] = enz;
                P.pr1[s] = fr + k.dphi * qnr; P.pim1[s] = fi + k.dphi * qni;
                double t1x = P.tx[s] + k.dtheta * enx, t1y = P.ty[s] + k.dtheta * eny, t1z = P.tz[s] + k.dtheta * enz;
                if (k.wrap) {
                    t1x = wrap_pi(t1x);
                    t1y = wrap_pi(t1y);
                    t1z = wrap_pi(t1z);
                }
                P.tx1[s] = t1x; P.ty1[s] = t1y; P.tz1[s] = t1z;
            }
        }
    }
    if (MEASURE) {
        // FP64 block reduction in a fixed order
        __shared__ double red[NT / 32][NQ];
        const int t = threadIdx.x + BX * threadIdx.y, lane = t & 31, wid = t >> 5;
        for (int off = 16; off > 0; off >>= 1) {
            for (int q = 0; q < NSUM; ++q) acc.s[q] += __shfl_xor_sync(0xffffffffu, acc.s[q], off);
            acc.gmax = fmax(acc.gmax, __shfl_xor_sync(0xffffffffu, acc.gmax, off));
            acc.wind += __shfl_xor_sync(0xffffffffu, acc.wind, off);
            acc.nf += __shfl_xor_sync(0xffffffffu, acc.nf, off);
        }
        if (lane == 0) {
            for (int q = 0; q < NSUM; ++q) red[wid][q] = acc.s[q];
            red[wid][Q_GMAX] = acc.gmax;
            red[wid][Q_WIND] = (double)acc.wind;
            red[wid][Q_NF] = (double)acc.nf;
            red[wid][14] = red[wid][15] = 0.0;
        }
        __syncthreads();
        if (t < NQ) {
            double v = red[0][t];
            for (int w = 1; w < NT / 32; ++w) v = (t == Q_GMAX) ? fmax(v, red[w][t]) : v + red[w][t];
            const size_t bi = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
            partials[bi * NQ + t] = v;
        }
    }
}

__global__ void init_fp64(double *pr, double *pim, size_t V, uint64_t seed, double sigma)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = (seed ^ splitmix64_device((uint64_t)i));
        const double u = (double)(splitmix64_device(z) >> 11) * (1.0 / 9007199254740992.0);
        double s, c;
        sincos(__dmul_rn(2.0 * kPiD, u), &s, &c);
        pr[i] = __dmul_rn(sigma, c);
        pim[i] = __dmul_rn(sigma, s);
    }
}

}  // namespace

StepShape step_shape_fp64(int N)
{
    StepShape s;
    s.by = BY;
    s.dz = N >= 256 ? 32 : N >= 64 ? 16 : (N < 8 ? N : 8);
    s.blocks = ((N + BX - 1) / BX) * ((N + BY - 1) / BY) * ((N + s.dz - 1) / s.dz);
    return s;
}

cudaError_t launch_step_fp64(const StepPtrs64 &p, const StepCoef64 &k, int N, bool measure, bool store,
                             double *partials, cudaStream_t st)
{
    const StepShape sh = step_shape_fp64(N);
    dim3 grid((N + BX - 1) / BX, (N + BY - 1) / BY, (N + sh.dz - 1) / sh.dz), block(BX, BY);
    if (measure && store) step_fp64<true, true><<<grid, block, 0, st>>>(p, k, N, sh.dz, partials);
    else if (measure) step_fp64<true, false><<<grid, block, 0, st>>>(p, k, N, sh.dz, partials);
    else if (store) step_fp64<false, true><<<grid, block, 0, st>>>(p, k, N, sh.dz, partials);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_init_fp64(double *pr, double *pim, int N, uint64_t seed, double sigma, cudaStream_t st)
{
    const size_t V = (size_t)N * N * N;
    const size_t want = (V + 255) / 256;
    init_fp64<<<(int)(want < (size_t)152 * 64 ? want : (size_t)152 * 64), 256, 0, st>>>(pr, pim, V, seed, sigma);
    return cudaGetLastError();
}

}  // namespace eng
