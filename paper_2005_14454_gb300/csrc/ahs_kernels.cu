// ahs_kernels.cu -- sm_103a kernels of the lattice Abelian-Higgs engine.
//
// Initial condition, standalone winding field, periodic box gather and the final
// FP64 reduction of the measurement partials.  The step kernel lives in
// ahs_step.cu.
#include "ahs_device.cuh"

#include <cmath>

namespace eng {

namespace {

// ---------------------------------------------------------------- init
__global__ void init_kernel(float *pr, float *pim, size_t V, uint64_t seed, double sigma)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
        const double u = (double)(splitmix64_device(seed ^ splitmix64_device((uint64_t)i)) >> 11) * (1.0 / 9007199254740992.0);
        const double th = __dmul_rn(2.0 * kPiD, u);
        double s, c;
        sincos(th, &s, &c);
        pr[i] = (float)__dmul_rn(sigma, c);
        pim[i] = (float)__dmul_rn(sigma, s);
    }
}

// ---------------------------------------------------------------- windings field
// W_ij(x) for every plaquette, from the same link phases (V = (cos, sin) of each
// link angle), plaquette products and branch handling as the fused measurement.
__device__ __forceinline__ float2 vphase(float th)
{
    float s, c;
    link_sincos(th, s, c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 plaq_q(float2 vi, float2 vj, float2 vjp, float2 vip)
{
    const float2 a = make_float2(vi.x * vj.x + vi.y * vj.y, vi.y * vj.x - vi.x * vj.y);
    const float2 b = make_float2(vjp.x * vip.x + vjp.y * vip.y, vjp.y * vip.x - vjp.x * vip.y);
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

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
    const float tyx = ty[sxp], tzx = tz[sxp], txy = tx[syp], tzy = tz[syp], txz = tx[szp], tyz = ty[szp];
    const float2 vx0 = vphase(tx0), vy0 = vphase(ty0), vz0 = vphase(tz0);
    const float2 vyx = vphase(tyx), vzx = vphase(tzx), vxy = vphase(txy), vzy = vphase(tzy), vxz = vphase(txz),
                 vyz = vphase(tyz);
    auto Y = [](float ar, float ai, float br, float bi, float2 v, float th) {
        return link_phase_v(ar, ai, br, bi, v.x, v.y, [&] { return th; });
    };
    const int Yx = Y(p0r, p0i, pxr, pxi, vx0, tx0);
    const int Yy = Y(p0r, p0i, pyr, pyi, vy0, ty0);
    const int Yz = Y(p0r, p0i, pzr, pzi, vz0, tz0);
    const int Yy_x = Y(pxr, pxi, pr[sxy], pim[sxy], vyx, tyx);
    const int Yz_x = Y(pxr, pxi, pr[sxz], pim[sxz], vzx, tzx);
    const int Yx_y = Y(pyr, pyi, pr[sxy], pim[sxy], vxy, txy);
    const int Yz_y = Y(pyr, pyi, pr[syz], pim[syz], vzy, tzy);
    const int Yx_z = Y(pzr, pzi, pr[sxz], pim[sxz], vxz, txz);
    const int Yy_z = Y(pzr, pzi, pr[syz], pim[syz], vyz, tyz);
    const float2 Qxy = plaq_q(vx0, vy0, vyx, vxy), Qxz = plaq_q(vx0, vz0, vzx, vxz), Qyz = plaq_q(vy0, vz0, vzy, vyz);
    const int wxy = wrap_from_q(Qxy.x, Qxy.y, [&](float &a, float &b, float &c, float &d) { a = tx0; b = tyx; c = txy; d = ty0; });
    const int wxz = wrap_from_q(Qxz.x, Qxz.y, [&](float &a, float &b, float &c, float &d) { a = tx0; b = tzx; c = txz; d = tz0; });
    const int wyz = wrap_from_q(Qyz.x, Qyz.y, [&](float &a, float &b, float &c, float &d) { a = ty0; b = tzy; c = tyz; d = tz0; });
    W[s] = (int8_t)winding(Yx, Yy_x, Yx_y, Yy, wxy);
    W[V + s] = (int8_t)winding(Yx, Yz_x, Yx_z, Yz, wxz);
    W[2 * V + s] = (int8_t)winding(Yy, Yz_y, Yy_z, Yz, wyz);
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

__device__ void reduce_rows(const double *__restrict__ part, int nb, const ObsScalars &sc, ahs_obs_t *rec)
{
    __shared__ double sh[RT][NQ + 1];
    const int t = threadIdx.x;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    auto add = [&](const double *x) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = (q == Q_GMAX) ? fmax(v[q], x[q]) : v[q] + x[q];
    };
    // rows t, t + RT, t + 2 RT, ... in that order; four rows' loads are issued
    // before their additions (a row is 16 doubles, 128-byte aligned: 8 x 16 bytes)
    int b = t;
    for (; b + 3 * RT < nb; b += 4 * RT) {
        double x[4][NQ];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 *row = reinterpret_cast<const double2 *>(part + (size_t)(b + k * RT) * NQ);
#pragma unroll
            for (int h = 0; h < NQ / 2; ++h) {
                const double2 d = __ldg(row + h);
                x[k][2 * h] = d.x;
                x[k][2 * h + 1] = d.y;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) add(x[k]);
    }
    for (; b < nb; b += RT) {
        double x[NQ];
        const double2 *row = reinterpret_cast<const double2 *>(part + (size_t)b * NQ);
#pragma unroll
        for (int h = 0; h < NQ / 2; ++h) {
            const double2 d = __ldg(row + h);
            x[2 * h] = d.x;
            x[2 * h + 1] = d.y;
        }
        add(x);
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
        // pierced plaquettes times dx, with the pi/6 correction for the Manhattan
        // overcount of lattice paths (the convention Table 1's xi_dot_W follows)
        o.string_length = (kPiD / 6.0) * sc.dx * (double)o.n_wind;
        o.xi_w = (o.n_wind > 0) ? sqrt(sc.volume / o.string_length) : INFINITY;
        o.gauss_rms = sqrt(S[Q_G2] / sc.sites);
        o.gauss_max = S[Q_GMAX];
        o.nonfinite = (int64_t)S[Q_NF];
        *rec = o;
    }
}

__global__ void __launch_bounds__(RT) reduce_kernel(const double *__restrict__ part, int nb, ObsScalars sc,
                                                    ahs_obs_t *rec)
{
    reduce_rows(part, nb, sc, rec);
}

// one CTA per member: the record of step *counter + dn for members still running
__global__ void __launch_bounds__(RT) batch_reduce_kernel(const double *__restrict__ part, const BatchMember *members,
                                                          const ObsScalars *obs, int obs_stride,
                                                          const int64_t *counter, int dn, int every,
                                                          ahs_obs_t *records, int rcap)
{
    const int m = blockIdx.x;
    const int64_t n = *counter + dn;
    const BatchMember &mb = members[m];
    if (n >= mb.n_end || every <= 0 || n % every != 0) return;
    const int slot = (int)(n / every);
    if (slot >= rcap || slot >= obs_stride) return;
    reduce_rows(part + (size_t)mb.row0 * NQ, mb.nrows, obs[(size_t)m * obs_stride + slot],
                records + (size_t)m * rcap + slot);
}

__global__ void advance_kernel(int64_t *counter, int64_t delta) { *counter += delta; }

}  // namespace

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

cudaError_t launch_batch_reduce(const double *partials, const BatchMember *members, int nmembers,
                                const ObsScalars *obs, int obs_stride, const int64_t *counter, int dn, int every,
                                ahs_obs_t *records, int rcap, cudaStream_t st)
{
    batch_reduce_kernel<<<nmembers, RT, 0, st>>>(partials, members, obs, obs_stride, counter, dn, every, records, rcap);
    return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *counter, int64_t delta, cudaStream_t st)
{
    advance_kernel<<<1, 1, 0, st>>>(counter, delta);
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
