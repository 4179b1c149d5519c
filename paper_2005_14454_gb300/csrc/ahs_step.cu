// ahs_step.cu -- the fused leapfrog step of the lattice Abelian-Higgs engine as a
// z-marching shared-memory stencil for sm_103a.
//
// One CTA owns a 32 x BY column of sites and marches it through a chunk of z
// planes.  For every plane it
//   A  turns the link angles of plane z+1 into link phases V_i = (cos th_i, sin th_i)
//      (one sincos per link, Eq. 13) and stages them with phi in shared memory,
//      over the tile plus a one-site ring (the halo);
//   B  forms the plaquettes of plane z as products of four link phases
//      (Eq. 15: Q_ij = V_i(x) V_j(x+i) V_i(x+j)^* V_j(x)^* = exp(i alpha_ij)),
//      so sin alpha_ij = Im Q_ij and cos alpha_ij = Re Q_ij, for the tile and its
//      backward ring;
//   C  kicks Pi (covariant Laplacian, Eq. 14, minus the potential) and E
//      (lattice curl of sin alpha plus the current Im[phi^* U phi(x+i)]) with the
//      Crank-Nicolson damping of Eqs. 7-8, drifts phi and theta (Eqs. 9-10), and
//      on measurement steps accumulates the diagnostics (Eqs. diagxi, diagvel),
//      the Gauss residual and the plaquette windings.
// Values a site needs from its z-1 neighbour (phi, V_z, sin alpha_xz/yz, E_z) are
// carried in registers from the previous plane; in-plane neighbours come from
// shared memory.  Every link phase and plaquette of the tile is computed once.
// Tile coordinates wrap modulo N, so ragged tiles and N < 32 need no special path.
#include "ahs_device.cuh"

#include <cstddef>

namespace eng {
namespace {

template <int BY_>
struct Tile {
    static constexpr int BX = 32, BY = BY_, NT = BX * BY;
    static constexpr int RX = BX + 2, RY = BY + 2, NR = RX * RY;  // links/phi: [-1, BX] x [-1, BY]
    static constexpr int SX = BX + 1, SY = BY + 1, NS = SX * SY;  // plaquettes: [-1, BX) x [-1, BY)
    static constexpr int YX = BX + 1, YY = BY + 1, NYW = YX * YY; // link phases Y: [0, BX] x [0, BY]
    static constexpr int NHA = 2 * RX + 2 * BY;                    // ring sites of phase A
    static constexpr int NHB = BX + BY;                            // backward ring sites of phase B
    static_assert(NHA <= NT && NHB <= NT, "ring items must fit one pass of the CTA");

    struct Plane {
        float vxc[NR], vxs[NR], vyc[NR], vys[NR], vzc[NR], vzs[NR], pr[NR], pi[NR];
    };
    struct Smem {
        Plane pl[2];
        float sxy[NS], sxz[NS], syz[NS];
        // measurement steps only
        float yx[NYW], yy[NYW], yz[NYW];
        float ex[NS], ey[NS];
    };
    static constexpr size_t kStepBytes = offsetof(Smem, yx);
    static constexpr size_t kMeasureBytes = sizeof(Smem);

    static __device__ __forceinline__ int r(int ex, int ey) { return (ey + 1) * RX + (ex + 1); }
    static __device__ __forceinline__ int q(int ex, int ey) { return (ey + 1) * SX + (ex + 1); }
    static __device__ __forceinline__ int w(int ex, int ey) { return ey * YX + ex; }
};

struct Raw {
    float tx, ty, tz, pr, pi;
};

struct PE {
    float qr, qi, ex, ey, ez;
};

__device__ __forceinline__ int wrapN(int v, int N)
{
    v %= N;
    return v < 0 ? v + N : v;
}

__device__ __forceinline__ Raw load_raw(const StepPtrs &P, size_t o)
{
    Raw a;
    a.tx = __ldg(P.tx + o);
    a.ty = __ldg(P.ty + o);
    a.tz = __ldg(P.tz + o);
    a.pr = __ldg(P.pr + o);
    a.pi = __ldg(P.pim + o);
    return a;
}

__device__ __forceinline__ PE load_pe(const StepPtrs &P, size_t o)
{
    PE a;
    a.qr = __ldg(P.qr + o);
    a.qi = __ldg(P.qi + o);
    a.ex = __ldg(P.ex + o);
    a.ey = __ldg(P.ey + o);
    a.ez = __ldg(P.ez + o);
    return a;
}

// complex helpers: (a) * (b), (a) * conj(b)
__device__ __forceinline__ void cmul(float ar, float ai, float br, float bi, float &cr, float &ci)
{
    cr = ar * br - ai * bi;
    ci = ar * bi + ai * br;
}
__device__ __forceinline__ void cmulc(float ar, float ai, float br, float bi, float &cr, float &ci)
{
    cr = ar * br + ai * bi;
    ci = ai * br - ar * bi;
}

// Q = V_i(x) conj(V_j(x)) * V_j(x+i) conj(V_i(x+j))
__device__ __forceinline__ void plaquette(float ic, float is, float jc, float js, float jpc, float jps, float ipc,
                                          float ips, float &qr, float &qi)
{
    float ar, ai, br, bi;
    cmulc(ic, is, jc, js, ar, ai);
    cmulc(jpc, jps, ipc, ips, br, bi);
    cmul(ar, ai, br, bi, qr, qi);
}

struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <int BY, bool MEASURE, bool STORE>
__global__ void __launch_bounds__(32 * BY) step_tiled(StepPtrs P, StepCoef k, int N, int Dz, double *partials)
{
    using T = Tile<BY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Smem &S = *reinterpret_cast<typename T::Smem *>(smem_raw);

    const int tx = threadIdx.x, ty = threadIdx.y, t = tx + 32 * ty;
    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * Dz;
    const int zend = min(z0 + Dz, N);
    const size_t NN = (size_t)N * N;

    // core item: this thread's own site; ring items of phase A and B
    const int cx = wrapN(x0 + tx, N), cy = wrapN(y0 + ty, N);
    const int coff = cx + N * cy;
    const bool valid = (x0 + tx < N) && (y0 + ty < N);
    int hax = 0, hay = 0;
    const bool hasA = t < T::NHA;
    if (hasA) {
        if (t < T::RX) { hax = t - 1; hay = -1; }
        else if (t < 2 * T::RX) { hax = t - T::RX - 1; hay = BY; }
        else if (t < 2 * T::RX + BY) { hax = -1; hay = t - 2 * T::RX; }
        else { hax = T::BX; hay = t - 2 * T::RX - BY; }
    }
    const int haoff = wrapN(x0 + hax, N) + N * wrapN(y0 + hay, N);
    int hbx = 0, hby = 0;
    const bool hasB = t < T::NHB;
    if (hasB) {
        if (t < T::BX) { hbx = t; hby = -1; }
        else { hbx = -1; hby = t - T::BX; }
    }
    // measurement: forward ring of the link phases Y (row BY for Y_x/Y_z, column BX for Y_y/Y_z)
    int hyx = 0, hyy = 0;
    if (MEASURE && hasB) {
        if (t < T::BX) { hyx = t; hyy = BY; }
        else { hyx = T::BX; hyy = t - T::BX; }
    }

    auto zoff = [&](int z) { return (size_t)wrapN(z, N) * NN; };

    // phase A for one item into plane buffer b
    auto phaseA = [&](const Raw &a, int ri, typename T::Plane &pl) {
        float s, c;
        sincosf(a.tx, &s, &c);
        pl.vxc[ri] = c; pl.vxs[ri] = s;
        sincosf(a.ty, &s, &c);
        pl.vyc[ri] = c; pl.vys[ri] = s;
        sincosf(a.tz, &s, &c);
        pl.vzc[ri] = c; pl.vzs[ri] = s;
        pl.pr[ri] = a.pr;
        pl.pi[ri] = a.pi;
    };

    // phase B for one site (ex, ey) of plane buffer b0 with the next plane b1
    auto phaseB = [&](int ex, int ey, const typename T::Plane &p0, const typename T::Plane &p1, float &qxyr,
                      float &qxyi, float &qxzr, float &qxzi, float &qyzr, float &qyzi) {
        const int r0 = T::r(ex, ey), rxp = T::r(ex + 1, ey), ryp = T::r(ex, ey + 1);
        const float vxc = p0.vxc[r0], vxs = p0.vxs[r0], vyc = p0.vyc[r0], vys = p0.vys[r0];
        const float vzc = p0.vzc[r0], vzs = p0.vzs[r0];
        plaquette(vxc, vxs, vyc, vys, p0.vyc[rxp], p0.vys[rxp], p0.vxc[ryp], p0.vxs[ryp], qxyr, qxyi);
        plaquette(vxc, vxs, vzc, vzs, p0.vzc[rxp], p0.vzs[rxp], p1.vxc[r0], p1.vxs[r0], qxzr, qxzi);
        plaquette(vyc, vys, vzc, vzs, p0.vzc[ryp], p0.vzs[ryp], p1.vyc[r0], p1.vys[r0], qyzr, qyzi);
    };

    // ---------------------------------------------------------------- prologue
    Raw rc = load_raw(P, zoff(z0 - 1) + coff);
    Raw rh = hasA ? load_raw(P, zoff(z0 - 1) + haoff) : Raw{};
    phaseA(rc, T::r(tx, ty), S.pl[0]);
    if (hasA) phaseA(rh, T::r(hax, hay), S.pl[0]);
    float thx = rc.tx, thy = rc.ty, thz = rc.tz;   // own theta of the current plane
    rc = load_raw(P, zoff(z0) + coff);
    if (hasA) rh = load_raw(P, zoff(z0) + haoff);
    PE pe_next{}, pe_cur{};
    float ezPrev = 0.f;
    if (MEASURE) ezPrev = __ldg(P.ez + zoff(z0 - 1) + coff);

    // carried from plane z-1 (own column)
    float phPrevR = 0.f, phPrevI = 0.f, vzPrevC = 1.f, vzPrevS = 0.f, sxzPrev = 0.f, syzPrev = 0.f;

    Acc acc;
    KSum ks[NSUM];
    if (MEASURE) acc_zero(acc);

    int b = 0;   // plane buffer holding plane zz
    for (int zz = z0 - 1; zz < zend; ++zz) {
        typename T::Plane &pc = S.pl[b];
        typename T::Plane &pn = S.pl[b ^ 1];
        // ---- A: link phases and phi of plane zz+1
        phaseA(rc, T::r(tx, ty), pn);
        if (hasA) phaseA(rh, T::r(hax, hay), pn);
        const float nthx = rc.tx, nthy = rc.ty, nthz = rc.tz;
        if (zz + 2 <= zend) {
            rc = load_raw(P, zoff(zz + 2) + coff);
            if (hasA) rh = load_raw(P, zoff(zz + 2) + haoff);
        }
        pe_cur = pe_next;
        if (zz + 1 < zend) pe_next = load_pe(P, zoff(zz + 1) + coff);
        __syncthreads();

        // ---- B: plaquettes of plane zz (tile + backward ring)
        float qxyr, qxyi, qxzr, qxzi, qyzr, qyzi;
        phaseB(tx, ty, pc, pn, qxyr, qxyi, qxzr, qxzi, qyzr, qyzi);
        {
            const int qi0 = T::q(tx, ty);
            S.sxy[qi0] = qxyi;
            S.sxz[qi0] = qxzi;
            S.syz[qi0] = qyzi;
        }
        if (hasB) {
            float a1, a2, a3, a4, a5, a6;
            phaseB(hbx, hby, pc, pn, a1, a2, a3, a4, a5, a6);
            const int qh = T::q(hbx, hby);
            S.sxy[qh] = a2;
            S.sxz[qh] = a4;
            S.syz[qh] = a6;
        }
        if (MEASURE && zz >= z0) {
            // link phases Y_i of plane zz on the tile and its forward ring
            const size_t zo = zoff(zz);
            const int r0 = T::r(tx, ty), wi = T::w(tx, ty);
            const float p0r = pc.pr[r0], p0i = pc.pi[r0];
            S.yx[wi] = link_phase_v(p0r, p0i, pc.pr[T::r(tx + 1, ty)], pc.pi[T::r(tx + 1, ty)], pc.vxc[r0], pc.vxs[r0], thx);
            S.yy[wi] = link_phase_v(p0r, p0i, pc.pr[T::r(tx, ty + 1)], pc.pi[T::r(tx, ty + 1)], pc.vyc[r0], pc.vys[r0], thy);
            S.yz[wi] = link_phase_v(p0r, p0i, pn.pr[r0], pn.pi[r0], pc.vzc[r0], pc.vzs[r0], thz);
            S.ex[T::q(tx, ty)] = pe_cur.ex;
            S.ey[T::q(tx, ty)] = pe_cur.ey;
            if (hasB) {
                const int rh0 = T::r(hyx, hyy), wh = T::w(hyx, hyy);
                const size_t ho = zo + wrapN(x0 + hyx, N) + (size_t)N * wrapN(y0 + hyy, N);
                const float hr = pc.pr[rh0], hi = pc.pi[rh0];
                if (t < T::BX) {   // row BY: Y_x and Y_z
                    S.yx[wh] = link_phase_v(hr, hi, pc.pr[T::r(hyx + 1, hyy)], pc.pi[T::r(hyx + 1, hyy)], pc.vxc[rh0],
                                            pc.vxs[rh0], __ldg(P.tx + ho));
                } else {           // column BX: Y_y and Y_z
                    S.yy[wh] = link_phase_v(hr, hi, pc.pr[T::r(hyx, hyy + 1)], pc.pi[T::r(hyx, hyy + 1)], pc.vyc[rh0],
                                            pc.vys[rh0], __ldg(P.ty + ho));
                }
                S.yz[wh] = link_phase_v(hr, hi, pn.pr[rh0], pn.pi[rh0], pc.vzc[rh0], pc.vzs[rh0], __ldg(P.tz + ho));
                // old E of the backward ring for the Gauss residual
                const size_t eo = zo + wrapN(x0 + hbx, N) + (size_t)N * wrapN(y0 + hby, N);
                if (t < T::BX) S.ey[T::q(hbx, hby)] = __ldg(P.ey + eo);
                else S.ex[T::q(hbx, hby)] = __ldg(P.ex + eo);
            }
        }
        __syncthreads();

        // ---- C: kick and drift of plane zz
        const int r0 = T::r(tx, ty);
        const float p0r = pc.pr[r0], p0i = pc.pi[r0];
        const float vzc = pc.vzc[r0], vzs = pc.vzs[r0];
        if (zz >= z0 && valid) {
            const float vxc = pc.vxc[r0], vxs = pc.vxs[r0], vyc = pc.vyc[r0], vys = pc.vys[r0];
            const int rxm = T::r(tx - 1, ty), rxp = T::r(tx + 1, ty), rym = T::r(tx, ty - 1), ryp = T::r(tx, ty + 1);
            // forward hops U_i(x) phi(x+i) = conj(V_i) phi(x+i)
            float hxr, hxi, hyr, hyi, hzr, hzi;
            cmulc(pc.pr[rxp], pc.pi[rxp], vxc, vxs, hxr, hxi);
            cmulc(pc.pr[ryp], pc.pi[ryp], vyc, vys, hyr, hyi);
            cmulc(pn.pr[r0], pn.pi[r0], vzc, vzs, hzr, hzi);
            // backward hops U_i(x-i)^* phi(x-i) = V_i(x-i) phi(x-i)
            float bxr, bxi, byr, byi, bzr, bzi;
            cmul(pc.vxc[rxm], pc.vxs[rxm], pc.pr[rxm], pc.pi[rxm], bxr, bxi);
            cmul(pc.vyc[rym], pc.vys[rym], pc.pr[rym], pc.pi[rym], byr, byi);
            cmul(vzPrevC, vzPrevS, phPrevR, phPrevI, bzr, bzi);
            const float hsr = ((hxr + bxr) + (hyr + byr)) + (hzr + bzr);
            const float hsi = ((hxi + bxi) + (hyi + byi)) + (hzi + bzi);
            const float mod2 = p0r * p0r + p0i * p0i;
            const float potf = k.kpi_pot * (mod2 - k.sigma2);
            const float qnr = k.cpi * pe_cur.qr + k.kpi_lap * (hsr - 6.f * p0r) - potf * p0r;
            const float qni = k.cpi * pe_cur.qi + k.kpi_lap * (hsi - 6.f * p0i) - potf * p0i;
            // currents J_i = Im(conj(phi) U_i phi(x+i))
            const float jx = p0r * hxi - p0i * hxr;
            const float jy = p0r * hyi - p0i * hyr;
            const float jz = p0r * hzi - p0i * hzr;
            const int qi0 = T::q(tx, ty);
            const float sxy = qxyi, sxz = qxzi, syz = qyzi;
            const float cxv = -(sxy - S.sxy[T::q(tx, ty - 1)]) - (sxz - sxzPrev);
            const float cyv = (sxy - S.sxy[T::q(tx - 1, ty)]) - (syz - syzPrev);
            const float czv = (sxz - S.sxz[T::q(tx - 1, ty)]) + (syz - S.syz[T::q(tx, ty - 1)]);
            (void)qi0;
            const float enx = k.ce * pe_cur.ex + k.ke_curl * cxv + k.ke_cur * jx;
            const float eny = k.ce * pe_cur.ey + k.ke_curl * cyv + k.ke_cur * jy;
            const float enz = k.ce * pe_cur.ez + k.ke_curl * czv + k.ke_cur * jz;

            if (MEASURE) {
                const float pbr = 0.5f * (pe_cur.qr + qnr), pbi = 0.5f * (pe_cur.qi + qni);
                const float K = pbr * pbr + pbi * pbi;
                const float gxr = hxr - p0r, gxi = hxi - p0i, gyr = hyr - p0r, gyi = hyi - p0i;
                const float gzr = hzr - p0r, gzi = hzi - p0i;
                const float G = k.m_grad * ((gxr * gxr + gxi * gxi) + (gyr * gyr + gyi * gyi) + (gzr * gzr + gzi * gzi));
                const float dm = mod2 - k.sigma2;
                const float V = k.m_pot * dm * dm;
                const float ebx = 0.5f * (pe_cur.ex + enx), eby = 0.5f * (pe_cur.ey + eny), ebz = 0.5f * (pe_cur.ez + enz);
                const float El = k.m_el * (ebx * ebx + eby * eby + ebz * ebz);
                const float B = k.m_mag * ((1.f - qxyr) + (1.f - qxzr) + (1.f - qyzr));
                const float L = K - G - V + El - B;
                const float rho = K + G + V + El + B;
                const float pres = K - G * (1.f / 3.f) - V + (El + B) * (1.f / 3.f);
                const float div = ((pe_cur.ex - S.ex[T::q(tx - 1, ty)]) + (pe_cur.ey - S.ey[T::q(tx, ty - 1)]) +
                                   (pe_cur.ez - ezPrev)) * k.inv_dx;
                const float g = div - k.m_gauss * (p0r * pe_cur.qi - p0i * pe_cur.qr);
                ks[Q_K].add(K); ks[Q_G].add(G); ks[Q_V].add(V); ks[Q_EL].add(El); ks[Q_B].add(B);
                ks[Q_L].add(L); ks[Q_KL].add(K * L); ks[Q_GL].add(G * L); ks[Q_PL].add(pres * L);
                ks[Q_RL].add(rho * L); ks[Q_G2].add(g * g);
                acc.gmax = fmaxf(acc.gmax, fabsf(g));
                if (!isfinite(rho) || !isfinite(L) || !isfinite(g)) acc.nf += 1;

                // plaquette windings with lower corner x
                const int wi = T::w(tx, ty);
                const float Yx = S.yx[wi], Yy = S.yy[wi], Yz = S.yz[wi];
                const size_t o = zoff(zz) + coff;
                const size_t oxp = zoff(zz) + wrapN(cx + 1, N) + (size_t)N * cy;
                const size_t oyp = zoff(zz) + cx + (size_t)N * wrapN(cy + 1, N);
                const size_t ozp = zoff(zz + 1) + coff;
                // Y_x, Y_y of plane zz+1 (own column)
                const int rxpn = T::r(tx + 1, ty), rypn = T::r(tx, ty + 1);
                const float Yxn = link_phase_v(pn.pr[r0], pn.pi[r0], pn.pr[rxpn], pn.pi[rxpn], pn.vxc[r0], pn.vxs[r0], nthx);
                const float Yyn = link_phase_v(pn.pr[r0], pn.pi[r0], pn.pr[rypn], pn.pi[rypn], pn.vyc[r0], pn.vys[r0], nthy);
                (void)o;
                const float wxy = wrap_from_q(qxyr, qxyi, thx, __ldg(P.ty + oxp), __ldg(P.tx + oyp), thy);
                const float wxz = wrap_from_q(qxzr, qxzi, thx, __ldg(P.tz + oxp), nthx, thz);
                const float wyz = wrap_from_q(qyzr, qyzi, thy, __ldg(P.tz + oyp), nthy, thz);
                const int nxy = winding(Yx, S.yy[T::w(tx + 1, ty)], S.yx[T::w(tx, ty + 1)], Yy, wxy);
                const int nxz = winding(Yx, S.yz[T::w(tx + 1, ty)], Yxn, Yz, wxz);
                const int nyz = winding(Yy, S.yz[T::w(tx, ty + 1)], Yyn, Yz, wyz);
                acc.wind += abs(nxy) + abs(nxz) + abs(nyz);
                (void)ozp;
            }

            if (STORE) {
                const size_t o = zoff(zz) + coff;
                P.qr1[o] = qnr;
                P.qi1[o] = qni;
                P.ex1[o] = enx;
                P.ey1[o] = eny;
                P.ez1[o] = enz;
                P.pr1[o] = p0r + k.dphi * qnr;
                P.pim1[o] = p0i + k.dphi * qni;
                float t1x = thx + k.dtheta * enx, t1y = thy + k.dtheta * eny, t1z = thz + k.dtheta * enz;
                if (k.wrap) {
                    t1x += kTwoPiF * floorf((kPiF - t1x) * kInvTwoPiF);
                    t1y += kTwoPiF * floorf((kPiF - t1y) * kInvTwoPiF);
                    t1z += kTwoPiF * floorf((kPiF - t1z) * kInvTwoPiF);
                }
                P.tx1[o] = t1x;
                P.ty1[o] = t1y;
                P.tz1[o] = t1z;
            }
        }
        // carry plane zz's own-column values to plane zz+1
        phPrevR = p0r; phPrevI = p0i;
        vzPrevC = vzc; vzPrevS = vzs;
        sxzPrev = qxzi; syzPrev = qyzi;
        if (MEASURE && zz >= z0) ezPrev = pe_cur.ez;
        thx = nthx; thy = nthy; thz = nthz;
        b ^= 1;
        __syncthreads();
    }

    if (MEASURE) {
#pragma unroll
        for (int qq = 0; qq < NSUM; ++qq) acc.s[qq] = ks[qq].s;
        const size_t bi = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
        block_reduce_store<32 * BY>(acc, partials + bi * NQ);
    }
}

template <int BY, bool M, bool S>
cudaError_t launch_variant(const StepPtrs &p, const StepCoef &k, int N, int Dz, double *partials, cudaStream_t st)
{
    using T = Tile<BY>;
    const size_t bytes = M ? T::kMeasureBytes : T::kStepBytes;
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(step_tiled<BY, M, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    dim3 block(32, BY);
    dim3 grid((N + 31) / 32, (N + BY - 1) / BY, (N + Dz - 1) / Dz);
    step_tiled<BY, M, S><<<grid, block, bytes, st>>>(p, k, N, Dz, partials);
    return cudaGetLastError();
}

template <int BY>
cudaError_t launch_by(const StepPtrs &p, const StepCoef &k, int N, int Dz, bool measure, bool store,
                      double *partials, cudaStream_t st)
{
    if (measure && store) return launch_variant<BY, true, true>(p, k, N, Dz, partials, st);
    if (measure) return launch_variant<BY, true, false>(p, k, N, Dz, partials, st);
    if (store) return launch_variant<BY, false, true>(p, k, N, Dz, partials, st);
    return cudaErrorInvalidValue;
}

}  // namespace

StepShape step_shape(int N, int tile_y, int zchunk)
{
    StepShape s;
    s.by = (tile_y == 8 || tile_y == 16) ? tile_y : 8;
    if (zchunk > 0) {
        s.dz = zchunk < N ? zchunk : N;
    } else {
        // several waves of CTAs on 152 SMs, marches long enough to amortise the two
        // prologue planes of each chunk
        s.dz = N >= 512 ? 64 : N >= 256 ? 32 : N >= 64 ? 16 : (N < 8 ? N : 8);
    }
    s.blocks = ((N + 31) / 32) * ((N + s.by - 1) / s.by) * ((N + s.dz - 1) / s.dz);
    return s;
}

cudaError_t launch_step(const StepPtrs &p, const StepCoef &k, int N, const StepShape &sh, bool measure, bool store,
                        double *partials, cudaStream_t st)
{
    if (sh.by == 16) return launch_by<16>(p, k, N, sh.dz, measure, store, partials, st);
    return launch_by<8>(p, k, N, sh.dz, measure, store, partials, st);
}

}  // namespace eng
