// ahs_step2.cu -- two leapfrog steps per pass over the fields: temporal blocking
// of the z-marching step (plain float32 steps).
//
// The plain step moves 80 bytes per site-update (every field read at time n and
// written at n+1), so at best it runs at the HBM copy rate.  step_two advances two
// consecutive plain steps n -> n+1 -> n+2 in one launch: the fields are read once
// at n and written once at n+2, 40 + 40 bytes for two site-updates.  The price is
// arithmetic: the second step of a tile needs the first step's phi^{n+1} and
// theta^{n+1} on a one-site ring around the tile, so the first step runs on the
// tile plus that ring, from link phases of the tile plus a two-site ring.
//
// A CTA owns a 32 x 8 column of sites and marches it through a z-chunk with two
// stages in flight:
//   stage 1 (step n) at plane zz on the 34 x 10 sites [-1, 32] x [-1, 8]: link
//     phases of plane zz+1 over 36 x 12 sites (phase A), plaquettes of plane zz
//     over the 34 x 10 sites and their backward ring (phase B), kick and drift
//     (phase C) -- the first step's phi^{n+1} and link phases V(theta^{n+1}) go to
//     shared memory, the own site's Pi^{n+1/2}, E^{n+1/2} and theta^{n+1} stay in
//     registers;
//   stage 2 (step n+1) at plane zz-2 on the tile: plaquettes (phase B) and kick
//     and drift (phase C) from stage 1's planes zz-2 and zz-1, stored to the
//     output buffer.
// Stage 2 lags two planes behind stage 1, so both stages share the two CTA
// barriers of a plane: everything stage 2 reads was written before the barrier
// that opens the current plane.  Shared memory holds three rotating time-n planes
// and three rotating time-(n+1) planes (stage 1 writes plane zz while stage 2 reads
// zz-2 and zz-1).  The arithmetic of each site-update is that of tile_step, in the
// same order, so the fields equal those of two plain steps.
#include "ahs_stencil.cuh"

namespace eng {
namespace {

struct Tile2Step {
    static constexpr int BX = 32, BY = 8, NT = BX * BY;
    static constexpr int AX = BX + 4, AY = BY + 4, NA = AX * AY;  // time-n sites: [-2, BX+1] x [-2, BY+1]
    static constexpr int HX = BX + 2, HY = BY + 2, NH = HX * HY;  // stage-1 sites: [-1, BX] x [-1, BY]
    static constexpr int P1X = BX + 3, NP1 = P1X * (BY + 3);     // stage-1 plaquettes: [-2, BX] x [-2, BY]
    static constexpr int P2X = BX + 1, NP2 = P2X * (BY + 1);     // stage-2 plaquettes: [-1, BX) x [-1, BY)
    static constexpr int NR1 = 2 * HX + 2 * BY;                   // stage-1 ring sites (84)
    static constexpr int NR2 = 2 * AX + 2 * HY;                   // second ring of time-n sites (92)
    static constexpr int NB1 = HX + HY;                           // stage-1 backward-ring plaquette sites (44)
    static constexpr int NB2 = BX + BY;                           // stage-2 backward-ring plaquette sites (40)
    // thread ranges of the ring work: ring-1 sites (phase A, stage 1), ring-2 sites
    // (phase A), stage-2 backward ring (phase B), stage-1 backward ring (phase B)
    static constexpr int T_R2 = NR1, T_B2 = NR1, T_B1 = NR1 + NR2;
    static_assert(NR1 + NR2 <= NT && T_B1 + NB1 <= NT && T_B2 + NB2 <= T_B1, "ring items must fit one pass");

    struct Plane0 {
        float2 vx[NA], vy[NA], vz[NA], ph[NA];
    };
    struct Plane1 {
        float2 vx[NH], vy[NH], vz[NH], ph[NH];
    };
    struct Smem {
        Plane0 p0[3];
        Plane1 p1[3];
        float s1xy[NP1], s1xz[NP1], s1yz[NP1];
        float s2xy[NP2], s2xz[NP2], s2yz[NP2];
    };
    static __device__ __forceinline__ int a(int ex, int ey) { return AHS_INDEX((ey + 2) * AX + (ex + 2), NA); }
    static __device__ __forceinline__ int h(int ex, int ey) { return AHS_INDEX((ey + 1) * HX + (ex + 1), NH); }
    static __device__ __forceinline__ int q1(int ex, int ey) { return AHS_INDEX((ey + 2) * P1X + (ex + 2), NP1); }
    static __device__ __forceinline__ int q2(int ex, int ey) { return AHS_INDEX((ey + 1) * P2X + (ex + 1), NP2); }
};

// a site's own values that stage 1 hands to stage 2: Pi^{n+1/2}, E^{n+1/2}, theta^{n+1}
struct Own {
    float qr, qi, ex, ey, ez, tx, ty, tz;
};

// Kick and drift of one site (tile_step's plain float32 arithmetic, Eqs. 7-10):
// the new momenta from the hops, the potential and the curls of sin alpha, then
// phi and theta one step on.  Arguments: phi and the link phases V_i of the site;
// phi at x+i (pxp, pyp, pzp); V_i and phi at x-i (vxm/pxm, vym/pym, vzm/pzm); the
// old momenta; sin alpha_ij of the site's plaquettes (sxy, sxz, syz) and of those
// one site behind (sxy_ym at x-y, sxy_xm and sxz_xm at x-x, syz_ym at x-y, sxz_zm
// and syz_zm at x-z); the site's theta.
struct Kicked {
    float qr, qi, ex, ey, ez;
    float pr, pi, tx, ty, tz;
};

__device__ __forceinline__ Kicked kick_drift(const StepCoef &k, float2 p0, float2 vx0, float2 vy0, float2 vz0,
                                             float2 pxp, float2 pyp, float2 pzp, float2 vxm, float2 pxm,
                                             float2 vym, float2 pym, float2 vzm, float2 pzm, float qr, float qi,
                                             float e0x, float e0y, float e0z, float sxy, float sxz, float syz,
                                             float sxy_ym, float sxy_xm, float sxz_xm, float syz_ym, float sxz_zm,
                                             float syz_zm, float thx, float thy, float thz)
{
    Kicked o;
    // forward hops U_i(x) phi(x+i) = conj(V_i) phi(x+i), backward V_i(x-i) phi(x-i)
    const float2 hx = cmulc(pxp, vx0);
    const float2 hy = cmulc(pyp, vy0);
    const float2 hz = cmulc(pzp, vz0);
    const float2 bxh = cmul(vxm, pxm);
    const float2 byh = cmul(vym, pym);
    const float2 bzh = cmul(vzm, pzm);
    const float hsr = ((hx.x + bxh.x) + (hy.x + byh.x)) + (hz.x + bzh.x);
    const float hsi = ((hx.y + bxh.y) + (hy.y + byh.y)) + (hz.y + bzh.y);
    const float mod2 = p0.x * p0.x + p0.y * p0.y;
    const float potf = k.kpi_pot * (mod2 - k.sigma2);
    o.qr = k.cpi * qr + k.kpi_lap * (hsr - float(6) * p0.x) - potf * p0.x;
    o.qi = k.cpi * qi + k.kpi_lap * (hsi - float(6) * p0.y) - potf * p0.y;
    // currents J_i = Im(conj(phi) U_i phi(x+i)) and the curl of sin alpha
    const float jx = p0.x * hx.y - p0.y * hx.x;
    const float jy = p0.x * hy.y - p0.y * hy.x;
    const float jz = p0.x * hz.y - p0.y * hz.x;
    const float cxv = -(sxy - sxy_ym) - (sxz - sxz_zm);
    const float cyv = (sxy - sxy_xm) - (syz - syz_zm);
    const float czv = (sxz - sxz_xm) + (syz - syz_ym);
    o.ex = k.ce * e0x + k.ke_curl * cxv + k.ke_cur * jx;
    o.ey = k.ce * e0y + k.ke_curl * cyv + k.ke_cur * jy;
    o.ez = k.ce * e0z + k.ke_curl * czv + k.ke_cur * jz;
    o.pr = p0.x + k.dphi * o.qr;
    o.pi = p0.y + k.dphi * o.qi;
    o.tx = thx + k.dtheta * o.ex;
    o.ty = thy + k.dtheta * o.ey;
    o.tz = thz + k.dtheta * o.ez;
    if (k.wrap) {
        o.tx += kTwoPiF * floorf((kPiF - o.tx) * kInvTwoPiF);
        o.ty += kTwoPiF * floorf((kPiF - o.ty) * kInvTwoPiF);
        o.tz += kTwoPiF * floorf((kPiF - o.tz) * kInvTwoPiF);
    }
    return o;
}

__global__ void __launch_bounds__(256, 2)
    step_two(StepPtrs P, StepCoef k1, StepCoef k2, int N, int Dz)
{
    using T = Tile2Step;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T::Smem &S = *reinterpret_cast<T::Smem *>(smem_raw);
    const ParamFields F{P, (uint32_t)N * (uint32_t)N * (uint32_t)N};
    const int tx = threadIdx.x, ty = threadIdx.y, t = tx + 32 * ty;
    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * T::BY, z0 = blockIdx.z * Dz;
    const int zend = min(z0 + Dz, N);
    const uint32_t NN = (uint32_t)N * (uint32_t)N;
    auto off = [&](int ex, int ey) {
        return (uint32_t)wrapN(x0 + ex, N) + (uint32_t)N * (uint32_t)wrapN(y0 + ey, N);
    };

    // core site; the thread's ring site of phase A (ring 1 for t < NR1, which the
    // thread also carries through stage 1, or ring 2)
    const uint32_t coff = off(tx, ty);
    const bool valid = (x0 + tx < N) && (y0 + ty < N);
    const bool hasA = t < T::NR1 + T::NR2;
    const bool ring1 = t < T::NR1;
    int hax = 0, hay = 0;
    if (ring1) {
        const int u = t;
        if (u < T::HX) { hax = u - 1; hay = -1; }
        else if (u < 2 * T::HX) { hax = u - T::HX - 1; hay = T::BY; }
        else if (u < 2 * T::HX + T::BY) { hax = -1; hay = u - 2 * T::HX; }
        else { hax = T::BX; hay = u - 2 * T::HX - T::BY; }
    } else if (hasA) {
        const int u = t - T::T_R2;
        if (u < T::AX) { hax = u - 2; hay = -2; }
        else if (u < 2 * T::AX) { hax = u - T::AX - 2; hay = T::BY + 1; }
        else if (u < 2 * T::AX + T::HY) { hax = -2; hay = u - 2 * T::AX - 1; }
        else { hax = T::BX + 1; hay = u - 2 * T::AX - T::HY - 1; }
    }
    const uint32_t haoff = off(hax, hay);
    // backward-ring plaquettes: stage 1 (row -2 over x in [-1, BX], column -2 over
    // y in [-1, BY]) and stage 2 (row -1 over x in [0, BX), column -1 over y in [0, BY))
    const bool hasB1 = t >= T::T_B1 && t < T::T_B1 + T::NB1;
    const bool rowB1 = t - T::T_B1 < T::HX;
    const int b1x = rowB1 ? t - T::T_B1 - 1 : -2, b1y = rowB1 ? -2 : t - T::T_B1 - T::HX - 1;
    const bool hasB2 = t >= T::T_B2 && t < T::T_B2 + T::NB2;
    const bool rowB2 = t - T::T_B2 < T::BX;
    const int b2x = rowB2 ? t - T::T_B2 : -1, b2y = rowB2 ? -1 : t - T::T_B2 - T::BX;

    auto phaseA = [&](const Raw<float> &r, int ai, T::Plane0 &pl) {
        float s, c;
        link_sincos(r.tx, s, c);
        pl.vx[ai] = make_float2(c, s);
        link_sincos(r.ty, s, c);
        pl.vy[ai] = make_float2(c, s);
        link_sincos(r.tz, s, c);
        pl.vz[ai] = make_float2(c, s);
        pl.ph[ai] = make_float2(r.pr, r.pi);
    };
    // stage-1 output of a site: phi^{n+1} and its link phases V(theta^{n+1})
    auto put1 = [&](const Kicked &o, int hi, T::Plane1 &pl) {
        float s, c;
        link_sincos(o.tx, s, c);
        pl.vx[hi] = make_float2(c, s);
        link_sincos(o.ty, s, c);
        pl.vy[hi] = make_float2(c, s);
        link_sincos(o.tz, s, c);
        pl.vz[hi] = make_float2(c, s);
        pl.ph[hi] = make_float2(o.pr, o.pi);
    };
    // stage-1 kick and drift of the site (ex, ey) at the time-n planes pc (zz) and
    // pn (zz+1), with its z-1 values carried
    auto stage1 = [&](int ex, int ey, const T::Plane0 &pc, const T::Plane0 &pn, const PE<float> &pe, float2 phm,
                      float2 vzm, float sxzm, float syzm, float thx, float thy, float thz) {
        const int r0 = T::a(ex, ey);
        const int q0 = T::q1(ex, ey);
        return kick_drift(k1, pc.ph[r0], pc.vx[r0], pc.vy[r0], pc.vz[r0], pc.ph[T::a(ex + 1, ey)],
                          pc.ph[T::a(ex, ey + 1)], pn.ph[r0], pc.vx[T::a(ex - 1, ey)], pc.ph[T::a(ex - 1, ey)],
                          pc.vy[T::a(ex, ey - 1)], pc.ph[T::a(ex, ey - 1)], vzm, phm, pe.qr, pe.qi, pe.ex, pe.ey,
                          pe.ez, S.s1xy[q0], S.s1xz[q0], S.s1yz[q0], S.s1xy[T::q1(ex, ey - 1)],
                          S.s1xy[T::q1(ex - 1, ey)], S.s1xz[T::q1(ex - 1, ey)], S.s1yz[T::q1(ex, ey - 1)], sxzm,
                          syzm, thx, thy, thz);
    };

    const int zs = z0 - 2;   // first plane of the march (stage 1's carries)
    int zc = wrapN(zs, N);
    int z1 = next_plane(zc, N);
    int z2 = next_plane(z1, N);

    // ---------------------------------------------------------------- prologue
    Raw<float> rc = load_raw(F, (uint32_t)zc * NN + coff);
    Raw<float> rh = hasA ? load_raw(F, (uint32_t)zc * NN + haoff) : Raw<float>{};
    phaseA(rc, T::a(tx, ty), S.p0[0]);
    if (hasA) phaseA(rh, T::a(hax, hay), S.p0[0]);
    float thx = rc.tx, thy = rc.ty, thz = rc.tz;   // own time-n theta of plane zz
    float rthx = rh.tx, rthy = rh.ty, rthz = rh.tz; // the same of the ring-1 site
    rc = load_raw(F, (uint32_t)z1 * NN + coff);
    if (hasA) rh = load_raw(F, (uint32_t)z1 * NN + haoff);
    PE<float> pe_next{}, pe_cur{}, rpe_next{}, rpe_cur{};

    // carried from plane zz-1: stage 1 (own site and ring-1 site), stage 2 (own site)
    float2 phPrev1 = make_float2(0.f, 0.f), vzPrev1 = make_float2(1.f, 0.f);
    float sxzPrev1 = 0.f, syzPrev1 = 0.f;
    float2 rphPrev1 = make_float2(0.f, 0.f), rvzPrev1 = make_float2(1.f, 0.f);
    float rsxzPrev1 = 0.f, rsyzPrev1 = 0.f;
    float2 phPrev2 = make_float2(0.f, 0.f), vzPrev2 = make_float2(1.f, 0.f);
    float sxzPrev2 = 0.f, syzPrev2 = 0.f;
    Own own1{}, own2{};   // stage-1 results of the own site at planes zz-1 and zz-2

    int b0 = 0;   // time-n buffer of plane zz
    int b1 = 0;   // time-(n+1) buffer of plane zz (zz-1, zz-2 in the two before it)
    for (int zz = zs; zz <= zend + 1; ++zz) {
        const int b0n = b0 == 2 ? 0 : b0 + 1;
        const int b1m1 = b1 == 0 ? 2 : b1 - 1;
        const int b1m2 = b1m1 == 0 ? 2 : b1m1 - 1;
        T::Plane0 &pc = S.p0[b0];
        T::Plane0 &pn = S.p0[b0n];
        const bool doB1 = zz <= zend;                  // stage-1 plaquettes, planes [z0-2, zend]
        const bool doC1 = zz >= z0 - 1 && zz <= zend;  // stage-1 updates, planes [z0-1, zend]
        const bool doB2 = zz >= z0 + 1;                // stage-2 plaquettes, planes [z0-1, zend)
        const bool doC2 = zz >= z0 + 2;                // stage-2 updates, planes [z0, zend)

        // ---- A: time-n link phases and phi of plane zz+1
        float nthx = 0.f, nthy = 0.f, nthz = 0.f, rnthx = 0.f, rnthy = 0.f, rnthz = 0.f;
        if (doB1) {
            phaseA(rc, T::a(tx, ty), pn);
            if (hasA) phaseA(rh, T::a(hax, hay), pn);
            nthx = rc.tx; nthy = rc.ty; nthz = rc.tz;
            rnthx = rh.tx; rnthy = rh.ty; rnthz = rh.tz;
            if (zz + 2 <= zend + 1) {
                const uint32_t o2 = (uint32_t)z2 * NN;
                rc = load_raw(F, o2 + coff);
                if (hasA) rh = load_raw(F, o2 + haoff);
            }
        }
        pe_cur = pe_next;
        rpe_cur = rpe_next;
        if (zz + 1 >= z0 - 1 && zz + 1 <= zend) {
            const uint32_t o1 = (uint32_t)z1 * NN;
            pe_next = load_pe<false>(F, o1 + coff);
            if (ring1) rpe_next = load_pe<false>(F, o1 + haoff);
        }
        __syncthreads();

        // ---- B: stage-1 plaquettes of plane zz, stage-2 plaquettes of plane zz-2
        float2 Qxz1 = make_float2(1.f, 0.f), Qyz1 = make_float2(1.f, 0.f);
        float2 rQxz1 = make_float2(1.f, 0.f), rQyz1 = make_float2(1.f, 0.f);
        if (doB1) {
            auto plaq1 = [&](int ex, int ey, float2 &qxz, float2 &qyz) {
                const int r0 = T::a(ex, ey), rxp = T::a(ex + 1, ey), ryp = T::a(ex, ey + 1);
                const float2 vx0 = pc.vx[r0], vy0 = pc.vy[r0], vz0 = pc.vz[r0];
                const float2 qxy = plaquette(vx0, vy0, pc.vy[rxp], pc.vx[ryp]);
                qxz = plaquette(vx0, vz0, pc.vz[rxp], pn.vx[r0]);
                qyz = plaquette(vy0, vz0, pc.vz[ryp], pn.vy[r0]);
                const int qi = T::q1(ex, ey);
                S.s1xy[qi] = qxy.y;
                S.s1xz[qi] = qxz.y;
                S.s1yz[qi] = qyz.y;
            };
            plaq1(tx, ty, Qxz1, Qyz1);
            if (ring1) plaq1(hax, hay, rQxz1, rQyz1);
            if (hasB1) {
                const int rb = T::a(b1x, b1y), rbx = T::a(b1x + 1, b1y), rby = T::a(b1x, b1y + 1);
                const float2 bx = pc.vx[rb], by = pc.vy[rb], bz = pc.vz[rb];
                const int qh = T::q1(b1x, b1y);
                S.s1xy[qh] = plaquette(bx, by, pc.vy[rbx], pc.vx[rby]).y;
                if (rowB1) S.s1yz[qh] = plaquette(by, bz, pc.vz[rby], pn.vy[rb]).y;
                else S.s1xz[qh] = plaquette(bx, bz, pc.vz[rbx], pn.vx[rb]).y;
            }
        }
        float2 Qxz2 = make_float2(1.f, 0.f), Qyz2 = make_float2(1.f, 0.f);
        if (doB2) {
            const T::Plane1 &qc = S.p1[b1m2], &qn = S.p1[b1m1];
            const int r0 = T::h(tx, ty), rxp = T::h(tx + 1, ty), ryp = T::h(tx, ty + 1);
            const float2 vx0 = qc.vx[r0], vy0 = qc.vy[r0], vz0 = qc.vz[r0];
            const float2 qxy = plaquette(vx0, vy0, qc.vy[rxp], qc.vx[ryp]);
            Qxz2 = plaquette(vx0, vz0, qc.vz[rxp], qn.vx[r0]);
            Qyz2 = plaquette(vy0, vz0, qc.vz[ryp], qn.vy[r0]);
            const int qi = T::q2(tx, ty);
            S.s2xy[qi] = qxy.y;
            S.s2xz[qi] = Qxz2.y;
            S.s2yz[qi] = Qyz2.y;
            if (hasB2) {
                const int rb = T::h(b2x, b2y), rbx = T::h(b2x + 1, b2y), rby = T::h(b2x, b2y + 1);
                const float2 bx = qc.vx[rb], by = qc.vy[rb], bz = qc.vz[rb];
                const int qh = T::q2(b2x, b2y);
                S.s2xy[qh] = plaquette(bx, by, qc.vy[rbx], qc.vx[rby]).y;
                if (rowB2) S.s2yz[qh] = plaquette(by, bz, qc.vz[rby], qn.vy[rb]).y;
                else S.s2xz[qh] = plaquette(bx, bz, qc.vz[rbx], qn.vx[rb]).y;
            }
        }
        __syncthreads();

        // ---- C: stage-1 kick and drift of plane zz (tile and ring 1; every column,
        // ragged-tile images too, since stage 2 reads them), stage-2 of plane zz-2
        Own own0{};
        if (doC1) {
            const Kicked o = stage1(tx, ty, pc, pn, pe_cur, phPrev1, vzPrev1, sxzPrev1, syzPrev1, thx, thy, thz);
            put1(o, T::h(tx, ty), S.p1[b1]);
            own0 = Own{o.qr, o.qi, o.ex, o.ey, o.ez, o.tx, o.ty, o.tz};
            if (ring1) {
                const Kicked r = stage1(hax, hay, pc, pn, rpe_cur, rphPrev1, rvzPrev1, rsxzPrev1, rsyzPrev1, rthx,
                                        rthy, rthz);
                put1(r, T::h(hax, hay), S.p1[b1]);
            }
        }
        if (doC2 && valid) {
            const T::Plane1 &qc = S.p1[b1m2], &qn = S.p1[b1m1];
            const int r0 = T::h(tx, ty), q0 = T::q2(tx, ty);
            const Kicked o = kick_drift(
                k2, qc.ph[r0], qc.vx[r0], qc.vy[r0], qc.vz[r0], qc.ph[T::h(tx + 1, ty)], qc.ph[T::h(tx, ty + 1)],
                qn.ph[r0], qc.vx[T::h(tx - 1, ty)], qc.ph[T::h(tx - 1, ty)], qc.vy[T::h(tx, ty - 1)],
                qc.ph[T::h(tx, ty - 1)], vzPrev2, phPrev2, own2.qr, own2.qi, own2.ex, own2.ey, own2.ez, S.s2xy[q0],
                S.s2xz[q0], S.s2yz[q0], S.s2xy[T::q2(tx, ty - 1)], S.s2xy[T::q2(tx - 1, ty)],
                S.s2xz[T::q2(tx - 1, ty)], S.s2yz[T::q2(tx, ty - 1)], sxzPrev2, syzPrev2, own2.tx, own2.ty, own2.tz);
            const uint32_t go = (uint32_t)wrapN(zz - 2, N) * NN + coff;
            F.out(FQR, go, o.qr);
            F.out(FQI, go, o.qi);
            F.out(FEX, go, o.ex);
            F.out(FEY, go, o.ey);
            F.out(FEZ, go, o.ez);
            F.out(FPR, go, o.pr);
            F.out(FPI, go, o.pi);
            F.out(FTX, go, o.tx);
            F.out(FTY, go, o.ty);
            F.out(FTZ, go, o.tz);
        }

        // carry plane zz's (stage 1) and plane zz-2's (stage 2) own values on
        if (doB1) {
            const int r0 = T::a(tx, ty);
            phPrev1 = pc.ph[r0];
            vzPrev1 = pc.vz[r0];
            sxzPrev1 = Qxz1.y;
            syzPrev1 = Qyz1.y;
            if (ring1) {
                const int rr = T::a(hax, hay);
                rphPrev1 = pc.ph[rr];
                rvzPrev1 = pc.vz[rr];
                rsxzPrev1 = rQxz1.y;
                rsyzPrev1 = rQyz1.y;
            }
        }
        if (doB2) {
            const T::Plane1 &qc = S.p1[b1m2];
            phPrev2 = qc.ph[T::h(tx, ty)];
            vzPrev2 = qc.vz[T::h(tx, ty)];
            sxzPrev2 = Qxz2.y;
            syzPrev2 = Qyz2.y;
        }
        own2 = own1;
        own1 = own0;
        thx = nthx; thy = nthy; thz = nthz;
        rthx = rnthx; rthy = rnthy; rthz = rnthz;
        zc = z1; z1 = z2; z2 = next_plane(z2, N);
        b0 = b0n;
        b1 = b1 == 2 ? 0 : b1 + 1;
    }
}

}  // namespace

cudaError_t launch_step_two(const StepPtrs &p, const StepCoef &k1, const StepCoef &k2, int N, int Dz,
                            cudaStream_t st)
{
    using T = Tile2Step;
    const size_t bytes = sizeof(T::Smem);
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(step_two, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    dim3 grid((N + T::BX - 1) / T::BX, (N + T::BY - 1) / T::BY, (N + Dz - 1) / Dz);
    step_two<<<grid, dim3(32, T::BY), bytes, st>>>(p, k1, k2, N, Dz);
    return cudaGetLastError();
}

AHS_BOUNDS_COUNTER(bounds_errors_step2)

}  // namespace eng
