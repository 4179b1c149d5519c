// ahs_step.cu -- the fused leapfrog step of the lattice Abelian-Higgs engine as a
// z-marching shared-memory stencil for sm_103a.
//
// One CTA owns a 32 x BY column of sites and marches it through a chunk of z
// planes.  For every plane it
//   A  turns the link angles of plane z+1 into link phases V_i = (cos th_i, sin th_i)
//      (one sincos per link, Eq. 13) and stages them with phi in shared memory,
//      over the tile plus a one-site ring;
//   B  forms the plaquettes of plane z as products of four link phases
//      (Eq. 15: Q_ij = V_i(x) V_j(x+i) V_i(x+j)^* V_j(x)^* = exp(i alpha_ij)),
//      so sin alpha_ij = Im Q_ij and cos alpha_ij = Re Q_ij, for the tile and the
//      backward ring (row -1 needs xy and yz, column -1 needs xy and xz);
//   C  kicks Pi (covariant Laplacian, Eq. 14, minus the potential) and E
//      (lattice curl of sin alpha plus the current Im[phi^* U phi(x+i)]) with the
//      Crank-Nicolson damping of Eqs. 7-8, drifts phi and theta (Eqs. 9-10), and
//      on measurement steps accumulates the diagnostics (Eqs. diagxi, diagvel),
//      the Gauss residual and the plaquette windings.
// Values a site needs from its z-1 neighbour (phi, V_z, sin alpha_xz/yz, E_z) are
// carried in registers from the previous plane; in-plane neighbours come from
// shared memory.  Every link phase and plaquette of the tile is computed once.
// One CTA barrier per plane (between B and C).  Phase B reads the link phases of
// plane z+1 only at sites the same thread wrote in phase A (its own column, and
// the ring sites of the backward-ring plaquettes and forward-ring link phases,
// which go to the thread that loaded them); everything else it reads is at least
// a plane old.  The link phases rotate through three plane buffers, so phase A of
// plane z+1 never writes a buffer a thread still in phase C of plane z-1 reads,
// and the arrays written in B and read in C (plaquette sines, measurement data)
// alternate between two buffers, so phase B of plane z+1 never writes the one a
// thread still in phase C of plane z reads.
// Tile coordinates wrap modulo N, so ragged tiles and N < 32 need no special path.
// Site offsets are 32-bit (the handle limits N^3 below 2^32).
// Kernels: step_tiled (any step, float32 and compensated, one site per thread),
// step_pair (the plain float32 step on even N, two x-adjacent sites per thread on
// 64-wide tiles, 8-byte field accesses), step_tiled64 (FP64 precision), batch_step
// (a persistent launch over the tiles of an ensemble), and gauss_tiled (the Gauss
// residual alone, ahead of a measuring step that updates Pi and E in place).
#include "ahs_stencil.cuh"

namespace eng {
namespace {

template <int BY_, class R = float>
struct Tile {
    static constexpr int BX = 32, BY = BY_, NT = BX * BY;
    static constexpr int RX = BX + 2, RY = BY + 2, NR = RX * RY;  // links/phi: [-1, BX] x [-1, BY]
    static constexpr int SX = BX + 1, SY = BY + 1, NS = SX * SY;  // plaquettes: [-1, BX) x [-1, BY)
    static constexpr int YX = BX + 1, YY = BY + 1, NYW = YX * YY; // link phases Y: [0, BX] x [0, BY]
    static constexpr int NHA = 2 * RX + 2 * BY;                    // ring sites of phase A
    static_assert(NHA <= NT, "ring items must fit one pass of the CTA");

    using V2 = typename Real<R>::V2;
    struct Plane {
        V2 vx[NR], vy[NR], vz[NR], ph[NR];
    };
    // The arrays written in phase B and read in phase C: NB = 2 buffers by the parity
    // of the plane (the plain step, one barrier per plane), NB = 1 (the measuring
    // step, two barriers per plane)
    template <int NB>
    struct SmemT {
        Plane pl[3];
        R sxy[NB][NS], sxz[NB][NS], syz[NB][NS];
        // measurement steps only: old E for the Gauss residual, octant codes of the
        // link phases Y
        R ex[NB][NS], ey[NB][NS];
        int yx[NB][NYW], yy[NB][NYW], yz[NB][NYW];
    };
    template <bool MEASURE>
    using Smem = SmemT<MEASURE ? 1 : 2>;
    static constexpr size_t kStepBytes = offsetof(SmemT<2>, ex);
    static constexpr size_t kMeasureBytes = sizeof(SmemT<1>);

    static __device__ __forceinline__ int r(int ex, int ey) { return AHS_INDEX((ey + 1) * RX + (ex + 1), NR); }
    static __device__ __forceinline__ int q(int ex, int ey) { return AHS_INDEX((ey + 1) * SX + (ex + 1), NS); }
    static __device__ __forceinline__ int w(int ex, int ey) { return AHS_INDEX(ey * YX + ex, NYW); }
};

// One tile: the 32 x BY column at (x0, y0), planes [z0, zend).  All threads of the
// CTA call it together (it contains CTA barriers); with MEASURE the CTA's FP64
// partial sums go to `partial_row`.
template <int BY, bool MEASURE, bool STORE, bool COMP, class FA>
__device__ __forceinline__ void tile_step(typename Tile<BY, typename FA::real>::template Smem<MEASURE> &S,
                                          const FA &P,
                                          const typename Real<typename FA::real>::Coef &k, int N,
                                          int x0, int y0, int z0, int zend, double *partial_row)
{
    using R = typename FA::real;
    using V2 = typename Real<R>::V2;
    using T = Tile<BY, R>;
    const int tx = threadIdx.x, ty = threadIdx.y, t = tx + 32 * ty;
    const uint32_t NN = (uint32_t)N * (uint32_t)N;

    // core item: this thread's own site; ring items of phases A and B
    const int cx = wrapN(x0 + tx, N), cy = wrapN(y0 + ty, N);
    const uint32_t coff = (uint32_t)cx + (uint32_t)N * (uint32_t)cy;
    const bool valid = (x0 + tx < N) && (y0 + ty < N);
    int hax = 0, hay = 0;
    const bool hasA = t < T::NHA;
    if (hasA) {
        if (t < T::RX) { hax = t - 1; hay = -1; }
        else if (t < 2 * T::RX) { hax = t - T::RX - 1; hay = BY; }
        else if (t < 2 * T::RX + BY) { hax = -1; hay = t - 2 * T::RX; }
        else { hax = T::BX; hay = t - 2 * T::RX - BY; }
    }
    const uint32_t haoff = (uint32_t)wrapN(x0 + hax, N) + (uint32_t)N * (uint32_t)wrapN(y0 + hay, N);
    // phase B ring (backward plaquettes: row -1 over x in [0, BX), column -1 over y in
    // [0, BY)).  The plain step (one barrier per plane) gives each ring site to the
    // thread that loaded it in phase A; the measuring step (two barriers) gives the
    // ring to the first BX + BY threads, which also take the forward ring of the
    // measurement (Y_x/Y_z on row BY, Y_y/Y_z on column BX) -- fewer warps with ring
    // work, measured faster there.
    const bool ringRow = MEASURE ? t < T::BX : (t >= 1 && t <= T::BX);
    const bool hasB = MEASURE ? t < T::BX + BY : ringRow || (t >= 2 * T::RX && t < 2 * T::RX + BY);
    const int hbx = ringRow ? (MEASURE ? t : t - 1) : -1;
    const int hby = ringRow ? -1 : (MEASURE ? t - T::BX : t - 2 * T::RX);
    const bool yRow = ringRow;
    const bool hasY = hasB;
    const int hyx = yRow ? hbx : T::BX, hyy = yRow ? BY : hby;
    // and the old E of the backward ring for the Gauss residual
    uint32_t hboff = 0;
    if (MEASURE && hasB) hboff = (uint32_t)wrapN(x0 + hbx, N) + (uint32_t)N * (uint32_t)wrapN(y0 + hby, N);
    const uint32_t cxpoff = (uint32_t)wrapN(cx + 1, N) + (uint32_t)N * (uint32_t)cy;
    const uint32_t cypoff = (uint32_t)cx + (uint32_t)N * (uint32_t)wrapN(cy + 1, N);

    auto phaseA = [&](const Raw<R> &a, int ri, typename T::Plane &pl) {
        R s, c;
        Real<R>::link(a.tx, s, c);
        pl.vx[ri] = Real<R>::v2(c, s);
        Real<R>::link(a.ty, s, c);
        pl.vy[ri] = Real<R>::v2(c, s);
        Real<R>::link(a.tz, s, c);
        pl.vz[ri] = Real<R>::v2(c, s);
        pl.ph[ri] = Real<R>::v2(a.pr, a.pi);
    };

    // plane indices (wrapped) of zz, zz+1, zz+2, maintained incrementally
    int zc = wrapN(z0 - 1, N);
    int z1 = next_plane(zc, N);
    int z2 = next_plane(z1, N);

    // ---------------------------------------------------------------- prologue
    Raw<R> rc = load_raw(P, (uint32_t)zc * NN + coff);
    Raw<R> rh = hasA ? load_raw(P, (uint32_t)zc * NN + haoff) : Raw<R>{};
    phaseA(rc, T::r(tx, ty), S.pl[0]);
    if (hasA) phaseA(rh, T::r(hax, hay), S.pl[0]);
    R thx = rc.tx, thy = rc.ty, thz = rc.tz;   // own theta of plane zz
    rc = load_raw(P, (uint32_t)z1 * NN + coff);
    if (hasA) rh = load_raw(P, (uint32_t)z1 * NN + haoff);
    PE<R> pe_next{}, pe_cur{};
    R ezPrev = 0;
    // the Gauss residual of a measuring step, unless an earlier launch wrote it
    const bool gauss = MEASURE && k.gauss != 0;
    if (gauss) ezPrev = P.in(FEZ, (uint32_t)zc * NN + coff);
    // old E of this thread's backward-ring site (Gauss residual), loaded one plane ahead
    R eRing = 0, eRingNext = 0;

    // carried from plane zz-1 (own column)
    V2 phPrev = Real<R>::v2(0, 0), vzPrev = Real<R>::v2(1, 0);
    R sxzPrev = 0, syzPrev = 0;
    int YxCar = 0, YyCar = 0;   // octant codes of Y_x, Y_y of plane zz (measurement)

    AccT<R> acc;
    if (MEASURE) acc_zero(acc);
    if (!MEASURE) __syncthreads();   // the prologue's plane, read at neighbours in the first phase B

    int b = 0;    // plane buffer holding plane zz
    int pb = 0;   // buffer of the phase-B arrays of plane zz (always 0 when measuring)
    for (int zz = z0 - 1; zz < zend; ++zz, pb = MEASURE ? 0 : pb ^ 1) {
        const int bn = b == 2 ? 0 : b + 1;   // third buffer: see the barrier note at the top
        typename T::Plane &pc = S.pl[b];
        typename T::Plane &pn = S.pl[bn];
        R(&Sxy)[T::NS] = S.sxy[pb];
        R(&Sxz)[T::NS] = S.sxz[pb];
        R(&Syz)[T::NS] = S.syz[pb];
        int(&Syx)[T::NYW] = S.yx[pb];
        int(&Syy)[T::NYW] = S.yy[pb];
        int(&Syzw)[T::NYW] = S.yz[pb];
        R(&Sex)[T::NS] = S.ex[pb];
        R(&Sey)[T::NS] = S.ey[pb];
        const uint32_t oc = (uint32_t)zc * NN, o1 = (uint32_t)z1 * NN, o2 = (uint32_t)z2 * NN;
        // ---- A: link phases and phi of plane zz+1
        phaseA(rc, T::r(tx, ty), pn);
        if (hasA) phaseA(rh, T::r(hax, hay), pn);
        const R nthx = rc.tx, nthy = rc.ty, nthz = rc.tz;
        if (zz + 2 <= zend) {
            rc = load_raw(P, o2 + coff);
            if (hasA) rh = load_raw(P, o2 + haoff);
        }
        pe_cur = pe_next;
        if (zz + 1 < zend) pe_next = load_pe<COMP>(P, o1 + coff);
        if (MEASURE) {
            eRing = eRingNext;
            if (gauss && hasB && zz + 1 < zend) eRingNext = P.in(ringRow ? FEY : FEX, o1 + hboff);
            __syncthreads();   // the measuring step's ring reads other threads' phase A
        }

        // ---- B: plaquettes of plane zz (tile + backward ring)
        const int r0 = T::r(tx, ty), rxp = T::r(tx + 1, ty), ryp = T::r(tx, ty + 1);
        const V2 vx0 = pc.vx[r0], vy0 = pc.vy[r0], vz0 = pc.vz[r0];
        // plane zz+1 at the own site (written by this thread in phase A): kept for the
        // measurement's link phases of plane zz+1 after the barrier
        const V2 vxn = pn.vx[r0], vyn = pn.vy[r0];
        const V2 pn0 = MEASURE ? pn.ph[r0] : Real<R>::v2(0, 0);
        const V2 Qxy = plaquette(vx0, vy0, pc.vy[rxp], pc.vx[ryp]);
        const V2 Qxz = plaquette(vx0, vz0, pc.vz[rxp], vxn);
        const V2 Qyz = plaquette(vy0, vz0, pc.vz[ryp], vyn);
        {
            const int qi0 = T::q(tx, ty);
            Sxy[qi0] = Qxy.y;
            Sxz[qi0] = Qxz.y;
            Syz[qi0] = Qyz.y;
        }
        if (hasB) {
            const int rb = T::r(hbx, hby), rbx = T::r(hbx + 1, hby), rby = T::r(hbx, hby + 1);
            const V2 bx = pc.vx[rb], by = pc.vy[rb], bz = pc.vz[rb];
            const int qh = T::q(hbx, hby);
            Sxy[qh] = plaquette(bx, by, pc.vy[rbx], pc.vx[rby]).y;
            if (ringRow) Syz[qh] = plaquette(by, bz, pc.vz[rby], pn.vy[rb]).y;
            else Sxz[qh] = plaquette(bx, bz, pc.vz[rbx], pn.vx[rb]).y;
        }
        V2 hzB = Real<R>::v2(0, 0);
        R jzB = 0;
        if (MEASURE && zz >= z0) {
            // link phases Y_i of plane zz on the tile (Y_x, Y_y carried from the
            // previous plane) and on its forward ring; old E of the backward ring.
            // Y_z = arg(conj(phi) U_z phi(x+z)) from the hop U_z phi(x+z) and the
            // current J_z = Im(conj(phi) U_z phi(x+z)) the kick of phase C uses
            const int wi = T::w(tx, ty);
            const V2 p0 = pc.ph[r0];
            hzB = cmulc(pn0, vz0);
            jzB = p0.x * hzB.y - p0.y * hzB.x;
            Syx[wi] = YxCar;
            Syy[wi] = YyCar;
            Syzw[wi] = flagged_octant(p0.x * hzB.x + p0.y * hzB.y, jzB);
            if (gauss) {
                Sex[T::q(tx, ty)] = pe_cur.ex;
                Sey[T::q(tx, ty)] = pe_cur.ey;
            }
            if (hasY) {
                const int rh0 = T::r(hyx, hyy), wh = T::w(hyx, hyy);
                const V2 hp = pc.ph[rh0];
                if (yRow) {   // row BY: Y_x
                    const V2 q = pc.ph[T::r(hyx + 1, hyy)], v = pc.vx[rh0];
                    Syx[wh] = link_code(hp.x, hp.y, q.x, q.y, v.x, v.y);
                } else {      // column BX: Y_y
                    const V2 q = pc.ph[T::r(hyx, hyy + 1)], v = pc.vy[rh0];
                    Syy[wh] = link_code(hp.x, hp.y, q.x, q.y, v.x, v.y);
                }
                const V2 q = pn.ph[rh0], v = pc.vz[rh0];
                Syzw[wh] = link_code(hp.x, hp.y, q.x, q.y, v.x, v.y);
            }
            if (gauss && hasB) {
                if (ringRow) Sey[T::q(hbx, hby)] = eRing;
                else Sex[T::q(hbx, hby)] = eRing;
            }
        }
        __syncthreads();

        // measurement: link phases Y_x, Y_y of plane zz+1 on every column of the tile
        // (ragged-tile columns too: they are the periodic images the ring reads)
        int YxNext = 0, YyNext = 0;
        if (MEASURE) {
            const V2 qxn = pn.ph[rxp], qyn = pn.ph[ryp];
            YxNext = link_code(pn0.x, pn0.y, qxn.x, qxn.y, vxn.x, vxn.y);
            YyNext = link_code(pn0.x, pn0.y, qyn.x, qyn.y, vyn.x, vyn.y);
        }

        // ---- C: kick and drift of plane zz
        const V2 p0 = pc.ph[r0];
        if (zz >= z0 && valid) {
            const int rxm = T::r(tx - 1, ty), rym = T::r(tx, ty - 1);
            // forward hops U_i(x) phi(x+i) = conj(V_i) phi(x+i)
            const V2 hx = cmulc(pc.ph[rxp], vx0);
            const V2 hy = cmulc(pc.ph[ryp], vy0);
            const V2 hz = MEASURE ? hzB : cmulc(pn.ph[r0], vz0);
            // backward hops U_i(x-i)^* phi(x-i) = V_i(x-i) phi(x-i)
            const V2 bxh = cmul(pc.vx[rxm], pc.ph[rxm]);
            const V2 byh = cmul(pc.vy[rym], pc.ph[rym]);
            const V2 bzh = cmul(vzPrev, phPrev);
            const R hsr = ((hx.x + bxh.x) + (hy.x + byh.x)) + (hz.x + bzh.x);
            const R hsi = ((hx.y + bxh.y) + (hy.y + byh.y)) + (hz.y + bzh.y);
            const R mod2 = p0.x * p0.x + p0.y * p0.y;
            const R potf = k.kpi_pot * (mod2 - k.sigma2);
            R qnr, qni, qnrl = 0, qnil = 0;
            if constexpr (COMP) {
                comp_update(k.cpi, pe_cur.qr, pe_cur.qrl, k.kpi_lap * (hsr - 6.f * p0.x) - potf * p0.x, qnr, qnrl);
                comp_update(k.cpi, pe_cur.qi, pe_cur.qil, k.kpi_lap * (hsi - 6.f * p0.y) - potf * p0.y, qni, qnil);
            } else {
                qnr = k.cpi * pe_cur.qr + k.kpi_lap * (hsr - R(6) * p0.x) - potf * p0.x;
                qni = k.cpi * pe_cur.qi + k.kpi_lap * (hsi - R(6) * p0.y) - potf * p0.y;
            }
            // currents J_i = Im(conj(phi) U_i phi(x+i))
            const R jx = p0.x * hx.y - p0.y * hx.x;
            const R jy = p0.x * hy.y - p0.y * hy.x;
            const R jz = MEASURE ? jzB : p0.x * hz.y - p0.y * hz.x;
            const R sxy = Qxy.y, sxz = Qxz.y, syz = Qyz.y;
            const R cxv = -(sxy - Sxy[T::q(tx, ty - 1)]) - (sxz - sxzPrev);
            const R cyv = (sxy - Sxy[T::q(tx - 1, ty)]) - (syz - syzPrev);
            const R czv = (sxz - Sxz[T::q(tx - 1, ty)]) + (syz - Syz[T::q(tx, ty - 1)]);
            R enx, eny, enz, enxl = 0, enyl = 0, enzl = 0;
            if constexpr (COMP) {
                comp_update(k.ce, pe_cur.ex, pe_cur.exl, k.ke_curl * cxv + k.ke_cur * jx, enx, enxl);
                comp_update(k.ce, pe_cur.ey, pe_cur.eyl, k.ke_curl * cyv + k.ke_cur * jy, eny, enyl);
                comp_update(k.ce, pe_cur.ez, pe_cur.ezl, k.ke_curl * czv + k.ke_cur * jz, enz, enzl);
            } else {
                enx = k.ce * pe_cur.ex + k.ke_curl * cxv + k.ke_cur * jx;
                eny = k.ce * pe_cur.ey + k.ke_curl * cyv + k.ke_cur * jy;
                enz = k.ce * pe_cur.ez + k.ke_curl * czv + k.ke_cur * jz;
            }

            if (MEASURE) {
                // diagnostics (Eqs. diagxi, diagvel) with explicit roundings: the
                // momenta at n are the means of those at n -+ 1/2.  A mean is half the
                // sum, so its square is a quarter of the sum's -- scalings by powers of
                // two are exact, so K = |sum|^2 / 4 and El = (m_el / 4) |sum|^2 (m_el
                // carries the 1/4) give the bits of squaring the means
                const R quarter = R(0.25), third = R(1) / R(3), one = R(1);
                auto sum = [&](R a, R al, R b, R bl) {
                    return COMP ? rn_add(rn_add(a, b), rn_add(al, bl)) : rn_add(a, b);
                };
                auto sq2 = [](R a, R b) { return rn_fma(a, a, rn_mul(b, b)); };
                const R K = rn_mul(quarter, sq2(sum(pe_cur.qr, pe_cur.qrl, qnr, qnrl), sum(pe_cur.qi, pe_cur.qil, qni, qnil)));
                const R G = rn_mul(k.m_grad, rn_add(rn_add(sq2(rn_sub(hx.x, p0.x), rn_sub(hx.y, p0.y)),
                                                           sq2(rn_sub(hy.x, p0.x), rn_sub(hy.y, p0.y))),
                                                    sq2(rn_sub(hz.x, p0.x), rn_sub(hz.y, p0.y))));
                const R dm = rn_sub(mod2, k.sigma2);
                const R V = rn_mul(rn_mul(k.m_pot, dm), dm);
                const R ebx = sum(pe_cur.ex, pe_cur.exl, enx, enxl);
                const R eby = sum(pe_cur.ey, pe_cur.eyl, eny, enyl);
                const R ebz = sum(pe_cur.ez, pe_cur.ezl, enz, enzl);
                const R El = rn_mul(k.m_el, rn_fma(ebz, ebz, sq2(ebx, eby)));
                const R B = rn_mul(k.m_mag, rn_add(rn_add(rn_sub(one, Qxy.x), rn_sub(one, Qxz.x)), rn_sub(one, Qyz.x)));
                const R L = rn_sub(rn_add(rn_sub(rn_sub(K, G), V), El), B);
                const R rho = rn_add(rn_add(rn_add(rn_add(K, G), V), El), B);
                const R pres = rn_add(rn_sub(rn_sub(K, rn_mul(G, third)), V), rn_mul(rn_add(El, B), third));
                const R g = gauss ? gauss_site(pe_cur.ex, Sex[T::q(tx - 1, ty)], pe_cur.ey, Sey[T::q(tx, ty - 1)],
                                               pe_cur.ez, ezPrev, k.inv_dx, k.m_gauss, p0.x, p0.y, pe_cur.qr,
                                               pe_cur.qi)
                                  : R(0);
                acc.s[Q_K] = rn_add(acc.s[Q_K], K);
                acc.s[Q_G] = rn_add(acc.s[Q_G], G);
                acc.s[Q_V] = rn_add(acc.s[Q_V], V);
                acc.s[Q_EL] = rn_add(acc.s[Q_EL], El);
                acc.s[Q_B] = rn_add(acc.s[Q_B], B);
                acc.s[Q_L] = rn_add(acc.s[Q_L], L);
                acc.s[Q_KL] = rn_fma(K, L, acc.s[Q_KL]);
                acc.s[Q_GL] = rn_fma(G, L, acc.s[Q_GL]);
                acc.s[Q_PL] = rn_fma(pres, L, acc.s[Q_PL]);
                acc.s[Q_RL] = rn_fma(rho, L, acc.s[Q_RL]);
                acc.s[Q_G2] = square_add(g, acc.s[Q_G2]);
                acc.gmax = fmax(acc.gmax, fabs(g));
                if (!isfinite(rho) || !isfinite(L) || !isfinite(g)) acc.nf += 1;

                // plaquette windings with lower corner x, from the flagged codes of
                // their twelve distinct phases; a flagged one is recomputed in FP64
                const int wi = T::w(tx, ty);
                const int Yx = YxCar, Yy = YyCar, Yz = Syzw[wi];
                const int Yyx = Syy[T::w(tx + 1, ty)], Yxy = Syx[T::w(tx, ty + 1)];
                const int Yzx = Syzw[T::w(tx + 1, ty)], Yzy = Syzw[T::w(tx, ty + 1)];
                const int cxy = flagged_octant(Qxy.x, Qxy.y), cxz = flagged_octant(Qxz.x, Qxz.y);
                const int cyz = flagged_octant(Qyz.x, Qyz.y);
                int nxy, nxz, nyz;
                if (((Yx | Yy | Yz | Yyx | Yxy | Yzx | Yzy | YxNext | YyNext | cxy | cxz | cyz) & 8) == 0) {
                    nxy = winding_codes(Yx, Yyx, Yxy, Yy, cxy);
                    nxz = winding_codes(Yx, Yzx, YxNext, Yz, cxz);
                    nyz = winding_codes(Yy, Yzy, YyNext, Yz, cyz);
                } else {
                    const uint32_t cxypoff = (uint32_t)wrapN(cx + 1, N) + (uint32_t)N * (uint32_t)wrapN(cy + 1, N);
                    unsigned long long codes = 0;
                    const int cs[12] = {Yx, Yy, Yz, Yyx, Yxy, Yzx, Yzy, YxNext, YyNext, cxy, cxz, cyz};
#pragma unroll
                    for (int c = 0; c < 12; ++c) codes |= (unsigned long long)(cs[c] & 15) << (4 * c);
                    const int3 w = site_windings_flagged(P.src(FPR), P.src(FPI), P.src(FTX), P.src(FTY), P.src(FTZ),
                                                         NN * (uint32_t)N, oc + coff, oc + cxpoff, oc + cypoff,
                                                         o1 + coff, oc + cxypoff, o1 + cxpoff, o1 + cypoff, codes);
                    nxy = w.x;
                    nxz = w.y;
                    nyz = w.z;
                }
                acc.wind += abs(nxy) + abs(nxz) + abs(nyz);
            }

            if (STORE) {
                const uint32_t o = oc + coff;
                P.out(FQR, o, qnr);
                P.out(FQI, o, qni);
                P.out(FEX, o, enx);
                P.out(FEY, o, eny);
                P.out(FEZ, o, enz);
                P.out(FPR, o, p0.x + k.dphi * (COMP ? qnr + qnrl : qnr));
                P.out(FPI, o, p0.y + k.dphi * (COMP ? qni + qnil : qni));
                if constexpr (COMP) {
                    P.out(FQRL, o, qnrl);
                    P.out(FQIL, o, qnil);
                    P.out(FEXL, o, enxl);
                    P.out(FEYL, o, enyl);
                    P.out(FEZL, o, enzl);
                }
                R t1x = thx + k.dtheta * (COMP ? enx + enxl : enx);
                R t1y = thy + k.dtheta * (COMP ? eny + enyl : eny);
                R t1z = thz + k.dtheta * (COMP ? enz + enzl : enz);
                if (k.wrap) {
                    if constexpr (std::is_same<R, float>::value) {
                        t1x += kTwoPiF * floorf((kPiF - t1x) * kInvTwoPiF);
                        t1y += kTwoPiF * floorf((kPiF - t1y) * kInvTwoPiF);
                        t1z += kTwoPiF * floorf((kPiF - t1z) * kInvTwoPiF);
                    } else {
                        t1x += 2.0 * kPiD * floor((kPiD - t1x) / (2.0 * kPiD));
                        t1y += 2.0 * kPiD * floor((kPiD - t1y) / (2.0 * kPiD));
                        t1z += 2.0 * kPiD * floor((kPiD - t1z) / (2.0 * kPiD));
                    }
                }
                P.out(FTX, o, t1x);
                P.out(FTY, o, t1y);
                P.out(FTZ, o, t1z);
            }
        }
        // carry plane zz's own-column values to plane zz+1
        phPrev = p0;
        vzPrev = vz0;
        sxzPrev = Qxz.y;
        syzPrev = Qyz.y;
        if (gauss && zz >= z0) ezPrev = pe_cur.ez;
        YxCar = YxNext;
        YyCar = YyNext;
        thx = nthx; thy = nthy; thz = nthz;
        zc = z1; z1 = z2; z2 = next_plane(z2, N);
        b = bn;
    }

    if (MEASURE) block_reduce_store<32 * BY>(acc, partial_row, gauss ? ROW_ALL : ROW_NO_GAUSS);
}

// Residency: a plain step fits 64 registers, so four 8-warp CTAs share an SM
// (32 warps); the measuring step needs 128 (two CTAs).
template <int BY, bool MEASURE, bool STORE, bool COMP>
__global__ void __launch_bounds__(32 * BY, (MEASURE ? 16 : 32) / BY)
    step_tiled(StepPtrs P, StepCoef k, int N, int Dz, double *partials)
{
    using T = Tile<BY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::template Smem<MEASURE> &S = *reinterpret_cast<typename T::template Smem<MEASURE> *>(smem_raw);
    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * Dz;
    const size_t bi = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    tile_step<BY, MEASURE, STORE, COMP>(S, ParamFields{P, (uint32_t)N * (uint32_t)N * (uint32_t)N}, k, N, x0, y0, z0, min(z0 + Dz, N),
                                        MEASURE ? partials + bi * NQ : nullptr);
}

// Persistent batched step: every CTA claims tiles of the work list one at a time
// from the step's ticket counter (so tiles of unequal cost balance dynamically)
// and runs them; the list is ordered by the members' last step, so at step n the
// tiles of members still running form the prefix live[n].  The member's field
// base and coefficients are staged per tile.
// FP64 precision: the same tile march in double (8-row tiles; two CTAs per SM for
// a plain step, one for a measuring step).
template <bool MEASURE, bool STORE>
__global__ void __launch_bounds__(256, MEASURE ? 1 : 2)
    step_tiled64(StepPtrs64 P, StepCoef64 k, int N, int Dz, double *partials)
{
    using T = Tile<8, double>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::template Smem<MEASURE> &S = *reinterpret_cast<typename T::template Smem<MEASURE> *>(smem_raw);
    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * 8, z0 = blockIdx.z * Dz;
    const size_t bi = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    tile_step<8, MEASURE, STORE, false>(S, ParamFields64{P, (uint32_t)N * (uint32_t)N * (uint32_t)N}, k, N, x0, y0, z0, min(z0 + Dz, N),
                                        MEASURE ? partials + bi * NQ : nullptr);
}

template <int BY, bool MEASURE>
__global__ void __launch_bounds__(32 * BY, (MEASURE ? 16 : 32) / BY) batch_step(BatchLaunch L, int dn)
{
    using T = Tile<BY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::template Smem<MEASURE> &S = *reinterpret_cast<typename T::template Smem<MEASURE> *>(smem_raw);
    __shared__ StepCoef sk;
    __shared__ int s_w;
    const int64_t n = *L.counter + dn;
    const int par = (int)(n & 1);
    const int live = L.live[n];
    const int t = threadIdx.x + 32 * threadIdx.y;
    for (;;) {
        __syncthreads();   // everyone is done with s_w and sk of the previous tile
        if (t == 0) s_w = atomicAdd(L.tickets + n, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= live) break;
        const BatchTile tl = L.tiles[w];
        const BatchMember &m = L.members[tl.member];
        if (t < (int)(sizeof(StepCoef) / sizeof(float)))
            reinterpret_cast<float *>(&sk)[t] = reinterpret_cast<const float *>(L.coef + (size_t)tl.member * L.coef_stride + n)[t];
        const uint32_t V = (uint32_t)m.N * (uint32_t)m.N * (uint32_t)m.N;
        const ArenaFields fa{m.base, par ? 10u * V : 0u, par ? 0u : 10u * V, V};
        __syncthreads();
        tile_step<BY, MEASURE, true, false>(S, fa, sk, m.N, tl.x0, tl.y0, tl.z0, tl.zend,
                                     MEASURE ? L.partials + (size_t)w * NQ : nullptr);
    }
}

template <int BY, bool MEASURE>
int batch_occupancy()
{
    using T = Tile<BY>;
    const size_t bytes = MEASURE ? T::kMeasureBytes : T::kStepBytes;
    if (cudaFuncSetAttribute(batch_step<BY, MEASURE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step<BY, MEASURE>, 32 * BY, bytes) != cudaSuccess)
        return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return per_sm * sms;
}

template <int BY, bool MEASURE>
cudaError_t launch_batch_variant(const BatchLaunch &L, int dn, int grid, cudaStream_t st)
{
    // the dynamic shared-memory limit was raised by batch_occupancy() when the
    // launch was sized, before any launch or graph capture
    using T = Tile<BY>;
    const size_t bytes = MEASURE ? T::kMeasureBytes : T::kStepBytes;
    batch_step<BY, MEASURE><<<grid, dim3(32, BY), bytes, st>>>(L, dn);
    return cudaGetLastError();
}

template <int BY, bool M, bool S, bool C>
cudaError_t launch_variant(const StepPtrs &p, const StepCoef &k, int N, int Dz, double *partials, cudaStream_t st)
{
    using T = Tile<BY>;
    const size_t bytes = M ? T::kMeasureBytes : T::kStepBytes;
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(step_tiled<BY, M, S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    dim3 block(32, BY);
    dim3 grid((N + 31) / 32, (N + BY - 1) / BY, (N + Dz - 1) / Dz);
    step_tiled<BY, M, S, C><<<grid, block, bytes, st>>>(p, k, N, Dz, partials);
    return cudaGetLastError();
}

template <bool M, bool S>
cudaError_t launch_variant64(const StepPtrs64 &p, const StepCoef64 &k, int N, int Dz, double *partials,
                             cudaStream_t st)
{
    using T = Tile<8, double>;
    const size_t bytes = M ? T::kMeasureBytes : T::kStepBytes;
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(step_tiled64<M, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    dim3 grid((N + 31) / 32, (N + 7) / 8, (N + Dz - 1) / Dz);
    step_tiled64<M, S><<<grid, dim3(32, 8), bytes, st>>>(p, k, N, Dz, partials);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- paired plain step
// The plain step (no measurement, float32) on 64 x BY tiles with two x-adjacent
// sites per thread: each field of the pair is one 8-byte load or store, the link
// phases of the pair go to shared memory as one 16-byte store per component, and
// the per-plane bookkeeping serves two sites.  The arithmetic of each site is that
// of tile_step, so the fields are bit-identical.  Needs an even N: a pair then
// never straddles the periodic wrap and its offset is even (8-byte aligned).
template <int BY_>
struct Tile2 {
    static constexpr int BX = 64, BY = BY_, NT = 32 * BY;
    static constexpr int RX = BX + 2;                                // ring sites per row: x in [-1, BX]
    static constexpr int RXP = BX + 4, RY = BY + 2, NR = RXP * RY;   // x in [-2, BX+1] (-2, BX+1: padding)
    static constexpr int SXP = BX + 2, NS = SXP * (BY + 1);          // plaquettes: x in [-2, BX), y in [-1, BY)
    static constexpr int NHA = 2 * RX + 2 * BY;
    static_assert(NHA <= NT, "ring items must fit one pass of the CTA");
    struct Plane {
        float2 vx[NR], vy[NR], vz[NR], ph[NR];
    };
    // plaquette sines: written in phase B, read in phase C, two buffers by the
    // parity of the plane
    struct Sines {
        alignas(16) float sxy[NS];
        alignas(16) float sxz[NS];
        alignas(16) float syz[NS];
    };
    struct Smem {
        Plane pl[3];
        Sines sn[2];
    };
    // the pair reads and writes link phases and phi as float4, plaquette sines as
    // float2, at even indices
    static_assert(sizeof(Plane) % 16 == 0 && (NR * sizeof(float2)) % 16 == 0 && SXP % 2 == 0 &&
                      sizeof(Sines) % 16 == 0,
                  "pair accesses must stay aligned");
    // even for even ex: the pair (ex, ex+1) is one aligned float4 / float2
    static __device__ __forceinline__ int r(int ex, int ey) { return AHS_INDEX((ey + 1) * RXP + (ex + 2), NR); }
    static __device__ __forceinline__ int q(int ex, int ey) { return AHS_INDEX((ey + 1) * SXP + (ex + 2), NS); }
};

// One paired tile: the 64 x BY column at (x0, y0), planes [z0, zend), plain step.
// All threads of the CTA call it together (it contains CTA barriers).
template <int BY, class FA>
__device__ __forceinline__ void pair_tile(typename Tile2<BY>::Smem &S, const FA &F, const StepCoef &k, int N, int x0,
                                          int y0, int z0, int zend)
{
    using T = Tile2<BY>;
    using V2 = float2;
    const int tx = threadIdx.x, ty = threadIdx.y, t = tx + 32 * ty;
    const uint32_t NN = (uint32_t)N * (uint32_t)N;

    // core pair: sites ex and ex+1 of row ty
    const int ex = 2 * tx;
    const int cx = wrapN(x0 + ex, N), cy = wrapN(y0 + ty, N);
    const uint32_t coff = (uint32_t)cx + (uint32_t)N * (uint32_t)cy;
    const bool valid = (x0 + ex < N) && (y0 + ty < N);
    // ring items (single sites) of phases A and B
    int hax = 0, hay = 0;
    const bool hasA = t < T::NHA;
    if (hasA) {
        if (t < T::RX) { hax = t - 1; hay = -1; }
        else if (t < 2 * T::RX) { hax = t - T::RX - 1; hay = BY; }
        else if (t < 2 * T::RX + BY) { hax = -1; hay = t - 2 * T::RX; }
        else { hax = T::BX; hay = t - 2 * T::RX - BY; }
    }
    const uint32_t haoff = (uint32_t)wrapN(x0 + hax, N) + (uint32_t)N * (uint32_t)wrapN(y0 + hay, N);
    // phase B ring (row -1 over x in [0, BX), column -1 over y in [0, BY)): each
    // site goes to the thread that loaded it in phase A
    const bool ringRow = t >= 1 && t <= T::BX;
    const bool hasB = ringRow || (t >= 2 * T::RX && t < 2 * T::RX + BY);
    const int hbx = ringRow ? t - 1 : -1, hby = ringRow ? -1 : t - 2 * T::RX;

    struct Raw2 {
        float2 tx, ty, tz, pr, pi;   // .x site ex, .y site ex+1
    };
    struct PE2 {
        float2 qr, qi, ex, ey, ez;
    };
    auto load_raw2 = [&](uint32_t o) {
        Raw2 a;
        a.tx = F.in2(FTX, o); a.ty = F.in2(FTY, o); a.tz = F.in2(FTZ, o);
        a.pr = F.in2(FPR, o); a.pi = F.in2(FPI, o);
        return a;
    };
    auto load_pe2 = [&](uint32_t o) {
        PE2 a;
        a.qr = F.in2(FQR, o); a.qi = F.in2(FQI, o);
        a.ex = F.in2(FEX, o); a.ey = F.in2(FEY, o); a.ez = F.in2(FEZ, o);
        return a;
    };
    auto phaseA2 = [&](const Raw2 &a, typename T::Plane &pl) {
        const int ri = T::r(ex, ty);
        float s0, c0, s1, c1;
        link_sincos(a.tx.x, s0, c0);
        link_sincos(a.tx.y, s1, c1);
        *reinterpret_cast<float4 *>(&pl.vx[ri]) = make_float4(c0, s0, c1, s1);
        link_sincos(a.ty.x, s0, c0);
        link_sincos(a.ty.y, s1, c1);
        *reinterpret_cast<float4 *>(&pl.vy[ri]) = make_float4(c0, s0, c1, s1);
        link_sincos(a.tz.x, s0, c0);
        link_sincos(a.tz.y, s1, c1);
        *reinterpret_cast<float4 *>(&pl.vz[ri]) = make_float4(c0, s0, c1, s1);
        *reinterpret_cast<float4 *>(&pl.ph[ri]) = make_float4(a.pr.x, a.pi.x, a.pr.y, a.pi.y);
    };
    auto phaseA1 = [&](const Raw<float> &a, typename T::Plane &pl) {
        const int ri = T::r(hax, hay);
        float s, c;
        link_sincos(a.tx, s, c);
        pl.vx[ri] = make_float2(c, s);
        link_sincos(a.ty, s, c);
        pl.vy[ri] = make_float2(c, s);
        link_sincos(a.tz, s, c);
        pl.vz[ri] = make_float2(c, s);
        pl.ph[ri] = make_float2(a.pr, a.pi);
    };

    int zc = wrapN(z0 - 1, N);
    int z1 = next_plane(zc, N);
    int z2 = next_plane(z1, N);

    Raw2 rc = load_raw2((uint32_t)zc * NN + coff);
    Raw<float> rh = hasA ? load_raw(F, (uint32_t)zc * NN + haoff) : Raw<float>{};
    phaseA2(rc, S.pl[0]);
    if (hasA) phaseA1(rh, S.pl[0]);
    float2 thx = rc.tx, thy = rc.ty, thz = rc.tz;   // own theta pair of plane zz
    rc = load_raw2((uint32_t)z1 * NN + coff);
    if (hasA) rh = load_raw(F, (uint32_t)z1 * NN + haoff);
    PE2 pe_next{}, pe_cur{};

    // carried from plane zz-1 (own columns), per site of the pair
    V2 phPrev[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    V2 vzPrev[2] = {make_float2(1.f, 0.f), make_float2(1.f, 0.f)};
    float sxzPrev[2] = {0.f, 0.f}, syzPrev[2] = {0.f, 0.f};

    __syncthreads();   // the prologue's plane, read at neighbours in the first phase B

    int b = 0, pb = 0;
    for (int zz = z0 - 1; zz < zend; ++zz, pb ^= 1) {
        const int bn = b == 2 ? 0 : b + 1;
        typename T::Plane &pc = S.pl[b];
        typename T::Plane &pn = S.pl[bn];
        typename T::Sines &Sn = S.sn[pb];
        const uint32_t oc = (uint32_t)zc * NN, o1 = (uint32_t)z1 * NN, o2 = (uint32_t)z2 * NN;
        // ---- A: link phases and phi of plane zz+1
        phaseA2(rc, pn);
        if (hasA) phaseA1(rh, pn);
        const float2 nthx = rc.tx, nthy = rc.ty, nthz = rc.tz;
        if (zz + 2 <= zend) {
            rc = load_raw2(o2 + coff);
            if (hasA) rh = load_raw(F, o2 + haoff);
        }
        pe_cur = pe_next;
        if (zz + 1 < zend) pe_next = load_pe2(o1 + coff);

        // ---- B: plaquettes of plane zz (the pair + backward ring)
        V2 Qxy[2], Qxz[2], Qyz[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r0 = T::r(ex + j, ty), rxp = r0 + 1, ryp = r0 + T::RXP;
            const V2 vx0 = pc.vx[r0], vy0 = pc.vy[r0], vz0 = pc.vz[r0];
            Qxy[j] = plaquette(vx0, vy0, pc.vy[rxp], pc.vx[ryp]);
            Qxz[j] = plaquette(vx0, vz0, pc.vz[rxp], pn.vx[r0]);
            Qyz[j] = plaquette(vy0, vz0, pc.vz[ryp], pn.vy[r0]);
        }
        {
            const int qi0 = T::q(ex, ty);
            *reinterpret_cast<float2 *>(&Sn.sxy[qi0]) = make_float2(Qxy[0].y, Qxy[1].y);
            *reinterpret_cast<float2 *>(&Sn.sxz[qi0]) = make_float2(Qxz[0].y, Qxz[1].y);
            *reinterpret_cast<float2 *>(&Sn.syz[qi0]) = make_float2(Qyz[0].y, Qyz[1].y);
        }
        if (hasB) {
            const int rb = T::r(hbx, hby), rbx = T::r(hbx + 1, hby), rby = T::r(hbx, hby + 1);
            const V2 bx = pc.vx[rb], by = pc.vy[rb], bz = pc.vz[rb];
            const int qh = T::q(hbx, hby);
            Sn.sxy[qh] = plaquette(bx, by, pc.vy[rbx], pc.vx[rby]).y;
            if (ringRow) Sn.syz[qh] = plaquette(by, bz, pc.vz[rby], pn.vy[rb]).y;
            else Sn.sxz[qh] = plaquette(bx, bz, pc.vz[rbx], pn.vx[rb]).y;
        }
        __syncthreads();

        // ---- C: kick and drift of plane zz, both sites
        V2 p0s[2], vz0s[2];
        if (zz >= z0 && valid) {
            float qn[2][2], en[2][3];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r0 = T::r(ex + j, ty), rxp = r0 + 1, ryp = r0 + T::RXP;
                const int rxm = r0 - 1, rym = r0 - T::RXP;
                const V2 p0 = pc.ph[r0], vx0 = pc.vx[r0], vy0 = pc.vy[r0], vz0 = pc.vz[r0];
                const float qr = j ? pe_cur.qr.y : pe_cur.qr.x, qi = j ? pe_cur.qi.y : pe_cur.qi.x;
                const float e0x = j ? pe_cur.ex.y : pe_cur.ex.x, e0y = j ? pe_cur.ey.y : pe_cur.ey.x;
                const float e0z = j ? pe_cur.ez.y : pe_cur.ez.x;
                const V2 hx = cmulc(pc.ph[rxp], vx0);
                const V2 hy = cmulc(pc.ph[ryp], vy0);
                const V2 hz = cmulc(pn.ph[r0], vz0);
                const V2 bxh = cmul(pc.vx[rxm], pc.ph[rxm]);
                const V2 byh = cmul(pc.vy[rym], pc.ph[rym]);
                const V2 bzh = cmul(vzPrev[j], phPrev[j]);
                const float hsr = ((hx.x + bxh.x) + (hy.x + byh.x)) + (hz.x + bzh.x);
                const float hsi = ((hx.y + bxh.y) + (hy.y + byh.y)) + (hz.y + bzh.y);
                const float mod2 = p0.x * p0.x + p0.y * p0.y;
                const float potf = k.kpi_pot * (mod2 - k.sigma2);
                qn[j][0] = k.cpi * qr + k.kpi_lap * (hsr - float(6) * p0.x) - potf * p0.x;
                qn[j][1] = k.cpi * qi + k.kpi_lap * (hsi - float(6) * p0.y) - potf * p0.y;
                const float jx = p0.x * hx.y - p0.y * hx.x;
                const float jy = p0.x * hy.y - p0.y * hy.x;
                const float jz = p0.x * hz.y - p0.y * hz.x;
                const float sxy = Qxy[j].y, sxz = Qxz[j].y, syz = Qyz[j].y;
                const float cxv = -(sxy - Sn.sxy[T::q(ex + j, ty - 1)]) - (sxz - sxzPrev[j]);
                const float cyv = (sxy - Sn.sxy[T::q(ex + j - 1, ty)]) - (syz - syzPrev[j]);
                const float czv = (sxz - Sn.sxz[T::q(ex + j - 1, ty)]) + (syz - Sn.syz[T::q(ex + j, ty - 1)]);
                en[j][0] = k.ce * e0x + k.ke_curl * cxv + k.ke_cur * jx;
                en[j][1] = k.ce * e0y + k.ke_curl * cyv + k.ke_cur * jy;
                en[j][2] = k.ce * e0z + k.ke_curl * czv + k.ke_cur * jz;
                p0s[j] = p0;
                vz0s[j] = vz0;
            }
            const uint32_t o = oc + coff;
            F.out2(FQR, o, qn[0][0], qn[1][0]);
            F.out2(FQI, o, qn[0][1], qn[1][1]);
            F.out2(FEX, o, en[0][0], en[1][0]);
            F.out2(FEY, o, en[0][1], en[1][1]);
            F.out2(FEZ, o, en[0][2], en[1][2]);
            F.out2(FPR, o, p0s[0].x + k.dphi * qn[0][0], p0s[1].x + k.dphi * qn[1][0]);
            F.out2(FPI, o, p0s[0].y + k.dphi * qn[0][1], p0s[1].y + k.dphi * qn[1][1]);
            float t1[2][3];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                t1[j][0] = (j ? thx.y : thx.x) + k.dtheta * en[j][0];
                t1[j][1] = (j ? thy.y : thy.x) + k.dtheta * en[j][1];
                t1[j][2] = (j ? thz.y : thz.x) + k.dtheta * en[j][2];
                if (k.wrap) {
                    t1[j][0] += kTwoPiF * floorf((kPiF - t1[j][0]) * kInvTwoPiF);
                    t1[j][1] += kTwoPiF * floorf((kPiF - t1[j][1]) * kInvTwoPiF);
                    t1[j][2] += kTwoPiF * floorf((kPiF - t1[j][2]) * kInvTwoPiF);
                }
            }
            F.out2(FTX, o, t1[0][0], t1[1][0]);
            F.out2(FTY, o, t1[0][1], t1[1][1]);
            F.out2(FTZ, o, t1[0][2], t1[1][2]);
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r0 = T::r(ex + j, ty);
                p0s[j] = pc.ph[r0];
                vz0s[j] = pc.vz[r0];
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            phPrev[j] = p0s[j];
            vzPrev[j] = vz0s[j];
            sxzPrev[j] = Qxz[j].y;
            syzPrev[j] = Qyz[j].y;
        }
        thx = nthx; thy = nthy; thz = nthz;
        zc = z1; z1 = z2; z2 = next_plane(z2, N);
        b = bn;
    }
}

template <int BY>
__global__ void __launch_bounds__(32 * BY, 16 / BY) step_pair(StepPtrs P, StepCoef k, int N, int Dz)
{
    using T = Tile2<BY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Smem &S = *reinterpret_cast<typename T::Smem *>(smem_raw);
    const int x0 = blockIdx.x * T::BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * Dz;
    pair_tile<BY>(S, ParamFields{P, (uint32_t)N * (uint32_t)N * (uint32_t)N}, k, N, x0, y0, z0, min(z0 + Dz, N));
}

// Persistent batched plain step on paired tiles (members of even side): the
// ticketed loop of batch_step over a list of 64 x BY tiles.
template <int BY>
__global__ void __launch_bounds__(32 * BY, 16 / BY) batch_pair_step(BatchLaunch L, int dn)
{
    using T = Tile2<BY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Smem &S = *reinterpret_cast<typename T::Smem *>(smem_raw);
    __shared__ StepCoef sk;
    __shared__ int s_w;
    const int64_t n = *L.counter + dn;
    const int par = (int)(n & 1);
    const int live = L.live[n];
    const int t = threadIdx.x + 32 * threadIdx.y;
    for (;;) {
        __syncthreads();   // everyone is done with s_w, sk and the shared planes of the previous tile
        if (t == 0) s_w = atomicAdd(L.tickets + n, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= live) break;
        const BatchTile tl = L.tiles[w];
        const BatchMember &m = L.members[tl.member];
        if (t < (int)(sizeof(StepCoef) / sizeof(float)))
            reinterpret_cast<float *>(&sk)[t] = reinterpret_cast<const float *>(L.coef + (size_t)tl.member * L.coef_stride + n)[t];
        const uint32_t V = (uint32_t)m.N * (uint32_t)m.N * (uint32_t)m.N;
        const ArenaFields fa{m.base, par ? 10u * V : 0u, par ? 0u : 10u * V, V};
        __syncthreads();
        pair_tile<BY>(S, fa, sk, m.N, tl.x0, tl.y0, tl.z0, tl.zend);
    }
}

int batch_pair_occupancy()
{
    using T = Tile2<8>;
    const size_t bytes = sizeof(typename T::Smem);
    if (cudaFuncSetAttribute(batch_pair_step<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_pair_step<8>, 256, bytes) != cudaSuccess)
        return 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return per_sm * sms;
}

template <int BY>
cudaError_t launch_pair(const StepPtrs &p, const StepCoef &k, int N, int Dz, cudaStream_t st)
{
    using T = Tile2<BY>;
    const size_t bytes = sizeof(typename T::Smem);
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(step_pair<BY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    dim3 grid((N + T::BX - 1) / T::BX, (N + BY - 1) / BY, (N + Dz - 1) / Dz);
    step_pair<BY><<<grid, dim3(32, BY), bytes, st>>>(p, k, N, Dz);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Gauss residual alone
// The Gauss residual of a measuring step (Eq. 5 in discrete form: the stored
// momenta at n - 1/2 with phi^n) for a measuring launch that overwrites E in place:
// the same tiles, z-chunks, per-thread order of accumulation and block reduction
// as the measuring step, writing only the Q_G2 and Q_GMAX slots of its partial
// rows, so the record equals the one the fused measurement gives.
template <int BY>
__global__ void __launch_bounds__(32 * BY) gauss_tiled(StepPtrs P, StepCoef k, int N, int Dz, double *partials)
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * BY, z0 = blockIdx.z * Dz;
    const int zend = min(z0 + Dz, N);
    const uint32_t NN = (uint32_t)N * (uint32_t)N;
    const int cx = wrapN(x0 + tx, N), cy = wrapN(y0 + ty, N);
    const uint32_t coff = (uint32_t)cx + (uint32_t)N * (uint32_t)cy;
    const uint32_t xmoff = (uint32_t)wrapN(cx - 1, N) + (uint32_t)N * (uint32_t)cy;
    const uint32_t ymoff = (uint32_t)cx + (uint32_t)N * (uint32_t)wrapN(cy - 1, N);
    const bool valid = (x0 + tx < N) && (y0 + ty < N);
    AccT<float> acc;
    acc_zero(acc);
    const uint32_t V = NN * (uint32_t)N;   // the extent of the bounds-check build's offset checks
    (void)V;
    float ezPrev = __ldg(P.ez + AHS_INDEX((uint32_t)wrapN(z0 - 1, N) * NN + coff, V));
    for (int zz = z0; zz < zend; ++zz) {
        const uint32_t o = (uint32_t)zz * NN;
        const uint32_t oc = AHS_INDEX(o + coff, V);
        const float ex = __ldg(P.ex + oc), ey = __ldg(P.ey + oc), ez = __ldg(P.ez + oc);
        if (valid) {
            const float exm = __ldg(P.ex + AHS_INDEX(o + xmoff, V)), eym = __ldg(P.ey + AHS_INDEX(o + ymoff, V));
            const float pr = __ldg(P.pr + oc), pim = __ldg(P.pim + oc);
            const float qr = __ldg(P.qr + oc), qi = __ldg(P.qi + oc);
            const float g = gauss_site(ex, exm, ey, eym, ez, ezPrev, k.inv_dx, k.m_gauss, pr, pim, qr, qi);
            acc.s[Q_G2] = square_add(g, acc.s[Q_G2]);
            acc.gmax = fmax(acc.gmax, fabs(g));
        }
        ezPrev = ez;
    }
    const size_t bi = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    block_reduce_store<32 * BY>(acc, partials + bi * NQ, ROW_GAUSS_ONLY);
}

template <int BY, bool C>
cudaError_t launch_by(const StepPtrs &p, const StepCoef &k, int N, int Dz, bool measure, bool store,
                      double *partials, cudaStream_t st)
{
    if (measure && store) return launch_variant<BY, true, true, C>(p, k, N, Dz, partials, st);
    if (measure) return launch_variant<BY, true, false, C>(p, k, N, Dz, partials, st);
    if (store) return launch_variant<BY, false, true, C>(p, k, N, Dz, partials, st);
    return cudaErrorInvalidValue;
}

// measuring launches only (the 4-row tiles serve nothing else)
template <int BY, bool C>
cudaError_t launch_measure_by(const StepPtrs &p, const StepCoef &k, int N, int Dz, bool store, double *partials,
                              cudaStream_t st)
{
    if (store) return launch_variant<BY, true, true, C>(p, k, N, Dz, partials, st);
    return launch_variant<BY, true, false, C>(p, k, N, Dz, partials, st);
}

StepShape make_shape(int N, int by, int zchunk)
{
    StepShape s;
    s.by = by;
    if (zchunk > 0) {
        s.dz = zchunk < N ? zchunk : N;
    } else {
        // several waves of CTAs on 152 SMs, marches long enough to amortise the two
        // prologue planes of each chunk; from 512^3 on, the chunk with the shortest
        // period of nine plain steps and one measuring step among those timed at
        // 512^3 (96), 768^3 (128), 1024^3 (192) and 1536^3 (128)
        s.dz = N >= 1280 ? 128 : N >= 896 ? 192 : N >= 640 ? 128 : N >= 512 ? 96 : N >= 256 ? 32 : N >= 64 ? 16
                                                                                       : (N < 8 ? N : 8);
    }
    s.blocks = ((N + 31) / 32) * ((N + s.by - 1) / s.by) * ((N + s.dz - 1) / s.dz);
    return s;
}

}  // namespace

StepShape step_shape(int N, int tile_y, int zchunk)
{
    return make_shape(N, (tile_y == 8 || tile_y == 16) ? tile_y : 8, zchunk);
}

StepShape measure_shape(int N, int tile_y, int zchunk)
{
    // 32 x 4 tiles by default: the measuring step holds two CTAs of 8 warps per SM
    // (its registers), or four of 4 warps, which wait less at the two barriers of
    // each plane and overlap each other's waits (26.2 against 27.0 ms at 1024^3,
    // 3-6% faster from 256^3 up) although the ring is relatively twice as large
    return make_shape(N, (tile_y == 4 || tile_y == 8 || tile_y == 16) ? tile_y : 4, zchunk);
}

int batch_grid(int by, bool measure)
{
    if (by == 4) return measure ? batch_occupancy<4, true>() : 0;   // 4-row tiles: measuring steps only
    if (by == 16) return measure ? batch_occupancy<16, true>() : batch_occupancy<16, false>();
    return measure ? batch_occupancy<8, true>() : batch_occupancy<8, false>();
}

int batch_pair_grid() { return batch_pair_occupancy(); }

cudaError_t launch_batch_pair_step(const BatchLaunch &L, int dn, int grid, cudaStream_t st)
{
    // the dynamic shared-memory limit was raised by batch_pair_grid() when the
    // launch was sized, before any launch or graph capture
    if (grid < 1) return cudaErrorInvalidConfiguration;
    batch_pair_step<8><<<grid, dim3(32, 8), sizeof(typename Tile2<8>::Smem), st>>>(L, dn);
    return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchLaunch &L, int by, int dn, bool measure, int grid, cudaStream_t st)
{
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (by == 4) return measure ? launch_batch_variant<4, true>(L, dn, grid, st) : cudaErrorInvalidValue;
    if (by == 16) return measure ? launch_batch_variant<16, true>(L, dn, grid, st) : launch_batch_variant<16, false>(L, dn, grid, st);
    return measure ? launch_batch_variant<8, true>(L, dn, grid, st) : launch_batch_variant<8, false>(L, dn, grid, st);
}

cudaError_t launch_step(const StepPtrs &p, const StepCoef &k, int N, const StepShape &sh, bool measure, bool store,
                        double *partials, cudaStream_t st, bool compensated)
{
    if (measure && sh.by == 4)
        return compensated ? launch_measure_by<4, true>(p, k, N, sh.dz, store, partials, st)
                           : launch_measure_by<4, false>(p, k, N, sh.dz, store, partials, st);
    if (sh.by != 8 && sh.by != 16) return cudaErrorInvalidValue;
    if (compensated) {
        if (sh.by == 16) return launch_by<16, true>(p, k, N, sh.dz, measure, store, partials, st);
        return launch_by<8, true>(p, k, N, sh.dz, measure, store, partials, st);
    }
    if (!measure && store && N % 2 == 0 && sh.by == 8) return launch_pair<8>(p, k, N, sh.dz, st);
    if (sh.by == 16) return launch_by<16, false>(p, k, N, sh.dz, measure, store, partials, st);
    return launch_by<8, false>(p, k, N, sh.dz, measure, store, partials, st);
}

cudaError_t launch_step64(const StepPtrs64 &p, const StepCoef64 &k, int N, const StepShape &sh, bool measure,
                          bool store, double *partials, cudaStream_t st)
{
    if (sh.by != 8) return cudaErrorInvalidValue;
    if (measure && store) return launch_variant64<true, true>(p, k, N, sh.dz, partials, st);
    if (measure) return launch_variant64<true, false>(p, k, N, sh.dz, partials, st);
    if (store) return launch_variant64<false, true>(p, k, N, sh.dz, partials, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_gauss(const StepPtrs &p, const StepCoef &k, int N, const StepShape &sh, double *partials,
                         cudaStream_t st)
{
    dim3 grid((N + 31) / 32, (N + sh.by - 1) / sh.by, (N + sh.dz - 1) / sh.dz);
    if (sh.by == 16) gauss_tiled<16><<<grid, dim3(32, 16), 0, st>>>(p, k, N, sh.dz, partials);
    else if (sh.by == 8) gauss_tiled<8><<<grid, dim3(32, 8), 0, st>>>(p, k, N, sh.dz, partials);
    else if (sh.by == 4) gauss_tiled<4><<<grid, dim3(32, 4), 0, st>>>(p, k, N, sh.dz, partials);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

AHS_BOUNDS_COUNTER(bounds_errors_step)

}  // namespace eng
