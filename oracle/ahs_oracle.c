/*
 * ahs_oracle.c -- plain FP64 CPU oracle of the lattice Abelian-Higgs evolution of
 * Correia & Martins, "Abelian-Higgs cosmic string evolution with multiple GPUs"
 * (arXiv:2005.14454), Sec. 2.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant with the CUDA engine; the engine never calls it.
 *
 * Everything is double precision on a periodic N^3 lattice, site index
 * idx = x + N*(y + N*z).  A state is ten contiguous planes of N^3 doubles:
 *   0 Re phi, 1 Im phi, 2 Re Pi, 3 Im Pi, 4 theta_x, 5 theta_y, 6 theta_z,
 *   7 E_x, 8 E_y, 9 E_z
 * with phi, theta at integer time n and Pi, E at n-1/2 (staggered leapfrog).
 * theta_i = dx * A_i is the compact link angle; the link variable is
 * U_i(x) = exp(-i theta_i(x))  (Eq. 13, with the dx of Eq. 16).
 *
 * Where the paper is silent or garbled, the reading taken is stated beside the
 * code it affects.
 *
 * Each function is a literal transcription of one definition: no blocking, no
 * fusion, loops in site order.  OpenMP only splits independent site loops;
 * sums are taken per z-plane and then added in plane order, so results do not
 * depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int N;
    double dx, dt, lambda0, e0, sigma, s;
    int era;        /* conformal expansion exponent p: a = (eta/eta0)^p */
    double alpha;   /* damping form factor of Eq. 11, 2 in the paper  */
    double tau0;    /* initial conformal time eta0, 1 in the paper     */
    double cool;    /* > 0: cooling run, a = 1 and delta = omega = cool (see orc_scalars) */
    double s_cg;    /* core growth: s of the steps with eta < tau_cg (see orc_scalars)  */
    double tau_cg;  /* end of the core-growth period; <= tau0: none                   */
} orc_params_t;

typedef struct {
    int64_t step;
    double tau, a;
    int64_t n_wind;
    double string_length, xi_w, xi_l, lagrangian;
    double v2_phi, v2_omega;
    double e_kin, e_grad, e_pot, e_elec, e_mag, e_total;
    double gauss_rms, gauss_max;
    int64_t nonfinite;
    /* raw site sums (no dx^3 factor) */
    double sum_K, sum_G, sum_V, sum_El, sum_B, sum_L;
    double sum_KL, sum_GL, sum_pL, sum_rhoL;
} orc_obs_t;

enum { F_PR = 0, F_PI, F_QR, F_QI, F_TX, F_TY, F_TZ, F_EX, F_EY, F_EZ, F_COUNT };

static inline int64_t vol(int N) { return (int64_t)N * N * N; }

static inline int64_t at(int N, int x, int y, int z)
{
    x %= N; if (x < 0) x += N;
    y %= N; if (y < 0) y += N;
    z %= N; if (z < 0) z += N;
    return (int64_t)x + (int64_t)N * ((int64_t)y + (int64_t)N * z);
}

/* neighbour of (x,y,z) displaced by d along axis i */
static inline int64_t nb(int N, int x, int y, int z, int i, int d)
{
    return at(N, x + (i == 0 ? d : 0), y + (i == 1 ? d : 0), z + (i == 2 ? d : 0));
}

/* ---------------------------------------------------------------------------
 * time-dependent scalars (Eqs. 7, 8, 11, 12).
 *   eta_n = eta0 + n dt,  a_n = (eta_n/eta0)^p,
 *   delta_n = (alpha/2) p dt/eta_n   (d ln a / d ln eta = p),
 *   omega_n = delta_n (1 - s),  c_n = a_n^{2s}.
 * out = {eta, a, delta, omega, c}
 * ------------------------------------------------------------------------- */
void orc_scalars(const orc_params_t *p, int64_t n, double out[5])
{
    double eta = p->tau0 + (double)n * p->dt;
    double a = pow(eta / p->tau0, (double)p->era);
    double delta = 0.5 * p->alpha * (double)p->era * p->dt / eta;
    /* Core growth (Sec. 2, after Eq. 6): a negative s lets the comoving string
     * width grow before the true equations (s = 1) shrink it again.  Read as the
     * exponent s_cg for the steps with eta < tau_cg and s after them, in omega and
     * in c, with c continuous at tau_cg (the couplings change their rate of
     * change, they do not jump): c = a^{2 s_cg} before, a_cg^{2 s_cg} (a/a_cg)^{2 s}
     * after, a_cg = a(tau_cg).  tau_cg <= tau0: constant s. */
    int grow = p->tau_cg > p->tau0;
    double s = grow && eta < p->tau_cg ? p->s_cg : p->s;
    double omega = delta * (1.0 - s);
    double c;
    if (grow && eta >= p->tau_cg) {
        double acg = pow(p->tau_cg / p->tau0, (double)p->era);
        c = pow(acg, 2.0 * p->s_cg) * pow(a / acg, 2.0 * p->s);
    } else {
        c = pow(a, 2.0 * s);
    }
    /* Cooling (the artificial damping period Sec. 2 mentions without details):
     * read as a static background, a = 1, with the same constant Crank-Nicolson
     * damping on both momenta, delta = omega = cool. */
    if (p->cool > 0.0) {
        a = 1.0;
        delta = omega = p->cool;
        c = 1.0;
    }
    out[0] = eta; out[1] = a; out[2] = delta; out[3] = omega; out[4] = c;
}

/* ---------------------------------------------------------------------------
 * SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state += golden gamma, then
 * the published 64-bit finaliser.  Used for the random-phase initial
 * condition:  u = (sm64(seed ^ sm64(idx)) >> 11) * 2^-53,  vartheta = 2 pi u.
 * ------------------------------------------------------------------------- */
static uint64_t sm64(uint64_t v)
{
    uint64_t z = v + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t idx)
{
    return (double)(sm64(seed ^ sm64(idx)) >> 11) * (1.0 / 9007199254740992.0);
}

/* random-phase initial condition (Sec. 2): phi = sigma e^{i vartheta},
 * every other field zero. */
void orc_init(const orc_params_t *p, uint64_t seed, double *F)
{
    int64_t V = vol(p->N);
    memset(F, 0, sizeof(double) * (size_t)(V * F_COUNT));
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < V; ++i) {
        double th = 2.0 * M_PI * orc_uniform(seed, (uint64_t)i);
        F[F_PR * V + i] = p->sigma * cos(th);
        F[F_PI * V + i] = p->sigma * sin(th);
    }
}

/* link variable U_i(x) = exp(-i theta) */
static inline void link(double th, double *ur, double *ui) { *ur = cos(th); *ui = -sin(th); }

/* complex product (ar + i ai)(br + i bi) */
static inline void cmul(double ar, double ai, double br, double bi, double *cr, double *ci)
{
    *cr = ar * br - ai * bi;
    *ci = ar * bi + ai * br;
}

/* plaquette angle alpha_ij(x) = theta_i(x) + theta_j(x+i) - theta_i(x+j) - theta_j(x),
 * the phase of Xi_ij of Eq. 15 (written with the standard oriented link order). */
static inline double plaq(const double *F, int N, int x, int y, int z, int i, int j)
{
    int64_t V = vol(N);
    const double *ti = F + (F_TX + i) * V;
    const double *tj = F + (F_TX + j) * V;
    return ti[at(N, x, y, z)] + tj[nb(N, x, y, z, i, 1)]
         - ti[nb(N, x, y, z, j, 1)] - tj[at(N, x, y, z)];
}

/* ---------------------------------------------------------------------------
 * Forces at integer time n (the bracketed terms of Eqs. 7 and 8), per site:
 *   FPi   = D_j^- D_j^+ phi - (lambda0/2) c_n (|phi|^2 - sigma^2) phi
 *   FE_i  = -(1/dx^3) sum_{j != i} [sin alpha_ij(x) - sin alpha_ij(x - j)]
 *           + (2 e0^2 c_n / dx) Im[phi*(x) U_i(x) phi(x+i)]
 * The covariant Laplacian is Eq. 14.  The field-strength term is the compact
 * (sine) form of -d_j^- F_ij; the current is 2 e0^2 a^{2s} Im[phi* D_i^+ phi]
 * with D_i^+ phi = (U_i phi(x+i) - phi(x))/dx.
 * out: 5 planes {Re FPi, Im FPi, FE_x, FE_y, FE_z}
 * ------------------------------------------------------------------------- */
void orc_forces(const orc_params_t *p, int64_t n, const double *F, double *out)
{
    const int N = p->N;
    const int64_t V = vol(N);
    double sc[5];
    orc_scalars(p, n, sc);
    const double c = sc[4];
    const double dx = p->dx, dx2 = dx * dx, dx3 = dx2 * dx;
    const double *pr = F + F_PR * V, *pim = F + F_PI * V;

    #pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
        int64_t s0 = at(N, x, y, z);
        double fr = pr[s0], fi = pim[s0];
        /* Eq. 14 */
        double lr = 0.0, li = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double *th = F + (F_TX + i) * V;
            int64_t sp = nb(N, x, y, z, i, 1), sm = nb(N, x, y, z, i, -1);
            double ur, ui, hr, hi;
            link(th[s0], &ur, &ui);
            cmul(ur, ui, pr[sp], pim[sp], &hr, &hi);          /* U_i(x) phi(x+i) */
            lr += hr; li += hi;
            link(th[sm], &ur, &ui);
            cmul(ur, -ui, pr[sm], pim[sm], &hr, &hi);         /* U_i(x-i)^* phi(x-i) */
            lr += hr; li += hi;
            lr -= 2.0 * fr; li -= 2.0 * fi;
        }
        lr /= dx2; li /= dx2;
        double m2 = fr * fr + fi * fi - p->sigma * p->sigma;
        out[0 * V + s0] = lr - 0.5 * p->lambda0 * c * m2 * fr;
        out[1 * V + s0] = li - 0.5 * p->lambda0 * c * m2 * fi;

        for (int i = 0; i < 3; ++i) {
            double curl = 0.0;
            for (int j = 0; j < 3; ++j) {
                if (j == i) continue;
                int xm = x - (j == 0), ym = y - (j == 1), zm = z - (j == 2);
                curl += sin(plaq(F, N, x, y, z, i, j)) - sin(plaq(F, N, xm, ym, zm, i, j));
            }
            const double *th = F + (F_TX + i) * V;
            int64_t sp = nb(N, x, y, z, i, 1);
            double ur, ui, hr, hi, jr, ji;
            link(th[s0], &ur, &ui);
            cmul(ur, ui, pr[sp], pim[sp], &hr, &hi);
            cmul(fr, -fi, hr, hi, &jr, &ji);                  /* phi^*(x) U_i(x) phi(x+i) */
            out[(2 + i) * V + s0] = -curl / dx3 + 2.0 * p->e0 * p->e0 * c * ji / dx;
        }
    }
}

/* ---------------------------------------------------------------------------
 * kick of step n (Eqs. 7, 8): Crank-Nicolson damping, leapfrog force.
 *   (1+delta) Pi^{n+1/2}  = (1-delta) Pi^{n-1/2}  + dt FPi
 *   (1+omega) E_i^{n+1/2} = (1-omega) E_i^{n-1/2} + dt FE_i
 * Writes the new momenta into out (5 planes: Re Pi, Im Pi, E_x, E_y, E_z);
 * F is left unchanged.
 * ------------------------------------------------------------------------- */
void orc_kick(const orc_params_t *p, int64_t n, const double *F, double *out)
{
    const int64_t V = vol(p->N);
    double sc[5];
    orc_scalars(p, n, sc);
    const double dl = sc[2], om = sc[3];
    orc_forces(p, n, F, out);
    #pragma omp parallel for schedule(static)
    for (int64_t s0 = 0; s0 < V; ++s0) {
        for (int k = 0; k < 2; ++k)
            out[k * V + s0] = ((1.0 - dl) * F[(F_QR + k) * V + s0] + p->dt * out[k * V + s0]) / (1.0 + dl);
        for (int i = 0; i < 3; ++i)
            out[(2 + i) * V + s0] = ((1.0 - om) * F[(F_EX + i) * V + s0] + p->dt * out[(2 + i) * V + s0]) / (1.0 + om);
    }
}

/* drift (Eqs. 9, 10): phi += dt Pi^{n+1/2}, theta_i += dt dx E_i^{n+1/2}. */
void orc_drift(const orc_params_t *p, double *F)
{
    const int64_t V = vol(p->N);
    #pragma omp parallel for schedule(static)
    for (int64_t s0 = 0; s0 < V; ++s0) {
        F[F_PR * V + s0] += p->dt * F[F_QR * V + s0];
        F[F_PI * V + s0] += p->dt * F[F_QI * V + s0];
        for (int i = 0; i < 3; ++i)
            F[(F_TX + i) * V + s0] += p->dt * p->dx * F[(F_EX + i) * V + s0];
    }
}

/* Kick only: replace Pi, E in F by their step-n update (used by the
 * time-reversal pin). work: 5 planes. */
void orc_kick_inplace(const orc_params_t *p, int64_t n, double *F, double *work)
{
    const int64_t V = vol(p->N);
    orc_kick(p, n, F, work);
    memcpy(F + F_QR * V, work, sizeof(double) * (size_t)(2 * V));
    memcpy(F + F_EX * V, work + 2 * V, sizeof(double) * (size_t)(3 * V));
}

/* One full leapfrog step n -> n+1: kick with the old phi, theta (all sites
 * read the same time level), then drift.  work: 5 planes of scratch. */
void orc_step(const orc_params_t *p, int64_t n, double *F, double *work)
{
    orc_kick_inplace(p, n, F, work);
    orc_drift(p, F);
}

void orc_run(const orc_params_t *p, int64_t n0, int64_t steps, double *F, double *work)
{
    for (int64_t k = 0; k < steps; ++k) orc_step(p, n0 + k, F, work);
}

/* wrap to (-pi, pi]: a + 2 pi floor((pi - a) / 2 pi) */
double orc_wrap(double a)
{
    return a + 2.0 * M_PI * floor((M_PI - a) / (2.0 * M_PI));
}

/* ---------------------------------------------------------------------------
 * plaquette windings (gauge-invariant lattice winding of Kajantie et al.
 * 1998, cited by the paper for xi_W).  With
 *   Y_i(x) = arg( phi*(x) U_i(x) phi(x+i) )  in (-pi, pi]
 *   W_ij(x) = ( Y_i(x) + Y_j(x+i) - Y_i(x+j) - Y_j(x) + [alpha_ij(x)]_pi ) / 2pi
 * which is an integer.  W holds 3 planes of int8 (xy, xz, yz); returns
 * sum |W|.
 * ------------------------------------------------------------------------- */
static double link_phase(const double *F, int N, int x, int y, int z, int i)
{
    int64_t V = vol(N);
    int64_t s0 = at(N, x, y, z), sp = nb(N, x, y, z, i, 1);
    double ur, ui, hr, hi, zr, zi;
    link(F[(F_TX + i) * V + s0], &ur, &ui);
    cmul(ur, ui, F[F_PR * V + sp], F[F_PI * V + sp], &hr, &hi);
    cmul(F[F_PR * V + s0], -F[F_PI * V + s0], hr, hi, &zr, &zi);
    return atan2(zi, zr);
}

int64_t orc_windings(const orc_params_t *p, const double *F, int8_t *W)
{
    const int N = p->N;
    const int64_t V = vol(N);
    static const int PI_[3] = {0, 0, 1}, PJ_[3] = {1, 2, 2};
    int64_t *plane = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
        for (int k = 0; k < 3; ++k) {
            int i = PI_[k], j = PJ_[k];
            int xi = x + (i == 0), yi = y + (i == 1), zi = z + (i == 2);
            int xj = x + (j == 0), yj = y + (j == 1), zj = z + (j == 2);
            double sum = link_phase(F, N, x, y, z, i) + link_phase(F, N, xi, yi, zi, j)
                       - link_phase(F, N, xj, yj, zj, i) - link_phase(F, N, x, y, z, j)
                       + orc_wrap(plaq(F, N, x, y, z, i, j));
            long w = lround(sum / (2.0 * M_PI));
            if (W) W[k * V + at(N, x, y, z)] = (int8_t)w;
            plane[z] += (w < 0 ? -w : w);
        }
    }
    int64_t tot = 0;
    for (int z = 0; z < N; ++z) tot += plane[z];
    free(plane);
    return tot;
}

/* ---------------------------------------------------------------------------
 * Gauss-law residual of the momenta stored in F (time n-1/2), evaluated
 * with phi^n:
 *   G(x) = sum_i (E_i(x) - E_i(x-i))/dx - 2 e0^2 kappa Im[phi*(x) Pi(x)]
 * where kappa = c_{n-1} (1+delta_{n-1})/(1+omega_{n-1}) is the factor the
 * kick of step n-1 leaves on the charge density (Eq. 5 in discrete form).
 * G is the per-site residual (N^3 doubles) or NULL; returns rms, max|G|.
 * ------------------------------------------------------------------------- */
void orc_gauss(const orc_params_t *p, int64_t n, const double *F, double *G, double out[2])
{
    const int N = p->N;
    const int64_t V = vol(N);
    double sc[5];
    orc_scalars(p, n - 1, sc);
    const double kappa = sc[4] * (1.0 + sc[2]) / (1.0 + sc[3]);
    double *s2 = (double *)calloc((size_t)N, sizeof(double));
    double *mx = (double *)calloc((size_t)N, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
        int64_t s0 = at(N, x, y, z);
        double div = 0.0;
        for (int i = 0; i < 3; ++i)
            div += (F[(F_EX + i) * V + s0] - F[(F_EX + i) * V + nb(N, x, y, z, i, -1)]) / p->dx;
        double im = F[F_PR * V + s0] * F[F_QI * V + s0] - F[F_PI * V + s0] * F[F_QR * V + s0];
        double g = div - 2.0 * p->e0 * p->e0 * kappa * im;
        if (G) G[s0] = g;
        s2[z] += g * g;
        if (fabs(g) > mx[z]) mx[z] = fabs(g);
    }
    double t = 0.0, m = 0.0;
    for (int z = 0; z < N; ++z) { t += s2[z]; if (mx[z] > m) m = mx[z]; }
    out[0] = sqrt(t / (double)V);
    out[1] = m;
    free(s2); free(mx);
}

/* ---------------------------------------------------------------------------
 * measurement at integer time n, from phi^n, theta^n and the momenta
 * averaged over the kick of step n:  Pibar = (Pi^{n-1/2} + Pi^{n+1/2})/2,
 * Ebar likewise.  Per site (Lagrangian of Eq. 1 on the lattice, with the
 * coupling scalings of Eqs. 7, 8 absorbed in c_n = a^{2s}):
 *   K = |Pibar|^2,  G = sum_i |D_i^+ phi|^2,  V = (lambda0 c/4)(|phi|^2-sigma^2)^2
 *   El = sum_i Ebar_i^2 / (2 e0^2 c),  B = sum_{i<j} (1 - cos alpha_ij)/(e0^2 c dx^4)
 *   L = K - G - V + El - B,  rho = K + G + V + El + B,
 *   p = K - G/3 - V + (El + B)/3
 * Observables (Eqs. diagxi, diagvel):
 *   xi_L = sqrt(-mu Vol / (dx^3 sum L)), mu = 2 pi sigma^2
 *   xi_W = sqrt(Vol / (dx n_wind))
 *   R = sum K L / sum G L,  <v^2>_phi = 2R/(1+R)
 *   <v^2>_omega = (1 + 3 sum p L / sum rho L)/2   (weight W = L)
 * work: 5 planes of scratch.  Gauss residual per orc_gauss.
 * ------------------------------------------------------------------------- */
void orc_measure(const orc_params_t *p, int64_t n, const double *F, double *work, orc_obs_t *o)
{
    const int N = p->N;
    const int64_t V = vol(N);
    double sc[5];
    orc_scalars(p, n, sc);
    const double c = sc[4];
    const double dx = p->dx, dx2 = dx * dx, dx3 = dx2 * dx, dx4 = dx2 * dx2;
    const double e02 = p->e0 * p->e0;
    orc_kick(p, n, F, work);            /* Pi^{n+1/2}, E^{n+1/2} */

    enum { QK, QG, QV, QEL, QB, QL, QKL, QGL, QPL, QRL, QNF, NQ };
    double *acc = (double *)calloc((size_t)N * NQ, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
        int64_t s0 = at(N, x, y, z);
        double fr = F[F_PR * V + s0], fi = F[F_PI * V + s0];
        double qr = 0.5 * (F[F_QR * V + s0] + work[0 * V + s0]);
        double qi = 0.5 * (F[F_QI * V + s0] + work[1 * V + s0]);
        double K = qr * qr + qi * qi;
        double G = 0.0, El = 0.0, B = 0.0;
        for (int i = 0; i < 3; ++i) {
            int64_t sp = nb(N, x, y, z, i, 1);
            double ur, ui, hr, hi;
            link(F[(F_TX + i) * V + s0], &ur, &ui);
            cmul(ur, ui, F[F_PR * V + sp], F[F_PI * V + sp], &hr, &hi);
            double dr = (hr - fr) / dx, di = (hi - fi) / dx;
            G += dr * dr + di * di;
            double e = 0.5 * (F[(F_EX + i) * V + s0] + work[(2 + i) * V + s0]);
            El += e * e / (2.0 * e02 * c);
            for (int j = i + 1; j < 3; ++j)
                B += (1.0 - cos(plaq(F, N, x, y, z, i, j))) / (e02 * c * dx4);
        }
        double m2 = fr * fr + fi * fi - p->sigma * p->sigma;
        double Vp = 0.25 * p->lambda0 * c * m2 * m2;
        double L = K - G - Vp + El - B;
        double rho = K + G + Vp + El + B;
        double pres = K - G / 3.0 - Vp + (El + B) / 3.0;
        double *a = acc + (size_t)z * NQ;
        a[QK] += K; a[QG] += G; a[QV] += Vp; a[QEL] += El; a[QB] += B; a[QL] += L;
        a[QKL] += K * L; a[QGL] += G * L; a[QPL] += pres * L; a[QRL] += rho * L;
        if (!isfinite(rho) || !isfinite(L)) a[QNF] += 1.0;
    }
    double t[NQ] = {0};
    for (int z = 0; z < N; ++z)
        for (int q = 0; q < NQ; ++q) t[q] += acc[(size_t)z * NQ + q];
    free(acc);

    memset(o, 0, sizeof(*o));
    o->step = n; o->tau = sc[0]; o->a = sc[1];
    o->sum_K = t[QK]; o->sum_G = t[QG]; o->sum_V = t[QV]; o->sum_El = t[QEL];
    o->sum_B = t[QB]; o->sum_L = t[QL]; o->sum_KL = t[QKL]; o->sum_GL = t[QGL];
    o->sum_pL = t[QPL]; o->sum_rhoL = t[QRL];
    o->nonfinite = (int64_t)t[QNF];
    o->e_kin = dx3 * t[QK]; o->e_grad = dx3 * t[QG]; o->e_pot = dx3 * t[QV];
    o->e_elec = dx3 * t[QEL]; o->e_mag = dx3 * t[QB];
    o->e_total = o->e_kin + o->e_grad + o->e_pot + o->e_elec + o->e_mag;
    o->lagrangian = dx3 * t[QL];
    double volume = pow((double)N * dx, 3.0);
    double mu = 2.0 * M_PI * p->sigma * p->sigma;
    o->xi_l = (o->lagrangian < 0.0) ? sqrt(-mu * volume / o->lagrangian) : INFINITY;
    double R = t[QKL] / t[QGL];
    o->v2_phi = 2.0 * R / (1.0 + R);
    o->v2_omega = 0.5 * (1.0 + 3.0 * t[QPL] / t[QRL]);

    o->n_wind = orc_windings(p, F, NULL);
    /* string length from the pierced plaquettes with the pi/6 correction for the
     * Manhattan overcount of lattice paths (Eq. diagxi is silent on
     * the length unit; the xi_dot_W of Table 1 is reproduced with this factor,
     * not with the bare count) */
    o->string_length = (M_PI / 6.0) * dx * (double)o->n_wind;
    o->xi_w = (o->n_wind > 0) ? sqrt(volume / o->string_length) : INFINITY;

    double g[2];
    orc_gauss(p, n, F, NULL, g);
    o->gauss_rms = g[0]; o->gauss_max = g[1];
}

/* ---------------------------------------------------------------------------
 * Lattice Hamiltonian at time n (the energy of the measurement with the stored momenta
 * taken as they are, no averaging):
 *   H = dx^3 sum_x [ |Pi|^2 + G + V + El + B ]
 * Used by the force and energy-conservation pins.
 * ------------------------------------------------------------------------- */
double orc_hamiltonian(const orc_params_t *p, int64_t n, const double *F, int include_kinetic)
{
    const int N = p->N;
    const int64_t V = vol(N);
    double sc[5];
    orc_scalars(p, n, sc);
    const double c = sc[4];
    const double dx = p->dx, dx2 = dx * dx, dx3 = dx2 * dx, dx4 = dx2 * dx2;
    const double e02 = p->e0 * p->e0;
    double *acc = (double *)calloc((size_t)N, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
        int64_t s0 = at(N, x, y, z);
        double fr = F[F_PR * V + s0], fi = F[F_PI * V + s0];
        double h = 0.0;
        if (include_kinetic) {
            h += F[F_QR * V + s0] * F[F_QR * V + s0] + F[F_QI * V + s0] * F[F_QI * V + s0];
            for (int i = 0; i < 3; ++i)
                h += F[(F_EX + i) * V + s0] * F[(F_EX + i) * V + s0] / (2.0 * e02 * c);
        }
        for (int i = 0; i < 3; ++i) {
            int64_t sp = nb(N, x, y, z, i, 1);
            double ur, ui, hr, hi;
            link(F[(F_TX + i) * V + s0], &ur, &ui);
            cmul(ur, ui, F[F_PR * V + sp], F[F_PI * V + sp], &hr, &hi);
            double dr = (hr - fr) / dx, di = (hi - fi) / dx;
            h += dr * dr + di * di;
            for (int j = i + 1; j < 3; ++j)
                h += (1.0 - cos(plaq(F, N, x, y, z, i, j))) / (e02 * c * dx4);
        }
        double m2 = fr * fr + fi * fi - p->sigma * p->sigma;
        h += 0.25 * p->lambda0 * c * m2 * m2;
        acc[z] += h;
    }
    double t = 0.0;
    for (int z = 0; z < N; ++z) t += acc[z];
    free(acc);
    return dx3 * t;
}
