// ahs_host.h -- host-side helpers shared by the single-lattice and batched entry
// points: lattice parameters and the FP64 per-step scalars of Eqs. 7, 8, 11, 12,
// rounded once to the float32 kernel coefficients.
#pragma once

#include <cmath>
#include <cstdint>

#include "ahs_internal.cuh"

namespace eng {

struct LatticeParams {
    int N = 0;
    double dx = 0.5, dt = 0.1, lambda0 = 2.0, e0 = 1.0, sigma = 1.0, s = 0.0;
    int era = 1;
    double alpha = 2.0, tau0 = 1.0;
    int wrap = 0;
    double cooling = 0.0;   // > 0: cooling run, a = 1 and delta = omega = cooling
    double s_cg = 0.0;      // core growth: s of the steps with eta < tau_cg
    double tau_cg = 0.0;    // end of the core-growth period (<= tau0: none)
};

// FP64 scalars of step n (Eqs. 7, 8, 11, 12): eta, a, delta, omega, c = a^{2s}
struct Scalars {
    double eta, a, delta, omega, c;
};

inline Scalars scalars(const LatticeParams *h, int64_t n)
{
    Scalars r;
    r.eta = h->tau0 + (double)n * h->dt;
    r.a = std::pow(r.eta / h->tau0, (double)h->era);
    r.delta = 0.5 * h->alpha * (double)h->era * h->dt / r.eta;
    // core growth (Sec. 2, after Eq. 6): exponent s_cg before tau_cg and s after
    // it, in omega and in c, with c continuous at tau_cg:
    // c = a^{2 s_cg} before, a_cg^{2 s_cg} (a / a_cg)^{2 s} after
    const bool grow = h->tau_cg > h->tau0;
    const double s = grow && r.eta < h->tau_cg ? h->s_cg : h->s;
    r.omega = r.delta * (1.0 - s);
    if (grow && r.eta >= h->tau_cg) {
        const double acg = std::pow(h->tau_cg / h->tau0, (double)h->era);
        r.c = std::pow(acg, 2.0 * h->s_cg) * std::pow(r.a / acg, 2.0 * h->s);
    } else {
        r.c = std::pow(r.a, 2.0 * s);
    }
    if (h->cooling > 0.0) {
        // cooling (the artificial damping period of Sec. 2): static background with
        // the same constant Crank-Nicolson damping on both momenta
        r.a = 1.0;
        r.delta = r.omega = h->cooling;
        r.c = 1.0;
    }
    return r;
}

inline StepCoef coefficients(const LatticeParams *h, int64_t n)
{
    const Scalars S = scalars(h, n);
    const double dx = h->dx, dt = h->dt;
    StepCoef k;
    k.cpi = (float)((1.0 - S.delta) / (1.0 + S.delta));
    k.kpi_lap = (float)(dt / ((1.0 + S.delta) * dx * dx));
    k.kpi_pot = (float)(dt * 0.5 * h->lambda0 * S.c / (1.0 + S.delta));
    k.sigma2 = (float)(h->sigma * h->sigma);
    k.ce = (float)((1.0 - S.omega) / (1.0 + S.omega));
    k.ke_curl = (float)(dt / ((1.0 + S.omega) * dx * dx * dx));
    k.ke_cur = (float)(dt * 2.0 * h->e0 * h->e0 * S.c / ((1.0 + S.omega) * dx));
    k.dphi = (float)dt;
    k.dtheta = (float)(dt * dx);
    k.wrap = h->wrap;
    k.m_grad = (float)(1.0 / (dx * dx));
    k.m_pot = (float)(0.25 * h->lambda0 * S.c);
    k.m_el = (float)(1.0 / (2.0 * h->e0 * h->e0 * S.c));
    k.m_mag = (float)(1.0 / (h->e0 * h->e0 * S.c * dx * dx * dx * dx));
    const Scalars P = scalars(h, n - 1);   // the kick that produced the stored momenta
    const double kappa = P.c * (1.0 + P.delta) / (1.0 + P.omega);
    k.m_gauss = (float)(2.0 * h->e0 * h->e0 * kappa);
    k.inv_dx = (float)(1.0 / dx);
    k.gauss = 1;
    return k;
}

inline StepCoef64 coefficients64(const LatticeParams *h, int64_t n)
{
    const Scalars S = scalars(h, n);
    const double dx = h->dx, dt = h->dt;
    StepCoef64 k;
    k.cpi = (1.0 - S.delta) / (1.0 + S.delta);
    k.kpi_lap = dt / ((1.0 + S.delta) * dx * dx);
    k.kpi_pot = dt * 0.5 * h->lambda0 * S.c / (1.0 + S.delta);
    k.sigma2 = h->sigma * h->sigma;
    k.ce = (1.0 - S.omega) / (1.0 + S.omega);
    k.ke_curl = dt / ((1.0 + S.omega) * dx * dx * dx);
    k.ke_cur = dt * 2.0 * h->e0 * h->e0 * S.c / ((1.0 + S.omega) * dx);
    k.dphi = dt;
    k.dtheta = dt * dx;
    k.wrap = h->wrap;
    k.m_grad = 1.0 / (dx * dx);
    k.m_pot = 0.25 * h->lambda0 * S.c;
    k.m_el = 1.0 / (2.0 * h->e0 * h->e0 * S.c);
    k.m_mag = 1.0 / (h->e0 * h->e0 * S.c * dx * dx * dx * dx);
    const Scalars P = scalars(h, n - 1);
    k.m_gauss = 2.0 * h->e0 * h->e0 * P.c * (1.0 + P.delta) / (1.0 + P.omega);
    k.inv_dx = 1.0 / dx;
    k.gauss = 1;
    return k;
}

inline ObsScalars obs_scalars(const LatticeParams *h, int64_t n)
{
    const Scalars S = scalars(h, n);
    ObsScalars o;
    o.step = n;
    o.tau = S.eta;
    o.a = S.a;
    o.dx = h->dx;
    o.sites = (double)h->N * (double)h->N * (double)h->N;
    o.volume = std::pow((double)h->N * h->dx, 3.0);
    o.mu = 2.0 * 3.141592653589793238 * h->sigma * h->sigma;
    return o;
}

}  // namespace eng
