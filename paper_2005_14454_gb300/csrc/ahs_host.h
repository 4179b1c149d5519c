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

// core growth (Sec. 2, after Eq. 6): the width exponent in force at conformal time
// eta -- s_cg before tau_cg, s after it
inline double width_exponent(const LatticeParams *h, double eta)
{
    return h->tau_cg > h->tau0 && eta < h->tau_cg ? h->s_cg : h->s;
}

// c = a^{2s} at conformal time eta (a = (eta/eta0)^p), continuous at tau_cg:
// a^{2 s_cg} before, a_cg^{2 s_cg} (a / a_cg)^{2 s} after
inline double coupling_factor(const LatticeParams *h, double eta)
{
    const double a = std::pow(eta / h->tau0, (double)h->era);
    if (h->tau_cg > h->tau0 && eta >= h->tau_cg) {
        const double acg = std::pow(h->tau_cg / h->tau0, (double)h->era);
        return std::pow(acg, 2.0 * h->s_cg) * std::pow(a / acg, 2.0 * h->s);
    }
    return std::pow(a, 2.0 * width_exponent(h, eta));
}

inline Scalars scalars(const LatticeParams *h, int64_t n)
{
    Scalars r;
    r.eta = h->tau0 + (double)n * h->dt;
    r.a = std::pow(r.eta / h->tau0, (double)h->era);
    r.delta = 0.5 * h->alpha * (double)h->era * h->dt / r.eta;
    r.omega = r.delta * (1.0 - width_exponent(h, r.eta));
    r.c = coupling_factor(h, r.eta);
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
    StepCoef k{};
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
    k.m_el = (float)(0.25 / (2.0 * h->e0 * h->e0 * S.c));   // applied to the sum of the half-step E
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
    StepCoef64 k{};
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
    k.m_el = 0.25 / (2.0 * h->e0 * h->e0 * S.c);
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
    ObsScalars o{};
    o.step = n;
    o.tau = S.eta;
    o.a = S.a;
    o.dx = h->dx;
    o.sites = (double)h->N * (double)h->N * (double)h->N;
    o.volume = std::pow((double)h->N * h->dx, 3.0);
    o.mu = 2.0 * 3.141592653589793238 * h->sigma * h->sigma;
    return o;
}

// Largest stable leapfrog step up to conformal time tau_end, times `safety`: the
// scheme is stable while dt omega_max < 2, with omega_max^2 = 12/dx^2 (the largest
// eigenvalue of the lattice Laplacian, and of the lattice curl-curl) plus the larger
// mass squared, max(lambda0, 2 e0^2) sigma^2 c, at the largest c of the run.  c is
// monotonic in eta on each side of tau_cg, so its largest value is at tau0, tau_end
// or tau_cg.
inline double stable_dt(const LatticeParams *h, double tau_end, double safety)
{
    double c_max = coupling_factor(h, h->tau0);
    const double c_end = coupling_factor(h, tau_end);
    if (c_end > c_max) c_max = c_end;
    if (h->tau_cg > h->tau0 && h->tau_cg < tau_end) {
        const double c_cg = coupling_factor(h, h->tau_cg);
        if (c_cg > c_max) c_max = c_cg;
    }
    const double m2 = (h->lambda0 > 2.0 * h->e0 * h->e0 ? h->lambda0 : 2.0 * h->e0 * h->e0) * h->sigma * h->sigma;
    const double w2 = 12.0 / (h->dx * h->dx) + m2 * c_max;
    return safety * 2.0 / std::sqrt(w2);
}

}  // namespace eng
