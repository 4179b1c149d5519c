// ahs_noalloc.cu -- measurement of caller-owned fields without any device
// allocation.
//
// The regular entry points allocate their device memory with cudaMalloc when a
// handle is created.  Some callers cannot do that: their whole device memory is
// owned by another allocator (a framework's caching allocator, or a pool that a
// job reserved up front) and a side allocation would fail, fragment that pool or
// stall on the allocator's device-wide synchronisation.  ahs_measure_noalloc
// serves them: the caller passes device buffers for the fields and for the
// result, and the only scratch the measurement needs -- one row of FP64 partial
// sums per CTA -- lives in the static device array below, which every GPU that
// loads this library holds until the process exits.
#include "ahs_internal.cuh"

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

constexpr int kMaxDevices = 64;

// AHS_NOALLOC_MAX_ROWS rows of NQ doubles (2 MiB).  Every CTA of a measurement
// writes its whole row before the final reduction reads it, so nothing has to be
// cleared between calls.
__device__ __align__(256) double g_noalloc_partials[AHS_NOALLOC_MAX_ROWS * eng::NQ];

std::mutex g_setup_mutex;
void *g_scratch[kMaxDevices] = {};

// device address of the static scratch on the current device (looked up once per
// device; the host-side name of the array is not a device address)
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "cudaGetDevice: %s", cudaGetErrorString(e));
        return eng::report_error(AHS_ECUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return eng::report_error(AHS_EINVAL, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            char msg[160];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            return eng::report_error(AHS_ECUDA, msg);
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return AHS_OK;
}

}  // namespace

extern "C" int ahs_measure_noalloc(int N, double dx, double dt, double lambda0, double e0, double sigma, double s,
                                   int era, double alpha, double tau0, int64_t step, const float *fields,
                                   ahs_obs_t *out, void *stream)
{
    using namespace eng;
    if (N < 4 || N > 1600) return report_error(AHS_EINVAL, "N outside [4, 1600]");
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt) || !std::isfinite(lambda0) ||
        !std::isfinite(e0) || e0 == 0 || !std::isfinite(sigma) || !std::isfinite(s) || !std::isfinite(alpha) ||
        !(tau0 > 0) || era < 0 || era > 2)
        return report_error(AHS_EINVAL, "invalid lattice parameters");
    if (!fields || !out) return report_error(AHS_EINVAL, "null device buffer");

    // launch shape: the automatic one, with longer z marches if its CTAs would not
    // all fit the static scratch
    StepShape sh = step_shape(N, 8, 0);
    if (sh.blocks > AHS_NOALLOC_MAX_ROWS) {
        const int tiles = ((N + 31) / 32) * ((N + 7) / 8);
        const int chunks = AHS_NOALLOC_MAX_ROWS / tiles;
        if (chunks < 1) return report_error(AHS_EINVAL, "lattice too large for the static measurement scratch");
        sh = step_shape(N, 8, (N + chunks - 1) / chunks);
        if (sh.blocks > AHS_NOALLOC_MAX_ROWS)
            return report_error(AHS_EINVAL, "lattice too large for the static measurement scratch");
    }
    void *scratch = nullptr;
    if (int r = scratch_address(&scratch)) return r;

    // FP64 scalars of step n (Eqs. 7, 8, 11, 12) and the measurement factors
    auto scal = [&](int64_t n, double &eta, double &a, double &delta, double &omega, double &c) {
        eta = tau0 + (double)n * dt;
        a = std::pow(eta / tau0, (double)era);
        delta = 0.5 * alpha * (double)era * dt / eta;
        omega = delta * (1.0 - s);
        c = std::pow(a, 2.0 * s);
    };
    double eta, a, delta, omega, c, etap, ap, deltap, omegap, cp;
    scal(step, eta, a, delta, omega, c);
    scal(step - 1, etap, ap, deltap, omegap, cp);
    StepCoef k;
    k.cpi = (float)((1.0 - delta) / (1.0 + delta));
    k.kpi_lap = (float)(dt / ((1.0 + delta) * dx * dx));
    k.kpi_pot = (float)(dt * 0.5 * lambda0 * c / (1.0 + delta));
    k.sigma2 = (float)(sigma * sigma);
    k.ce = (float)((1.0 - omega) / (1.0 + omega));
    k.ke_curl = (float)(dt / ((1.0 + omega) * dx * dx * dx));
    k.ke_cur = (float)(dt * 2.0 * e0 * e0 * c / ((1.0 + omega) * dx));
    k.dphi = (float)dt;
    k.dtheta = (float)(dt * dx);
    k.wrap = 0;
    k.m_grad = (float)(1.0 / (dx * dx));
    k.m_pot = (float)(0.25 * lambda0 * c);
    k.m_el = (float)(1.0 / (2.0 * e0 * e0 * c));
    k.m_mag = (float)(1.0 / (e0 * e0 * c * dx * dx * dx * dx));
    k.m_gauss = (float)(2.0 * e0 * e0 * cp * (1.0 + deltap) / (1.0 + omegap));
    k.inv_dx = (float)(1.0 / dx);

    const size_t V = (size_t)N * N * N;
    StepPtrs p = {};
    p.pr = fields;
    p.pim = fields + V;
    p.qr = fields + 2 * V;
    p.qi = fields + 3 * V;
    p.tx = fields + 4 * V;
    p.ty = fields + 5 * V;
    p.tz = fields + 6 * V;
    p.ex = fields + 7 * V;
    p.ey = fields + 8 * V;
    p.ez = fields + 9 * V;

    ObsScalars o;
    o.step = step;
    o.tau = eta;
    o.a = a;
    o.dx = dx;
    o.sites = (double)V;
    o.volume = std::pow((double)N * dx, 3.0);
    o.mu = 2.0 * 3.141592653589793238 * sigma * sigma;

    cudaStream_t st = (cudaStream_t)stream;
    double *partials = static_cast<double *>(scratch);
    cudaError_t e = launch_step(p, k, N, sh, true, false, partials, st);
    if (e == cudaSuccess) e = launch_reduce(partials, sh.blocks, o, out, st);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "measurement launch: %s", cudaGetErrorString(e));
        return report_error(AHS_ECUDA, msg);
    }
    return report_ok();
}
