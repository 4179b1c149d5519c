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
#include "ahs_host.h"

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

    // launch shape: the automatic measuring one (4-row tiles), with longer z marches
    // if its CTAs would not all fit the static scratch, else 8-row tiles
    StepShape sh{};
    bool fits = false;
    for (int by : {4, 8}) {
        sh = measure_shape(N, by, 0);
        if (sh.blocks > AHS_NOALLOC_MAX_ROWS) {
            const int tiles = ((N + 31) / 32) * ((N + by - 1) / by);
            const int chunks = AHS_NOALLOC_MAX_ROWS / tiles;
            if (chunks < 1) continue;
            sh = measure_shape(N, by, (N + chunks - 1) / chunks);
        }
        if (sh.blocks <= AHS_NOALLOC_MAX_ROWS) {
            fits = true;
            break;
        }
    }
    if (!fits) return report_error(AHS_EINVAL, "lattice too large for the static measurement scratch");
    void *scratch = nullptr;
    if (int r = scratch_address(&scratch)) return r;

    // the coefficients and record scalars of step n from the same FP64 helpers the
    // handle-based entry points use (Eqs. 7, 8, 11, 12), so the record equals the
    // one ahs_measure gives for the same launch shape
    LatticeParams lp;
    lp.N = N;
    lp.dx = dx;
    lp.dt = dt;
    lp.lambda0 = lambda0;
    lp.e0 = e0;
    lp.sigma = sigma;
    lp.s = s;
    lp.era = era;
    lp.alpha = alpha;
    lp.tau0 = tau0;
    const StepCoef k = coefficients(&lp, step);
    const ObsScalars o = obs_scalars(&lp, step);

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
