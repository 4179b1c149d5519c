// ahs_abi.cu -- host side of the C ABI declared in include/ahs.h.
//
// Owns the device state of one lattice, turns the step index into the FP64
// scalars of Eqs. 7-8 and 11-12 (rounded once to float32 for the stencil), and
// sequences the step, reduction and copy launches on the handle's stream.
#include "ahs_host.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

using namespace eng;

namespace {

thread_local int g_last = AHS_OK;
thread_local char g_msg[512] = "";

int fail(int code, const char *fmt, ...)
{
    g_last = code;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

int ok()
{
    g_last = AHS_OK;
    g_msg[0] = 0;
    return AHS_OK;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(AHS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kFields = 10;   // Re phi, Im phi, Re Pi, Im Pi, theta_xyz, E_xyz
constexpr int kLowPlanes = 5; // compensated precision: low words of Re Pi, Im Pi, E_xyz

}  // namespace

namespace eng {
// error reporting for entry points defined in other translation units
int report_error(int code, const char *msg) { return fail(code, "%s", msg); }
int report_ok() { return ok(); }
}  // namespace eng

struct ahs : eng::LatticeParams {
    size_t V = 0;
    int measure_every = 10;
    int profile = 0;
    int64_t n = 0;        // integer time level of phi/theta in buffer `cur`
    int cur = 0;
    bool ready = false;   // fields defined
    int device = 0;

    int precision = AHS_PREC_FP32;
    int planes = kFields;            // planes per buffer (15 with low words)
    size_t esize = sizeof(float);    // bytes per stored value
    int inplace = 0;                 // Pi and E stored once (AHS_OPT_MOMENTA_IN_PLACE)
    void *base = nullptr;            // 2 buffers of `planes` planes of V values; in place:
                                     // buffer 0 (10 planes), then phi and theta of buffer 1
    double *partials = nullptr;      // nblocks * NQ
    int nblocks = 0;                 // capacity of partials in rows
    int tile_y = 0, zchunk = 0;      // launch-shape overrides (0: automatic)
    int measure_tile_y = 0;          // tile height of measuring launches (0: automatic)
    ahs_obs_t *rec_dev = nullptr;    // device records of one ahs_step call
    int rec_cap = 0;
    ahs_obs_t *rec_host = nullptr;   // pinned staging
    std::vector<ahs_obs_t> log;

    cudaStream_t stream = nullptr;
    int steps_per_pass = 1;          // 2: pairs of plain steps as one launch
    std::vector<cudaEvent_t> ev;     // profiling event pool (pairs)
    double prof_ms[3] = {0.0, 0.0, 0.0};  // [plain step, measuring step, two-step launch]
    int64_t prof_launches[3] = {0, 0, 0};

    // index of plane f of buffer buf in the allocation
    size_t plane_index(int buf, int f) const
    {
        if (!inplace || buf == 0) return (size_t)buf * planes + f;
        if (f < 2) return kFields + f;                 // phi of buffer 1
        if (f >= 4 && f < 7) return kFields + f - 2;   // theta of buffer 1
        return f;                                      // Pi, E: the single copy
    }
    size_t total_planes() const { return inplace ? kFields + 5 : 2 * (size_t)planes; }
    float *plane(int buf, int f) const { return (float *)base + plane_index(buf, f) * V; }
    double *plane64(int buf, int f) const { return (double *)base + plane_index(buf, f) * V; }
    size_t field_bytes() const { return esize * V * total_planes(); }
};

namespace {

StepPtrs pointers(const ahs_t *h)
{
    const int a = h->cur, b = 1 - h->cur;
    StepPtrs p;
    p.pr = h->plane(a, 0); p.pim = h->plane(a, 1);
    p.qr = h->plane(a, 2); p.qi = h->plane(a, 3);
    p.tx = h->plane(a, 4); p.ty = h->plane(a, 5); p.tz = h->plane(a, 6);
    p.ex = h->plane(a, 7); p.ey = h->plane(a, 8); p.ez = h->plane(a, 9);
    p.pr1 = h->plane(b, 0); p.pim1 = h->plane(b, 1);
    p.qr1 = h->plane(b, 2); p.qi1 = h->plane(b, 3);
    p.tx1 = h->plane(b, 4); p.ty1 = h->plane(b, 5); p.tz1 = h->plane(b, 6);
    p.ex1 = h->plane(b, 7); p.ey1 = h->plane(b, 8); p.ez1 = h->plane(b, 9);
    const bool lo = h->precision == AHS_PREC_FP32_COMPENSATED;
    p.qrl = lo ? h->plane(a, 10) : nullptr; p.qil = lo ? h->plane(a, 11) : nullptr;
    p.exl = lo ? h->plane(a, 12) : nullptr; p.eyl = lo ? h->plane(a, 13) : nullptr;
    p.ezl = lo ? h->plane(a, 14) : nullptr;
    p.qrl1 = lo ? h->plane(b, 10) : nullptr; p.qil1 = lo ? h->plane(b, 11) : nullptr;
    p.exl1 = lo ? h->plane(b, 12) : nullptr; p.eyl1 = lo ? h->plane(b, 13) : nullptr;
    p.ezl1 = lo ? h->plane(b, 14) : nullptr;
    return p;
}

StepPtrs64 pointers64(const ahs_t *h)
{
    const int a = h->cur, b = 1 - h->cur;
    StepPtrs64 p;
    p.pr = h->plane64(a, 0); p.pim = h->plane64(a, 1);
    p.qr = h->plane64(a, 2); p.qi = h->plane64(a, 3);
    p.tx = h->plane64(a, 4); p.ty = h->plane64(a, 5); p.tz = h->plane64(a, 6);
    p.ex = h->plane64(a, 7); p.ey = h->plane64(a, 8); p.ez = h->plane64(a, 9);
    p.pr1 = h->plane64(b, 0); p.pim1 = h->plane64(b, 1);
    p.qr1 = h->plane64(b, 2); p.qi1 = h->plane64(b, 3);
    p.tx1 = h->plane64(b, 4); p.ty1 = h->plane64(b, 5); p.tz1 = h->plane64(b, 6);
    p.ex1 = h->plane64(b, 7); p.ey1 = h->plane64(b, 8); p.ez1 = h->plane64(b, 9);
    return p;
}

// the launch shape of a plain or a measuring step (FP64: 8-row tiles for both)
StepShape shape_of(const ahs_t *h, bool measure)
{
    if (h->precision == AHS_PREC_FP64) return step_shape(h->N, 8, h->zchunk);
    return measure ? measure_shape(h->N, h->measure_tile_y, h->zchunk) : step_shape(h->N, h->tile_y, h->zchunk);
}

// CTAs (rows of partials) of the current measuring launch
int launch_blocks(const ahs_t *h) { return shape_of(h, true).blocks; }

// one step launch (measure: diagnostics into the partials; store: write n+1;
// gauss false: the Gauss residual's slots were written by launch_gauss)
cudaError_t launch_current(const ahs_t *h, bool measure, bool store, bool gauss = true)
{
    if (h->precision == AHS_PREC_FP64)
        return launch_step64(pointers64(h), coefficients64(h, h->n), h->N, shape_of(h, measure), measure, store,
                             h->partials, h->stream);
    StepCoef k = coefficients(h, h->n);
    k.gauss = gauss ? 1 : 0;
    return launch_step(pointers(h), k, h->N, shape_of(h, measure), measure, store, h->partials, h->stream,
                       h->precision == AHS_PREC_FP32_COMPENSATED);
}

// the storage layout of the handle's precision and storage mode; frees any field
// storage (the fields are then undefined until ahs_init or ahs_set_fields)
void reset_fields(ahs_t *h)
{
    if (h->base) cudaFree(h->base);
    h->base = nullptr;
    h->ready = false;
    h->cur = 0;
    h->planes = h->precision == AHS_PREC_FP32_COMPENSATED ? kFields + kLowPlanes : kFields;
    h->esize = h->precision == AHS_PREC_FP64 ? sizeof(double) : sizeof(float);
}

// allocate the field storage on first use (ahs_init, ahs_set_fields), so that the
// precision and storage options are set before the bytes are committed
int alloc_fields(ahs_t *h)
{
    if (h->base) return AHS_OK;
    const size_t bytes = h->field_bytes();
    cudaError_t e = cudaMalloc(&h->base, bytes);
    if (e != cudaSuccess) {
        h->base = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? AHS_ENOMEM : AHS_ECUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    return AHS_OK;
}

// field selector -> (first plane, number of planes)
bool selector(int which, int *first, int *count)
{
    switch (which) {
    case AHS_FIELD_PHI: *first = 0; *count = 2; return true;
    case AHS_FIELD_PI: *first = 2; *count = 2; return true;
    case AHS_FIELD_THETA: *first = 4; *count = 3; return true;
    case AHS_FIELD_E: *first = 7; *count = 3; return true;
    case AHS_FIELD_ALL: *first = 0; *count = 10; return true;
    case AHS_FIELD_LOW: *first = 10; *count = 5; return true;
    default: return false;
    }
}

int ensure_records(ahs_t *h, int count)
{
    if (count <= h->rec_cap) return AHS_OK;
    int cap = h->rec_cap ? h->rec_cap : 64;
    while (cap < count) cap *= 2;
    if (h->rec_dev) cudaFree(h->rec_dev);
    if (h->rec_host) cudaFreeHost(h->rec_host);
    h->rec_dev = nullptr;
    h->rec_host = nullptr;
    h->rec_cap = 0;
    if (cudaMalloc(&h->rec_dev, sizeof(ahs_obs_t) * cap) != cudaSuccess)
        return fail(AHS_ENOMEM, "cannot allocate %d device records", cap);
    if (cudaMallocHost(&h->rec_host, sizeof(ahs_obs_t) * cap) != cudaSuccess)
        return fail(AHS_ENOMEM, "cannot allocate %d pinned records", cap);
    h->rec_cap = cap;
    return AHS_OK;
}

// grow the measurement partials to the CTA count of the current launch shape
int ensure_partials(ahs_t *h, int blocks)
{
    if (blocks <= h->nblocks) return AHS_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->partials);
    h->partials = nullptr;
    h->nblocks = 0;
    if (cudaMalloc(&h->partials, sizeof(double) * NQ * (size_t)blocks) != cudaSuccess) {
        cudaGetLastError();
        return fail(AHS_ENOMEM, "cannot allocate %d measurement partials", blocks);
    }
    h->nblocks = blocks;
    return AHS_OK;
}

cudaEvent_t event_at(ahs_t *h, size_t i)
{
    while (h->ev.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev.push_back(e);
    }
    return h->ev[i];
}

int set_device(const ahs_t *h)
{
    CU(cudaSetDevice(h->device));
    return AHS_OK;
}

}  // namespace

extern "C" {

int ahs_last_error(void) { return g_last; }
const char *ahs_last_error_message(void) { return g_msg; }
size_t ahs_sizeof_obs(void) { return sizeof(ahs_obs_t); }

const char *ahs_strerror(int status)
{
    switch (status) {
    case AHS_OK: return "ok";
    case AHS_EINVAL: return "invalid argument";
    case AHS_ENOMEM: return "out of memory";
    case AHS_ECUDA: return "CUDA error";
    case AHS_ESTATE: return "invalid state";
    case AHS_ENONFINITE: return "non-finite field value";
    case AHS_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

ahs_t *ahs_create(int N, double dx, double dt, double lambda0, double e0, double sigma, double s, int era)
{
    if (N < 4 || N > 1600) { fail(AHS_EINVAL, "N=%d outside [4, 1600]", N); return nullptr; }
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt)) {
        fail(AHS_EINVAL, "dx and dt must be positive");
        return nullptr;
    }
    if (!std::isfinite(lambda0) || !std::isfinite(e0) || !(e0 != 0) || !std::isfinite(sigma) || !std::isfinite(s)) {
        fail(AHS_EINVAL, "couplings must be finite and e0 non-zero");
        return nullptr;
    }
    if (era < 0 || era > 2) { fail(AHS_EINVAL, "era=%d not in {0,1,2}", era); return nullptr; }
    ahs_t *h = new (std::nothrow) ahs_t;
    if (!h) { fail(AHS_ENOMEM, "host allocation"); return nullptr; }
    h->N = N;
    h->V = (size_t)N * N * N;
    h->dx = dx; h->dt = dt; h->lambda0 = lambda0; h->e0 = e0; h->sigma = sigma; h->s = s; h->era = era;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        fail(AHS_ECUDA, "no CUDA device");
        delete h;
        return nullptr;
    }
    reset_fields(h);
    h->nblocks = measure_shape(N, 0, 0).blocks;
    cudaError_t e = cudaMalloc(&h->partials, sizeof(double) * NQ * (size_t)h->nblocks);
    if (e != cudaSuccess) {
        fail(AHS_ENOMEM, "cudaMalloc(partials): %s", cudaGetErrorString(e));
        cudaGetLastError();
        delete h;
        return nullptr;
    }
    if (ensure_records(h, 64) != AHS_OK) {
        cudaFree(h->partials);
        delete h;
        return nullptr;
    }
    ok();
    return h;
}

void ahs_destroy(ahs_t *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->rec_dev) cudaFree(h->rec_dev);
    if (h->rec_host) cudaFreeHost(h->rec_host);
    if (h->partials) cudaFree(h->partials);
    if (h->base) cudaFree(h->base);
    delete h;
}

int ahs_set_stream(ahs_t *h, void *stream)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    h->stream = (cudaStream_t)stream;
    return ok();
}

int ahs_device_bytes(ahs_t *h, size_t *bytes)
{
    if (!h || !bytes) return fail(AHS_EINVAL, "null argument");
    *bytes = h->field_bytes() + sizeof(double) * NQ * (size_t)h->nblocks +
             sizeof(ahs_obs_t) * (size_t)h->rec_cap;
    return ok();
}

int ahs_init(ahs_t *h, uint64_t seed)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    if (int r = set_device(h)) return r;
    if (int r = alloc_fields(h)) return r;
    h->cur = 0;
    h->n = 0;
    if (h->precision == AHS_PREC_FP64) {
        CU(cudaMemsetAsync(h->plane64(0, 2), 0, sizeof(double) * h->V * (h->planes - 2), h->stream));
        CU(launch_init_fp64(h->plane64(0, 0), h->plane64(0, 1), h->N, seed, h->sigma, h->stream));
    } else {
        CU(cudaMemsetAsync(h->plane(0, 2), 0, sizeof(float) * h->V * (h->planes - 2), h->stream));
        CU(launch_init(h->plane(0, 0), h->plane(0, 1), h->N, seed, h->sigma, h->stream));
    }
    CU(cudaStreamSynchronize(h->stream));
    h->ready = true;
    h->log.clear();
    return ok();
}

int ahs_set_option(ahs_t *h, int key, double v)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    switch (key) {
    case AHS_OPT_MEASURE_EVERY:
        if (!(v >= 0) || v > 1e9 || v != std::floor(v)) return fail(AHS_EINVAL, "measure_every must be a non-negative integer");
        h->measure_every = (int)v;
        return ok();
    case AHS_OPT_ALPHA:
        if (!std::isfinite(v)) return fail(AHS_EINVAL, "alpha must be finite");
        h->alpha = v;
        return ok();
    case AHS_OPT_TAU0:
        if (!(v > 0) || !std::isfinite(v)) return fail(AHS_EINVAL, "tau0 must be positive");
        h->tau0 = v;
        return ok();
    case AHS_OPT_STEP:
        if (v != std::floor(v) || std::fabs(v) > 9e15) return fail(AHS_EINVAL, "step must be an integer");
        h->n = (int64_t)v;
        return ok();
    case AHS_OPT_WRAP_THETA:
        if (v != 0 && v != 1) return fail(AHS_EINVAL, "wrap_theta must be 0 or 1");
        h->wrap = (int)v;
        return ok();
    case AHS_OPT_PROFILE:
        if (v != 0 && v != 1) return fail(AHS_EINVAL, "profile must be 0 or 1");
        h->profile = (int)v;
        return ok();
    case AHS_OPT_TILE_Y:
        if (v != 0 && v != 8 && v != 16) return fail(AHS_EINVAL, "tile_y must be 0, 8 or 16");
        h->tile_y = (int)v;
        return ok();
    case AHS_OPT_MEASURE_TILE_Y:
        if (v != 0 && v != 4 && v != 8 && v != 16) return fail(AHS_EINVAL, "measure_tile_y must be 0, 4, 8 or 16");
        h->measure_tile_y = (int)v;
        return ok();
    case AHS_OPT_ZCHUNK:
        if (!(v >= 0) || v > h->N || v != std::floor(v)) return fail(AHS_EINVAL, "zchunk must be an integer in [0, N]");
        h->zchunk = (int)v;
        return ok();
    case AHS_OPT_PRECISION: {
        if (v != AHS_PREC_FP32 && v != AHS_PREC_FP32_COMPENSATED && v != AHS_PREC_FP64)
            return fail(AHS_EINVAL, "precision must be AHS_PREC_FP32, _FP32_COMPENSATED or _FP64");
        if ((int)v == h->precision) return ok();
        if (h->inplace && v != AHS_PREC_FP32) return fail(AHS_EINVAL, "in-place momenta need float32 precision");
        if (h->steps_per_pass == 2) return fail(AHS_EINVAL, "two steps per pass need float32 precision");
        if (int r = set_device(h)) return r;
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
        h->precision = (int)v;
        reset_fields(h);
        return ok();
    }
    case AHS_OPT_COOLING:
        if (!(v >= 0) || !std::isfinite(v) || v >= 1.0) return fail(AHS_EINVAL, "cooling damping must be in [0, 1)");
        h->cooling = v;
        return ok();
    case AHS_OPT_CORE_GROWTH_S:
        if (!std::isfinite(v)) return fail(AHS_EINVAL, "core-growth s must be finite");
        h->s_cg = v;
        return ok();
    case AHS_OPT_CORE_GROWTH_TAU:
        if (!std::isfinite(v)) return fail(AHS_EINVAL, "core-growth end must be finite");
        h->tau_cg = v;
        return ok();
    case AHS_OPT_MOMENTA_IN_PLACE: {
        if (v != 0 && v != 1) return fail(AHS_EINVAL, "momenta_in_place must be 0 or 1");
        if ((int)v == h->inplace) return ok();
        if (v == 1 && h->precision != AHS_PREC_FP32) return fail(AHS_EINVAL, "in-place momenta need float32 precision");
        if (v == 1 && h->steps_per_pass == 2) return fail(AHS_EINVAL, "two steps per pass need double-buffered momenta");
        if (int r = set_device(h)) return r;
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
        h->inplace = (int)v;
        reset_fields(h);
        return ok();
    }
    case AHS_OPT_STEPS_PER_PASS:
        if (v != 1 && v != 2) return fail(AHS_EINVAL, "steps_per_pass must be 1 or 2");
        if (v == 2 && (h->precision != AHS_PREC_FP32 || h->inplace))
            return fail(AHS_EINVAL, "two steps per pass need float32 precision and double-buffered momenta");
        h->steps_per_pass = (int)v;
        return ok();
    case AHS_OPT_N:
        return fail(AHS_EINVAL, "N is read only");
    default:
        return fail(AHS_EINVAL, "unknown option %d", key);
    }
}

int ahs_get_option(ahs_t *h, int key, double *v)
{
    if (!h || !v) return fail(AHS_EINVAL, "null argument");
    switch (key) {
    case AHS_OPT_MEASURE_EVERY: *v = h->measure_every; break;
    case AHS_OPT_ALPHA: *v = h->alpha; break;
    case AHS_OPT_TAU0: *v = h->tau0; break;
    case AHS_OPT_STEP: *v = (double)h->n; break;
    case AHS_OPT_WRAP_THETA: *v = h->wrap; break;
    case AHS_OPT_PROFILE: *v = h->profile; break;
    case AHS_OPT_N: *v = h->N; break;
    case AHS_OPT_PRECISION: *v = h->precision; break;
    case AHS_OPT_COOLING: *v = h->cooling; break;
    case AHS_OPT_MOMENTA_IN_PLACE: *v = h->inplace; break;
    case AHS_OPT_CORE_GROWTH_S: *v = h->s_cg; break;
    case AHS_OPT_CORE_GROWTH_TAU: *v = h->tau_cg; break;
    case AHS_OPT_STEPS_PER_PASS: *v = h->steps_per_pass; break;
    case AHS_OPT_TILE_Y: *v = shape_of(h, false).by; break;
    case AHS_OPT_MEASURE_TILE_Y: *v = shape_of(h, true).by; break;
    case AHS_OPT_ZCHUNK: *v = step_shape(h->N, h->tile_y, h->zchunk).dz; break;
    default: return fail(AHS_EINVAL, "unknown option %d", key);
    }
    return ok();
}

int ahs_step(ahs_t *h, int nsteps)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    if (nsteps < 0) return fail(AHS_EINVAL, "negative step count");
    if (!h->ready) return fail(AHS_ESTATE, "fields not initialised");
    if (int r = set_device(h)) return r;
    int nrec = 0;
    if (h->measure_every > 0) {
        for (int i = 0; i < nsteps; ++i)
            if ((h->n + i) % h->measure_every == 0) ++nrec;
    }
    if (int r = ensure_records(h, nrec)) return r;
    if (int r = ensure_partials(h, launch_blocks(h))) return r;
    size_t nev = 0;
    int ri = 0;
    std::vector<char> kind;          // per event pair: the AHS_KERNEL_* kind of the launch
    auto measures = [h](int64_t n) { return h->measure_every > 0 && (n % h->measure_every == 0); };
    for (int i = 0; i < nsteps; ++i) {
        const bool meas = measures(h->n);
        const bool pair = h->steps_per_pass == 2 && !meas && i + 1 < nsteps && !measures(h->n + 1);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->profile) {
            e0 = event_at(h, nev++);
            e1 = event_at(h, nev++);
            kind.push_back(pair ? AHS_KERNEL_STEP_PAIR : meas ? AHS_KERNEL_STEP_MEASURE : AHS_KERNEL_STEP);
            if (!e0 || !e1) return fail(AHS_ECUDA, "cudaEventCreate failed");
            CU(cudaEventRecord(e0, h->stream));
        }
        if (pair) {
            // steps n and n+1 in one pass: buffer cur (time n) -> the other (n+2)
            CU(launch_step_two(pointers(h), coefficients(h, h->n), coefficients(h, h->n + 1), h->N,
                               step_shape(h->N, 8, h->zchunk).dz, h->stream));
            if (h->profile) CU(cudaEventRecord(e1, h->stream));
            h->cur = 1 - h->cur;
            h->n += 2;
            ++i;
            continue;
        }
        const int nb = launch_blocks(h);
        if (meas && h->inplace) {
            // the Gauss residual reads neighbours' old E, which an in-place step
            // overwrites: it goes first, into the measuring launch's partial rows
            CU(launch_gauss(pointers(h), coefficients(h, h->n), h->N, shape_of(h, true), h->partials, h->stream));
            CU(launch_current(h, true, true, false));
        } else {
            CU(launch_current(h, meas, true));
        }
        if (h->profile) CU(cudaEventRecord(e1, h->stream));
        if (meas) {
            CU(launch_reduce(h->partials, nb, obs_scalars(h, h->n), h->rec_dev + ri, h->stream));
            ++ri;
        }
        h->cur = 1 - h->cur;
        h->n += 1;
    }
    if (ri > 0) CU(cudaMemcpyAsync(h->rec_host, h->rec_dev, sizeof(ahs_obs_t) * ri, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (h->profile) {
        for (size_t j = 0; j + 1 < nev; j += 2) {
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, h->ev[j], h->ev[j + 1]));
            h->prof_ms[(int)kind[j / 2]] += ms;
            h->prof_launches[(int)kind[j / 2]] += 1;
        }
    }
    bool bad = false;
    for (int j = 0; j < ri; ++j) {
        h->log.push_back(h->rec_host[j]);
        if (h->rec_host[j].nonfinite != 0) bad = true;
    }
    if (bad) return fail(AHS_ENONFINITE, "a measurement counted non-finite sites");
    return ok();
}

int ahs_measure(ahs_t *h, ahs_obs_t *out)
{
    if (!h || !out) return fail(AHS_EINVAL, "null argument");
    if (!h->ready) return fail(AHS_ESTATE, "fields not initialised");
    if (int r = set_device(h)) return r;
    if (int r = ensure_partials(h, launch_blocks(h))) return r;
    const int nb = launch_blocks(h);
    CU(launch_current(h, true, false));
    CU(launch_reduce(h->partials, nb, obs_scalars(h, h->n), h->rec_dev, h->stream));
    CU(cudaMemcpyAsync(h->rec_host, h->rec_dev, sizeof(ahs_obs_t), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    *out = h->rec_host[0];
    return ok();
}

int ahs_records(ahs_t *h, ahs_obs_t *out, int max)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    if (max < 0 || (max > 0 && !out)) return fail(AHS_EINVAL, "bad output buffer");
    if (max == 0) {
        ok();
        return (int)h->log.size();
    }
    const int m = (int)h->log.size() < max ? (int)h->log.size() : max;
    for (int i = 0; i < m; ++i) out[i] = h->log[i];
    h->log.erase(h->log.begin(), h->log.begin() + m);
    ok();
    return m;
}

int ahs_fields(ahs_t *h, int which, void *dst, size_t bytes)
{
    if (!h || !dst) return fail(AHS_EINVAL, "null argument");
    int first, count;
    if (!selector(which, &first, &count) || first + count > h->planes)
        return fail(AHS_EINVAL, "field selector %d not available in this precision", which);
    const size_t pb = h->esize * h->V;
    if (bytes != pb * count) return fail(AHS_EINVAL, "buffer is %zu bytes, field needs %zu", bytes, pb * count);
    if (!h->ready) return fail(AHS_ESTATE, "fields not initialised");
    if (int r = set_device(h)) return r;
    for (int i = 0; i < count; ++i)
        CU(cudaMemcpyAsync((char *)dst + (size_t)i * pb, (char *)h->base + h->plane_index(h->cur, first + i) * pb,
                           pb, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return ok();
}

int ahs_set_fields(ahs_t *h, int which, const void *src, size_t bytes)
{
    if (!h || !src) return fail(AHS_EINVAL, "null argument");
    int first, count;
    if (!selector(which, &first, &count) || first + count > h->planes)
        return fail(AHS_EINVAL, "field selector %d not available in this precision", which);
    const size_t pb = h->esize * h->V;
    if (bytes != pb * count) return fail(AHS_EINVAL, "buffer is %zu bytes, field needs %zu", bytes, pb * count);
    if (int r = set_device(h)) return r;
    if (int r = alloc_fields(h)) return r;
    if (!h->ready) {
        // a partial set on a fresh handle leaves the other fields zero
        for (int f = 0; f < h->planes; ++f)
            CU(cudaMemsetAsync((char *)h->base + h->plane_index(h->cur, f) * pb, 0, pb, h->stream));
    } else if (h->precision == AHS_PREC_FP32_COMPENSATED && which != AHS_FIELD_LOW &&
               (which == AHS_FIELD_PI || which == AHS_FIELD_E || which == AHS_FIELD_ALL)) {
        // new momenta replace their low words too
        const int lf = which == AHS_FIELD_E ? 12 : 10, lc = which == AHS_FIELD_PI ? 2 : which == AHS_FIELD_E ? 3 : 5;
        CU(cudaMemsetAsync((char *)h->base + h->plane_index(h->cur, lf) * pb, 0, pb * lc, h->stream));
    }
    for (int i = 0; i < count; ++i)
        CU(cudaMemcpyAsync((char *)h->base + h->plane_index(h->cur, first + i) * pb, (const char *)src + (size_t)i * pb,
                           pb, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->ready = true;
    return ok();
}

int ahs_fields_box(ahs_t *h, int which, int x0, int y0, int z0, int nx, int ny, int nz, void *dst, size_t bytes)
{
    if (!h || !dst) return fail(AHS_EINVAL, "null argument");
    int first, count;
    if (!selector(which, &first, &count)) return fail(AHS_EINVAL, "unknown field selector %d", which);
    const int N = h->N;
    if (nx < 1 || ny < 1 || nz < 1 || nx > N || ny > N || nz > N) return fail(AHS_EINVAL, "box extent outside [1, N]");
    const size_t per = (size_t)nx * ny * nz;
    if (bytes != sizeof(float) * per * count) return fail(AHS_EINVAL, "buffer is %zu bytes, box needs %zu", bytes, sizeof(float) * per * count);
    if (!h->ready) return fail(AHS_ESTATE, "fields not initialised");
    if (h->precision == AHS_PREC_FP64) return fail(AHS_EINVAL, "box copies are float32 only");
    if (int r = set_device(h)) return r;
    auto md = [N](int v) { v %= N; return v < 0 ? v + N : v; };
    const float *planes[10];
    for (int i = 0; i < count; ++i) planes[i] = h->plane(h->cur, first + i);
    float *tmp = nullptr;
    CU(cudaMallocAsync(&tmp, sizeof(float) * per * count, h->stream));
    cudaError_t e = launch_gather_box(planes, count, N, md(x0), md(y0), md(z0), nx, ny, nz, tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(tmp, h->stream);
    if (e != cudaSuccess) return fail(AHS_ECUDA, "box copy: %s", cudaGetErrorString(e));
    CU(cudaStreamSynchronize(h->stream));
    return ok();
}

int ahs_windings(ahs_t *h, int8_t *dst, size_t bytes, int64_t *n_wind)
{
    if (!h || !dst) return fail(AHS_EINVAL, "null argument");
    if (bytes != 3 * h->V) return fail(AHS_EINVAL, "buffer is %zu bytes, windings need %zu", bytes, 3 * h->V);
    if (!h->ready) return fail(AHS_ESTATE, "fields not initialised");
    if (h->precision == AHS_PREC_FP64) return fail(AHS_EINVAL, "the winding field is float32 only (the FP64 measurement counts windings)");
    if (int r = set_device(h)) return r;
    int8_t *W = nullptr;
    CU(cudaMallocAsync(&W, bytes, h->stream));
    const int c = h->cur;
    cudaError_t e = launch_windings(h->plane(c, 0), h->plane(c, 1), h->plane(c, 4), h->plane(c, 5), h->plane(c, 6), h->N,
                                    W, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, W, bytes, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(W, h->stream);
    if (e != cudaSuccess) return fail(AHS_ECUDA, "windings: %s", cudaGetErrorString(e));
    CU(cudaStreamSynchronize(h->stream));
    if (n_wind) {
        int64_t t = 0;
        for (size_t i = 0; i < bytes; ++i) t += dst[i] < 0 ? -dst[i] : dst[i];
        *n_wind = t;
    }
    return ok();
}

int ahs_autotune(ahs_t *h)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    if (!h->ready) return fail(AHS_ESTATE, "fields not initialised");
    if (h->precision == AHS_PREC_FP64) return fail(AHS_EINVAL, "the FP64 kernel has a fixed launch shape");
    if (h->inplace) return fail(AHS_ESTATE, "autotuning times real steps, which would advance in-place momenta");
    if (int r = set_device(h)) return r;
    const StepCoef k = coefficients(h, h->n);
    const StepPtrs p = pointers(h);
    const bool comp = h->precision == AHS_PREC_FP32_COMPENSATED;
    cudaEvent_t e0 = event_at(h, 0), e1 = event_at(h, 1);
    if (!e0 || !e1) return fail(AHS_ECUDA, "cudaEventCreate failed");
    const int bys[2] = {8, 16}, dzs[8] = {0, 4, 8, 16, 32, 64, 128, 256};   // 0: the automatic chunk
    double best = 1e300;
    int best_by = 8, best_dz = 0;
    for (int by : bys)
        for (int dz : dzs) {
            if (dz > h->N) continue;
            const StepShape sh = step_shape(h->N, by, dz);
            CU(launch_step(p, k, h->N, sh, false, true, nullptr, h->stream, comp));   // warm-up
            float tot = 0.f, ms = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                CU(cudaEventRecord(e0, h->stream));
                CU(launch_step(p, k, h->N, sh, false, true, nullptr, h->stream, comp));
                CU(cudaEventRecord(e1, h->stream));
                CU(cudaEventSynchronize(e1));
                CU(cudaEventElapsedTime(&ms, e0, e1));
                tot += ms;
            }
            if (tot < best) {
                best = tot;
                best_by = by;
                best_dz = dz;
            }
        }
    // then the measuring step's tile height at that z-chunk, by timing measure-only
    // launches (they write only the partial rows)
    StepCoef km = k;
    km.gauss = 1;
    double mbest = 1e300;
    int best_mby = 4;
    for (int mby : {4, 8, 16}) {
        const StepShape sh = measure_shape(h->N, mby, best_dz);
        if (int r = ensure_partials(h, sh.blocks)) return r;
        CU(launch_step(p, km, h->N, sh, true, false, h->partials, h->stream, comp));   // warm-up
        float tot = 0.f, ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            CU(cudaEventRecord(e0, h->stream));
            CU(launch_step(p, km, h->N, sh, true, false, h->partials, h->stream, comp));
            CU(cudaEventRecord(e1, h->stream));
            CU(cudaEventSynchronize(e1));
            CU(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        if (tot < mbest) {
            mbest = tot;
            best_mby = mby;
        }
    }
    h->tile_y = best_by;
    h->zchunk = best_dz;
    h->measure_tile_y = best_mby;
    return ok();
}

int ahs_stable_dt(double dx, double lambda0, double e0, double sigma, double s, int era, double tau0,
                  double tau_end, double s_cg, double tau_cg, double safety, double *dt)
{
    if (!dt) return fail(AHS_EINVAL, "null argument");
    if (!(dx > 0) || !std::isfinite(dx) || !std::isfinite(lambda0) || !std::isfinite(e0) || !std::isfinite(sigma) ||
        !std::isfinite(s) || !std::isfinite(s_cg) || !std::isfinite(tau_cg))
        return fail(AHS_EINVAL, "dx must be positive and the couplings finite");
    if (era < 0 || era > 2) return fail(AHS_EINVAL, "era=%d not in {0,1,2}", era);
    if (!(tau0 > 0) || !std::isfinite(tau0) || !(tau_end >= tau0) || !std::isfinite(tau_end))
        return fail(AHS_EINVAL, "need 0 < tau0 <= tau_end");
    if (!(safety > 0) || !(safety <= 1)) return fail(AHS_EINVAL, "safety must be in (0, 1]");
    eng::LatticeParams lp;
    lp.dx = dx;
    lp.lambda0 = lambda0;
    lp.e0 = e0;
    lp.sigma = sigma;
    lp.s = s;
    lp.era = era;
    lp.tau0 = tau0;
    lp.s_cg = s_cg;
    lp.tau_cg = tau_cg;
    const double v = eng::stable_dt(&lp, tau_end, safety);
    if (!(v > 0) || !std::isfinite(v)) return fail(AHS_EINVAL, "no stable step for these parameters");
    *dt = v;
    return ok();
}

int ahs_bounds_check(int op, int64_t *count)
{
    if (!count || op < 0 || op > 2) return fail(AHS_EINVAL, "need a count pointer and op 0, 1 or 2");
    unsigned long long a = 0, b = 0;
    cudaError_t e = bounds_errors_step(&a, op);
    if (e == cudaErrorNotSupported)
        return fail(AHS_ESTATE, "index checks are compiled only into the bounds-check build (-DAHS_BOUNDS_CHECK)");
    if (e == cudaSuccess) e = bounds_errors_step2(&b, op);
    if (e != cudaSuccess) return fail(AHS_ECUDA, "bounds counters: %s", cudaGetErrorString(e));
    *count = (int64_t)(a + b);
    return ok();
}

int ahs_kernel_time(ahs_t *h, int kind, double *ms, int64_t *launches, int reset)
{
    if (!h) return fail(AHS_EINVAL, "null handle");
    if (kind != AHS_KERNEL_STEP && kind != AHS_KERNEL_STEP_MEASURE && kind != AHS_KERNEL_STEP_PAIR)
        return fail(AHS_EINVAL, "unknown kernel kind %d", kind);
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_launches[kind];
    if (reset) {
        h->prof_ms[kind] = 0.0;
        h->prof_launches[kind] = 0;
    }
    return ok();
}

}  // extern "C"
