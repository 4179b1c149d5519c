// ahs_batch.cu -- batched ensembles: many independent realisations of uneven box
// sizes and eras advanced together by one persistent step launch per leapfrog
// step, recorded once into a CUDA graph of one measurement period and replayed.
//
// Every member runs the same step as a single lattice (Eqs. 7-10, the z-marching
// tile of ahs_step.cu) with the same FP64 per-step coefficients, so a member's
// fields are bit-identical to a single-lattice run of the same seed and launch
// shape.  Members stop at their own last step (half light-crossing, Sec. 2, by
// default) while the others continue.  Three work lists: the measuring steps of
// all members on one-site 32 x mby tiles (their partial rows are the rows of a
// single lattice's measuring launch, so the records match too); the plain steps
// of members of even side on paired 64 x 8 tiles (the single lattice's plain step
// on even N); the plain steps of members of odd side on one-site tiles.
#include "ahs_host.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

using namespace eng;

namespace {

int bfail(int code, const char *msg) { return report_error(code, msg); }

int cuda_fail(const char *what, cudaError_t e)
{
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return report_error(e == cudaErrorMemoryAllocation ? AHS_ENOMEM : AHS_ECUDA, msg);
}

#define BCU(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
    } while (0)

constexpr int kFields = 10;

}  // namespace

struct ahs_batch {
    int count = 0;
    std::vector<LatticeParams> prm;
    std::vector<uint64_t> seed;
    std::vector<int64_t> n_end;
    std::vector<size_t> off;      // float offset of each member in the arena
    std::vector<int> dz;          // z-chunk per member
    int by = 8;                   // one-site plain tiles (odd sides)
    int mby = 4;                  // measuring tiles
    int measure_every = 10;
    int use_graph = 1;
    int profile = 0;
    int device = 0;

    float *arena = nullptr;
    size_t arena_floats = 0;

    // device tables
    BatchMember *d_members = nullptr;
    BatchTile *d_tiles = nullptr; // measuring steps: one-site tiles of every member
    int ntiles = 0;
    int *d_live = nullptr;        // live tiles per step
    int *d_tickets = nullptr;     // tile tickets per step
    BatchTile *d_ptiles = nullptr;   // plain steps, even side: paired tiles
    int nptiles = 0;
    int *d_plive = nullptr, *d_ptickets = nullptr;
    BatchTile *d_otiles = nullptr;   // plain steps, odd side: one-site tiles
    int notiles = 0;
    int *d_olive = nullptr, *d_otickets = nullptr;
    double *d_partials = nullptr;
    int rows_cap = 0;
    StepCoef *d_coef = nullptr;
    int coef_stride = 0;
    ObsScalars *d_obs = nullptr;
    int obs_stride = 0;
    int64_t *d_counter = nullptr;
    ahs_obs_t *d_records = nullptr;
    ahs_obs_t *h_records = nullptr;
    int rcap = 0;
    std::vector<BatchMember> members;
    bool tables_dirty = true;
    bool tiles_dirty = true;

    int grid_plain = 0, grid_meas = 0, grid_pair = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t gexec = nullptr;
    bool graph_dirty = true;

    // on-demand measurement of one member (ahs_batch_measure)
    double *d_mpart = nullptr;
    int mpart_rows = 0;
    ahs_obs_t *d_mrec = nullptr, *h_mrec = nullptr;

    int64_t n = 0;
    bool ready = false;
    std::vector<std::vector<ahs_obs_t>> log;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double prof_ms = 0.0;
    int64_t prof_steps = 0;

    int64_t max_end() const
    {
        int64_t m = 0;
        for (int64_t e : n_end) m = std::max(m, e);
        return m;
    }
    int64_t member_time(int m) const { return std::min(n, n_end[m]); }
    float *plane(int m, int buf, int f) const
    {
        const size_t V = (size_t)prm[m].N * prm[m].N * prm[m].N;
        return arena + off[m] + ((size_t)buf * kFields + f) * V;
    }
};

namespace {

int period(const ahs_batch_t *b) { return b->measure_every > 0 ? b->measure_every : 10; }

void free_lists(ahs_batch_t *b)
{
    cudaFree(b->d_members); b->d_members = nullptr;
    for (BatchTile **t : {&b->d_tiles, &b->d_ptiles, &b->d_otiles}) {
        cudaFree(*t);
        *t = nullptr;
    }
    for (int **a : {&b->d_live, &b->d_tickets, &b->d_plive, &b->d_ptickets, &b->d_olive, &b->d_otickets}) {
        cudaFree(*a);
        *a = nullptr;
    }
    b->ntiles = b->nptiles = b->notiles = 0;
}

void free_tables(ahs_batch_t *b)
{
    free_lists(b);
    cudaFree(b->d_partials); b->d_partials = nullptr;
    cudaFree(b->d_coef); b->d_coef = nullptr;
    cudaFree(b->d_obs); b->d_obs = nullptr;
    cudaFree(b->d_records); b->d_records = nullptr;
    if (b->h_records) cudaFreeHost(b->h_records);
    b->h_records = nullptr;
}

void drop_graph(ahs_batch_t *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_dirty = true;
}

StepPtrs member_ptrs(const ahs_batch_t *b, int m, int buf)
{
    StepPtrs p;
    const int o = 1 - buf;
    p.pr = b->plane(m, buf, 0); p.pim = b->plane(m, buf, 1);
    p.qr = b->plane(m, buf, 2); p.qi = b->plane(m, buf, 3);
    p.tx = b->plane(m, buf, 4); p.ty = b->plane(m, buf, 5); p.tz = b->plane(m, buf, 6);
    p.ex = b->plane(m, buf, 7); p.ey = b->plane(m, buf, 8); p.ez = b->plane(m, buf, 9);
    p.pr1 = b->plane(m, o, 0); p.pim1 = b->plane(m, o, 1);
    p.qr1 = b->plane(m, o, 2); p.qi1 = b->plane(m, o, 3);
    p.tx1 = b->plane(m, o, 4); p.ty1 = b->plane(m, o, 5); p.tz1 = b->plane(m, o, 6);
    p.ex1 = b->plane(m, o, 7); p.ey1 = b->plane(m, o, 8); p.ez1 = b->plane(m, o, 9);
    return p;
}

// work lists: members in decreasing order of their last step (ties: larger first),
// each member's tiles in (z-chunk, y, x) order; live[n] counts the tiles of the
// members with n < n_end, a prefix of the list
int upload_list(ahs_batch_t *b, const std::vector<BatchTile> &tiles, const std::vector<int> &live, BatchTile **d_t,
                int **d_live, int **d_tickets)
{
    const size_t steps = live.size();
    if (tiles.empty()) return AHS_OK;
    BCU(cudaMalloc(d_t, sizeof(BatchTile) * tiles.size()));
    BCU(cudaMalloc(d_live, sizeof(int) * steps));
    BCU(cudaMalloc(d_tickets, sizeof(int) * steps));
    BCU(cudaMemcpy(*d_t, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice));
    BCU(cudaMemcpy(*d_live, live.data(), sizeof(int) * steps, cudaMemcpyHostToDevice));
    BCU(cudaMemset(*d_tickets, 0, sizeof(int) * steps));
    return AHS_OK;
}

int build_tiles(ahs_batch_t *b)
{
    b->members.assign(b->count, BatchMember{});
    std::vector<int> order(b->count);
    for (int m = 0; m < b->count; ++m) order[m] = m;
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
        if (b->n_end[i] != b->n_end[j]) return b->n_end[i] > b->n_end[j];
        return b->prm[i].N > b->prm[j].N;
    });
    const int64_t steps = b->max_end() + 1;
    // the tiles of the members `use` accepts, wx sites wide and by rows high
    auto make = [&](auto use, int wx, int by, std::vector<BatchTile> &tiles, std::vector<int> &live, bool rows) {
        live.assign((size_t)steps, 0);
        for (int m : order) {
            if (!use(m)) continue;
            const int N = b->prm[m].N, dz = std::max(1, std::min(b->dz[m], N));
            const int first = (int)tiles.size();
            for (int z0 = 0; z0 < N; z0 += dz)
                for (int y0 = 0; y0 < N; y0 += by)
                    for (int x0 = 0; x0 < N; x0 += wx) tiles.push_back(BatchTile{m, x0, y0, z0, std::min(z0 + dz, N), 0});
            const int cnt = (int)tiles.size() - first;
            if (rows) {
                b->members[m].row0 = first;
                b->members[m].nrows = cnt;
            }
            for (int64_t n = 0; n < std::min<int64_t>(steps, b->n_end[m]); ++n) live[(size_t)n] += cnt;
        }
    };
    for (int m = 0; m < b->count; ++m) {
        BatchMember &mb = b->members[m];
        mb.base = b->plane(m, 0, 0);
        mb.N = b->prm[m].N;
        mb.n_end = b->n_end[m];
    }
    std::vector<BatchTile> tm, tp, to;
    std::vector<int> lm, lp, lo;
    make([](int) { return true; }, 32, b->mby, tm, lm, true);
    make([&](int m) { return b->prm[m].N % 2 == 0; }, 64, 8, tp, lp, false);
    make([&](int m) { return b->prm[m].N % 2 != 0; }, 32, b->by, to, lo, false);
    BatchMember *keep_members = nullptr;
    std::swap(keep_members, b->d_members);
    free_lists(b);
    b->d_members = keep_members;
    if (!b->d_members) BCU(cudaMalloc(&b->d_members, sizeof(BatchMember) * b->count));
    BCU(cudaMemcpy(b->d_members, b->members.data(), sizeof(BatchMember) * b->count, cudaMemcpyHostToDevice));
    if (int r = upload_list(b, tm, lm, &b->d_tiles, &b->d_live, &b->d_tickets)) return r;
    if (int r = upload_list(b, tp, lp, &b->d_ptiles, &b->d_plive, &b->d_ptickets)) return r;
    if (int r = upload_list(b, to, lo, &b->d_otiles, &b->d_olive, &b->d_otickets)) return r;
    b->ntiles = (int)tm.size();
    b->nptiles = (int)tp.size();
    b->notiles = (int)to.size();
    if (b->ntiles > b->rows_cap) {
        cudaFree(b->d_partials);
        b->d_partials = nullptr;
        BCU(cudaMalloc(&b->d_partials, sizeof(double) * NQ * (size_t)b->ntiles));
        b->rows_cap = b->ntiles;
    }
    b->grid_meas = std::min(batch_grid(b->mby, true), b->ntiles);
    b->grid_plain = b->notiles ? std::min(batch_grid(b->by, false), b->notiles) : 0;
    b->grid_pair = b->nptiles ? std::min(batch_pair_grid(), b->nptiles) : 0;
    if (b->grid_meas < 1 || (b->notiles && b->grid_plain < 1) || (b->nptiles && b->grid_pair < 1))
        return bfail(AHS_ECUDA, "cannot size the persistent batch launch");
    b->tiles_dirty = false;
    drop_graph(b);
    return AHS_OK;
}

// FP64 per-step coefficients and measurement scalars of every member
int build_tables(ahs_batch_t *b)
{
    const int64_t steps = b->max_end() + 1;
    const int G = b->measure_every;
    b->coef_stride = (int)steps;
    b->obs_stride = G > 0 ? (int)(steps / G + 1) : 1;
    b->rcap = b->obs_stride;
    std::vector<StepCoef> coef((size_t)b->count * steps);
    std::vector<ObsScalars> obs((size_t)b->count * b->obs_stride);
    for (int m = 0; m < b->count; ++m) {
        for (int64_t n = 0; n < steps; ++n) coef[(size_t)m * steps + n] = coefficients(&b->prm[m], n);
        for (int sl = 0; sl < b->obs_stride; ++sl)
            obs[(size_t)m * b->obs_stride + sl] = obs_scalars(&b->prm[m], (int64_t)sl * (G > 0 ? G : 1));
    }
    cudaFree(b->d_coef); b->d_coef = nullptr;
    cudaFree(b->d_obs); b->d_obs = nullptr;
    cudaFree(b->d_records); b->d_records = nullptr;
    if (b->h_records) cudaFreeHost(b->h_records);
    b->h_records = nullptr;
    BCU(cudaMalloc(&b->d_coef, sizeof(StepCoef) * coef.size()));
    BCU(cudaMalloc(&b->d_obs, sizeof(ObsScalars) * obs.size()));
    BCU(cudaMalloc(&b->d_records, sizeof(ahs_obs_t) * (size_t)b->count * b->rcap));
    BCU(cudaMallocHost(&b->h_records, sizeof(ahs_obs_t) * (size_t)b->count * b->rcap));
    BCU(cudaMemcpy(b->d_coef, coef.data(), sizeof(StepCoef) * coef.size(), cudaMemcpyHostToDevice));
    BCU(cudaMemcpy(b->d_obs, obs.data(), sizeof(ObsScalars) * obs.size(), cudaMemcpyHostToDevice));
    b->tables_dirty = false;
    drop_graph(b);
    return AHS_OK;
}

// the launch arguments of one work list: measuring (0), plain paired (1), plain
// one-site of odd sides (2)
BatchLaunch launch_args(const ahs_batch_t *b, int list = 0)
{
    BatchLaunch L;
    L.tiles = list == 1 ? b->d_ptiles : list == 2 ? b->d_otiles : b->d_tiles;
    L.ntiles = list == 1 ? b->nptiles : list == 2 ? b->notiles : b->ntiles;
    L.live = list == 1 ? b->d_plive : list == 2 ? b->d_olive : b->d_live;
    L.tickets = list == 1 ? b->d_ptickets : list == 2 ? b->d_otickets : b->d_tickets;
    L.members = b->d_members;
    L.nmembers = b->count;
    L.coef = b->d_coef;
    L.coef_stride = b->coef_stride;
    L.counter = b->d_counter;
    L.partials = b->d_partials;
    return L;
}

// one plain step of every member: the paired launch (even sides) and the one-site
// launch (odd sides), each only if it has tiles
cudaError_t enqueue_plain(const ahs_batch_t *b, int d, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (b->nptiles) e = launch_batch_pair_step(launch_args(b, 1), d, b->grid_pair, st);
    if (e == cudaSuccess && b->notiles) e = launch_batch_step(launch_args(b, 2), b->by, d, false, b->grid_plain, st);
    return e;
}

// enqueue steps n .. n+len-1 (the first measures when it is a measurement step)
cudaError_t enqueue_steps(ahs_batch_t *b, int64_t n0, int len, cudaStream_t st)
{
    const BatchLaunch L = launch_args(b);
    const int G = b->measure_every;
    for (int d = 0; d < len; ++d) {
        const bool meas = G > 0 && ((n0 + d) % G == 0);
        cudaError_t e = meas ? launch_batch_step(L, b->mby, d, true, b->grid_meas, st) : enqueue_plain(b, d, st);
        if (e != cudaSuccess) return e;
        if (meas) {
            e = launch_batch_reduce(b->d_partials, b->d_members, b->count, b->d_obs, b->obs_stride, b->d_counter, d, G,
                                    b->d_records, b->rcap, st);
            if (e != cudaSuccess) return e;
        }
    }
    return launch_advance(b->d_counter, len, st);
}

int ensure_graph(ahs_batch_t *b)
{
    if (!b->graph_dirty && b->gexec) return AHS_OK;
    drop_graph(b);
    cudaGraph_t g = nullptr;
    BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_steps(b, 0, period(b), b->stream);   // n0 = 0: the period starts on a measurement step
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail("graph capture", e);
    }
    if (e2 != cudaSuccess) return cuda_fail("cudaStreamEndCapture", e2);
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        return cuda_fail("cudaGraphInstantiate", e);
    }
    b->graph_dirty = false;
    return AHS_OK;
}

int check_member(const ahs_batch_t *b, int m)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    if (m < 0 || m >= b->count) return bfail(AHS_EINVAL, "member index out of range");
    return AHS_OK;
}

bool selector(int which, int *first, int *count)
{
    switch (which) {
    case AHS_FIELD_PHI: *first = 0; *count = 2; return true;
    case AHS_FIELD_PI: *first = 2; *count = 2; return true;
    case AHS_FIELD_THETA: *first = 4; *count = 3; return true;
    case AHS_FIELD_E: *first = 7; *count = 3; return true;
    case AHS_FIELD_ALL: *first = 0; *count = 10; return true;
    default: return false;
    }
}

}  // namespace

extern "C" {

ahs_batch_t *ahs_batch_create(int count, const int *N, const int *era, const uint64_t *seed, const int64_t *n_end,
                              double dx, double dt, double lambda0, double e0, double sigma, double s)
{
    if (count < 1 || count > 4096 || !N || !era || !seed) {
        bfail(AHS_EINVAL, "count must be in [1, 4096] and N, era, seed non-NULL");
        return nullptr;
    }
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt) || !std::isfinite(lambda0) ||
        !std::isfinite(e0) || e0 == 0 || !std::isfinite(sigma) || !std::isfinite(s)) {
        bfail(AHS_EINVAL, "invalid couplings or spacings");
        return nullptr;
    }
    ahs_batch_t *b = new (std::nothrow) ahs_batch_t;
    if (!b) {
        bfail(AHS_ENOMEM, "host allocation");
        return nullptr;
    }
    b->count = count;
    size_t total = 0;
    for (int m = 0; m < count; ++m) {
        if (N[m] < 4 || N[m] > 512 || era[m] < 0 || era[m] > 2) {
            bfail(AHS_EINVAL, "member N outside [4, 512] or era not in {0,1,2}");
            delete b;
            return nullptr;
        }
        LatticeParams p;
        p.N = N[m]; p.dx = dx; p.dt = dt; p.lambda0 = lambda0; p.e0 = e0; p.sigma = sigma; p.s = s; p.era = era[m];
        b->prm.push_back(p);
        b->seed.push_back(seed[m]);
        int64_t e = n_end ? n_end[m] : (int64_t)std::llround((0.5 * dx * N[m] - p.tau0) / dt);
        if (e < 0 || e > (int64_t)1 << 30) {
            bfail(AHS_EINVAL, "member end step out of range");
            delete b;
            return nullptr;
        }
        b->n_end.push_back(e);
        b->off.push_back(total);
        b->dz.push_back(step_shape(N[m], 8, 0).dz);
        total += (size_t)2 * kFields * N[m] * N[m] * N[m];
    }
    b->arena_floats = total;
    b->log.assign(count, {});
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        bfail(AHS_ECUDA, "no CUDA device");
        delete b;
        return nullptr;
    }
    cudaError_t e = cudaMalloc(&b->arena, sizeof(float) * total);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->own_stream = true;
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e != cudaSuccess) {
        cuda_fail("batch allocation", e);
        cudaGetLastError();
        ahs_batch_destroy(b);
        return nullptr;
    }
    if (build_tiles(b) != AHS_OK || build_tables(b) != AHS_OK) {
        ahs_batch_destroy(b);
        return nullptr;
    }
    report_ok();
    return b;
}

void ahs_batch_destroy(ahs_batch_t *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    free_tables(b);
    cudaFree(b->d_counter);
    cudaFree(b->arena);
    cudaFree(b->d_mpart);
    cudaFree(b->d_mrec);
    if (b->h_mrec) cudaFreeHost(b->h_mrec);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int ahs_batch_init(ahs_batch_t *b)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    BCU(cudaSetDevice(b->device));
    for (int m = 0; m < b->count; ++m) {
        const size_t V = (size_t)b->prm[m].N * b->prm[m].N * b->prm[m].N;
        BCU(cudaMemsetAsync(b->plane(m, 0, 2), 0, sizeof(float) * V * 8, b->stream));
        BCU(launch_init(b->plane(m, 0, 0), b->plane(m, 0, 1), b->prm[m].N, b->seed[m], b->prm[m].sigma, b->stream));
    }
    b->n = 0;
    BCU(cudaMemsetAsync(b->d_counter, 0, sizeof(int64_t), b->stream));
    for (int *t : {b->d_tickets, b->d_ptickets, b->d_otickets})
        if (t) BCU(cudaMemsetAsync(t, 0, sizeof(int) * (size_t)(b->max_end() + 1), b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    for (auto &l : b->log) l.clear();
    b->ready = true;
    return report_ok();
}

int ahs_batch_run(ahs_batch_t *b, int max_steps)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    if (max_steps < 0) return bfail(AHS_EINVAL, "negative step count");
    if (!b->ready) return bfail(AHS_ESTATE, "batch not initialised");
    BCU(cudaSetDevice(b->device));
    if (b->tiles_dirty)
        if (int r = build_tiles(b)) return r;
    if (b->tables_dirty)
        if (int r = build_tables(b)) return r;
    const int64_t left = b->max_end() - b->n;
    const int64_t S = std::min<int64_t>(max_steps, std::max<int64_t>(left, 0));
    if (S == 0) return report_ok(), 0;
    const int P = period(b);
    const int64_t n_first = b->n;
    if (b->profile) BCU(cudaEventRecord(b->ev0, b->stream));
    int64_t done = 0;
    while (done < S) {
        const int64_t n = b->n;
        if (b->use_graph && n % P == 0 && S - done >= P) {
            if (int r = ensure_graph(b)) return r;
            BCU(cudaGraphLaunch(b->gexec, b->stream));
            b->n += P;
            done += P;
        } else {
            BCU(enqueue_steps(b, n, 1, b->stream));
            b->n += 1;
            done += 1;
        }
    }
    if (b->profile) BCU(cudaEventRecord(b->ev1, b->stream));
    // measurement records of the steps just run
    const int G = b->measure_every;
    bool bad = false;
    if (G > 0) {
        const int64_t s0 = (n_first + G - 1) / G, s1 = (b->n - 1) / G;   // slots of measured steps
        if (s1 >= s0) {
            for (int m = 0; m < b->count; ++m)
                BCU(cudaMemcpyAsync(b->h_records + (size_t)m * b->rcap + s0, b->d_records + (size_t)m * b->rcap + s0,
                                    sizeof(ahs_obs_t) * (size_t)(s1 - s0 + 1), cudaMemcpyDeviceToHost, b->stream));
        }
        BCU(cudaStreamSynchronize(b->stream));
        for (int m = 0; m < b->count; ++m)
            for (int64_t sl = s0; sl <= s1; ++sl) {
                const int64_t step = sl * G;
                if (step < n_first || step >= b->n || step >= b->n_end[m]) continue;
                const ahs_obs_t &r = b->h_records[(size_t)m * b->rcap + sl];
                b->log[m].push_back(r);
                if (r.nonfinite) bad = true;
            }
    } else {
        BCU(cudaStreamSynchronize(b->stream));
    }
    if (b->profile) {
        float ms = 0.f;
        BCU(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        b->prof_ms += ms;
        b->prof_steps += S;
    }
    if (bad) return bfail(AHS_ENONFINITE, "a member's measurement counted non-finite sites");
    report_ok();
    return (int)S;
}

int ahs_batch_records(ahs_batch_t *b, int m, ahs_obs_t *out, int max)
{
    if (int r = check_member(b, m)) return r;
    if (max < 0 || (max > 0 && !out)) return bfail(AHS_EINVAL, "bad output buffer");
    auto &l = b->log[m];
    if (max == 0) {
        report_ok();
        return (int)l.size();
    }
    const int k = std::min<int>(max, (int)l.size());
    std::copy(l.begin(), l.begin() + k, out);
    l.erase(l.begin(), l.begin() + k);
    report_ok();
    return k;
}

int ahs_batch_fields(ahs_batch_t *b, int m, int which, void *dst, size_t bytes)
{
    if (int r = check_member(b, m)) return r;
    int first, cnt;
    if (!dst || !selector(which, &first, &cnt)) return bfail(AHS_EINVAL, "bad field selector or buffer");
    const size_t V = (size_t)b->prm[m].N * b->prm[m].N * b->prm[m].N;
    if (bytes != sizeof(float) * V * cnt) return bfail(AHS_EINVAL, "buffer size does not match the field");
    if (!b->ready) return bfail(AHS_ESTATE, "batch not initialised");
    BCU(cudaSetDevice(b->device));
    const int cur = (int)(b->member_time(m) & 1);
    for (int i = 0; i < cnt; ++i)
        BCU(cudaMemcpyAsync((float *)dst + (size_t)i * V, b->plane(m, cur, first + i), sizeof(float) * V,
                            cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return report_ok();
}

int ahs_batch_set_fields(ahs_batch_t *b, int m, int which, const void *src, size_t bytes)
{
    if (int r = check_member(b, m)) return r;
    int first, cnt;
    if (!src || !selector(which, &first, &cnt)) return bfail(AHS_EINVAL, "bad field selector or buffer");
    const size_t V = (size_t)b->prm[m].N * b->prm[m].N * b->prm[m].N;
    if (bytes != sizeof(float) * V * cnt) return bfail(AHS_EINVAL, "buffer size does not match the field");
    if (!b->ready) return bfail(AHS_ESTATE, "initialise the batch before replacing a member's fields");
    BCU(cudaSetDevice(b->device));
    const int cur = (int)(b->member_time(m) & 1);
    for (int i = 0; i < cnt; ++i)
        BCU(cudaMemcpyAsync(b->plane(m, cur, first + i), (const float *)src + (size_t)i * V, sizeof(float) * V,
                            cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return report_ok();
}

int ahs_batch_measure(ahs_batch_t *b, int m, ahs_obs_t *out)
{
    if (int r = check_member(b, m)) return r;
    if (!out) return bfail(AHS_EINVAL, "null output record");
    if (!b->ready) return bfail(AHS_ESTATE, "batch not initialised");
    BCU(cudaSetDevice(b->device));
    const LatticeParams &P = b->prm[m];
    const int64_t t = b->member_time(m);
    const StepShape sh = measure_shape(P.N, b->mby, b->dz[m]);
    BCU(cudaStreamSynchronize(b->stream));
    if (sh.blocks > b->mpart_rows) {
        cudaFree(b->d_mpart);
        b->d_mpart = nullptr;
        b->mpart_rows = 0;
        BCU(cudaMalloc(&b->d_mpart, sizeof(double) * NQ * (size_t)sh.blocks));
        b->mpart_rows = sh.blocks;
    }
    if (!b->d_mrec) BCU(cudaMalloc(&b->d_mrec, sizeof(ahs_obs_t)));
    if (!b->h_mrec) BCU(cudaMallocHost(&b->h_mrec, sizeof(ahs_obs_t)));
    // the measurement launch of a single lattice (the kick of step t kept in
    // registers, nothing written) on the member's current buffer
    BCU(launch_step(member_ptrs(b, m, (int)(t & 1)), coefficients(&P, t), P.N, sh, true, false, b->d_mpart,
                    b->stream));
    BCU(launch_reduce(b->d_mpart, sh.blocks, obs_scalars(&P, t), b->d_mrec, b->stream));
    BCU(cudaMemcpyAsync(b->h_mrec, b->d_mrec, sizeof(ahs_obs_t), cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    *out = *b->h_mrec;
    return report_ok();
}

int ahs_batch_step_info(ahs_batch_t *b, int m, int64_t *n, int64_t *n_end)
{
    if (int r = check_member(b, m)) return r;
    if (n) *n = b->member_time(m);
    if (n_end) *n_end = b->n_end[m];
    return report_ok();
}

int ahs_batch_set_option(ahs_batch_t *b, int key, double v)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    switch (key) {
    case AHS_OPT_MEASURE_EVERY:
        if (!(v >= 0) || v > 1e6 || v != std::floor(v)) return bfail(AHS_EINVAL, "measure_every must be a non-negative integer");
        if (b->n % (v > 0 ? (int64_t)v : 1) != 0) return bfail(AHS_ESTATE, "change the cadence on a multiple of it");
        b->measure_every = (int)v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_ALPHA:
        if (!std::isfinite(v)) return bfail(AHS_EINVAL, "alpha must be finite");
        for (auto &p : b->prm) p.alpha = v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_TAU0:
        if (!(v > 0) || !std::isfinite(v)) return bfail(AHS_EINVAL, "tau0 must be positive");
        for (auto &p : b->prm) p.tau0 = v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_WRAP_THETA:
        if (v != 0 && v != 1) return bfail(AHS_EINVAL, "wrap_theta must be 0 or 1");
        for (auto &p : b->prm) p.wrap = (int)v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_PROFILE:
        if (v != 0 && v != 1) return bfail(AHS_EINVAL, "profile must be 0 or 1");
        b->profile = (int)v;
        return report_ok();
    case AHS_OPT_COOLING:
        if (!(v >= 0) || !std::isfinite(v) || v >= 1.0) return bfail(AHS_EINVAL, "cooling damping must be in [0, 1)");
        for (auto &p : b->prm) p.cooling = v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_CORE_GROWTH_S:
        if (!std::isfinite(v)) return bfail(AHS_EINVAL, "core-growth s must be finite");
        for (auto &p : b->prm) p.s_cg = v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_CORE_GROWTH_TAU:
        if (!std::isfinite(v)) return bfail(AHS_EINVAL, "core-growth end must be finite");
        for (auto &p : b->prm) p.tau_cg = v;
        b->tables_dirty = true;
        return report_ok();
    case AHS_OPT_TILE_Y:
        if (v != 8 && v != 16) return bfail(AHS_EINVAL, "tile_y must be 8 or 16");
        b->by = (int)v;
        b->tiles_dirty = true;
        return report_ok();
    case AHS_OPT_MEASURE_TILE_Y:
        if (v != 0 && v != 4 && v != 8 && v != 16) return bfail(AHS_EINVAL, "measure_tile_y must be 0, 4, 8 or 16");
        b->mby = v == 0 ? 4 : (int)v;
        b->tiles_dirty = true;
        return report_ok();
    case AHS_OPT_ZCHUNK:
        if (!(v >= 0) || v > 1600 || v != std::floor(v)) return bfail(AHS_EINVAL, "zchunk must be an integer in [0, 1600]");
        for (int m = 0; m < b->count; ++m) b->dz[m] = step_shape(b->prm[m].N, b->by, (int)v).dz;
        b->tiles_dirty = true;
        return report_ok();
    case AHS_OPT_GRAPH:
        if (v != 0 && v != 1) return bfail(AHS_EINVAL, "graph must be 0 or 1");
        b->use_graph = (int)v;
        return report_ok();
    case AHS_OPT_STEP:
        return bfail(AHS_EINVAL, "a batch's step is set by ahs_batch_init only");
    default:
        return bfail(AHS_EINVAL, "unknown or read-only option");
    }
}

int ahs_batch_get_option(ahs_batch_t *b, int key, double *v)
{
    if (!b || !v) return bfail(AHS_EINVAL, "null argument");
    switch (key) {
    case AHS_OPT_MEASURE_EVERY: *v = b->measure_every; break;
    case AHS_OPT_ALPHA: *v = b->prm[0].alpha; break;
    case AHS_OPT_TAU0: *v = b->prm[0].tau0; break;
    case AHS_OPT_WRAP_THETA: *v = b->prm[0].wrap; break;
    case AHS_OPT_PROFILE: *v = b->profile; break;
    case AHS_OPT_COOLING: *v = b->prm[0].cooling; break;
    case AHS_OPT_CORE_GROWTH_S: *v = b->prm[0].s_cg; break;
    case AHS_OPT_CORE_GROWTH_TAU: *v = b->prm[0].tau_cg; break;
    case AHS_OPT_TILE_Y: *v = b->by; break;
    case AHS_OPT_MEASURE_TILE_Y: *v = b->mby; break;
    case AHS_OPT_GRAPH: *v = b->use_graph; break;
    case AHS_OPT_STEP: *v = (double)b->n; break;
    default: return bfail(AHS_EINVAL, "unknown option");
    }
    return report_ok();
}

int ahs_batch_member_zchunk(ahs_batch_t *b, int m, int *dz)
{
    if (int r = check_member(b, m)) return r;
    if (dz) *dz = b->dz[m];
    return report_ok();
}

// Time one plain batched step (the persistent launches over all members, CUDA
// events, state unchanged: the step reads one buffer and writes the other and the
// step counter is not advanced) for each tile height (8 only when every side is
// even), and then per member size for each z-chunk with the other sizes held
// fixed; keep the fastest.
int ahs_batch_autotune(ahs_batch_t *b)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    if (!b->ready) return bfail(AHS_ESTATE, "batch not initialised");
    BCU(cudaSetDevice(b->device));
    if (b->tables_dirty)
        if (int r = build_tables(b)) return r;
    auto time_step = [&](float *out) -> int {
        if (b->tiles_dirty)
            if (int r = build_tiles(b)) return r;
        const int64_t n = std::min<int64_t>(b->n, b->max_end());   // the step's tile counters
        auto reset = [&]() -> int {
            for (int *t : {b->d_ptickets, b->d_otickets})
                if (t) BCU(cudaMemsetAsync(t + n, 0, sizeof(int), b->stream));
            return AHS_OK;
        };
        if (int r = reset()) return r;
        BCU(enqueue_plain(b, 0, b->stream));   // warm-up
        float best = 1e30f, ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            if (int r = reset()) return r;
            BCU(cudaEventRecord(b->ev0, b->stream));
            BCU(enqueue_plain(b, 0, b->stream));
            BCU(cudaEventRecord(b->ev1, b->stream));
            BCU(cudaEventSynchronize(b->ev1));
            BCU(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
            best = std::min(best, ms);
        }
        *out = best;
        return AHS_OK;
    };
    std::vector<int> sizes;
    for (auto &p : b->prm)
        if (std::find(sizes.begin(), sizes.end(), p.N) == sizes.end()) sizes.push_back(p.N);
    const int dzs[6] = {4, 8, 16, 32, 64, 128};
    float best_total = 1e30f;
    int best_by = b->by;
    std::vector<int> best_dz = b->dz;
    // the tile height shapes only the one-site plain tiles (members of odd side) of
    // a plain step; without those the measuring steps keep 8-row tiles
    bool any_odd = false;
    for (auto &p : b->prm) any_odd = any_odd || p.N % 2 != 0;
    for (int by : {8, 16}) {
        if (by == 16 && !any_odd) break;
        b->by = by;
        for (int m = 0; m < b->count; ++m) b->dz[m] = std::min(32, b->prm[m].N);
        b->tiles_dirty = true;
        float t = 0.f;
        for (int N : sizes) {
            int keep = std::min(32, N);
            float tbest = 1e30f;
            for (int dz : dzs) {
                if (dz > N) continue;
                for (int m = 0; m < b->count; ++m)
                    if (b->prm[m].N == N) b->dz[m] = dz;
                b->tiles_dirty = true;
                if (int r = time_step(&t)) return r;
                if (t < tbest) {
                    tbest = t;
                    keep = dz;
                }
            }
            for (int m = 0; m < b->count; ++m)
                if (b->prm[m].N == N) b->dz[m] = keep;
            b->tiles_dirty = true;
        }
        if (int r = time_step(&t)) return r;
        if (t < best_total) {
            best_total = t;
            best_by = by;
            best_dz = b->dz;
        }
    }
    b->by = best_by;
    b->dz = best_dz;
    b->tiles_dirty = true;   // rebuilt (with zeroed tickets) before the next run
    return report_ok();
}

int ahs_batch_kernel_time(ahs_batch_t *b, double *ms, int64_t *steps, int reset)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    if (ms) *ms = b->prof_ms;
    if (steps) *steps = b->prof_steps;
    if (reset) {
        b->prof_ms = 0.0;
        b->prof_steps = 0;
    }
    return report_ok();
}

int ahs_batch_set_stream(ahs_batch_t *b, void *stream)
{
    if (!b) return bfail(AHS_EINVAL, "null batch");
    if (!stream) return bfail(AHS_EINVAL, "a batch needs a non-default stream (graph capture)");
    BCU(cudaStreamSynchronize(b->stream));
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->stream = (cudaStream_t)stream;
    b->own_stream = false;
    drop_graph(b);
    return report_ok();
}

}  // extern "C"
