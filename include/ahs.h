/*
 * ahs.h -- C ABI of the GB300 engine for the lattice Abelian-Higgs string
 * evolution of Correia & Martins, "Abelian-Higgs cosmic string evolution with
 * multiple GPUs" (arXiv:2005.14454).
 *
 * One handle = one periodic comoving N^3 lattice on the current CUDA device:
 * a complex scalar phi on sites and compact U(1) link angles theta_i = dx A_i
 * (U_i = exp(-i theta_i), Eq. 13 with the dx of Eq. 16), evolved by the
 * staggered leapfrog of Eqs. 7-10 in an expanding background a = (eta/eta0)^p
 * with Crank-Nicolson damping (Eqs. 11-12), plus the string and velocity
 * diagnostics of Eqs. diagxi and diagvel.
 *
 * Conventions
 *  - Every function returns AHS_OK (0) or a negative status; ahs_create returns
 *    NULL on error.  The status of the failing call on this thread is kept in
 *    ahs_last_error(), with a message in ahs_last_error_message().  No C++
 *    exception crosses the ABI.
 *  - The library owns all device memory of a handle (cudaMalloc at create/init,
 *    cudaFree at destroy).  The caller owns every host buffer it passes; the
 *    library never keeps a host pointer after a call returns.
 *  - Calls that move data or produce observables (init, step, measure, fields,
 *    set_fields, windings, records) synchronise the handle's stream before they
 *    return.  A handle is not thread-safe; distinct handles are independent.
 *  - Field storage is float32 (FP64 in the FP64 precision mode), structure of
 *    arrays: one plane of N^3 values per real component, site index
 *    x + N*(y + N*z) (x fastest).
 */
#ifndef AHS_H
#define AHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
    AHS_OK = 0,
    AHS_EINVAL = -1,      /* bad argument (size, selector, pointer, range)          */
    AHS_ENOMEM = -2,      /* device or host allocation failed                       */
    AHS_ECUDA = -3,       /* a CUDA runtime call failed; message has the CUDA error */
    AHS_ESTATE = -4,      /* call not valid in the handle's state (e.g. not init)   */
    AHS_ENONFINITE = -5,  /* a measurement found a non-finite field value           */
    AHS_ETIMEOUT = -6     /* reserved: no kernel of this library waits on another   */
};

/* ---- expansion eras: the value is p in a = (eta/eta0)^p (Eq. defm in
 *      conformal time; p = m/(1-m) for a physical-time exponent m) ------- */
enum { AHS_MINKOWSKI = 0, AHS_RADIATION = 1, AHS_MATTER = 2 };

/* ---- field selectors ------------------------------------------------------
 * number of float32 planes: PHI 2 (Re, Im), PI 2 (Re, Im), THETA 3 (x, y, z),
 * E 3 (x, y, z), ALL 10 in the order phi, Pi, theta, E.  phi and theta live at
 * the integer time n, Pi and E at n - 1/2. */
enum { AHS_FIELD_PHI = 0, AHS_FIELD_PI = 1, AHS_FIELD_THETA = 2, AHS_FIELD_E = 3,
       AHS_FIELD_ALL = 4,
       AHS_FIELD_LOW = 5   /* compensated precision only: 5 planes, low words of Re Pi, Im Pi, E_xyz */ };

/* ---- precision modes (AHS_OPT_PRECISION; changing it discards the fields) ----
 * FP32: float32 storage and arithmetic, FP64 reductions (80 bytes/site).
 * FP32_COMPENSATED: as FP32, with Pi and E held as float32 high + low words and
 *   updated by compensated (error-free product and sum) arithmetic (120 bytes/site).
 * FP64: double storage and arithmetic for every step (160 bytes/site); field copies
 *   then move 8-byte values; box copies, the winding field and autotuning are not
 *   available. */
enum { AHS_PREC_FP32 = 0, AHS_PREC_FP32_COMPENSATED = 1, AHS_PREC_FP64 = 2 };

/* ---- options for ahs_set_option / ahs_get_option ------------------------ */
enum {
    AHS_OPT_MEASURE_EVERY = 0, /* fuse a measurement into every k-th step (0: never); default 10 */
    AHS_OPT_ALPHA = 1,         /* damping form factor alpha of Eq. 11; default 2               */
    AHS_OPT_TAU0 = 2,          /* initial conformal time eta0; default 1                       */
    AHS_OPT_STEP = 3,          /* current integer time level n (eta = eta0 + n dt)             */
    AHS_OPT_WRAP_THETA = 4,    /* 1: keep theta in (-pi, pi] after each drift; default 0       */
    AHS_OPT_PROFILE = 5,       /* 1: time every step-kernel launch with CUDA events            */
    AHS_OPT_N = 6,             /* lattice side (read only)                                     */
    AHS_OPT_TILE_Y = 7,        /* plain-step tile height: 8 or 16 rows of 32 sites; 0 = auto    */
    AHS_OPT_ZCHUNK = 8,        /* z planes one CTA marches through, 1..N; 0 = auto            */
    AHS_OPT_GRAPH = 9,         /* batches: 1 = replay each measurement period as a CUDA graph  */
    AHS_OPT_PRECISION = 10,    /* AHS_PREC_*; default FP32                                     */
    AHS_OPT_COOLING = 11,      /* > 0: cooling steps, a = 1 and delta = omega = value (the
                                  artificial damping period Sec. 2 mentions); 0 = off       */
    AHS_OPT_MOMENTA_IN_PLACE = 12, /* 1: keep one copy of Pi and E and update it in place */
    AHS_OPT_CORE_GROWTH_S = 13,   /* s of the core-growth period (see below); default 0    */
    AHS_OPT_CORE_GROWTH_TAU = 14, /* end eta_cg of the period; <= eta0 (default): none     */
    AHS_OPT_STEPS_PER_PASS = 15,  /* 1 (default) or 2: temporal blocking, see below          */
    AHS_OPT_MEASURE_TILE_Y = 16   /* tile height of measuring steps (and of ahs_measure): 4, 8
                                     or 16 rows of 32 sites; 0 = auto (4; FP64 precision: 8) */
};

/* AHS_OPT_STEPS_PER_PASS = 2 (float32 precision with double-buffered momenta only).
 * Two consecutive plain steps (neither of them a measuring step) run as one launch
 * that reads every field once at n and writes it once at n+2 (40 + 40 bytes per
 * two site-updates instead of 80 + 80, the paper's remark that the kernels are
 * memory bound, Sec. 5).  The second step of a tile needs the first step's phi and
 * theta on a one-site ring, so the first step is computed on the tile plus that
 * ring (34 x 10 sites for a 32 x 8 tile) from link phases over a two-site ring:
 * about 16% more arithmetic per site-update.  Fields are those of two single
 * steps.  A measuring step, or a step left over at the end of an ahs_step call,
 * runs alone.  The launch uses 32 x 8 tiles whatever AHS_OPT_TILE_Y says, and the
 * z-chunk of AHS_OPT_ZCHUNK.  Setting it with another precision or with in-place
 * momenta (where the first step of a neighbouring tile would overwrite momenta the
 * ring still reads) returns AHS_EINVAL, as does changing those while it is 2. */

/* Core growth (Sec. 2, after Eq. 6): a negative s makes the comoving string width
 * grow, so that the true equations (s = 1) can later shrink it without it falling
 * below the lattice spacing.  Steps with eta_n < AHS_OPT_CORE_GROWTH_TAU use the
 * exponent s_cg = AHS_OPT_CORE_GROWTH_S in omega = delta (1 - s) and c = a^{2 s};
 * later steps use the s of ahs_create, with c kept continuous at eta_cg:
 * c = a_cg^{2 s_cg} (a / a_cg)^{2 s}, a_cg = a(eta_cg).  (The paper gives no
 * switching rule; a jump of c would quench the string cores.)  Gauss's law is
 * kept exactly only where constant s keeps it (see ahs_obs_t.gauss_rms). */

/* AHS_OPT_MOMENTA_IN_PLACE (float32 precision only; changing it discards the
 * fields).  The kicks of Eqs. 7-8 give each site's new Pi and E from its own old
 * values, so Pi and E need no second buffer; phi and theta, which the stencil
 * reads at neighbours, stay double-buffered.  Device storage drops from 80 to 60
 * bytes per site (a 1536^3 lattice takes 217 GB).  The fields, records and the
 * results of every call are bit-identical to the default storage.  Costs: a
 * measuring step runs as two launches (the Gauss residual first, since it reads
 * the old E of neighbouring sites that the fused step overwrites, then the step
 * with the rest of the measurement); ahs_autotune returns AHS_ESTATE (it times
 * real steps, which would advance the momenta). */

typedef struct ahs ahs_t;

/* ---- one measurement (all FP64 reductions) --------------------------------
 * Taken at an integer time n from phi^n, theta^n and the momenta averaged over
 * the kick of step n (Pibar = (Pi^{n-1/2} + Pi^{n+1/2})/2, Ebar likewise).
 * Per site, with c = a^{2s}:
 *   K = |Pibar|^2, G = sum_i |D_i^+ phi|^2, V = (lambda0 c/4)(|phi|^2 - sigma^2)^2,
 *   El = sum_i Ebar_i^2/(2 e0^2 c), B = sum_{i<j} (1 - cos alpha_ij)/(e0^2 c dx^4),
 *   L = K - G - V + El - B, rho = K + G + V + El + B, p = K - G/3 - V + (El+B)/3.
 * xi_l = sqrt(-mu Vol/(dx^3 sum L)) with mu = 2 pi sigma^2 (Eq. diagxi, left);
 * xi_w = sqrt(Vol/string_length), string_length = (pi/6) dx n_wind, n_wind = sum
 * |W_ij| over all plaquettes (Eq. diagxi, right; pi/6 corrects the Manhattan
 * overcount of lattice paths, the convention of the paper's Table 1); v2_phi = 2R/(1+R), R = sum K L/sum G L
 * and v2_omega = (1 + 3 sum p L/sum rho L)/2 (Eq. diagvel, weight L).
 * gauss_*: residual of Gauss's law (Eq. 5 in discrete form) of the stored
 * momenta at n - 1/2 with phi^n.  nonfinite: number of sites whose diagnostic
 * was not finite.  Energies carry the dx^3 volume factor; sum_* do not. */
typedef struct ahs_obs {
    int64_t step;
    double tau, a;
    int64_t n_wind;
    double string_length, xi_w, xi_l, lagrangian;
    double v2_phi, v2_omega;
    double e_kin, e_grad, e_pot, e_elec, e_mag, e_total;
    double gauss_rms, gauss_max;
    int64_t nonfinite;
    double sum_K, sum_G, sum_V, sum_El, sum_B, sum_L;
    double sum_KL, sum_GL, sum_pL, sum_rhoL;
} ahs_obs_t;

/* ahs_create -- a lattice of side N (4 <= N <= 1600, so N^3 < 2^32) with spacing dx, time step
 * dt, couplings lambda0 and e0 (Eqs. 7-8), vacuum expectation value sigma, width
 * exponent s (lambda = lambda0 a^{-2(1-s)}, e = e0 a^{-(1-s)}, so the potential
 * and the current carry a^{2s}; Eq. 6 read with Eqs. 7-8), and era p in
 * {0, 1, 2}.  The field storage -- 80 bytes of device memory per site by
 * default: all ten field components double buffered, so a step reads one copy
 * and writes the other (see AHS_OPT_PRECISION and AHS_OPT_MOMENTA_IN_PLACE for
 * the other layouts) -- is allocated by the first ahs_init or ahs_set_fields,
 * which return AHS_ENOMEM if it does not fit; options that change the layout
 * free it.  Fields are undefined until ahs_init or ahs_set_fields.  NULL on
 * error (EINVAL, ENOMEM, ECUDA). */
ahs_t *ahs_create(int N, double dx, double dt, double lambda0, double e0,
                  double sigma, double s, int era);

/* ahs_init -- random-phase initial condition of Sec. 2 at n = 0: phi(x) =
 * sigma e^{i vartheta(x)}, Pi = theta = E = 0, with vartheta = 2 pi u and
 * u = (sm64(seed ^ sm64(idx)) >> 11) 2^-53, sm64 one SplitMix64 step (Steele,
 * Lea & Flood 2014); phase and cos/sin in FP64, stored rounded to float32.
 * Clears the measurement log. */
int ahs_init(ahs_t *h, uint64_t seed);

/* ahs_step -- n >= 0 leapfrog steps (Eqs. 7-10): kick Pi and E at n -> n+1/2
 * with the old phi, theta, then drift phi and theta to n+1.  Steps whose index
 * is a multiple of AHS_OPT_MEASURE_EVERY also measure (fused into the same
 * kernel) the state they start from and append the record to the log (see
 * ahs_records).  Returns AHS_ENONFINITE (after completing all n steps) if any
 * measurement of this call counted a non-finite site. */
int ahs_step(ahs_t *h, int n);

/* ahs_measure -- measure the current state (integer time n) without changing
 * it: the kick of step n runs with its results kept in registers. */
int ahs_measure(ahs_t *h, ahs_obs_t *out);

/* ahs_records -- move up to max records of the measurement log (oldest first)
 * into out; returns the number moved (>= 0) or a negative status.  out may be
 * NULL with max 0 to query the number pending. */
int ahs_records(ahs_t *h, ahs_obs_t *out, int max);

/* ahs_fields / ahs_set_fields -- copy one field (see the selectors) between the
 * device and a host buffer of exactly planes * N^3 * 4 bytes (8 in FP64 precision),
 * planes in the selector's order.  set_fields leaves the time level n unchanged;
 * in compensated precision, setting Pi or E clears their low words. */
int ahs_fields(ahs_t *h, int which, void *host_dst, size_t bytes);
int ahs_set_fields(ahs_t *h, int which, const void *host_src, size_t bytes);

/* ahs_fields_box -- copy the periodic sub-box [x0, x0+nx) x [y0, y0+ny) x
 * [z0, z0+nz) (coordinates taken modulo N, 1 <= n* <= N) of one field into a
 * host buffer of planes * nx * ny * nz * 4 bytes, x fastest. */
int ahs_fields_box(ahs_t *h, int which, int x0, int y0, int z0, int nx, int ny,
                   int nz, void *host_dst, size_t bytes);

/* ahs_windings -- the plaquette windings W_ij of the current state (gauge
 * invariant form of Kajantie et al. 1998, cited for xi_W): 3 int8 planes
 * (xy, xz, yz) of N^3, W_ij(x) for the plaquette with lower corner x.  bytes
 * must be 3 * N^3.  Writes the total sum |W| to *n_wind when non-NULL. */
int ahs_windings(ahs_t *h, int8_t *host_dst, size_t bytes, int64_t *n_wind);

/* ahs_set_option / ahs_get_option -- see AHS_OPT_*.  Values are validated
 * (EINVAL).  AHS_OPT_N is read only. */
int ahs_set_option(ahs_t *h, int key, double value);
int ahs_get_option(ahs_t *h, int key, double *value);

/* ahs_set_stream -- run this handle's work on an existing CUDA stream
 * (cudaStream_t passed as void*; NULL selects the legacy default stream).  The
 * stream must belong to the device the handle was created on and outlive it. */
int ahs_set_stream(ahs_t *h, void *cuda_stream);

/* ahs_kernel_time -- with AHS_OPT_PROFILE on: total device time (ms, CUDA
 * events recorded on the handle's stream around each launch) and number of
 * launches of the step kernel since the last reset.  kind selects the plain
 * step kernel (AHS_KERNEL_STEP), the step kernel with the fused measurement
 * (AHS_KERNEL_STEP_MEASURE) or the two-step kernel of AHS_OPT_STEPS_PER_PASS = 2
 * (AHS_KERNEL_STEP_PAIR, one launch per two steps); reset != 0 zeroes that
 * counter after reading. */
enum { AHS_KERNEL_STEP = 0, AHS_KERNEL_STEP_MEASURE = 1, AHS_KERNEL_STEP_PAIR = 2 };
int ahs_kernel_time(ahs_t *h, int kind, double *ms_total, int64_t *launches, int reset);

/* ahs_stable_dt -- the largest leapfrog time step that stays stable from eta0 =
 * tau0 up to conformal time tau_end, times safety (0 < safety <= 1), into *dt.
 * The staggered leapfrog of Eqs. 7-10 is stable while dt omega_max < 2; omega_max^2
 * = 12/dx^2 (largest eigenvalue of the lattice Laplacian of Eq. 14 and of the
 * lattice curl-curl of Eq. 8) + max(lambda0, 2 e0^2) sigma^2 c_max, the Higgs and
 * gauge masses squared at the largest c = a^{2s} of the run (a = (eta/tau0)^era;
 * with a core-growth period, s_cg before tau_cg and c continuous there, as
 * AHS_OPT_CORE_GROWTH_S / _TAU; tau_cg <= tau0 means none).  The paper keeps a
 * fixed dt = 0.1; this bound matters where s = 1 makes c grow (a^2 in the
 * radiation era, a^4 in the matter era).  Host arithmetic only, no device call.
 * Returns AHS_EINVAL for dx <= 0, non-finite couplings, era outside {0,1,2},
 * tau_end < tau0 or safety outside (0, 1]. */
int ahs_stable_dt(double dx, double lambda0, double e0, double sigma, double s, int era, double tau0,
                  double tau_end, double s_cg, double tau_cg, double safety, double *dt);

/* ahs_bounds_check -- the index checks of the bounds-check build of this library
 * (compiled with -DAHS_BOUNDS_CHECK: _ahs_check.so beside _ahs.so), a test aid
 * with no counterpart in the paper.  There every global offset of the step
 * kernels' tile loaders, rings and stores, and every shared-memory index of their
 * tiles, is checked against the extent it addresses; an index outside it is
 * counted and replaced by 0, so the access stays in range and no kernel traps.
 *   op 0: *count = the indices counted on the current device since the library was
 *         loaded or last reset; 1: the same, then zero the count; 2: first run a
 *         self-test that passes one out-of-range index through the check of each
 *         kernel translation unit (touching no memory), then as 1.
 * Returns AHS_ESTATE in the production build, which compiles the checks away;
 * AHS_EINVAL for a NULL count or another op. */
int ahs_bounds_check(int op, int64_t *count);

/* ahs_device_bytes -- device memory of the handle: its field storage (allocated
 * or, before the first ahs_init / ahs_set_fields, to be allocated), measurement
 * partials and records. */
int ahs_device_bytes(ahs_t *h, size_t *bytes);

/* ---- batched ensembles ---------------------------------------------------
 * Many independent realisations (members) of possibly different sides N and
 * eras, sharing dx, dt, lambda0, e0, sigma and s, advanced together: every
 * leapfrog step is one persistent launch over the tiles of all members (a plain
 * step: paired 64 x 8 tiles for members of even side, and a second launch on
 * one-site tiles if some side is odd; a measuring step: one-site tiles), and each
 * measurement period (AHS_OPT_MEASURE_EVERY steps, 10 if measurements are off)
 * is replayed as one captured CUDA graph.  A member runs the same kernels and
 * coefficients as a single lattice, so its fields and records equal those of an
 * ahs_t run of the same seed and launch shape bit for bit.  All members start at n = 0; member
 * m stops at its last step n_end[m] (default: half light-crossing, eta_end =
 * N dx / 2, Sec. 2) while the others continue.  Device memory: 80 bytes per site
 * of every member plus small tables; the batch owns a non-blocking stream. */
typedef struct ahs_batch ahs_batch_t;

/* count members with sides N[m] in [4, 512], eras era[m], seeds seed[m] and last
 * steps n_end[m] (NULL: half light-crossing).  NULL on error. */
ahs_batch_t *ahs_batch_create(int count, const int *N, const int *era, const uint64_t *seed,
                              const int64_t *n_end, double dx, double dt, double lambda0, double e0,
                              double sigma, double s);
/* random-phase initial condition of every member from its seed (as ahs_init) */
int ahs_batch_init(ahs_batch_t *b);
/* advance every member that has not reached its last step by up to max_steps
 * steps; returns the number of steps advanced (0 when all are done) or a
 * negative status (AHS_ENONFINITE after the steps if a measurement found one). */
int ahs_batch_run(ahs_batch_t *b, int max_steps);
/* measurement log of member m (as ahs_records) */
int ahs_batch_records(ahs_batch_t *b, int m, ahs_obs_t *out, int max);
/* measure member m at its current time level without changing it (as ahs_measure:
 * the member's launch shape, a record equal to the one a single lattice of the
 * same launch shape reports); synchronous on the batch's stream */
int ahs_batch_measure(ahs_batch_t *b, int m, ahs_obs_t *out);
/* fields of member m at its current time (as ahs_fields / ahs_set_fields) */
int ahs_batch_fields(ahs_batch_t *b, int m, int which, void *host_dst, size_t bytes);
int ahs_batch_set_fields(ahs_batch_t *b, int m, int which, const void *host_src, size_t bytes);
/* current time level and last step of member m */
int ahs_batch_step_info(ahs_batch_t *b, int m, int64_t *n, int64_t *n_end);
/* options: MEASURE_EVERY (change only on a multiple of the old cadence), ALPHA,
 * TAU0, WRAP_THETA, PROFILE, TILE_Y (8/16: one-site plain tiles of odd sides),
 * MEASURE_TILE_Y (4/8/16, 0 = 4: measuring tiles), ZCHUNK (all members; 0 = auto), GRAPH */
int ahs_batch_set_option(ahs_batch_t *b, int key, double value);
int ahs_batch_get_option(ahs_batch_t *b, int key, double *value);
/* z-chunk member m currently uses */
int ahs_batch_member_zchunk(ahs_batch_t *b, int m, int *dz);
/* choose the tile height and each member size's z-chunk by timing the batched
 * plain step itself (CUDA events on the batch stream; the state is not changed):
 * per tile height, each size's z-chunk in turn with the others held fixed.  The
 * tile height shapes the one-site tiles (members of odd side, measuring steps);
 * when every side is even it stays 8.  Needs an initialised batch. */
int ahs_batch_autotune(ahs_batch_t *b);
/* with AHS_OPT_PROFILE: device time of ahs_batch_run calls (ms, CUDA events on the
 * batch stream) and the steps they advanced */
int ahs_batch_kernel_time(ahs_batch_t *b, double *ms_total, int64_t *steps, int reset);
/* run on the caller's non-default stream instead of the batch's own */
int ahs_batch_set_stream(ahs_batch_t *b, void *cuda_stream);
void ahs_batch_destroy(ahs_batch_t *b);

/* ahs_autotune -- choose AHS_OPT_TILE_Y and AHS_OPT_ZCHUNK of a single lattice by
 * timing its plain step, then AHS_OPT_MEASURE_TILE_Y at that z-chunk by timing
 * measure-only launches (CUDA events, the state is not changed); needs fields. */
int ahs_autotune(ahs_t *h);

/* ahs_measure_noalloc -- the measurement of ahs_measure on fields the caller
 * owns, without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, because all of their
 * device memory belongs to another allocator (a framework's caching allocator, or
 * a pool reserved for the job up front) and a side allocation would fail,
 * fragment that pool or stall on the allocator's device-wide synchronisation.
 *   fields: device pointer to the ten float32 planes of AHS_FIELD_ALL (phi and
 *           theta at the integer time `step`, Pi and E at step - 1/2), N^3 each,
 *           site index x + N*(y + N*z); read only.
 *   out:    device pointer to one ahs_obs_t, written by the call.
 *   N, dx, dt, lambda0, e0, sigma, s, era: as for ahs_create; alpha and tau0 as
 *           the AHS_OPT_ALPHA / AHS_OPT_TAU0 options.
 *   stream: cudaStream_t (as void*) to run on; NULL for the legacy default stream.
 * The call only enqueues work: synchronise the stream before reading *out.  Its
 * scratch is a static device array of AHS_NOALLOC_MAX_ROWS rows of FP64 partial
 * sums (2 MiB) that every GPU loading this library holds until the process
 * exits; every CTA overwrites its own row, so nothing carries over between calls,
 * but calls that overlap on the GPU (other streams, other threads) share the
 * array and race.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process; make that first call before any stream capture.  The kept
 * address is not valid after cudaDeviceReset (or any other re-creation of the
 * device's primary context): do not call this entry point after one.  The launch
 * takes the automatic measuring shape of ahs_measure (32 x 4 tiles) with its
 * z-chunks lengthened until the CTAs fit the scratch rows, or 32 x 8 tiles where
 * even one chunk of 4-row tiles would not fit (N > 1440): the record equals that
 * of ahs_measure at the same launch shape, and at another one up to the grouping
 * of the FP64 sums.  Returns AHS_EINVAL for N outside [4, 1600] (a
 * lattice whose CTAs cannot fit the scratch is rejected the same way), bad
 * parameters or NULL buffers, AHS_ECUDA if a launch fails. */
#define AHS_NOALLOC_MAX_ROWS 16384
int ahs_measure_noalloc(int N, double dx, double dt, double lambda0, double e0, double sigma, double s,
                        int era, double alpha, double tau0, int64_t step, const float *fields,
                        ahs_obs_t *out, void *stream);

void ahs_destroy(ahs_t *h);

int ahs_last_error(void);
const char *ahs_last_error_message(void);
const char *ahs_strerror(int status);
size_t ahs_sizeof_obs(void);

#ifdef __cplusplus
}
#endif
#endif /* AHS_H */
